// fim.cu -- the persistent active-list Fast Iterative Method (Algorithm 2
// with the local solver of Sec. II-B): one cooperative kernel that runs
// every iteration of the solve.  The kernels around it (per-tet precompute,
// onset seeding, parent pass) are in fim_aux.cu.
#include "gbp_internal.cuh"

namespace gbp {

// Vertex state written during the solve is read through L2 only (values of
// other SMs from earlier iterations; same-iteration values may be stale,
// which the chaotic relaxation of Algorithm 2 tolerates).
#define FIM_LD(p) __ldcg(p)

// ---------------------------------------------------------------------------
struct FimArgs {
    int64_t n_v;    // vertices per problem
    int64_t n_t;    // tets per problem
    int64_t n_tot;  // n_v x problems (entries of the active lists)
    const float4 *xyz;
    const int4 *tets;
    const float4 *tf;   // unit fibre per tet (shared by the batch)
    const float2 *tv;   // (1/ct, 1/cf - 1/ct) per problem and tet
    const float4 *tlip;
    const int *n2t_ptr, *n2t, *n2n_ptr, *n2n;
    const int4 *frec;   // per vertex->tet entry: face vertex ids (slot order) and tet*4 + slot
    int2 *pc;           // per vertex entry: (value bits, iteration of the last change)
    float *phi;
    int4 *rec;
    int *chg, *stamp, *lists;
    Control *ctl;
    BarGroup *grp;
    float eps;
    int max_iters;
    int n_f;
    long long *trace;  // optional: per iteration (active vertices, global timer ns)
    int2 *defer;       // faces deferred to the FP64 repair (DEFER kernels): (vertex entry, face record)
    int resume;        // continue from the state and list the repair left (iteration numbers go on)
};

// One iteration k = one Jacobi-style sweep of Algorithm 2 restricted to the
// active vertices (neighbours of the vertices that changed at k-1).  A group
// of FIM_G lanes owns one active vertex i: its lanes take i's face records
// (the three other vertices of an incident tet and the code tet*4 + slot, in
// vertex->tet order), read each face vertex's packed (value, change stamp),
// solve the local problem of every face E_{j\i} that has a vertex changed
// since k-1 (the optional mask of Algorithm 2) and reduce the minimum
// (Eq. hopflax_global).  A vertex that
// decreased by more than eps is marked changed and activates its neighbours
// for k+1 (each appended to the next list by the lane that stamps it
// first).  Reads of neighbour values may see this
// iteration's updates (chaotic relaxation); the operator is monotone, so the
// limit is the same fixed point.
#ifndef GBP_FIM_G
#define GBP_FIM_G 8  // lanes per active vertex
#endif
#ifndef GBP_FIM_BLOCK
#define GBP_FIM_BLOCK 1024  // threads per CTA
#endif
constexpr int FIM_G = GBP_FIM_G;
constexpr int FIM_BLOCK = GBP_FIM_BLOCK;
// One CTA of 1024 threads per SM (64 registers): the same 32 warps per SM as
// four CTAs of 256, with a quarter of the grid barrier's arrivals
#ifndef GBP_FIM_MINB
#define GBP_FIM_MINB 1  // CTAs per SM
#endif
constexpr int FIM_MINB = GBP_FIM_MINB;
// Appends to the next active list go straight to the global list, so that it
// holds the vertices in the order they were activated, and the next
// iteration takes first those reached first.  A per-CTA buffer flushed at the
// end of the iteration put its entries after every direct append: measured
// on 16 problems of the 72^3 cube, a 512-entry buffer cost 6 % more face
// solves (692 M against 652 M) and 5 % more time, a 2048-entry one more still.

// One active vertex (entry g of the list) handled by a group of G lanes:
// its faces in rounds of G, the (value, code) minimum over the group, the
// update of its state and the activation of its neighbours for k + 1.
// Two loads are issued one step ahead, off the dependent chain: the list
// entry of the group's next vertex (gi_pf, read when this vertex starts; the
// list was complete before the iteration's barrier) and each lane's face
// record of the next round (read before this round's solve).  Measured on 16
// problems of the 72^3 cube: 22.12 -> 21.65 ms (the record alone: 21.74 ms;
// also the next vertex's adjacency range: 21.88 ms; also the next round's
// velocity terms or face values: 22.9 / 22.5 ms).  L1 / L2 prefetch
// instructions for the fibre, the positions or the next velocity terms cost
// more issue slots than they saved (21.9 / 21.7 ms against 21.5).
// Register budget (64 at 32 warps per SM): only what the face loop needs is
// held across it; the vertex's own position is re-read per face (an L1
// hit), its own value and change stamp and its neighbour range after the
// loop, so that the solver's working set stays in registers (every value
// held across the loop was otherwise spilled to local memory, whose
// traffic through L1/L2 exceeded the kernel's DRAM traffic).
//
// DEFER: the exact solver does not take its rare FP64 interior step here; such
// a face contributes its boundary minimum (an upper bound of its value) and
// is recorded for the repair after the solve (launch_fim), which re-solves it
// in full and resumes the iteration from any vertex it lowers.  Any FP64 code
// in this kernel made the register allocator spill the face loop's state
// (measured: 9 % of the kernel's time).
template <int MODE, bool DEFER, int G>
__device__ __forceinline__ void fim_vertex(const FimArgs &a, int k, int g, bool act, const int *__restrict__ list,
                                           int *nlist, int nxt, int &fb_local,
                                           unsigned int &my_faces, int &gi_pf, int stride, int n_cand)
{
    const int n_v = (int)a.n_v;
    const int sub = threadIdx.x & (G - 1);
    // entry gi = b * n_v + i: vertex i of problem b
    int gi = 0, boff = 0, toff = 0, beg = 0, end = 0;
    if (act) {
        gi = gi_pf;
        const int b = gi / n_v;
        boff = b * n_v;
        toff = b * (int)a.n_t;  // b * n_t < 2^31 (checked at set-up)
        beg = __ldg(&a.n2t_ptr[gi - boff]);
        end = __ldg(&a.n2t_ptr[gi - boff + 1]);
    }
    gi_pf = g + stride < n_cand ? __ldcg(&list[g + stride]) : 0;
    const int maxdeg = __reduce_max_sync(0xffffffffu, end - beg);
    float best = GBP_INF;
    int best_code = 0x7fffffff;
    int4 fr_next = beg + sub < end ? __ldg(&a.frec[beg + sub]) : make_int4(0, 0, 0, -1);
    for (int e0 = 0; e0 < maxdeg; e0 += G) {
        // the face record (face vertex ids, code), then each face vertex's
        // packed value and change stamp
        const int e = beg + e0 + sub;
        const int4 fr = fr_next;
        fr_next = (e0 + G < maxdeg && e + G < end) ? __ldg(&a.frec[e + G]) : make_int4(0, 0, 0, -1);
        // the face's per-problem velocity terms (the one input of the solve
        // that is mostly not in L2 once a batch is in flight) depend only on
        // the face record: issued before the face values come back
        float2 vj = make_float2(0.f, 0.f);
        if (fr.w >= 0) vj = __ldg(&a.tv[toff + (fr.w >> 2)]);
        float ph[3] = {GBP_INF, GBP_INF, GBP_INF};
        bool mk = false;
        if (fr.w >= 0) {
            const int2 q0 = FIM_LD(&a.pc[boff + fr.x]), q1 = FIM_LD(&a.pc[boff + fr.y]),
                       q2 = FIM_LD(&a.pc[boff + fr.z]);
            ph[0] = __int_as_float(q0.x);
            ph[1] = __int_as_float(q1.x);
            ph[2] = __int_as_float(q2.x);
            mk = max(q0.y, max(q1.y, q2.y)) >= k - 1;
        }
        if (mk) {
            const int code_r = fr.w;
            const int j = code_r >> 2;
            ++my_faces;
            // metric: the fibre shared by the batch, the velocity terms of this problem
            const float4 fj = __ldg(&a.tf[j]);
            const float4 m = make_float4(fj.x, fj.y, fj.z, vj.x);
            const float sd = vj.y;
            const float4 xi = __ldg(&a.xyz[gi - boff]);
            const float4 x0 = __ldg(&a.xyz[fr.x]), x1 = __ldg(&a.xyz[fr.y]), x2 = __ldg(&a.xyz[fr.z]);
            float3 p[3];
            p[0] = xform(make_float3(x0.x - xi.x, x0.y - xi.y, x0.z - xi.z), m, sd);
            p[1] = xform(make_float3(x1.x - xi.x, x1.y - xi.y, x1.z - xi.z), m, sd);
            p[2] = xform(make_float3(x2.x - xi.x, x2.y - xi.y, x2.z - xi.z), m, sd);
            LocalRes res;
            if (MODE == GBP_LOCAL_FISTA) {
                const int s = code_r & 3;
                const float4 Lq = __ldg(&a.tlip[toff + j]);
                const float Lv = s == 0 ? Lq.x : s == 1 ? Lq.y : s == 2 ? Lq.z : Lq.w;
                res = local_fista(p, ph, Lv, a.n_f);
            } else if (DEFER) {
                bool need64 = false;
                res = local_exact<false, true>(p, ph, &fb_local, &need64);
                if (need64) {
                    const int pos = atomicAdd(&a.ctl->n_defer, 1);
                    if (pos < FIM_DEFER_CAP) a.defer[pos] = make_int2(gi, e);
                    else atomicExch(&a.ctl->defer_overflow, 1);
                }
            } else {
                res = local_exact(p, ph, &fb_local);
            }
            if (res.v < best || (res.v == best && code_r < best_code)) {
                best = res.v;
                best_code = code_r;
            }
        }
    }
    // the vertex's own value and change stamp and its neighbour range, issued
    // before the reduction so that their latency overlaps it (only this group
    // writes the vertex in this iteration, so the value read now is the one
    // the iteration began with)
    int2 own = make_int2(0, 0);
    int nb0 = 0, ne0 = 0;
    if (act) {
        own = FIM_LD(&a.pc[gi]);
        nb0 = __ldg(&a.n2n_ptr[gi - boff]);
        ne0 = __ldg(&a.n2n_ptr[gi - boff + 1]);
    }
    // lexicographic (value, code) minimum over the group
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, best, off);
        const int oc = __shfl_xor_sync(0xffffffffu, best_code, off);
        if (ov < best || (ov == best && oc < best_code)) {
            best = ov;
            best_code = oc;
        }
    }
    bool changed = false;
    int nb = 0, ne = 0;
    if (act) {
        const float phi_old = __int_as_float(own.x);
        if (best < phi_old) {
            changed = (phi_old == GBP_INF) || (phi_old - best > a.eps);
            if (sub == 0) {
                // value and change stamp in one 8-byte store: readers see a pair
                a.pc[gi] = make_int2(__float_as_int(best), changed ? k : own.y);
                a.rec[gi].x = best_code;
            }
        }
        if (changed) {
            nb = nb0;
            ne = ne0;
        }
    }
    // activate the neighbours of changed vertices for iteration k+1: two per
    // lane and pass (a Kuhn vertex has 14 neighbours: one pass of an 8-lane
    // group), so that the two stamps' atomics overlap (16 problems: 21.34 ->
    // 20.80 ms against one neighbour per lane and pass)
    const int maxn = __reduce_max_sync(0xffffffffu, ne - nb);
    for (int e0 = 0; e0 < maxn; e0 += 2 * G) {
        const int ea = nb + e0 + sub, eb = ea + G;
        const bool va = ea < ne, vb = eb < ne;
        const int ma = va ? boff + __ldg(&a.n2n[ea]) : 0;
        const int mb = vb ? boff + __ldg(&a.n2n[eb]) : 0;
        const int sa = va ? atomicMax(&a.stamp[ma], k + 1) : k + 1;
        const int sb = vb ? atomicMax(&a.stamp[mb], k + 1) : k + 1;
        if (sa < k + 1) nlist[atomicAdd(&a.ctl->count[nxt], 1)] = ma;
        if (sb < k + 1) nlist[atomicAdd(&a.ctl->count[nxt], 1)] = mb;
    }
}

// The persistent FIM.  DEFER (the exact solver's main solve) leaves the
// faces that need the FP64 interior step to the repair below; resume (the
// exact solver without DEFER, after the repair) continues the iteration from
// the list the repair built, numbering iterations on from the main solve.
template <int MODE, bool DEFER>
__global__ void __launch_bounds__(FIM_BLOCK, FIM_MINB) k_fim(FimArgs a)
{
    const int lane = threadIdx.x & 31;
    const int groups_per_block = blockDim.x / FIM_G;
    const int ggroup = blockIdx.x * groups_per_block + threadIdx.x / FIM_G;
    const int ngroups = gridDim.x * groups_per_block;
    const int gwarp = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int nwarps = gridDim.x * (blockDim.x / 32);
    __shared__ unsigned long long s_cand, s_faces;
    __shared__ int s_fb;
    if (threadIdx.x == 0) {
        s_cand = 0;
        s_faces = 0;
        s_fb = 0;
    }
    __syncthreads();
    unsigned int nbar = 0;
    // the first iteration: 1, or the one after the main solve's last
    const int k0 = a.resume ? ld_relaxed_i32(&a.ctl->iterations) + 1 : 1;
    int k = k0;
    int fb_local = 0;
    unsigned int my_faces = 0;
    __shared__ int s_ncand;
    // max_iters bounds the iteration numbers, so it bounds the main and the
    // resumed solve together
    for (; k <= a.max_iters; ++k) {
        const int cur = k % 3, nxt = (k + 1) % 3, nn = (k + 2) % 3;
        // one read of the list size per CTA (all warps reading the one word
        // queue at its L2 slice)
        if (threadIdx.x == 0) s_ncand = ld_relaxed_i32(&a.ctl->count[cur]);
        __syncthreads();
        const int n_cand = s_ncand;
        if (a.trace && blockIdx.x == 0 && threadIdx.x == 0) {
            unsigned long long tns;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(tns));
            a.trace[2 * (k - 1)] = n_cand;
            a.trace[2 * (k - 1) + 1] = (long long)tns;
        }
        if (n_cand == 0) break;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            a.ctl->count[nn] = 0;
            s_cand += (unsigned long long)n_cand;
        }
        const int *list = a.lists + (int64_t)cur * a.n_tot;
        int *nlist = a.lists + (int64_t)nxt * a.n_tot;
        // a front smaller than a third of the 8-lane groups: one warp per
        // vertex, so a vertex's faces take one round instead of three
        if (n_cand <= ngroups / 3) {
            int gi_pf = gwarp < n_cand ? __ldcg(&list[gwarp]) : 0;
            for (int g = gwarp;; g += nwarps) {
                const bool act = g < n_cand;
                if (!__any_sync(0xffffffffu, act)) break;
                fim_vertex<MODE, DEFER, 32>(a, k, g, act, list, nlist, nxt, fb_local, my_faces, gi_pf, nwarps,
                                            n_cand);
            }
        } else {
            int gi_pf = ggroup < n_cand ? __ldcg(&list[ggroup]) : 0;
            for (int g = ggroup;; g += ngroups) {
                const bool act = g < n_cand;
                if (!__any_sync(0xffffffffu, act)) break;
                fim_vertex<MODE, DEFER, FIM_G>(a, k, g, act, list, nlist, nxt, fb_local, my_faces, gi_pf, ngroups,
                                               n_cand);
            }
        }
        ++nbar;
        if (!grid_barrier(a.ctl, a.grp, nbar)) break;
    }
    // statistics
    unsigned int wf = my_faces;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) wf += __shfl_xor_sync(0xffffffffu, wf, off);
    int wfb = fb_local;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) wfb += __shfl_xor_sync(0xffffffffu, wfb, off);
    if (lane == 0) {
        if (wf) atomicAdd(&s_faces, (unsigned long long)wf);
        if (wfb) atomicAdd(&s_fb, wfb);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_cand) atomicAdd(&a.ctl->candidates, s_cand);
        if (s_faces) atomicAdd(&a.ctl->face_updates, s_faces);
        if (s_fb) atomicAdd(&a.ctl->fp64_fallbacks, (unsigned long long)s_fb);
        if (blockIdx.x == 0) {
            a.ctl->iterations = k - 1;
            if (k > a.max_iters && !ld_relaxed_i32(&a.ctl->abort))
                atomicCAS(&a.ctl->status, 0, (int)GBP_ERR_NOT_CONVERGED);
        }
    }
}

// ---------------------------------------------------------------------------
// FP64 repair of the faces the main solve deferred.  The main solve converged
// to a fixed point U of the operator that takes the boundary minimum of
// those faces (an upper bound of theirs), and each face's last evaluation
// used the final values of its vertices, so the deferred faces that matter
// are in the list.  Each is solved in full with U's values; a vertex whose
// value drops takes it (smallest (value, code) per vertex), and the exact
// iteration resumes from its neighbours: monotone iteration from an upper
// bound ends at the same fixed point the exact solve would.
// ---------------------------------------------------------------------------
__global__ void k_repair_init(FimArgs a, unsigned long long *keys)
{
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d < min(ld_relaxed_i32(&a.ctl->n_defer), FIM_DEFER_CAP)) keys[a.defer[d].x] = ~0ull;
}

__global__ void k_repair(FimArgs a, unsigned long long *keys)
{
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= min(ld_relaxed_i32(&a.ctl->n_defer), FIM_DEFER_CAP)) return;
    const int2 de = a.defer[d];
    const int gi = de.x, n_v = (int)a.n_v;
    const int b = gi / n_v, boff = b * n_v, toff = b * (int)a.n_t;
    const int4 fr = a.frec[de.y];
    const float ph[3] = {__int_as_float(a.pc[boff + fr.x].x), __int_as_float(a.pc[boff + fr.y].x),
                         __int_as_float(a.pc[boff + fr.z].x)};
    const int j = fr.w >> 2;
    const float2 vj = a.tv[toff + j];
    const float4 fj = a.tf[j];
    const float4 m = make_float4(fj.x, fj.y, fj.z, vj.x);
    const float4 xi = a.xyz[gi - boff];
    const float4 x0 = a.xyz[fr.x], x1 = a.xyz[fr.y], x2 = a.xyz[fr.z];
    float3 p[3];
    p[0] = xform(make_float3(x0.x - xi.x, x0.y - xi.y, x0.z - xi.z), m, vj.y);
    p[1] = xform(make_float3(x1.x - xi.x, x1.y - xi.y, x1.z - xi.z), m, vj.y);
    p[2] = xform(make_float3(x2.x - xi.x, x2.y - xi.y, x2.z - xi.z), m, vj.y);
    int fb = 0;
    const LocalRes res = local_exact(p, ph, &fb);
    if (fb) atomicAdd(&a.ctl->fp64_fallbacks, (unsigned long long)fb);
    if (res.v < __int_as_float(a.pc[gi].x))
        atomicMin(&keys[gi], ((unsigned long long)float_key(res.v) << 32) | (unsigned int)fr.w);
}

__global__ void k_repair_apply(FimArgs a, unsigned long long *keys)
{
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= min(ld_relaxed_i32(&a.ctl->n_defer), FIM_DEFER_CAP)) return;
    const int gi = a.defer[d].x;
    // one thread per vertex takes its key
    const unsigned long long K = atomicExch(&keys[gi], ~0ull);
    if (K == ~0ull) return;
    const float v = key_float((unsigned int)(K >> 32));
    const int code = (int)(K & 0xffffffffu);
    const int k0 = ld_relaxed_i32(&a.ctl->iterations) + 1;
    const int2 own = a.pc[gi];
    const float phi_old = __int_as_float(own.x);
    if (!(v < phi_old)) return;
    const bool changed = (phi_old == GBP_INF) || (phi_old - v > a.eps);
    a.pc[gi] = make_int2(__float_as_int(v), changed ? k0 - 1 : own.y);
    a.rec[gi].x = code;
    atomicAdd(&a.ctl->n_repaired, 1);
    if (!changed) return;
    const int n_v = (int)a.n_v, boff = (gi / n_v) * n_v, i = gi - boff;
    int *list = a.lists + (int64_t)(k0 % 3) * a.n_tot;
    for (int e = a.n2n_ptr[i]; e < a.n2n_ptr[i + 1]; ++e) {
        const int mm = boff + a.n2n[e];
        if (atomicMax(&a.stamp[mm], k0) < k0) list[atomicAdd(&a.ctl->count[k0 % 3], 1)] = mm;
    }
}

// More deferred faces than the list holds (not seen on the test meshes): the
// resumed exact iteration starts from every vertex, all faces masked in.
__global__ void k_repair_all(FimArgs a)
{
    if (!ld_relaxed_i32(&a.ctl->defer_overflow)) return;
    const int k0 = ld_relaxed_i32(&a.ctl->iterations) + 1;
    int *list = a.lists + (int64_t)(k0 % 3) * a.n_tot;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < (int)a.n_tot; g += gridDim.x * blockDim.x) {
        a.pc[g].y = k0 - 1;
        if (atomicMax(&a.stamp[g], k0) < k0) list[atomicAdd(&a.ctl->count[k0 % 3], 1)] = g;
    }
}

static int fim_grid(gbp_ctx *c, const void *fn)
{
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, FIM_BLOCK, 0);
    if (per_sm < 1) per_sm = 1;
    return per_sm * c->num_sms;
}

cudaError_t launch_fim(gbp_ctx *c, const gbp_solve_opts *o)
{
    cudaError_t err = launch_fim_seed(c);
    if (err) return err;
    const int64_t n_v = c->n_v;
    const int64_t n_tot = n_v * c->nb;  // all problems of the batch (< 2^31, checked at set-up)
    long long *trace = nullptr;
    if (c->trace_on) {
        if (c->trace_cap < o->max_iters + 2) {
            if (c->trace) cudaFree(c->trace);
            c->trace = nullptr;
            c->trace_cap = 0;
            if (cudaMalloc(&c->trace, sizeof(long long) * 2 * (o->max_iters + 2)) == cudaSuccess)
                c->trace_cap = o->max_iters + 2;
        }
        if (c->trace) {
            cudaMemsetAsync(c->trace, 0, sizeof(long long) * 2 * c->trace_cap, c->stream);
            trace = c->trace;
        }
    }
    FimArgs a;
    a.n_v = n_v;
    a.n_t = c->n_t;
    a.n_tot = n_tot;
    a.xyz = c->xyz;
    a.tets = c->tets;
    a.tf = c->tf;
    a.tv = c->tv;
    a.tlip = c->tlip;
    a.frec = c->frec;
    a.pc = c->pc;
    a.n2t_ptr = c->n2t_ptr;
    a.n2t = c->n2t;
    a.n2n_ptr = c->n2n_ptr;
    a.n2n = c->n2n;
    a.phi = c->phi;
    a.rec = c->rec;
    a.chg = c->chg;
    a.stamp = c->stamp;
    a.lists = c->lists;
    a.ctl = c->ctl;
    a.grp = c->bar_grp;
    a.eps = o->eps;
    a.max_iters = o->max_iters;
    a.n_f = o->n_f;
    a.trace = trace;
    a.defer = c->defer;
    a.resume = 0;
    err = cudaMemsetAsync(c->bar_grp, 0, sizeof(BarGroup) * GBP_BAR_GROUPS, c->stream);
    if (err) return err;
    const bool exact = o->local_solver != GBP_LOCAL_FISTA;
    const void *fn = exact ? (const void *)k_fim<GBP_LOCAL_EXACT, true> : (const void *)k_fim<GBP_LOCAL_FISTA, false>;
    int grid = fim_grid(c, fn);
    void *args[] = {&a};
    time_begin(c, 0);
    err = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(FIM_BLOCK), args, 0, c->stream);
    if (!err && exact) {
        // the deferred faces in FP64, then the exact iteration from what they
        // lowered (an empty list ends it at once)
        const unsigned bl = FIM_DEFER_CAP / 256;
        k_repair_init<<<bl, 256, 0, c->stream>>>(a, c->keys);
        k_repair<<<bl, 256, 0, c->stream>>>(a, c->keys);
        k_repair_apply<<<bl, 256, 0, c->stream>>>(a, c->keys);
        k_repair_all<<<c->num_sms, 256, 0, c->stream>>>(a);
        c->launches += 4;
        err = cudaGetLastError();
        // the resumed kernel numbers its grid barriers from 1 again: zero the
        // grid-level arrival count and the groups' words (the abort flag is
        // kept, so a main solve that gave up ends the resumed one at once)
        if (!err) err = cudaMemsetAsync(&c->ctl->barrier, 0, sizeof(unsigned int), c->stream);
        if (!err) err = cudaMemsetAsync(c->bar_grp, 0, sizeof(BarGroup) * GBP_BAR_GROUPS, c->stream);
        if (!err) {
            a.resume = 1;
            a.trace = nullptr;
            const void *fr = (const void *)k_fim<GBP_LOCAL_EXACT, false>;
            err = cudaLaunchCooperativeKernel(fr, dim3(fim_grid(c, fr)), dim3(FIM_BLOCK), args, 0, c->stream);
            c->launches++;
        }
    }
    time_end(c, 0);
    c->launches++;
    if (err) return err;
    return launch_unpack_state(c);
}

}  // namespace gbp
