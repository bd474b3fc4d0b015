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
// for k+1 (appended through a per-CTA shared-memory buffer, one global
// atomic per CTA and iteration).  Reads of neighbour values may see this
// iteration's updates (chaotic relaxation); the operator is monotone, so the
// limit is the same fixed point.
#ifndef GBP_FIM_G
#define GBP_FIM_G 8  // lanes per active vertex
#endif
#ifndef GBP_FIM_R
#define GBP_FIM_R 1  // faces per lane fetched together
#endif
#ifndef GBP_FIM_BLOCK
#define GBP_FIM_BLOCK 1024  // threads per CTA
#endif
constexpr int FIM_G = GBP_FIM_G;
constexpr int FIM_R = GBP_FIM_R;
constexpr int FIM_BLOCK = GBP_FIM_BLOCK;
// One CTA of 1024 threads per SM (64 registers): the same 32 warps per SM as
// four CTAs of 256, with a quarter of the grid barrier's arrivals and each
// CTA's appends gathered over four times the vertices
#ifndef GBP_FIM_MINB
#define GBP_FIM_MINB 1  // CTAs per SM
#endif
constexpr int FIM_MINB = GBP_FIM_MINB;
// Per-CTA append buffer for the next active list; appends beyond it go
// straight to the global list during the iteration.  A small buffer leaves
// less to the flush at the end of the iteration, which every CTA does
// before the grid barrier (16 problems: 512 entries 27.0 ms, 2048 28.2 ms).
#ifndef GBP_FIM_CAP
#define GBP_FIM_CAP 512
#endif
constexpr int FIM_CAP = GBP_FIM_CAP;

// One active vertex (entry g of the list) handled by a group of G lanes:
// its faces in rounds of G, the (value, code) minimum over the group, the
// update of its state and the activation of its neighbours for k + 1.
template <int MODE, int G>
__device__ __forceinline__ void fim_vertex(const FimArgs &a, int k, int64_t g, bool act, const int *__restrict__ list,
                                           int *nlist, int nxt, int *s_list, int *s_n, int &fb_local,
                                           unsigned int &my_faces)
{
    const int64_t n_v = a.n_v;
    const int sub = threadIdx.x & (G - 1);
    // entry gi = b * n_v + i: vertex i of problem b
    int gi = 0, i = 0, boff = 0, beg = 0, end = 0, nb = 0, ne = 0, chg_old = 0;
    int64_t toff = 0;
    float phi_old = 0.f;
    float4 xi = make_float4(0.f, 0.f, 0.f, 0.f);
    if (act) {
        gi = __ldcg(&list[g]);
        const int b = gi / (int)n_v;
        boff = b * (int)n_v;
        toff = (int64_t)b * a.n_t;
        i = gi - boff;
        const int2 own = FIM_LD(&a.pc[gi]);
        phi_old = __int_as_float(own.x);
        chg_old = own.y;
        beg = __ldg(&a.n2t_ptr[i]);
        end = __ldg(&a.n2t_ptr[i + 1]);
        nb = __ldg(&a.n2n_ptr[i]);
        ne = __ldg(&a.n2n_ptr[i + 1]);
        xi = __ldg(&a.xyz[i]);
    }
    const int maxdeg = __reduce_max_sync(0xffffffffu, end - beg);
    float best = GBP_INF;
    int best_code = 0x7fffffff;
    // FIM_R faces per lane at a time: their adjacency, tets and face
    // values are fetched together (three dependent loads for all of
    // them), then the masked ones are solved
    for (int e0 = 0; e0 < maxdeg; e0 += G * FIM_R) {
        // the face record (face vertex ids, code), then each face
        // vertex's packed value and change stamp
        int4 fr[FIM_R];
#pragma unroll
        for (int r = 0; r < FIM_R; ++r) {
            const int e = beg + e0 + r * G + sub;
            fr[r] = e < end ? __ldg(&a.frec[e]) : make_int4(0, 0, 0, -1);
        }
        // the face's per-problem velocity terms (the one input of the solve
        // that is mostly not in L2 once a batch is in flight) depend only on
        // the face record: issued before the face values come back
        float2 vj[FIM_R];
#pragma unroll
        for (int r = 0; r < FIM_R; ++r)
            if (fr[r].w >= 0) vj[r] = __ldg(&a.tv[toff + (fr[r].w >> 2)]);
        float ph[FIM_R][3];
        bool mk[FIM_R];
#pragma unroll
        for (int r = 0; r < FIM_R; ++r) {
            mk[r] = false;
            ph[r][0] = ph[r][1] = ph[r][2] = GBP_INF;
            if (fr[r].w >= 0) {
                const int2 q0 = FIM_LD(&a.pc[boff + fr[r].x]), q1 = FIM_LD(&a.pc[boff + fr[r].y]),
                           q2 = FIM_LD(&a.pc[boff + fr[r].z]);
                ph[r][0] = __int_as_float(q0.x);
                ph[r][1] = __int_as_float(q1.x);
                ph[r][2] = __int_as_float(q2.x);
                mk[r] = max(q0.y, max(q1.y, q2.y)) >= k - 1;
            }
        }
#pragma unroll
        for (int r = 0; r < FIM_R; ++r) {
            if (!mk[r]) continue;
            const int code_r = fr[r].w;
            const int j = code_r >> 2, s = code_r & 3;
            ++my_faces;
            // metric: the fibre shared by the batch, the velocity terms of this problem
            const float4 fj = __ldg(&a.tf[j]);
            const float4 m = make_float4(fj.x, fj.y, fj.z, vj[r].x);
            const float sd = vj[r].y;
            const float4 x0 = __ldg(&a.xyz[fr[r].x]), x1 = __ldg(&a.xyz[fr[r].y]),
                         x2 = __ldg(&a.xyz[fr[r].z]);
            float3 p[3];
            p[0] = xform(make_float3(x0.x - xi.x, x0.y - xi.y, x0.z - xi.z), m, sd);
            p[1] = xform(make_float3(x1.x - xi.x, x1.y - xi.y, x1.z - xi.z), m, sd);
            p[2] = xform(make_float3(x2.x - xi.x, x2.y - xi.y, x2.z - xi.z), m, sd);
            LocalRes res;
            if (MODE == GBP_LOCAL_FISTA) {
                const float4 Lq = __ldg(&a.tlip[toff + j]);
                const float Lv = s == 0 ? Lq.x : s == 1 ? Lq.y : s == 2 ? Lq.z : Lq.w;
                res = local_fista(p, ph[r], Lv, a.n_f);
            } else {
                res = local_exact(p, ph[r], &fb_local);
            }
            if (res.v < best || (res.v == best && code_r < best_code)) {
                best = res.v;
                best_code = code_r;
            }
        }
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
    if (act && best < phi_old) {
        changed = (phi_old == GBP_INF) || (phi_old - best > a.eps);
        if (sub == 0) {
            // value and change stamp in one 8-byte store: readers see a pair
            a.pc[gi] = make_int2(__float_as_int(best), changed ? k : chg_old);
            a.rec[gi].x = best_code;
        }
    }
    // activate the neighbours of changed vertices for iteration k+1
    if (!changed) nb = ne = 0;
    const int maxn = __reduce_max_sync(0xffffffffu, ne - nb);
    for (int e0 = 0; e0 < maxn; e0 += G) {
        const int e = nb + e0 + sub;
        if (e < ne) {
            const int m = boff + __ldg(&a.n2n[e]);
            if (atomicMax(&a.stamp[m], k + 1) < k + 1) {
                const int pos = atomicAdd(s_n, 1);
                if (pos < FIM_CAP) {
                    s_list[pos] = m;
                } else {
                    nlist[atomicAdd(&a.ctl->count[nxt], 1)] = m;
                }
            }
        }
    }
}

template <int MODE>
__global__ void __launch_bounds__(FIM_BLOCK, FIM_MINB) k_fim(FimArgs a)
{
    const int lane = threadIdx.x & 31;
    const int groups_per_block = blockDim.x / FIM_G;
    const int64_t ggroup = (int64_t)blockIdx.x * groups_per_block + threadIdx.x / FIM_G;
    const int64_t ngroups = (int64_t)gridDim.x * groups_per_block;
    const int64_t gwarp = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x / 32);
    __shared__ int s_list[FIM_CAP];
    __shared__ int s_n, s_cnt, s_base;
    __shared__ unsigned long long s_cand, s_faces;
    __shared__ int s_fb;
    if (threadIdx.x == 0) {
        s_n = 0;
        s_cand = 0;
        s_faces = 0;
        s_fb = 0;
    }
    __syncthreads();
    unsigned int nbar = 0;
    int k = 1;
    int fb_local = 0;
    unsigned int my_faces = 0;
    __shared__ int s_ncand;
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
        if ((int64_t)n_cand * 3 <= ngroups) {
            for (int64_t g = gwarp;; g += nwarps) {
                const bool act = g < n_cand;
                if (!__any_sync(0xffffffffu, act)) break;
                fim_vertex<MODE, 32>(a, k, g, act, list, nlist, nxt, s_list, &s_n, fb_local, my_faces);
            }
        } else {
            for (int64_t g = ggroup;; g += ngroups) {
                const bool act = g < n_cand;
                if (!__any_sync(0xffffffffu, act)) break;
                fim_vertex<MODE, FIM_G>(a, k, g, act, list, nlist, nxt, s_list, &s_n, fb_local, my_faces);
            }
        }
        // flush the CTA's appends with one global reservation
        __syncthreads();
        if (threadIdx.x == 0) {
            const int n = min(s_n, FIM_CAP);
            s_cnt = n;
            s_base = n ? atomicAdd(&a.ctl->count[nxt], n) : 0;
            s_n = 0;
        }
        __syncthreads();
        for (int q = threadIdx.x; q < s_cnt; q += blockDim.x) nlist[s_base + q] = s_list[q];
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
    err = cudaMemsetAsync(c->bar_grp, 0, sizeof(BarGroup) * GBP_BAR_GROUPS, c->stream);
    if (err) return err;
    const void *fn = o->local_solver == GBP_LOCAL_FISTA ? (const void *)k_fim<GBP_LOCAL_FISTA>
                                                        : (const void *)k_fim<GBP_LOCAL_EXACT>;
    int grid = fim_grid(c, fn);
    void *args[] = {&a};
    time_begin(c, 0);
    err = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(FIM_BLOCK), args, 0, c->stream);
    time_end(c, 0);
    c->launches++;
    if (err) return err;
    return launch_unpack_state(c);
}

}  // namespace gbp
