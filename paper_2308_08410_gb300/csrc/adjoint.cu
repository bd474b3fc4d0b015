// adjoint.cu -- Geodesic-BP gradient along the frozen parent graph
// (Sec. II-C, Eq. dto_grad, Eq. upwind_xi; velocities as in the
// conduction-tensor remark of Sec. IV).
//
// For a vertex i with face parent (j, slot) and barycentric alpha:
//   phi_i = sum_n alpha_n phi_{j_n} + ||w||_{D_j},  w = v_i - sum_n alpha_n v_{j_n},
// alpha frozen (first variation), so d phi_i / d phi_{j_n} = alpha_n and,
// with ||w||_D^2 = |w_perp|^2 / ct^2 + (f.w)^2 / cf^2,
//   d phi_i / d cf_j = -(f.w)^2 / (cf^3 ||w||_D),
//   d phi_i / d ct_j = -|w_perp|^2 / (ct^3 ||w||_D).
// Onset vertices: d phi / d t_k = 1; element onsets (Eq. upwind_xi) add
// d phi_v / d x_k = -D_E (v - x_k) / ||v - x_k||_{D_E} and the velocity
// derivatives of tet E with w = v - x_k.
//
// mu = (I - P^T)^{-1} dL/dphi is accumulated children-first: a vertex is
// processed once every child (vertex whose parent face holds it with
// alpha > 0) has pushed alpha * mu into it.  This runs as a dataflow with no
// grid barriers.  Each vertex owns one 64-bit word that packs its
// outstanding child count (top 9 bits) and the fixed-point sum of the pushes
// it has received (low 55 bits, two's complement, scale 2^e chosen from
// sum |dL/dphi| so that every partial sum stays below 2^53): one atomic add
// both delivers a child's contribution and decrements the count, and the
// child that brings the count to zero receives the complete sum in the
// atomic's return value.  No fence or re-read is needed on the chain, and
// the sums are exact integers, so mu does not depend on the order of the
// pushes.  That child continues with the parent itself; further parents it
// readies go to a work queue of (vertex, mu) pairs.  The critical path is
// the depth of the parent graph times one vertex's latency.  The parent
// graph of the discrete fixed point can hold short cycles (non-causal
// updates in anisotropic elements); the vertices they block (the longer
// cycles and all their ancestors) are finished by a bounded fixed-point
// (Jacobi) iteration on that sub-graph, which is closed under taking
// parents, in the words' fixed point and stopped per vertex (below).  Most of
// those cycles are 2-cycles (c's
// parent face holds p and p's holds c); they are solved exactly inside the
// dataflow instead: the edge between the two is left out of their counts,
// and once both have every other child, the second of the two to be ready
// solves mu_c = S_c + a_pc mu_p, mu_p = S_p + a_cp mu_c (S = lambda plus the
// other children's pushes) and carries on with both.  A pair caught in a
// longer cycle never becomes ready and goes to the iteration as before.
//
// Memory: a hop reads the vertex's 32-byte record written by the parent pass
// (parent vertices, alpha, the tet and its two velocity coefficients: one
// sector) and does its pushes into the parents' words, which also hold lambda
// in the same fixed point (so the vertex that completes a parent reads its
// whole mu from the atomic's return value).  Processed vertices are marked in
// a bitmap.  The gradient additions of the vertices with a face parent follow
// the dataflow in one pass in vertex order (their mu is then the sum in their
// word); only 2-cycle members and onset-parented vertices add theirs inline.
#include "gbp_internal.cuh"

namespace gbp {

// Batched: vertex entries g = b * n_v + i and tet entries b * n_t + j of
// problem b; the mesh and the onset sites are shared.
struct AdjArgs {
    int64_t n_v;    // vertices per problem
    int64_t n_t;    // tets per problem
    int64_t n_tot;  // n_v x problems
    int K;
    const float4 *xyz;
    const int4 *tets;
    const float4 *tf;  // unit fibre per tet (shared by the batch)
    const float *cf, *ct;
    const int4 *rec;       // (code, alpha bits) per vertex entry: the onset path
    const int4 *arec;      // the parent pass's 32-byte record per vertex entry
    int onset_kind;
    int site_per_problem;  // on_idx / on_bary hold one site set per problem
    BarGroup *grp;         // group words of the two-level grid barrier
    const int *pair;       // 2-cycle partner entry of each vertex entry, or -1
    unsigned long long *pairw;  // hand-over word of each 2-cycle, at its smaller entry
    int64_t qcap;          // 64-bit slots of the work queue
    const int *on_idx;
    const float *on_bary;
    const float *lam;
    float *mu;
    unsigned long long *xj, *acc, *acc2;  // cycle iteration: x and the pushes, in the words' fixed point
    unsigned long long *w;  // packed (child count, fixed-point lambda + push sum) per vertex
    unsigned int *done;     // processed vertex entries (bitmap)
    int *lists;
    float *d_cf, *d_ct, *d_t, *d_x;
    Control *ctl;
    int max_cycle_iters;
};

// The record of vertex entry v (see the parent pass): parent face vertices
// f[q] (within the problem, -1 where alpha is 0), alpha a[q], the tet (with
// the 2-cycle flag in bit 30) or a negative code, and the velocity
// coefficients.
constexpr int ADJ_PAIR_FLAG = 1 << 30;
struct ARec {
    int f[3];
    int jt;
    float a[3];
    float gcf, gct;
};

__device__ __forceinline__ ARec load_arec(const int4 *__restrict__ arec, int64_t v)
{
    const int4 h = __ldg(&arec[2 * v]);
    const int4 q = __ldg(&arec[2 * v + 1]);
    ARec r;
    r.f[0] = h.x;
    r.f[1] = h.y;
    r.f[2] = h.z;
    r.jt = h.w;
    r.a[0] = __int_as_float(q.x);
    r.a[1] = __int_as_float(q.y);
    r.a[2] = (1.f - r.a[0]) - r.a[1];
    r.gcf = __int_as_float(q.z);
    r.gct = __int_as_float(q.w);
    return r;
}

// weight of vertex i (within the problem) in the parent face of r (0 if absent)
__device__ __forceinline__ float face_weight(const ARec &r, int i)
{
    return r.f[0] == i ? r.a[0] : r.f[1] == i ? r.a[1] : r.f[2] == i ? r.a[2] : 0.f;
}

// gradient contributions of vertex i (of problem b) through its own parent
// (no pushes): the tet's velocity terms from the record, or the onset terms
__device__ __forceinline__ void local_terms(const AdjArgs &a, int b, int64_t i, const ARec &r, float m)
{
    const int64_t toff = (int64_t)b * a.n_t;
    if (r.jt >= 0) {
        const int64_t j = toff + (r.jt & (ADJ_PAIR_FLAG - 1));
        if (a.d_cf) atomicAdd(&a.d_cf[j], m * r.gcf);
        if (a.d_ct) atomicAdd(&a.d_ct[j], m * r.gct);
    } else if (r.jt != GBP_UNREACHED) {
        const int k = -1 - r.jt;
        const int bk = b * a.K + k;
        if (a.d_t) atomicAdd(&a.d_t[bk], m);
        if (a.onset_kind == GBP_ONSET_ELEMENT) {
            const int sk = a.site_per_problem ? bk : k;
            const int E = __ldg(&a.on_idx[sk]);
            const int4 tv = __ldg(&a.tets[E]);
            int ids[4] = {tv.x, tv.y, tv.z, tv.w};
            const float4 xi = __ldg(&a.xyz[i]);
            // w = v - x_k = sum_q b_q (v - v_q)
            float3 w = make_float3(0.f, 0.f, 0.f);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float bq = __ldg(&a.on_bary[4 * sk + q]);
                float4 xq = __ldg(&a.xyz[ids[q]]);
                w.x = fmaf(bq, xi.x - xq.x, w.x);
                w.y = fmaf(bq, xi.y - xq.y, w.y);
                w.z = fmaf(bq, xi.z - xq.z, w.z);
            }
            const float4 mm = __ldg(&a.tf[E]);
            const float cfe = __ldg(&a.cf[toff + E]), cte = __ldg(&a.ct[toff + E]);
            float fw = mm.x * w.x + mm.y * w.y + mm.z * w.z;
            float3 wp = make_float3(w.x - fw * mm.x, w.y - fw * mm.y, w.z - fw * mm.z);
            float wp2 = f3dot(wp, wp);
            float icf = 1.f / cfe, ict = 1.f / cte;
            float g = sqrtf(wp2 * ict * ict + fw * fw * icf * icf);
            if (g > 0.f) {
                // D w = wp / ct^2 + (f.w) f / cf^2
                float ig = 1.f / g;
                if (a.d_x) {
                    float c1 = ict * ict, c2 = fw * icf * icf;
                    atomicAdd(&a.d_x[3 * bk + 0], -m * (wp.x * c1 + c2 * mm.x) * ig);
                    atomicAdd(&a.d_x[3 * bk + 1], -m * (wp.y * c1 + c2 * mm.y) * ig);
                    atomicAdd(&a.d_x[3 * bk + 2], -m * (wp.z * c1 + c2 * mm.z) * ig);
                }
                if (a.d_cf) atomicAdd(&a.d_cf[toff + E], -m * fw * fw * icf * icf * icf * ig);
                if (a.d_ct) atomicAdd(&a.d_ct[toff + E], -m * wp2 * ict * ict * ict * ig);
            }
        }
    }
}

// Packed per-vertex word: W = count * 2^55 + S with |S| < 2^54, S the
// fixed-point sum of lambda and the pushes received.
constexpr int ADJ_CNT_SHIFT = 55;
constexpr unsigned long long ADJ_ONE = 1ull << ADJ_CNT_SHIFT;
constexpr int ADJ_MAX_CHILDREN = 511;

__device__ __forceinline__ unsigned int adj_count(unsigned long long W)
{
    return (unsigned int)((W + (1ull << (ADJ_CNT_SHIFT - 1))) >> ADJ_CNT_SHIFT);
}

__device__ __forceinline__ long long adj_sum(unsigned long long W)
{
    return (long long)(W - ((unsigned long long)adj_count(W) << ADJ_CNT_SHIFT));
}

// fixed-point scale from sum |dL/dphi| (rounded up, so every partial sum of
// lambda and pushes stays below 2^53 in magnitude)
__device__ __forceinline__ void adj_scale(const Control *ctl, double *scale, double *iscale)
{
    const double lsum = ld_relaxed_f64(&ctl->adj_lsum);
    const int ex = lsum > 0.0 ? ilogb(lsum) + 1 : 0;
    *scale = ldexp(1.0, 53 - ex);
    *iscale = ldexp(1.0, ex - 53);
}

__device__ __forceinline__ bool is_done(const unsigned int *done, int64_t v)
{
    return (__ldcg(&done[v >> 5]) >> (v & 31)) & 1u;
}

// Zero the words, mark the unreached vertices done and sum |dL/dphi|.  One
// thread per vertex entry; a warp covers 32 consecutive entries, i.e. one
// bitmap word.
__global__ void k_adj_init(int64_t n_v, const int4 *__restrict__ arec, const float *__restrict__ dphi,
                           unsigned long long *w, unsigned int *done, Control *ctl)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    bool reached = i < n_v && __ldg(&arec[2 * i]).w != GBP_UNREACHED;
    float l = reached ? fabsf(dphi[i]) : 0.f;
    if (i < n_v) w[i] = 0ull;
    const unsigned int word = __ballot_sync(0xffffffffu, !reached);
    if ((threadIdx.x & 31) == 0 && i < n_v) done[i >> 5] = word;
    __shared__ float red[32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) l += __shfl_xor_sync(0xffffffffu, l, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x < 32) {
        l = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) l += __shfl_xor_sync(0xffffffffu, l, off);
        // rounded up so that the sum stays an upper bound
        if (threadIdx.x == 0 && l > 0.f) atomicAdd(&ctl->adj_lsum, 1.001 * (double)l);
    }
}

// cand[c] = the parent p of c (weight > 0) whose own parent face holds c
// (weight > 0), when there is exactly one such parent; else -1
__global__ void k_adj_cand(int n_v, int n_tot, const int4 *__restrict__ arec, int *cand)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_tot) return;
    const ARec r = load_arec(arec, g);
    int c = -1, found = 0;
    if (r.jt >= 0) {
        const int boff = (g / n_v) * n_v;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            if (r.f[q] < 0) continue;
            const ARec rp = load_arec(arec, boff + r.f[q]);
            if (rp.jt >= 0 && face_weight(rp, g - boff) != 0.f) {
                c = boff + r.f[q];
                ++found;
            }
        }
    }
    cand[g] = found == 1 ? c : -1;
}

// pair[c] = cand[c] when the candidacy is mutual and 1 - a_cp a_pc is not
// tiny (the record of c gets the 2-cycle flag); also clears the pair's
// hand-over word
__global__ void k_adj_pair(int n_v, int n_tot, int4 *arec, const int *__restrict__ cand, int *pair,
                           unsigned long long *pairw)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_tot) return;
    int p = cand[g];
    if (p >= 0 && cand[p] == g) {
        const int boff = (g / n_v) * n_v;
        const ARec rg = load_arec(arec, g), rp = load_arec(arec, p);
        const float a_gp = face_weight(rg, p - boff), a_pg = face_weight(rp, g - boff);
        if (!(1.f - a_gp * a_pg > 1e-6f)) p = -1;
    } else {
        p = -1;
    }
    pair[g] = p;
    pairw[g] = 0ull;
    if (p >= 0) arec[2 * (int64_t)g].w |= ADJ_PAIR_FLAG;
}

// Children per parent word (one ADJ_ONE per face vertex with alpha > 0, the
// edge to a 2-cycle partner left out) and each vertex's own lambda in the
// fixed point.
__global__ void k_adj_count(int n_v, int n_tot, const int4 *__restrict__ arec, const int *__restrict__ pair,
                            const float *__restrict__ dphi, unsigned long long *w, const Control *ctl)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_tot) return;
    const ARec r = load_arec(arec, i);
    if (r.jt == GBP_UNREACHED) return;
    double scale, iscale;
    adj_scale(ctl, &scale, &iscale);
    const long long lf = __double2ll_rn((double)dphi[i] * scale);
    if (lf) atomicAdd(&w[i], (unsigned long long)lf);
    if (r.jt < 0) return;
    const int boff = (i / n_v) * n_v;
    const int partner = (r.jt & ADJ_PAIR_FLAG) ? pair[i] - boff : -1;
#pragma unroll
    for (int q = 0; q < 3; ++q)
        if (r.f[q] >= 0 && r.f[q] != partner) atomicAdd(&w[boff + r.f[q]], ADJ_ONE);
}

// queue slot: vertex id (low word) and mu bits (high word); empty = all ones
__device__ __forceinline__ unsigned long long adj_item(int v, float m)
{
    return (unsigned long long)(unsigned int)v | ((unsigned long long)__float_as_uint(m) << 32);
}

// vertices with no children start the dataflow: they go to the work queue
// (their mu is lambda)
__global__ void k_adj_seed(int64_t n_v, const unsigned long long *__restrict__ w, const unsigned int *__restrict__ done,
                           const float *__restrict__ dphi, unsigned long long *queue, Control *ctl)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    bool app = i < n_v && !((done[i >> 5] >> (i & 31)) & 1u) && adj_count(w[i]) == 0u;
    unsigned int mask = __ballot_sync(0xffffffffu, app);
    if (mask == 0) return;
    const int lane = threadIdx.x & 31, leader = __ffs(mask) - 1;
    int base = 0;
    if (lane == leader) {
        base = atomicAdd(&ctl->q_res, __popc(mask));
        atomicAdd(&ctl->q_active, __popc(mask));
        atomicAdd(&ctl->adj_levels, __popc(mask));  // number of seeds, reported in the stats
    }
    base = __shfl_sync(0xffffffffu, base, leader);
    if (app) queue[base + __popc(mask & ((1u << lane) - 1u))] = adj_item((int)i, dphi[i]);
}

// A vertex has more children than the packed count holds.
__global__ void k_adj_check(int64_t n_v, const unsigned long long *__restrict__ w, Control *ctl)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n_v && adj_count(w[i]) > (unsigned)ADJ_MAX_CHILDREN) atomicCAS(&ctl->status, 0, (int)GBP_ERR_INVALID_ARG);
}

__device__ __forceinline__ float ld_cg_f(const float *p) { return __ldcg(p); }

__device__ __forceinline__ int ld_acquire_i32(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

#ifndef GBP_ADJ_POST
#define GBP_ADJ_POST 4  // vertices per thread and step of the gradient pass after the dataflow
#endif
constexpr int ADJ_POST = GBP_ADJ_POST;
#ifndef GBP_ADJ_REFILL
#define GBP_ADJ_REFILL 8  // idle lanes that make a warp take new items while others are busy
#endif


__global__ void __launch_bounds__(256) k_adjoint(AdjArgs a)
{
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nth = (int64_t)gridDim.x * blockDim.x;
    const int64_t n_v = a.n_v, n_tot = a.n_tot;
    unsigned int nbar = 0;
    __shared__ int s_proc;
    if (threadIdx.x == 0) s_proc = 0;
    __syncthreads();
    bool ok = true;
    int mine = 0;
    if (tid == 0) asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(a.ctl->adj_ts[0]));
    // ---- dataflow phase (no grid barrier per level) ----
    // The vertices readied so far sit in a work queue of (vertex, mu) items
    // (lists[0..3 n_tot) as qcap = 1.5 n_tot 64-bit slots, empty = all ones:
    // every vertex is queued at most once, the second member of a 2-cycle at
    // most twice); q_res counts
    // the slots produced, q_head the slots handed out, and q_active the
    // queued items plus chains in progress (it reaches zero only when no
    // more work can appear).  Each warp runs up to 32 chains in lockstep:
    // every pass, idle lanes take the items that are available (one atomic
    // per warp), then every busy lane processes one vertex and moves on to
    // the first parent it readied, queueing any further ones.  A warp sleeps
    // only when none of its lanes has work.
    double scale, iscale;
    adj_scale(a.ctl, &scale, &iscale);
    unsigned long long *queue = reinterpret_cast<unsigned long long *>(a.lists);
    const int lane = threadIdx.x & 31;
    int v = -1;        // vertex this lane is processing
    float m = 0.f;     // its mu (or, for a 2-cycle member not yet solved, lambda + the other children's pushes)
    bool pre = false;  // v is a 2-cycle member whose pair is already solved (m is its mu)
    int pending = -1;  // a slot handed to this lane that was still empty
    unsigned int idle_spins = 0, sleep_ns = 32;
    for (;;) {
        // hand available slots to the idle lanes
        const unsigned int idle = __ballot_sync(0xffffffffu, v < 0 && pending < 0);
        // a refill costs the busy lanes a round trip: batch it
        if (idle && (__popc(idle) >= GBP_ADJ_REFILL || idle == 0xffffffffu ||
                     !__ballot_sync(0xffffffffu, v >= 0))) {
            int base = 0, got = 0;
            if (lane == 0) {
                const int avail = ld_relaxed_i32(&a.ctl->q_res) - ld_relaxed_i32(&a.ctl->q_head);
                got = min(__popc(idle), avail);
                if (got > 0) base = atomicAdd(&a.ctl->q_head, got);
            }
            got = __shfl_sync(0xffffffffu, got, 0);
            base = __shfl_sync(0xffffffffu, base, 0);
            const int rank = __popc(idle & ((1u << lane) - 1u));
            if (((idle >> lane) & 1u) && rank < got) pending = base + rank;
        }
        // a slot handed out may still be empty if other warps took the items
        // counted as available; it fills once its producer stores it
        if (pending >= 0) {
            const unsigned long long item = pending < a.qcap ? ld_relaxed_u64(&queue[pending]) : 0ull;
            if (pending >= a.qcap) {
                pending = -1;  // cannot happen: at most n_tot + n_tot / 2 items are ever queued
            } else if (item != ~0ull) {
                const unsigned int vv = (unsigned int)(item & 0xffffffffu);
                v = (int)(vv & 0x7fffffffu);
                pre = (vv >> 31) != 0u;
                m = __uint_as_float((unsigned int)(item >> 32));
                pending = -1;
            }
        }
        // one vertex per busy lane (entry v = b * n_v + vertex); the items it
        // queues are reserved for the whole warp at once below
        int ended = 0;
        unsigned long long pend[3];
        int npend = 0;
        if (v >= 0) {
            const int b = v / (int)n_v;
            const int boff = b * (int)n_v;
            const ARec r = load_arec(a.arec, v);
            const int partner = (r.jt >= 0 && (r.jt & ADJ_PAIR_FLAG)) ? __ldg(&a.pair[v]) : -1;
            bool go = true;
            if (partner >= 0 && !pre) {
                // 2-cycle: the first member to be ready leaves its sum in the
                // pair's word and stops; the second solves the pair
                const int slot = min(v, partner);
                const unsigned long long own = (2ull << 32) | __float_as_uint(m);
                const unsigned long long old = atomicCAS(&a.pairw[slot], 0ull, own);
                if (old == 0ull) {
                    go = false;
                } else {
                    const float mq = __uint_as_float((unsigned int)(old & 0xffffffffu));
                    const float a_vq = face_weight(r, partner - boff);                        // partner in v's face
                    const float a_qv = face_weight(load_arec(a.arec, partner), v - boff);  // v in partner's face
                    const float mv = (m + a_qv * mq) / (1.f - a_vq * a_qv);
                    m = mv;
                    pend[npend++] = adj_item((int)((unsigned int)partner | 0x80000000u), mq + a_vq * mv);
                }
            }
            pre = false;
            int next = -1;
            float mnext = 0.f;
            if (go) {
                atomicOr(&a.done[v >> 5], 1u << (v & 31));
                ++mine;
                if (r.jt >= 0) {
                    unsigned long long nw[3] = {0ull, 0ull, 0ull};
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        if (r.f[q] < 0 || boff + r.f[q] == partner) continue;
                        const long long c = __double2ll_rn((double)(r.a[q] * m) * scale);
                        const unsigned long long d = (unsigned long long)c - ADJ_ONE;
                        nw[q] = atomicAdd(&a.w[boff + r.f[q]], d) + d;
                    }
                    // a 2-cycle member's mu is not its word's sum: its
                    // gradient terms are added here; every other vertex's
                    // after the dataflow (below)
                    if (r.jt & ADJ_PAIR_FLAG) local_terms(a, b, v - boff, r, m);
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        if (r.f[q] < 0 || boff + r.f[q] == partner || adj_count(nw[q]) != 0u) continue;
                        // this push completed the parent: its mu is the whole sum
                        const float mp = (float)((double)adj_sum(nw[q]) * iscale);
                        if (next < 0) {
                            next = boff + r.f[q];
                            mnext = mp;
                        } else {
                            pend[npend++] = adj_item(boff + r.f[q], mp);
                        }
                    }
                } else {
                    local_terms(a, b, v - boff, r, m);
                }
            }
            v = next;
            m = mnext;
            ended = v < 0;
        }
        // queue this pass's extra items: one reservation for the warp (the
        // count of live work rises before any chain of the warp retires)
        const int wsum = __reduce_add_sync(0xffffffffu, npend);
        if (wsum) {
            int base = 0;
            if (lane == 0) {
                atomicAdd(&a.ctl->q_active, wsum);
                base = atomicAdd(&a.ctl->q_res, wsum);
            }
            base = __shfl_sync(0xffffffffu, base, 0);
            int incl = npend;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, off);
                if (lane >= off) incl += t;
            }
            const int pos = base + incl - npend;
            for (int k = 0; k < npend; ++k) st_relaxed_u64(&queue[pos + k], pend[k]);
        }
        // retire the chains that ended.  No fence: their pushes are atomics
        // that have returned, the items they queued were counted before, and
        // nothing in this loop reads the other writes (the bitmap, the
        // gradients), which the grid barrier after the loop orders.
        const unsigned int ends = __ballot_sync(0xffffffffu, ended);
        if (ends) {
            __syncwarp();
            if (lane == 0) atomicSub(&a.ctl->q_active, __popc(ends));
        }
        if (__ballot_sync(0xffffffffu, v >= 0)) {
            idle_spins = 0;
            sleep_ns = 32;
            continue;
        }
        // no lane is processing: finished when no work can appear any more
        int done = 0;
        if (lane == 0) {
            done = ld_acquire_i32(&a.ctl->q_active) == 0;
            if (!done && ld_relaxed_i32(&a.ctl->abort)) done = 2;
        }
        done = __shfl_sync(0xffffffffu, done, 0);
        if (done == 2) break;
        if (done) {
            // a pending slot can only have been filled before the count reached zero
            if (pending >= 0) {
                const unsigned long long item = ld_relaxed_u64(&queue[pending]);
                pending = -1;
                if (item != ~0ull) {
                    const unsigned int vv = (unsigned int)(item & 0xffffffffu);
                    v = (int)(vv & 0x7fffffffu);
                    pre = (vv >> 31) != 0u;
                    m = __uint_as_float((unsigned int)(item >> 32));
                }
            }
            if (!__ballot_sync(0xffffffffu, v >= 0)) break;
            continue;
        }
        if (++idle_spins > (1u << 21)) {
            if (lane == 0) {
                atomicExch(&a.ctl->abort, 1);
                atomicCAS(&a.ctl->status, 0, (int)GBP_ERR_TIMEOUT);
            }
            ok = false;
            break;
        }
        __nanosleep(sleep_ns);
        if (sleep_ns < 512) sleep_ns <<= 1;
    }
    if (mine) atomicAdd(&s_proc, mine);
    __syncthreads();
    if (threadIdx.x == 0 && s_proc) atomicAdd(&a.ctl->adj_processed, s_proc);
    ++nbar;
    if (!grid_barrier(a.ctl, a.grp, nbar) || !ok) return;
    if (tid == 0) {
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(a.ctl->adj_ts[1]));
        a.ctl->adj_ts[2] = a.ctl->adj_ts[1];
    }
    // ---- vertices blocked by cycles: fixed-point iteration ----
    // collect the unprocessed reached vertices R (closed under parents); the
    // barrier above ordered every write of the dataflow phase before this
    // The gradient terms of the vertices the dataflow finished with a face
    // parent (2-cycle members excepted), in vertex order: their mu is the
    // complete sum in their word.  Scattered through the dataflow, these float
    // atomics into the per-tet gradients (arrays larger than L2 at 16
    // problems) slowed its chains by ~30 %.  ADJ_POST vertices per thread
    // and step, every load issued before the atomics, so that the loads
    // overlap.
    for (int64_t base = 0; base < n_tot; base += ADJ_POST * nth) {
        ARec r[ADJ_POST];
        unsigned long long wv[ADJ_POST];
        bool ok[ADJ_POST];
#pragma unroll
        for (int u = 0; u < ADJ_POST; ++u) {
            const int64_t i = base + u * nth + tid;
            ok[u] = i < n_tot && is_done(a.done, i);
            if (ok[u]) {
                r[u] = load_arec(a.arec, i);
                wv[u] = __ldcg(&a.w[i]);
            }
        }
#pragma unroll
        for (int u = 0; u < ADJ_POST; ++u) {
            const int64_t i = base + u * nth + tid;
            if (ok[u] && r[u].jt >= 0 && !(r[u].jt & ADJ_PAIR_FLAG)) {
                const int b = (int)(i / n_v);
                local_terms(a, b, i - (int64_t)b * n_v, r[u], (float)((double)adj_sum(wv[u]) * iscale));
            }
        }
    }
    int *R = a.lists + 3 * n_tot;
    for (int64_t base = 0; base < n_tot; base += nth) {
        const int64_t i = base + tid;
        bool app = i < n_tot && !is_done(a.done, i);
        if (app) {
            // x starts from the base (lambda plus the pushes of the processed
            // children, the sum in the vertex's word); the base stays there
            a.xj[i] = (unsigned long long)adj_sum(__ldcg(&a.w[i]));
            a.acc[i] = 0ull;
            a.acc2[i] = 0ull;
        }
        warp_append(app, (int)i, R, &a.ctl->count[3]);
    }
    ++nbar;
    if (!grid_barrier(a.ctl, a.grp, nbar)) return;
    const int nR = ld_relaxed_i32(&a.ctl->count[3]);
    if (nR == 0) return;
    // x <- base + P_R^T x in the words' fixed point (integer sums: the result
    // does not depend on the order of the pushes, and a settled vertex stops
    // changing).  One barrier per iteration: the update of x reads the sums
    // pushed in the previous iteration (buffer cur) and pushes the new x into
    // the other buffer.  Stop when every vertex of R changed by at most
    // |x| 2^-23 + 8192 units (about 1e-7 relative, plus 2^-40 sum |lambda|).
    // A stop against the largest |x| of R instead left vertices with small mu,
    // and ancestors still receiving pushes, far from their fixed point.
    unsigned long long *acc_cur = a.acc, *acc_nxt = a.acc2;
    auto push = [&](int i, long long x, unsigned long long *dst) {
        const ARec r = load_arec(a.arec, i);
        if (r.jt < 0) return;
        const int boff = (i / (int)n_v) * (int)n_v;
#pragma unroll
        for (int q = 0; q < 3; ++q)
            if (r.f[q] >= 0)
                atomicAdd(&dst[boff + r.f[q]], (unsigned long long)__double2ll_rn((double)r.a[q] * (double)x));
    };
    for (int64_t w = tid; w < nR; w += nth) {
        const int i = __ldcg(&R[w]);
        push(i, (long long)__ldcg(&a.xj[i]), acc_cur);
    }
    ++nbar;
    if (!grid_barrier(a.ctl, a.grp, nbar)) return;
    int it = 0;
    for (; it < a.max_cycle_iters; ++it) {
        // slot (it+1)%3 was last read before the previous barrier
        if (blockIdx.x == 0 && threadIdx.x == 0) a.ctl->adj_delta[(it + 1) % 3] = 0.f;
        int viol = 0;
        for (int64_t w = tid; w < nR; w += nth) {
            const int i = __ldcg(&R[w]);
            const long long xn = adj_sum(__ldcg(&a.w[i])) + (long long)__ldcg(&acc_cur[i]);
            const long long xo = (long long)__ldcg(&a.xj[i]);
            acc_cur[i] = 0ull;
            const long long d = xn > xo ? xn - xo : xo - xn;
            const long long ax = xn < 0 ? -xn : xn;
            viol += d > (ax >> 23) + 8192;
            a.xj[i] = (unsigned long long)xn;
            push(i, xn, acc_nxt);
        }
        viol = __reduce_add_sync(0xffffffffu, viol);
        if ((threadIdx.x & 31) == 0 && viol) atomicAdd((int *)&a.ctl->adj_delta[it % 3], viol);
        ++nbar;
        if (!grid_barrier(a.ctl, a.grp, nbar)) return;
        const int gv = ld_relaxed_i32((const int *)&a.ctl->adj_delta[it % 3]);
        unsigned long long *t = acc_cur;
        acc_cur = acc_nxt;
        acc_nxt = t;
        if (gv == 0) {
            ++it;
            break;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(a.ctl->adj_ts[2]));
        a.ctl->adj_cycle_nodes = nR;
        a.ctl->adj_cycle_iters = it;
        if (it >= a.max_cycle_iters) atomicCAS(&a.ctl->status, 0, (int)GBP_ERR_NOT_CONVERGED);
    }
    for (int64_t w = tid; w < nR; w += nth) {
        const int i = __ldcg(&R[w]);
        const float x = (float)((double)(long long)__ldcg(&a.xj[i]) * iscale);
        a.mu[i] = x;
        atomicOr(&a.done[i >> 5], 1u << (i & 31));
        const int b = i / (int)n_v;
        local_terms(a, b, i - b * (int)n_v, load_arec(a.arec, i), x);
    }
}

cudaError_t launch_adjoint(gbp_ctx *c, const float *dphi, float *d_cf, float *d_ct, float *d_t, float *d_x)
{
    cudaError_t err;
    const int64_t n_v = c->n_v;
    // keep the solve's statistics, reset the adjoint counters
    err = cudaMemsetAsync(c->ctl->count, 0, sizeof(int) * 4, c->stream);
    if (err) return err;
    err = cudaMemsetAsync(&c->ctl->barrier, 0, sizeof(unsigned int) * 2, c->stream);  // arrivals, abort
    if (err) return err;
    err = cudaMemsetAsync(c->bar_grp, 0, sizeof(BarGroup) * GBP_BAR_GROUPS, c->stream);
    if (err) return err;
    err = cudaMemsetAsync(&c->ctl->q_head, 0, sizeof(int), c->stream);
    if (err) return err;
    err = cudaMemsetAsync(&c->ctl->q_res, 0, sizeof(int), c->stream);
    if (err) return err;
    err = cudaMemsetAsync(&c->ctl->q_active, 0, sizeof(int), c->stream);
    if (err) return err;
    const int64_t n_tot = n_v * c->nb;
    const int64_t qcap = (3 * n_tot) / 2;  // 64-bit queue slots in lists[0 .. 3 n_tot)
    err = cudaMemsetAsync(c->lists, 0xff, sizeof(unsigned long long) * qcap, c->stream);  // empty queue slots
    if (err) return err;
    err = cudaMemsetAsync(&c->ctl->adj_levels, 0, offsetof(Control, adj_ts) - offsetof(Control, adj_levels),
                          c->stream);
    if (err) return err;
    if (d_cf) cudaMemsetAsync(d_cf, 0, sizeof(float) * c->n_t * c->nb, c->stream);
    if (d_ct) cudaMemsetAsync(d_ct, 0, sizeof(float) * c->n_t * c->nb, c->stream);
    if (d_t) cudaMemsetAsync(d_t, 0, sizeof(float) * c->K * c->nb, c->stream);
    if (d_x) cudaMemsetAsync(d_x, 0, sizeof(float) * 3 * c->K * c->nb, c->stream);
    int th = 256;
    unsigned bl = (unsigned)((n_tot + th - 1) / th);
    time_begin(c, 4);
    k_adj_init<<<bl, th, 0, c->stream>>>(n_tot, c->adj_rec, dphi, c->adj_w, c->adj_done, c->ctl);
    k_adj_cand<<<bl, th, 0, c->stream>>>((int)n_v, (int)n_tot, c->adj_rec, c->adj_cand);
    k_adj_pair<<<bl, th, 0, c->stream>>>((int)n_v, (int)n_tot, c->adj_rec, c->adj_cand, c->adj_pair, c->adj_pairw);
    k_adj_count<<<bl, th, 0, c->stream>>>((int)n_v, (int)n_tot, c->adj_rec, c->adj_pair, dphi, c->adj_w, c->ctl);
    c->launches += 4;
    if (c->max_nbr > ADJ_MAX_CHILDREN) {
        k_adj_check<<<bl, th, 0, c->stream>>>(n_tot, c->adj_w, c->ctl);
        c->launches++;
    }
    k_adj_seed<<<bl, th, 0, c->stream>>>(n_tot, c->adj_w, c->adj_done, dphi,
                                         reinterpret_cast<unsigned long long *>(c->lists), c->ctl);
    c->launches++;
    if ((err = cudaGetLastError())) return err;
    AdjArgs a;
    a.n_v = n_v;
    a.n_t = c->n_t;
    a.n_tot = n_tot;
    a.K = c->K;
    a.xyz = c->xyz;
    a.tets = c->tets;
    a.tf = c->tf;
    a.cf = c->cf;
    a.ct = c->ct;
    a.rec = c->rec;
    a.arec = c->adj_rec;
    a.onset_kind = c->onset_kind;
    a.site_per_problem = c->site_b > 0;
    a.grp = c->bar_grp;
    a.pair = c->adj_pair;
    a.pairw = c->adj_pairw;
    a.qcap = qcap;
    a.on_idx = c->on_idx;
    a.on_bary = c->on_bary;
    a.lam = dphi;
    a.mu = c->mu;
    a.w = c->adj_w;
    a.done = c->adj_done;
    a.xj = c->jac_x;
    a.acc = c->jac_acc;
    a.acc2 = c->jac_acc2;
    a.lists = c->lists;
    a.d_cf = d_cf;
    a.d_ct = d_ct;
    a.d_t = d_t;
    a.d_x = d_x;
    a.ctl = c->ctl;
    a.max_cycle_iters = 4096;
    // one 256-thread CTA per SM: ~39k threads, several times the widest
    // ready front, few enough that idle consumers poll lightly
    // (2 or 4 per SM measured slower at 16 problems too: the consumers'
    // polling contends with the pushes)
    int grid = c->num_sms;
    void *args[] = {&a};
    err = cudaLaunchCooperativeKernel((const void *)k_adjoint, dim3(grid), dim3(256), args, 0, c->stream);
    time_end(c, 4);
    c->launches++;
    return err;
}

}  // namespace gbp
