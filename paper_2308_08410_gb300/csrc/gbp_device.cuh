// gbp_device.cuh -- device building blocks of libgbp: the control block,
// the local solvers (exact and FISTA), the bounded grid barrier and small
// helpers.  Shared by the translation units of the CUDA library only.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/gbp.h"

#define GBP_INF __int_as_float(0x7f800000)
#define GBP_UNREACHED ((int)0x80000000)

namespace gbp {

// ---------------------------------------------------------------------------
// device control block (one per context)
// ---------------------------------------------------------------------------
struct Control {
    // cache line 0: grid-barrier group arrivals (atomics) and the abort flag
    unsigned int barrier;         // groups arrived, monotonic per launch
    int abort;                    // set when a bounded wait ran out
    unsigned int pad0[30];
    // counters and statistics
    int count[4];                 // active-list sizes (3 rotating lists) + spare
    int status;                   // latched gbp_status of the last device phase
    int iterations;               // FIM iterations of the last solve
    unsigned long long candidates;
    unsigned long long face_updates;
    unsigned long long fp64_fallbacks;
    unsigned long long unreached;
    // work queue of the adjoint's dataflow phase: each counter on its own
    // cache line (consumers, producers and the termination count do not
    // contend)
    int q_head;                   // tickets handed to consumers
    int padq0[31];
    int q_res;                    // slots reserved by producers
    int padq1[31];
    int q_active;                 // chains queued or in progress
    int padq2[31];
    int adj_levels;
    int adj_cycle_nodes;
    int adj_cycle_iters;
    int adj_processed;
    float adj_delta[3];           // cycle iteration: vertices not yet settled, as int bits (rotating slots)
    float adj_xmax[3];            // spare
    double adj_lsum;              // sum |dL/dphi| (scale of the adjoint's fixed-point sums)
    unsigned long long adj_ts[3]; // global timer at adjoint start, end of dataflow, end
    int n_defer;                  // FIM faces deferred to the FP64 repair (entries written, may exceed the cap)
    int defer_overflow;           // more deferred faces than the list holds: the repair re-solves everything
    int n_repaired;               // vertices the repair lowered
    int param_status;             // latched by the metric precompute (kept across solves)
};

// ---------------------------------------------------------------------------
// metric: the local metric D = M^{-1} of Sec. II-A with
// M = ct^2 I + (cf^2 - ct^2) f f^T.  We keep R = D^{1/2} in factored form,
// R = sa I + sd f f^T with sa = 1/ct, sd = 1/cf - 1/ct, so that
// ||w||_D = |R w| is a plain Euclidean norm (no cancellation).
// Per tet: float4 (fx, fy, fz, sa) and float sd.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float3 xform(float3 e, float4 m, float sd)
{
    float fe = m.x * e.x + m.y * e.y + m.z * e.z;
    float k = sd * fe;
    return make_float3(fmaf(m.w, e.x, k * m.x), fmaf(m.w, e.y, k * m.y), fmaf(m.w, e.z, k * m.z));
}

__device__ __forceinline__ float3 f3sub(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float f3dot(float3 a, float3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ float3 f3cross(float3 a, float3 b)
{
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float3 f4to3(float4 a) { return make_float3(a.x, a.y, a.z); }

// Order-preserving map of a float onto an unsigned key, so that the smallest
// value (ties: the smaller low word of a packed 64-bit key) wins an atomicMin.
__device__ __forceinline__ unsigned int float_key(float v)
{
    unsigned int b = __float_as_uint(v);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float key_float(unsigned int k)
{
    unsigned int b = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
    return __uint_as_float(b);
}

// Square root for the local solver: x * rsqrt(x) (about 2.5 ulp) instead of
// the correctly rounded sqrtf, which costs several times more instructions.
// The solver's values feed comparisons with 1e-5 relative margins at most.
#ifndef GBP_FAST_SQRT
#define GBP_FAST_SQRT 1
#endif
__device__ __forceinline__ float lsqrt(float x)
{
#if GBP_FAST_SQRT
    return x > 0.f ? x * rsqrtf(x) : 0.f;
#else
    return sqrtf(x);
#endif
}

struct LocalRes {
    float v;
    float a0, a1, a2;
};

// value of the objective of Eq. (upwind_eq_lsqr) at alpha, computed relative
// to ref = smallest finite Phi: ref + sum a_n (Phi_n - ref) + |sum a_n p_n|.
__device__ __forceinline__ float eval_alpha(const float3 p[3], const float ph[3], float ref, float a0, float a1,
                                            float a2)
{
    float3 w = make_float3(0.f, 0.f, 0.f);
    float s = 0.f;
    if (a0 > 0.f) {
        s = fmaf(a0, ph[0] - ref, s);
        w.x = fmaf(a0, p[0].x, w.x); w.y = fmaf(a0, p[0].y, w.y); w.z = fmaf(a0, p[0].z, w.z);
    }
    if (a1 > 0.f) {
        s = fmaf(a1, ph[1] - ref, s);
        w.x = fmaf(a1, p[1].x, w.x); w.y = fmaf(a1, p[1].y, w.y); w.z = fmaf(a1, p[1].z, w.z);
    }
    if (a2 > 0.f) {
        s = fmaf(a2, ph[2] - ref, s);
        w.x = fmaf(a2, p[2].x, w.x); w.y = fmaf(a2, p[2].y, w.y); w.z = fmaf(a2, p[2].z, w.z);
    }
    return ref + (s + lsqrt(f3dot(w, w)));
}

// The objective in FP64 at a boundary candidate, from the FP32 face vectors
// and values: vertex `kind` (0..2), or edge kind - 3 = 0, 1, 2 for (0, 1),
// (0, 2), (1, 2) at weight lam on its first vertex and 1 - lam (formed in
// FP64, so that the weights sum to 1 exactly) on its second.
__device__ __forceinline__ double eval_candidate64(const float3 p[3], const float ph[3], float ref, int kind, float lam)
{
    double a[3] = {0.0, 0.0, 0.0};
    if (kind < 3) {
        a[kind] = 1.0;
    } else {
        const int e = kind - 3, n = e == 2 ? 1 : 0, m = e == 0 ? 1 : 2;
        a[n] = lam;
        a[m] = 1.0 - (double)lam;
    }
    double wx = 0.0, wy = 0.0, wz = 0.0, s = 0.0;
#pragma unroll
    for (int n = 0; n < 3; ++n) {
        if (!(a[n] > 0.0)) continue;
        s += a[n] * ((double)ph[n] - (double)ref);
        wx += a[n] * p[n].x;
        wy += a[n] * p[n].y;
        wz += a[n] * p[n].z;
    }
    return (double)ref + (s + sqrt(wx * wx + wy * wy + wz * wz));
}

#define GBP_TRY(a0_, a1_, a2_)                                   \
    do {                                                         \
        float v_ = eval_alpha(p, ph, ref, (a0_), (a1_), (a2_));  \
        if (v_ < r.v) {                                          \
            r.v = v_;                                            \
            r.a0 = (a0_); r.a1 = (a1_); r.a2 = (a2_);            \
        }                                                        \
    } while (0)

// Interior stationary point of the face (all three values finite), FP64.
// Same algebra as the FP32 branch below; used when the FP32 discriminant
// or the face is too close to degenerate.  Scalar arguments and a by-value
// result keep the caller's operands in registers; returns (beta0, beta1), or
// (-1, -1) when the point is not inside.  Inlined: an out-of-line call in the
// FIM's face loop made the register allocator spill the loop's state on every
// face; the FIM defers these solves to after its face loop instead
// (local_exact with DEFER64).
static __device__ __forceinline__ float2 interior_fp64(float p0x, float p0y, float p0z, float p1x, float p1y, float p1z,
                                                    float p2x, float p2y, float p2z, float ph0, float ph1, float ph2)
{
    const float2 none = make_float2(-1.f, -1.f);
    double d1x = (double)p0x - p2x, d1y = (double)p0y - p2y, d1z = (double)p0z - p2z;
    double d2x = (double)p1x - p2x, d2y = (double)p1y - p2y, d2z = (double)p1z - p2z;
    double Q00 = d1x * d1x + d1y * d1y + d1z * d1z;
    double Q01 = d1x * d2x + d1y * d2y + d1z * d2z;
    double Q11 = d2x * d2x + d2y * d2y + d2z * d2z;
    double nx = d1y * d2z - d1z * d2y, ny = d1z * d2x - d1x * d2z, nz = d1x * d2y - d1y * d2x;
    double det = nx * nx + ny * ny + nz * nz;
    if (!(det > 0.0)) return none;
    double q0 = d1x * p2x + d1y * p2y + d1z * p2z;
    double q1 = d2x * p2x + d2y * p2y + d2z * p2z;
    double D0 = (double)ph0 - ph2, D1 = (double)ph1 - ph2;
    double k = (Q11 * D0 * D0 - 2.0 * Q01 * D0 * D1 + Q00 * D1 * D1) / det;
    double tp = nx * p2x + ny * p2y + nz * p2z;
    double S = tp * tp / det;
    if (!(k < 1.0) || !(S > 0.0)) return none;
    double h = sqrt(S / (1.0 - k));
    double y0 = h * D0 + q0, y1 = h * D1 + q1;
    double b0 = -(Q11 * y0 - Q01 * y1) / det;
    double b1 = -(-Q01 * y0 + Q00 * y1) / det;
    if (!(b0 > 0.0 && b1 > 0.0 && b0 + b1 < 1.0)) return none;
    return make_float2((float)b0, (float)b1);
}

// The interior step is redone in FP64 when 1 - Delta^T Q^-1 Delta falls below
// this value (or the face is nearly degenerate).  The candidate is always
// evaluated at its own (feasible) point, so an FP32 location error only costs
// second order in the value.
#ifndef GBP_FP64_FALLBACK_TOL
#define GBP_FP64_FALLBACK_TOL 1e-3f
#endif

// Exact minimiser of Eq. (upwind_eq_lsqr) on one face (Sec. II-B).  The
// objective is convex on the simplex, so the minimum is at a KKT point: the
// stationary point of the face interior, of an edge, or a vertex.  A
// feasible interior stationary point is the minimiser, so it is tried first
// and ends the search; otherwise all feasible edge and vertex candidates are
// evaluated at their (feasible) point and the smallest value wins, vertices
// first, then edges, ties to the earlier one.  Locations (lambda, beta) use
// approximate reciprocals (a location error only costs second order in the
// value); values use IEEE square roots.  p[n] = R (v_{j_n} - v_i),
// ph[n] = Phi_n (+inf allowed).  fb counts FP64 fallbacks.
//
// ALPHA (the parent pass, where the minimiser alpha is an output): the
// boundary candidates are collected with their FP32 values, and when two or
// more lie within about 8 ulps of the best, those are re-evaluated in FP64
// at their (FP32) locations and the smallest FP64 value wins.  Near a
// vertex, or where two edges meet, candidates a few hundredths apart in
// alpha differ in value by less than FP32 resolves (a fraction of an ulp),
// while FP64 separates them; a plain FP32 comparison returns the same value
// but the other candidate's alpha.
//
// DEFER64 (the FIM's face loop): a face whose interior step needs FP64 is not
// solved in FP64 here; *need64 is set and the boundary minimum (an upper
// bound of the face's value) is returned, and the caller solves the face
// again in full where fewer registers are live.
template <bool ALPHA = false, bool DEFER64 = false>
__device__ __forceinline__ LocalRes local_exact(const float3 p[3], const float ph[3], int *fb, bool *need64 = nullptr)
{
    LocalRes r;
    r.v = GBP_INF;
    r.a0 = r.a1 = r.a2 = 0.f;
    bool ok0 = ph[0] < GBP_INF, ok1 = ph[1] < GBP_INF, ok2 = ph[2] < GBP_INF;
    if (!(ok0 || ok1 || ok2)) return r;
    float ref = fminf(fminf(ok0 ? ph[0] : GBP_INF, ok1 ? ph[1] : GBP_INF), ok2 ? ph[2] : GBP_INF);
    // interior
    if (ok0 && ok1 && ok2) {
        float3 d1 = f3sub(p[0], p[2]), d2 = f3sub(p[1], p[2]);
        float Q00 = f3dot(d1, d1), Q01 = f3dot(d1, d2), Q11 = f3dot(d2, d2);
        float3 nrm = f3cross(d1, d2);
        float det = f3dot(nrm, nrm);
        bool degenerate = !(det > 1e-6f * Q00 * Q11);
        float idet = __fdividef(1.f, det);
        float q0 = f3dot(d1, p[2]), q1 = f3dot(d2, p[2]);
        float D0 = ph[0] - ph[2], D1 = ph[1] - ph[2];
        float k = (Q11 * D0 * D0 - 2.f * Q01 * D0 * D1 + Q00 * D1 * D1) * idet;
        float tp = f3dot(nrm, p[2]);
        float S = tp * tp * idet;
        // The stationary point is x = x0 + w with x0 the foot of the
        // perpendicular from the origin to the face plane (|x0|^2 = S) and
        // |w|^2 = k S / (1 - k); inside the face requires |w| <= max_n |p_n|.
        // When 1 - k is too small for FP32, that necessary condition (with
        // a factor-2 and 1e-5 slack for the rounding of k) rules most faces
        // out before the FP64 redo.
        const bool near_singular = 1.f - k < GBP_FP64_FALLBACK_TOL;
        const float pmax2 = fmaxf(fmaxf(f3dot(p[0], p[0]), f3dot(p[1], p[1])), f3dot(p[2], p[2]));
        const bool outside = near_singular && k * S > 2.f * pmax2 * ((1.f - k) + 1e-5f);
        if ((k < 1.f && !outside) || degenerate) {
            float b0, b1;
            bool found = false;
            if ((degenerate || near_singular) && DEFER64) {
                *need64 = true;
            } else if (degenerate || near_singular) {
                ++*fb;
                const float2 bb = interior_fp64(p[0].x, p[0].y, p[0].z, p[1].x, p[1].y, p[1].z, p[2].x, p[2].y,
                                                p[2].z, ph[0], ph[1], ph[2]);
                b0 = bb.x;
                b1 = bb.y;
                found = b0 > 0.f;
            } else {
                float h = lsqrt(S * __fdividef(1.f, 1.f - k));
                float y0 = fmaf(h, D0, q0), y1 = fmaf(h, D1, q1);
                b0 = -(Q11 * y0 - Q01 * y1) * idet;
                b1 = -(Q00 * y1 - Q01 * y0) * idet;
                found = b0 > 0.f && b1 > 0.f && b0 + b1 < 1.f;
            }
            if (found) {
                GBP_TRY(b0, b1, 1.f - b0 - b1);
                return r;
            }
        }
    }
    // boundary candidates of the ALPHA variant: FP32 value, kind (vertex n or
    // edge 3 + e) and edge weight
    float cv[6], cl[6];
    int ck[6];
    int nc = 0;
    // vertices
    if (ALPHA) {
        if (ok0) { cv[nc] = eval_alpha(p, ph, ref, 1.f, 0.f, 0.f); ck[nc] = 0; cl[nc] = 1.f; ++nc; }
        if (ok1) { cv[nc] = eval_alpha(p, ph, ref, 0.f, 1.f, 0.f); ck[nc] = 1; cl[nc] = 1.f; ++nc; }
        if (ok2) { cv[nc] = eval_alpha(p, ph, ref, 0.f, 0.f, 1.f); ck[nc] = 2; cl[nc] = 1.f; ++nc; }
    } else {
        if (ok0) GBP_TRY(1.f, 0.f, 0.f);
        if (ok1) GBP_TRY(0.f, 1.f, 0.f);
        if (ok2) GBP_TRY(0.f, 0.f, 1.f);
    }
    // edges (n, m), lambda = weight on n
#pragma unroll
    for (int e = 0; e < 3; ++e) {
        const int n = e == 2 ? 1 : 0;
        const int m = e == 0 ? 1 : 2;
        bool okn = n == 0 ? ok0 : ok1;
        bool okm = m == 1 ? ok1 : ok2;
        if (!(okn && okm)) continue;
        float3 u = f3sub(p[n], p[m]);
        float A = f3dot(u, u);
        float iA = __fdividef(1.f, A);
        float dl = ph[n] - ph[m];
        float g = dl * dl * iA;
        if (!(g < 1.f)) continue;
        float3 cr = f3cross(u, p[m]);
        float S = f3dot(cr, cr) * iA;
        float h = lsqrt(S * __fdividef(1.f, 1.f - g));
        float lam = (-dl * h - f3dot(u, p[m])) * iA;
        if (!(lam > 0.f && lam < 1.f)) continue;
        float an = lam, am = 1.f - lam;
        if (ALPHA) {
            const float b0 = e == 2 ? 0.f : an, b1 = e == 0 ? am : e == 2 ? an : 0.f, b2 = e == 0 ? 0.f : am;
            cv[nc] = eval_alpha(p, ph, ref, b0, b1, b2);
            ck[nc] = 3 + e;
            cl[nc] = lam;
            ++nc;
            continue;
        }
        if (e == 0) GBP_TRY(an, am, 0.f);
        else if (e == 1) GBP_TRY(an, 0.f, am);
        else GBP_TRY(0.f, an, am);
    }
    if (ALPHA && nc > 0) {
        // the FP32 best, then an FP64 comparison among the near-ties
        int bq = 0;
        for (int q = 1; q < nc; ++q)
            if (cv[q] < cv[bq]) bq = q;
        const float thr = cv[bq] + 1e-6f * fabsf(cv[bq]);
        int ties = 0;
        for (int q = 0; q < nc; ++q) ties += cv[q] <= thr;
        if (ties > 1) {
            double best64 = 1e300;
            for (int q = 0; q < nc; ++q) {
                if (!(cv[q] <= thr)) continue;
                const double v64 = eval_candidate64(p, ph, ref, ck[q], cl[q]);
                if (v64 < best64) {
                    best64 = v64;
                    bq = q;
                }
            }
        }
        // alpha in the solver's own expressions: edge (n, m) at (lam, 1 - lam)
        const int kq = ck[bq];
        const float lq = cl[bq], mq = 1.f - lq;
        r.v = cv[bq];
        r.a0 = kq == 0 ? 1.f : (kq == 3 || kq == 4) ? lq : 0.f;
        r.a1 = kq == 1 ? 1.f : kq == 3 ? mq : kq == 5 ? lq : 0.f;
        r.a2 = kq == 2 ? 1.f : (kq == 4 || kq == 5) ? mq : 0.f;
    }
    return r;
}

// Euclidean projection onto the probability simplex (Duchi et al., Fig. 1,
// the closed form the paper cites for the prox step of Algorithm 1) of the
// k = 2 or 3 active coordinates selected by mask.
__device__ __forceinline__ void proj_simplex3(float v[3], const bool ok[3])
{
    float u0 = ok[0] ? v[0] : -GBP_INF, u1 = ok[1] ? v[1] : -GBP_INF, u2 = ok[2] ? v[2] : -GBP_INF;
    // sort descending (3-element network)
    float a = fmaxf(u0, u1), b = fminf(u0, u1);
    float s0 = fmaxf(a, u2), t = fminf(a, u2);
    float s1 = fmaxf(b, t), s2 = fminf(b, t);
    int k = (int)ok[0] + (int)ok[1] + (int)ok[2];
    float cs = s0, theta = s0 - 1.f;  // j = 1 always satisfies the test
    if (k >= 2) {
        cs += s1;
        float t2 = (cs - 1.f) * 0.5f;
        if (s1 - t2 > 0.f) theta = t2;
    }
    if (k >= 3) {
        cs += s2;
        float t3 = (cs - 1.f) * (1.f / 3.f);
        if (s2 - t3 > 0.f) theta = t3;
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) v[i] = ok[i] ? fmaxf(v[i] - theta, 0.f) : 0.f;
}

// Algorithm 1 (FISTA, beta_k = (k-1)/(k+1)) on the sub-face of finite
// values, with alpha_0 = hat alpha_0 = uniform.  Phi is shifted by its
// smallest finite entry, which leaves the projection (and so every iterate)
// unchanged.  Returns the objective at alpha_{n_f}.
__device__ __forceinline__ LocalRes local_fista(const float3 p[3], const float ph[3], float L, int n_f)
{
    LocalRes r;
    r.v = GBP_INF;
    r.a0 = r.a1 = r.a2 = 0.f;
    bool ok[3] = {ph[0] < GBP_INF, ph[1] < GBP_INF, ph[2] < GBP_INF};
    int k = (int)ok[0] + (int)ok[1] + (int)ok[2];
    if (k == 0) return r;
    float ref = fminf(fminf(ok[0] ? ph[0] : GBP_INF, ok[1] ? ph[1] : GBP_INF), ok[2] ? ph[2] : GBP_INF);
    if (k == 1) {
        r.a0 = ok[0] ? 1.f : 0.f;
        r.a1 = ok[1] ? 1.f : 0.f;
        r.a2 = ok[2] ? 1.f : 0.f;
        r.v = eval_alpha(p, ph, ref, r.a0, r.a1, r.a2);
        return r;
    }
    float G00 = f3dot(p[0], p[0]), G01 = f3dot(p[0], p[1]), G02 = f3dot(p[0], p[2]);
    float G11 = f3dot(p[1], p[1]), G12 = f3dot(p[1], p[2]), G22 = f3dot(p[2], p[2]);
    float sh[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) sh[i] = ok[i] ? ph[i] - ref : 0.f;
    float invk = 1.f / (float)k;
    float hat[3], prev[3], cur[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        hat[i] = ok[i] ? invk : 0.f;
        prev[i] = hat[i];
        cur[i] = hat[i];
    }
    float invL = 1.f / L;
    for (int it = 1; it <= n_f; ++it) {
        float y0 = G00 * hat[0] + G01 * hat[1] + G02 * hat[2];
        float y1 = G01 * hat[0] + G11 * hat[1] + G12 * hat[2];
        float y2 = G02 * hat[0] + G12 * hat[1] + G22 * hat[2];
        float h = sqrtf(hat[0] * y0 + hat[1] * y1 + hat[2] * y2);
        float ih = 1.f / h;
        cur[0] = (hat[0] - y0 * ih * invL) - sh[0] * invL;
        cur[1] = (hat[1] - y1 * ih * invL) - sh[1] * invL;
        cur[2] = (hat[2] - y2 * ih * invL) - sh[2] * invL;
        proj_simplex3(cur, ok);
        float beta = (float)(it - 1) / (float)(it + 1);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            hat[i] = fmaf(beta, cur[i] - prev[i], cur[i]);
            prev[i] = cur[i];
        }
    }
    r.a0 = cur[0];
    r.a1 = cur[1];
    r.a2 = cur[2];
    r.v = eval_alpha(p, ph, ref, r.a0, r.a1, r.a2);
    return r;
}

// Largest eigenvalue of a symmetric positive semi-definite 3x3 matrix by the
// closed form of the characteristic cubic (trigonometric solution).
__device__ __forceinline__ float sym3_lmax(float a00, float a01, float a02, float a11, float a12, float a22)
{
    float p1 = a01 * a01 + a02 * a02 + a12 * a12;
    float q = (a00 + a11 + a22) * (1.f / 3.f);
    float b00 = a00 - q, b11 = a11 - q, b22 = a22 - q;
    float p2 = b00 * b00 + b11 * b11 + b22 * b22 + 2.f * p1;
    if (!(p2 > 0.f)) return q;
    float pp = sqrtf(p2 * (1.f / 6.f));
    float ip = 1.f / pp;
    float c00 = b00 * ip, c11 = b11 * ip, c22 = b22 * ip, c01 = a01 * ip, c02 = a02 * ip, c12 = a12 * ip;
    float detB = c00 * (c11 * c22 - c12 * c12) - c01 * (c01 * c22 - c12 * c02) + c02 * (c01 * c12 - c11 * c02);
    float rr = fminf(fmaxf(0.5f * detB, -1.f), 1.f);
    float ang = acosf(rr) * (1.f / 3.f);
    return q + 2.f * pp * cosf(ang);
}

// Eq. (lipschitz_est) with the practical lower bound h_ = h_min / 1.1,
// h_min = min over the face of ||A alpha|| (exact, Phi = 0).
__device__ __forceinline__ float face_lipschitz(const float3 p[3])
{
    float G00 = f3dot(p[0], p[0]), G01 = f3dot(p[0], p[1]), G02 = f3dot(p[0], p[2]);
    float G11 = f3dot(p[1], p[1]), G12 = f3dot(p[1], p[2]), G22 = f3dot(p[2], p[2]);
    float lmax = sym3_lmax(G00, G01, G02, G11, G12, G22);
    float zero[3] = {0.f, 0.f, 0.f};
    int fb = 0;
    LocalRes m = local_exact(p, zero, &fb);
    float hl = m.v * (1.f / 1.1f);
    return lmax / hl * (1.f + sqrtf(lmax) / hl);
}

// ---------------------------------------------------------------------------
// grid barrier with a bounded wait (cooperative launches only)
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int *p)
{
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_relaxed_i32(const int *p)
{
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ double ld_relaxed_f64(const double *p)
{
    double v;
    asm volatile("ld.relaxed.gpu.global.f64 %0, [%1];" : "=d"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_u32(unsigned int *p, unsigned int v)
{
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier number `gen` (1, 2, ...) of a cooperative launch, in two
// levels: the CTAs form groups of gs (16, more for grids above 2048 CTAs);
// each group has an arrival counter and a release word on their own cache
// lines, so arrivals and polls spread over the groups' lines instead of all
// CTAs hitting one word.  The last CTA of a group adds one arrival to the grid
// counter (ctl->barrier); the last group's closes the barrier by releasing
// every group's word.  The wait is bounded: max_spins polls (2^22 by
// default) with a short sleep each; on timeout the abort flag and
// GBP_ERR_TIMEOUT are set and every CTA leaves.  Returns false on abort.
// grp: GBP_BAR_GROUPS zeroed entries per launch.
struct BarGroup {
    unsigned int arr;
    unsigned int pad0[31];
    unsigned int gen;
    unsigned int pad1[31];
};
constexpr unsigned int GBP_BAR_GROUPS = 128;

__device__ __forceinline__ bool grid_barrier(Control *ctl, BarGroup *grp, unsigned int gen,
                                             unsigned int max_spins = 1u << 22)
{
    __shared__ int s_ok2;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned int nblk = gridDim.x;
        const unsigned int gs = max(16u, (nblk + GBP_BAR_GROUPS - 1) / GBP_BAR_GROUPS);
        const unsigned int ng = (nblk + gs - 1) / gs;
        const unsigned int g = blockIdx.x / gs;
        const unsigned int size = min(gs, nblk - g * gs);
        __threadfence();
        const unsigned int arrived = atomicAdd(&grp[g].arr, 1u) + 1u;
        if (arrived == gen * size) {
            __threadfence();
            const unsigned int groups = atomicAdd(&ctl->barrier, 1u) + 1u;
            if (groups == gen * ng) {
                // one fence, then plain stores (a release pattern for the
                // waiters' acquire loads) so the stores issue back to back
                __threadfence();
                for (unsigned int h = 0; h < ng; ++h) st_relaxed_u32(&grp[h].gen, gen);
            }
        }
        unsigned int spins = 0;
        while (ld_acquire_u32(&grp[g].gen) < gen) {
            if (ld_relaxed_i32(&ctl->abort)) {
                ok = 0;
                break;
            }
            if (++spins > max_spins) {
                atomicExch(&ctl->abort, 1);
                atomicCAS(&ctl->status, 0, (int)GBP_ERR_TIMEOUT);
                ok = 0;
                break;
            }
            __nanosleep(20);
        }
        __threadfence();
        s_ok2 = ok;
    }
    __syncthreads();
    return s_ok2 != 0;
}

// warp-aggregated append of `pred` lanes to list (returns nothing)
__device__ __forceinline__ void warp_append(bool pred, int value, int *list, int *count)
{
    unsigned int mask = __ballot_sync(0xffffffffu, pred);
    if (mask == 0) return;
    int lane = threadIdx.x & 31;
    int leader = __ffs(mask) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(count, __popc(mask));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (pred) list[base + __popc(mask & ((1u << lane) - 1u))] = value;
}

// vertices of the face of tet tv opposite slot s, in increasing slot order
__device__ __forceinline__ void face_ids(int4 tv, int s, int &vi, int &f0, int &f1, int &f2)
{
    vi = s == 0 ? tv.x : s == 1 ? tv.y : s == 2 ? tv.z : tv.w;
    f0 = s == 0 ? tv.y : tv.x;
    f1 = s <= 1 ? tv.z : tv.y;
    f2 = s <= 2 ? tv.w : tv.z;
}

// transformed edge vectors p_n = R (v_{j_n} - v_i) of face (tet tv, opposite slot s)
__device__ __forceinline__ void face_vectors(const float4 *__restrict__ xyz, int4 tv, int s, float4 m, float sd,
                                             float3 p[3], int fv[3])
{
    int vi, f0, f1, f2;
    face_ids(tv, s, vi, f0, f1, f2);
    fv[0] = f0;
    fv[1] = f1;
    fv[2] = f2;
    const float4 xi = __ldg(&xyz[vi]);
    const float4 x0 = __ldg(&xyz[f0]), x1 = __ldg(&xyz[f1]), x2 = __ldg(&xyz[f2]);
    p[0] = xform(make_float3(x0.x - xi.x, x0.y - xi.y, x0.z - xi.z), m, sd);
    p[1] = xform(make_float3(x1.x - xi.x, x1.y - xi.y, x1.z - xi.z), m, sd);
    p[2] = xform(make_float3(x2.x - xi.x, x2.y - xi.y, x2.z - xi.z), m, sd);
}

}  // namespace gbp
