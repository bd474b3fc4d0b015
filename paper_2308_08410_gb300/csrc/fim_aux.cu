// fim_aux.cu -- the kernels around the FIM of fim.cu: per-tet metric
// precompute and FISTA Lipschitz estimates, onset seeding (Eq. upwind_xi)
// and vertex-state reset before the solve, the parent pass after it, and
// the batched local-solve diagnostic.
#include "gbp_internal.cuh"

namespace gbp {

// ---------------------------------------------------------------------------
// per-tet metric (Sec. II-A): R = D^{1/2} in factored form
// ---------------------------------------------------------------------------
// Batched: entry g = b * n_t + j of the per-problem arrays (cf, ct, tv).
// The metric of tet j in problem b is kept as the unit fibre tf[j] (shared by
// the batch) and tv[g] = (1/ct, 1/cf - 1/ct): R = D^{1/2} applied to e is
// e / ct + (1/cf - 1/ct) (f.e) f.
__global__ void k_precompute(int64_t n_t, int64_t n_tot, const float *__restrict__ fib, const float *__restrict__ cf,
                             const float *__restrict__ ct, float4 *__restrict__ tf, float2 *__restrict__ tv,
                             Control *ctl)
{
    int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= n_tot) return;
    const int64_t j = g % n_t;
    float fx = fib[3 * j], fy = fib[3 * j + 1], fz = fib[3 * j + 2];
    float nn = sqrtf(fx * fx + fy * fy + fz * fz);
    float vf = cf[g], vt = ct[g];
    bool bad = !(nn > 0.f) || !(vf > 0.f) || !(vt > 0.f) || !isfinite(vf) || !isfinite(vt) || !isfinite(nn);
    if (bad) {
        atomicCAS(&ctl->param_status, 0, (int)GBP_ERR_NOT_SPD);
        nn = 1.f; fx = 1.f; fy = fz = 0.f;
        vf = vt = 1.f;
    }
    float in = 1.f / nn;
    float sa = 1.f / vt;
    tv[g] = make_float2(sa, 1.f / vf - sa);
    if (g < n_t) tf[g] = make_float4(fx * in, fy * in, fz * in, 0.f);
}

cudaError_t launch_precompute(gbp_ctx *c)
{
    int th = 256;
    const int64_t n_tot = c->n_t * c->nb;
    int64_t bl = (n_tot + th - 1) / th;
    k_precompute<<<(unsigned)bl, th, 0, c->stream>>>(c->n_t, n_tot, c->fib, c->cf, c->ct, c->tf, c->tv,
                                                     c->ctl);
    c->launches++;
    return cudaGetLastError();
}

__global__ void k_lipschitz(int64_t n_t, int64_t n_tot, const float4 *__restrict__ xyz, const int4 *__restrict__ tets,
                            const float4 *__restrict__ tf, const float2 *__restrict__ tvel, float4 *__restrict__ tlip)
{
    int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g >= n_tot) return;
    int4 tv = tets[g % n_t];
    const float4 f = tf[g % n_t];
    const float2 v2 = tvel[g];
    const float4 m = make_float4(f.x, f.y, f.z, v2.x);
    const float sd = v2.y;
    float L[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        float3 p[3];
        int fv[3];
        face_vectors(xyz, tv, s, m, sd, p, fv);
        L[s] = face_lipschitz(p);
    }
    tlip[g] = make_float4(L[0], L[1], L[2], L[3]);
}

cudaError_t launch_lipschitz(gbp_ctx *c)
{
    int th = 256;
    const int64_t n_tot = c->n_t * c->nb;
    int64_t bl = (n_tot + th - 1) / th;
    k_lipschitz<<<(unsigned)bl, th, 0, c->stream>>>(c->n_t, n_tot, c->xyz, c->tets, c->tf, c->tv, c->tlip);
    c->launches++;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// onset seeding (Algorithm 2 initialisation, Eq. upwind_xi)
// ---------------------------------------------------------------------------

// Batched: thread g = b * K + k (onset times t [nb][K]; sites shared, or
// one set per problem when per_problem is set: idx [nb][K], bary [nb][K][4]).
// Vertices from n_real on (the apex of a lifted triangle mesh) take no key.
__global__ void k_onset_keys(int K, int nb, int per_problem, int kind, const int *__restrict__ idx,
                             const float *__restrict__ bary,
                             const float *__restrict__ t, int64_t n_v, int64_t n_real, int64_t n_t,
                             const float4 *__restrict__ xyz,
                             const int4 *__restrict__ tets, const float4 *__restrict__ tf,
                             const float2 *__restrict__ tvel, unsigned long long *keys_all, Control *ctl)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= K * nb) return;
    const int b = g / K, k = g - b * K;
    unsigned long long *keys = keys_all + (int64_t)b * n_v;
    const float tk = t[g];
    const int sk = per_problem ? g : k;
    int id = idx[sk];
    if (kind == GBP_ONSET_NODAL) {
        if (id < 0 || id >= n_real) {
            atomicCAS(&ctl->status, 0, (int)GBP_ERR_INVALID_ARG);
            return;
        }
        unsigned long long key = ((unsigned long long)float_key(tk) << 32) | (unsigned)k;
        atomicMin(&keys[id], key);
    } else {
        if (id < 0 || id >= n_t) {
            atomicCAS(&ctl->status, 0, (int)GBP_ERR_INVALID_ARG);
            return;
        }
        int4 tv = tets[id];
        int ids[4] = {tv.x, tv.y, tv.z, tv.w};
        float4 x[4];
        float3 xo = make_float3(0.f, 0.f, 0.f);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            x[q] = xyz[ids[q]];
            float b = bary[4 * sk + q];
            xo.x = fmaf(b, x[q].x, xo.x);
            xo.y = fmaf(b, x[q].y, xo.y);
            xo.z = fmaf(b, x[q].z, xo.z);
        }
        const float4 fe = tf[id];
        const float2 ve = tvel[(int64_t)b * n_t + id];
        const float4 m = make_float4(fe.x, fe.y, fe.z, ve.x);
        const float sd = ve.y;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float3 w = xform(make_float3(x[q].x - xo.x, x[q].y - xo.y, x[q].z - xo.z), m, sd);
            float v = tk + sqrtf(f3dot(w, w));
            unsigned long long key = ((unsigned long long)float_key(v) << 32) | (unsigned)k;
            if (ids[q] < n_real) atomicMin(&keys[ids[q]], key);
        }
    }
}

// Per vertex: decode the onset key, reset the FIM state.
__global__ void k_init_nodes(int64_t n_tot, const unsigned long long *__restrict__ keys, float *phi, int4 *rec,
                             int *chg, int *stamp, int2 *pc)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n_tot) return;
    unsigned long long key = keys[i];
    if (key != ~0ull) {
        phi[i] = key_float((unsigned int)(key >> 32));
        rec[i] = make_int4(-1 - (int)(key & 0xffffffffu), 0, 0, 0);
        chg[i] = 0;
    } else {
        phi[i] = GBP_INF;
        rec[i] = make_int4(GBP_UNREACHED, 0, 0, 0);
        chg[i] = -1000000;
    }
    stamp[i] = 0;
    pc[i] = make_int2(__float_as_int(phi[i]), chg[i]);
}

// phi of every vertex entry from the FIM's packed (value, change stamp) state
__global__ void k_unpack_pc(int64_t n_tot, const int2 *__restrict__ pc, float *phi)
{
    const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (g < n_tot) phi[g] = __int_as_float(pc[g].x);
}

// Seeded vertices put their neighbours on the first active list.
// Batched: vertex entry g = b * n_v + i (lists hold such entries).
__global__ void k_seed_lists(int n_v, int n_tot, const unsigned long long *__restrict__ keys,
                             const int *__restrict__ n2n_ptr, const int *__restrict__ n2n, int *stamp, int *list1,
                             Control *ctl)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_tot || keys[g] == ~0ull) return;
    const int b = g / n_v, i = g - b * n_v;
    for (int e = n2n_ptr[i]; e < n2n_ptr[i + 1]; ++e) {
        const int m = b * n_v + n2n[e];
        if (atomicMax(&stamp[m], 1) < 1) {
            int pos = atomicAdd(&ctl->count[1], 1);
            list1[pos] = m;
        }
    }
}

// ---------------------------------------------------------------------------
// persistent FIM (Algorithm 2)

// Before the FIM: reset the control block (counters, status; the
// precompute's status word, the last field, is kept) and the onset keys,
// seed the onset values, reset the vertex state and build the first active
// list (the neighbours of the onset vertices).
cudaError_t launch_fim_seed(gbp_ctx *c)
{
    const int64_t n_v = c->n_v;
    const int64_t n_tot = n_v * c->nb;
    cudaError_t err = cudaMemsetAsync(c->ctl, 0, offsetof(Control, param_status), c->stream);
    if (err) return err;
    err = cudaMemsetAsync(c->keys, 0xff, sizeof(unsigned long long) * n_tot, c->stream);
    if (err) return err;
    const int th = 256;
    k_onset_keys<<<(c->K * c->nb + th - 1) / th, th, 0, c->stream>>>(c->K, c->nb, c->site_b > 0,
                                                                      c->onset_kind, c->on_idx, c->on_bary,
                                                                      c->on_t, n_v, c->n_e, c->n_t, c->xyz,
                                                                      c->tets, c->tf, c->tv, c->keys, c->ctl);
    const unsigned bl = (unsigned)((n_tot + th - 1) / th);
    k_init_nodes<<<bl, th, 0, c->stream>>>(n_tot, c->keys, c->phi, c->rec, c->chg, c->stamp, c->pc);
    k_seed_lists<<<bl, th, 0, c->stream>>>((int)n_v, (int)n_tot, c->keys, c->n2n_ptr, c->n2n, c->stamp,
                                           c->lists + n_tot, c->ctl);
    c->launches += 3;
    return cudaGetLastError();
}

// After the FIM: the final values out of the packed vertex state.
cudaError_t launch_unpack_state(gbp_ctx *c)
{
    const int64_t n_tot = c->n_v * c->nb;
    k_unpack_pc<<<(unsigned)((n_tot + 255) / 256), 256, 0, c->stream>>>(n_tot, c->pc, c->phi);
    c->launches++;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// parent pass: alpha of the final parent face with the final values
// ---------------------------------------------------------------------------
// Batched: entry g = b * n_v + i.  Outputs (single problem only) and the
// unreached count cover the caller's vertices i < n_e; for a lifted triangle
// mesh (dim 2) the code is written as triangle * 3 + slot and alpha as the
// weights of the triangle's two other vertices (the apex weight is 0).
//
// It also writes the adjoint's 32-byte record of each vertex entry (two
// int4), so that one hop of the adjoint reads one sector:
//   (f0, f1, f2, jt): the parent face's vertices in slot order (within the
//     problem; -1 where alpha is 0) and the parent tet, or jt = the code for
//     an onset-held (-1 - k) or unreached vertex (f = -1);
//   (a0, a1, gcf, gct) as float bits: alpha of f0 and f1 (alpha of f2 is
//     (1 - a0) - a1, the expression the local solver gives it), and the
//     derivatives of phi_i = sum alpha_n phi_n + ||w||_D (w = v_i - sum
//     alpha_n v_n, alpha frozen) with respect to the tet's velocities:
//     gcf = -(f.w)^2 / (cf^3 ||w||_D), gct = -|w_perp|^2 / (ct^3 ||w||_D).
template <int MODE>
__global__ void k_parent_pass(int n_v, int n_e, int dim, int n_tot, int64_t n_t, const float4 *__restrict__ xyz,
                              const int4 *__restrict__ tets, const float4 *__restrict__ tf,
                              const float2 *__restrict__ tv_all, const float4 *__restrict__ tlip_all, int n_f,
                              const float *__restrict__ cf_all, const float *__restrict__ ct_all,
                              const float *__restrict__ phi_all, int4 *rec, int4 *arec, float *out_phi,
                              int32_t *out_parent, float *out_alpha, Control *ctl)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_tot) return;
    const int b = g / n_v;
    const float *phi = phi_all + (int64_t)b * n_v;
    const float2 *tvb = tv_all + (int64_t)b * n_t;
    const float4 *tlip = tlip_all + (int64_t)b * n_t;
    const int i = g;
    int4 r = rec[i];
    int code = r.x;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f;
    float pv = phi_all[i];
    int4 ar0 = make_int4(-1, -1, -1, code);
    int4 ar1 = make_int4(0, 0, 0, 0);
    if (code >= 0) {
        int j = code >> 2, s = code & 3;
        int4 tv = tets[j];
        float3 p[3];
        int fv[3];
        const float4 fj = tf[j];
        const float2 vj = tvb[j];
        face_vectors(xyz, tv, s, make_float4(fj.x, fj.y, fj.z, vj.x), vj.y, p, fv);
        float ph[3] = {phi[fv[0]], phi[fv[1]], phi[fv[2]]};
        LocalRes lr;
        int fb = 0;
        if (MODE == GBP_LOCAL_FISTA) {
            float4 Lq = tlip[j];
            float Lv = s == 0 ? Lq.x : s == 1 ? Lq.y : s == 2 ? Lq.z : Lq.w;
            lr = local_fista(p, ph, Lv, n_f);
        } else {
            lr = local_exact<true>(p, ph, &fb);
        }
        a0 = lr.a0;
        a1 = lr.a1;
        a2 = lr.a2;
        rec[i] = make_int4(code, __float_as_int(a0), __float_as_int(a1), __float_as_int(a2));
        // w = v_i - sum alpha_n v_n = -sum alpha_n (v_n - v_i)
        const float4 xi = xyz[i - b * n_v];
        const float al[3] = {a0, a1, a2};
        float3 w = make_float3(0.f, 0.f, 0.f);
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const float4 xq = xyz[fv[q]];
            w.x = fmaf(-al[q], xq.x - xi.x, w.x);
            w.y = fmaf(-al[q], xq.y - xi.y, w.y);
            w.z = fmaf(-al[q], xq.z - xi.z, w.z);
        }
        const float fw = fj.x * w.x + fj.y * w.y + fj.z * w.z;
        const float3 wp = make_float3(w.x - fw * fj.x, w.y - fw * fj.y, w.z - fw * fj.z);
        const float wp2 = f3dot(wp, wp);
        const float icf = 1.f / cf_all[(int64_t)b * n_t + j], ict = 1.f / ct_all[(int64_t)b * n_t + j];
        const float gg = sqrtf(wp2 * ict * ict + fw * fw * icf * icf);
        float gcf = 0.f, gct = 0.f;
        if (gg > 0.f) {
            const float ig = 1.f / gg;
            gcf = -fw * fw * icf * icf * icf * ig;
            gct = -wp2 * ict * ict * ict * ig;
        }
        ar0 = make_int4(a0 != 0.f ? fv[0] : -1, a1 != 0.f ? fv[1] : -1, a2 != 0.f ? fv[2] : -1, j);
        ar1 = make_int4(__float_as_int(a0), __float_as_int(a1), __float_as_int(gcf), __float_as_int(gct));
    }
    arec[2 * (int64_t)i] = ar0;
    arec[2 * (int64_t)i + 1] = ar1;
    if (i - b * n_v >= n_e) return;
    if (code == GBP_UNREACHED) atomicAdd(&ctl->unreached, 1ull);
    if (out_phi) out_phi[i] = pv;
    if (dim == 2) {
        if (out_parent) out_parent[i] = code >= 0 ? (code >> 2) * 3 + (code & 3) : code;
        if (out_alpha) {
            out_alpha[2 * i] = a0;
            out_alpha[2 * i + 1] = a1;
        }
        return;
    }
    if (out_parent) out_parent[i] = code;
    if (out_alpha) {
        out_alpha[3 * i] = a0;
        out_alpha[3 * i + 1] = a1;
        out_alpha[3 * i + 2] = a2;
    }
}

cudaError_t launch_parent_pass(gbp_ctx *c, int mode, int n_f, float *phi, int32_t *parent, float *alpha)
{
    int th = 256;
    const int n_tot = (int)(c->n_v * c->nb);
    unsigned bl = (unsigned)((n_tot + th - 1) / th);
    time_begin(c, 1);
    if (mode == GBP_LOCAL_FISTA)
        k_parent_pass<GBP_LOCAL_FISTA><<<bl, th, 0, c->stream>>>((int)c->n_v, (int)c->n_e, c->dim, n_tot, c->n_t,
                                                                 c->xyz, c->tets, c->tf, c->tv, c->tlip, n_f, c->cf,
                                                                 c->ct, c->phi, c->rec, c->adj_rec, phi, parent,
                                                                 alpha, c->ctl);
    else
        k_parent_pass<GBP_LOCAL_EXACT><<<bl, th, 0, c->stream>>>((int)c->n_v, (int)c->n_e, c->dim, n_tot, c->n_t,
                                                                 c->xyz, c->tets, c->tf, c->tv, c->tlip, n_f, c->cf,
                                                                 c->ct, c->phi, c->rec, c->adj_rec, phi, parent,
                                                                 alpha, c->ctl);
    time_end(c, 1);
    c->launches++;
    return cudaGetLastError();
}

// the activation map and parent record of problem b of the last solve, in
// the caller's layout (the output part of k_parent_pass: codes and alpha for
// d = 3, triangle codes and two weights for d = 2)
__global__ void k_export_solution(int n_e, int dim, const float *__restrict__ phi_b, const int4 *__restrict__ rec,
                                  float *out_phi, int32_t *out_parent, float *out_alpha)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_e) return;
    if (out_phi) out_phi[i] = phi_b[i];
    const int4 r = rec[i];
    const int code = r.x;
    if (dim == 2) {
        if (out_parent) out_parent[i] = code >= 0 ? (code >> 2) * 3 + (code & 3) : code;
        if (out_alpha) {
            out_alpha[2 * i] = __int_as_float(r.y);
            out_alpha[2 * i + 1] = __int_as_float(r.z);
        }
        return;
    }
    if (out_parent) out_parent[i] = code;
    if (out_alpha) {
        out_alpha[3 * i] = __int_as_float(r.y);
        out_alpha[3 * i + 1] = __int_as_float(r.z);
        out_alpha[3 * i + 2] = __int_as_float(r.w);
    }
}

cudaError_t launch_export_solution(gbp_ctx *c, int b, float *phi, int32_t *parent, float *alpha)
{
    const int n_e = (int)c->n_e;
    const int64_t off = (int64_t)b * c->n_v;
    k_export_solution<<<(n_e + 255) / 256, 256, 0, c->stream>>>(n_e, c->dim, c->phi + off, c->rec + off, phi, parent,
                                                                  alpha);
    c->launches++;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// local problems on independent faces (diagnostic entry point)
// ---------------------------------------------------------------------------
__global__ void k_local_batch(int64_t n, const float *__restrict__ e, const float *__restrict__ fib,
                              const float *__restrict__ cf, const float *__restrict__ ct,
                              const float *__restrict__ Phi, int mode, int n_f, float *value, float *alpha,
                              Control *ctl)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    float fx = fib[3 * i], fy = fib[3 * i + 1], fz = fib[3 * i + 2];
    float in = rsqrtf(fx * fx + fy * fy + fz * fz);
    float sa = 1.f / ct[i];
    float4 m = make_float4(fx * in, fy * in, fz * in, sa);
    float sd = 1.f / cf[i] - sa;
    float3 p[3];
    float ph[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        p[a] = xform(make_float3(e[9 * i + 3 * a], e[9 * i + 3 * a + 1], e[9 * i + 3 * a + 2]), m, sd);
        ph[a] = Phi[3 * i + a];
    }
    LocalRes r;
    int fb = 0;
    if (mode == GBP_LOCAL_FISTA) r = local_fista(p, ph, face_lipschitz(p), n_f);
    else r = local_exact<true>(p, ph, &fb);
    if (fb) atomicAdd(&ctl->fp64_fallbacks, (unsigned long long)fb);
    value[i] = r.v;
    alpha[3 * i] = r.a0;
    alpha[3 * i + 1] = r.a1;
    alpha[3 * i + 2] = r.a2;
}

cudaError_t launch_local_batch(gbp_ctx *c, int64_t n, const float *e, const float *fib, const float *cf,
                               const float *ct, const float *Phi, int mode, int n_f, float *value, float *alpha)
{
    int th = 128;
    unsigned bl = (unsigned)((n + th - 1) / th);
    k_local_batch<<<bl, th, 0, c->stream>>>(n, e, fib, cf, ct, Phi, mode, n_f, value, alpha, c->ctl);
    c->launches++;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// bounded-wait diagnostic: the grid barrier of the FIM and the adjoint with
// `absent` CTAs that never arrive, so that every other CTA's wait runs out
// after max_spins polls and latches GBP_ERR_TIMEOUT (absent = 0: the barrier
// completes and nothing is latched)
// ---------------------------------------------------------------------------
__global__ void k_barrier_probe(Control *ctl, BarGroup *grp, int absent, unsigned int max_spins)
{
    if ((int)blockIdx.x >= (int)gridDim.x - absent) return;
    grid_barrier(ctl, grp, 1u, max_spins);
}

cudaError_t launch_barrier_probe(gbp_ctx *c, int absent, unsigned int max_spins)
{
    cudaError_t err = cudaMemsetAsync(c->ctl, 0, offsetof(Control, param_status), c->stream);
    if (err) return err;
    err = cudaMemsetAsync(c->bar_grp, 0, sizeof(BarGroup) * GBP_BAR_GROUPS, c->stream);
    if (err) return err;
    Control *ctl = c->ctl;
    BarGroup *grp = c->bar_grp;
    void *args[] = {&ctl, &grp, &absent, &max_spins};
    err = cudaLaunchCooperativeKernel((const void *)k_barrier_probe, dim3(c->num_sms), dim3(32), args, 0, c->stream);
    c->launches++;
    return err;
}

}  // namespace gbp
