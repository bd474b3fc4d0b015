// ecg.cu -- lead-field ECG (Sec. II-D) and the misfit derivative, FP32
// CUDA-core path.
//
// Template of Eq. (tanh_waveform), read as U(xi) = K0 + (K1-K0)/2 (1 +
// tanh(2 xi / tau)).  Since (1 + tanh(y))/2 = sigma(2y) with the logistic
// sigma(z) = 1/(1 + e^-z), U(xi) = K0 + (K1 - K0) sigma(4 xi / tau), so
//   V_l(t) = K0 S_l + (K1 - K0) sum_n B_ln sigma(4 (t - phi_n) / tau),
// S_l = sum_n B_ln.  Not-yet-activated vertices contribute exactly 0 (no
// cancellation against the resting potential), and
//   U'(xi) = (K1 - K0) (4 / tau) sigma (1 - sigma).
#include "gbp_internal.cuh"

namespace gbp {

constexpr int ECG_NL = 16;   // max leads
constexpr int ECG_CH = 256;  // vertices staged per chunk

__device__ __forceinline__ float logistic(float z) { return __fdividef(1.f, 1.f + __expf(-z)); }

// Per CTA: a contiguous vertex range; thread (s_loc, g) accumulates sample
// s = s_base + s_loc over the vertices q = g mod G of each staged chunk.
// Writes part[cta][l][s] (deterministic second-stage reduction).
__global__ void __launch_bounds__(512) k_ecg_fwd(int64_t n_v, int N, int T, const float *__restrict__ L,
                                                 const float *__restrict__ phi, float t0, float dt, float c4,
                                                 int T_tile, int G, int64_t per_cta, float *__restrict__ part)
{
    extern __shared__ float sm[];
    float *sphi = sm;               // [ECG_CH]
    float *sL = sm + ECG_CH;        // [N][ECG_CH]
    float *red = sL + N * ECG_CH;   // [G][N][T_tile]
    const int tid = threadIdx.x;
    const int s_loc = tid % T_tile;
    const int g = tid / T_tile;
    const int64_t n0 = blockIdx.x * per_cta;
    const int64_t n1 = min(n0 + per_cta, n_v);
    for (int s_base = 0; s_base < T; s_base += T_tile) {
        const int s = s_base + s_loc;
        const float ts = fmaf((float)s, dt, t0);
        float acc[ECG_NL];
#pragma unroll
        for (int l = 0; l < ECG_NL; ++l) acc[l] = 0.f;
        for (int64_t c0 = n0; c0 < n1; c0 += ECG_CH) {
            const int cnt = (int)min((int64_t)ECG_CH, n1 - c0);
            __syncthreads();
            for (int q = tid; q < ECG_CH; q += blockDim.x) sphi[q] = q < cnt ? phi[c0 + q] : GBP_INF;
            for (int e = tid; e < N * ECG_CH; e += blockDim.x) {
                int l = e / ECG_CH, q = e - l * ECG_CH;
                sL[e] = q < cnt ? __ldg(&L[(int64_t)l * n_v + c0 + q]) : 0.f;
            }
            __syncthreads();
            if (s < T) {
                for (int q = g; q < cnt; q += G) {
                    const float sg = logistic((ts - sphi[q]) * c4);
                    if (sg == 0.f) continue;
#pragma unroll
                    for (int l = 0; l < ECG_NL; ++l)
                        if (l < N) acc[l] = fmaf(sL[l * ECG_CH + q], sg, acc[l]);
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int l = 0; l < ECG_NL; ++l)
            if (l < N) red[(g * N + l) * T_tile + s_loc] = acc[l];
        __syncthreads();
        for (int e = tid; e < N * T_tile; e += blockDim.x) {
            int l = e / T_tile, sl = e - l * T_tile;
            if (s_base + sl >= T) continue;
            float v = 0.f;
            for (int gg = 0; gg < G; ++gg) v += red[(gg * N + l) * T_tile + sl];
            part[((int64_t)blockIdx.x * N + l) * T + s_base + sl] = v;
        }
    }
}

// V[l][s] = K0 S_l + (K1 - K0) sum_cta part[cta][l][s]  (fixed order)
__global__ void k_ecg_reduce(int N, int T, int ncta, const float *__restrict__ part, const float *__restrict__ rowsum,
                             float K0, float dK, float *__restrict__ ecg)
{
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N * T) return;
    int l = e / T;
    float v = 0.f;
    for (int c = 0; c < ncta; ++c) v += part[(int64_t)c * N * T + e];
    ecg[e] = fmaf(K0, rowsum[l], dK * v);
}

static void ecg_fwd_shape(int T, int *T_tile, int *G)
{
    int tt = ((T + 31) / 32) * 32;
    if (tt > 512) tt = 512;
    *T_tile = tt;
    int g = 512 / tt;
    if (g < 1) g = 1;
    *G = g;
}

cudaError_t launch_ecg_forward_fp32(gbp_ctx *c, const float *phi, const gbp_template *t, float *ecg)
{
    const int N = c->N, T = t->T;
    int T_tile, G;
    ecg_fwd_shape(T, &T_tile, &G);
    int ncta = 2 * c->num_sms;
    int64_t per = (c->n_v + ncta - 1) / ncta;
    per = ((per + ECG_CH - 1) / ECG_CH) * ECG_CH;
    ncta = (int)((c->n_v + per - 1) / per);
    int64_t need = (int64_t)ncta * N * T;
    if (need > c->ecg_part_cap) {
        if (c->ecg_part) cudaFree(c->ecg_part);
        cudaError_t err = cudaMalloc(&c->ecg_part, sizeof(float) * need);
        if (err) {
            c->ecg_part = nullptr;
            c->ecg_part_cap = 0;
            return err;
        }
        c->ecg_part_cap = need;
    }
    size_t smem = sizeof(float) * (ECG_CH + (size_t)N * ECG_CH + (size_t)G * N * T_tile);
    cudaFuncSetAttribute(k_ecg_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    float c4 = 4.f / t->tau;
    time_begin(c, 2);
    k_ecg_fwd<<<ncta, T_tile * G, smem, c->stream>>>(c->n_v, N, T, c->L, phi, t->t0, t->dt, c4, T_tile, G, per,
                                                    c->ecg_part);
    k_ecg_reduce<<<(N * T + 255) / 256, 256, 0, c->stream>>>(N, T, ncta, c->ecg_part, c->Lrowsum, t->K0,
                                                            t->K1 - t->K0, ecg);
    time_end(c, 2);
    c->launches += 2;
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// misfit and its derivative in phi
// ---------------------------------------------------------------------------
// r = ecg - target; loss = 1/(N T) sum r^2 (Eq. inverse_ecg, rectangle rule).
__global__ void k_ecg_resid(int NT, const float *__restrict__ ecg, const float *__restrict__ target,
                            float *__restrict__ r, float inv_nt, float *__restrict__ loss)
{
    __shared__ double red[32];
    double acc = 0.0;
    for (int e = threadIdx.x; e < NT; e += blockDim.x) {
        float d = ecg[e] - target[e];
        r[e] = d;
        acc += (double)d * d;
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (threadIdx.x == 0) *loss = (float)(v * inv_nt);
    }
}

// lam_n = -2/(N T) (K1-K0)(4/tau) sum_s sigma(1-sigma)(z_s) sum_l B_ln r_l(s),
// z_s = 4 (t_s - phi_n)/tau.  Samples with |z| > 80 carry a weight below
// 2e-35 and are skipped (their terms vanish against the FP32 sum).
__global__ void __launch_bounds__(256) k_ecg_bwd(int64_t n_v, int N, int T, const float *__restrict__ L,
                                                 const float *__restrict__ phi, const float *__restrict__ r,
                                                 int r_in_smem, float t0, float dt, float tau, float scale,
                                                 float *__restrict__ dphi)
{
    extern __shared__ float sr[];
    if (r_in_smem) {
        for (int e = threadIdx.x; e < N * T; e += blockDim.x) sr[e] = r[e];
        __syncthreads();
    }
    const float *rr = r_in_smem ? sr : r;
    int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (n >= n_v) return;
    float p = phi[n];
    if (!(p < GBP_INF)) {
        dphi[n] = 0.f;
        return;
    }
    float Ln[ECG_NL];
#pragma unroll
    for (int l = 0; l < ECG_NL; ++l) Ln[l] = l < N ? __ldg(&L[(int64_t)l * n_v + n]) : 0.f;
    const float c4 = 4.f / tau;
    const float win = 20.f * tau;
    // clamp in float before converting, so huge phi cannot overflow the int
    const int s_lo = (int)fminf(fmaxf(ceilf((p - win - t0) / dt), 0.f), (float)T);
    const int s_hi = (int)fminf(fmaxf(floorf((p + win - t0) / dt), -1.f), (float)(T - 1));
    float acc = 0.f;
    for (int s = s_lo; s <= s_hi; ++s) {
        float z = (fmaf((float)s, dt, t0) - p) * c4;
        float e = __expf(-fabsf(z));
        float w = __fdividef(e, (1.f + e) * (1.f + e));
        float cs = 0.f;
#pragma unroll
        for (int l = 0; l < ECG_NL; ++l)
            if (l < N) cs = fmaf(Ln[l], rr[l * T + s], cs);
        acc = fmaf(w, cs, acc);
    }
    dphi[n] = scale * acc;
}

cudaError_t launch_ecg_backward(gbp_ctx *c, const float *phi, const float *ecg, const float *target,
                                const gbp_template *t, float *loss, float *dphi)
{
    const int N = c->N, T = t->T;
    int64_t NT = (int64_t)N * T;
    if (NT > c->resid_cap) {
        if (c->resid) cudaFree(c->resid);
        cudaError_t err = cudaMalloc(&c->resid, sizeof(float) * NT);
        if (err) {
            c->resid = nullptr;
            c->resid_cap = 0;
            return err;
        }
        c->resid_cap = NT;
    }
    time_begin(c, 3);
    k_ecg_resid<<<1, 1024, 0, c->stream>>>((int)NT, ecg, target, c->resid, 1.f / (float)NT, loss);
    size_t smem = sizeof(float) * NT;
    int in_smem = smem <= 160 * 1024;
    if (in_smem) cudaFuncSetAttribute(k_ecg_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    else smem = 0;
    float scale = -2.f / (float)NT * (t->K1 - t->K0) * (4.f / t->tau);
    int th = 256;
    k_ecg_bwd<<<(unsigned)((c->n_v + th - 1) / th), th, smem, c->stream>>>(c->n_v, N, T, c->L, phi, c->resid,
                                                                           in_smem, t->t0, t->dt, t->tau, scale,
                                                                           dphi);
    time_end(c, 3);
    c->launches += 2;
    return cudaGetLastError();
}

// dispatcher (the BF16 tensor-core path lives in ecg_bf16.cu)
cudaError_t launch_ecg_forward_bf16(gbp_ctx *c, const float *phi, const gbp_template *t, float *ecg);

cudaError_t launch_ecg_forward(gbp_ctx *c, const float *phi, const gbp_template *t, int prec, float *ecg)
{
    if (prec == GBP_PREC_BF16) return launch_ecg_forward_bf16(c, phi, t, ecg);
    return launch_ecg_forward_fp32(c, phi, t, ecg);
}

}  // namespace gbp
