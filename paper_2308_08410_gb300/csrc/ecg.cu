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

constexpr int ECG_CH = 256;  // vertices staged per chunk

// The accurate expf and an IEEE division: the ECG is a sum of up to 10^6
// terms that can cancel by several orders of magnitude (lead-field rows sum
// to zero), so the relative error of each sigma carries over multiplied by
// that condition number; the __expf intrinsic's error grows with |z| (tens
// of ulp at the |z| ~ 50 this sum still sees).
__device__ __forceinline__ float logistic(float z) { return 1.f / (1.f + expf(-z)); }

// Per CTA: a contiguous vertex range; thread (s_loc, g) accumulates sample
// s = s_base + s_loc over the vertices q = g mod G of each staged chunk.
// Writes part[cta][l][s] (deterministic second-stage reduction).  NL is the
// number of leads, a compile-time constant so the accumulators stay in
// registers.  Each chunk of ECG_CH vertices is summed in FP32 and the chunk
// sums in FP64: the terms of one lead can cancel by orders of magnitude
// (its lead-field row sums to zero), and a long FP32 running sum would
// carry its rounding times that cancellation into the result.
// Problem blockIdx.y of a batch reads phi + blockIdx.y * phi_stride and
// writes part + blockIdx.y * part_stride.
template <int NL>
__global__ void __launch_bounds__(512) k_ecg_fwd_t(int64_t n_v, int T, const float *__restrict__ L,
                                                   const float *__restrict__ phi, float t0, float dt, float c4,
                                                   int T_tile, int G, int64_t per_cta, double *__restrict__ part,
                                                   int64_t phi_stride, int64_t part_stride)
{
    phi += blockIdx.y * phi_stride;
    part += blockIdx.y * part_stride;
    extern __shared__ double smd[];
    double *red = smd;                                        // [G][NL][T_tile]
    float *sphi = reinterpret_cast<float *>(red + (size_t)G * NL * T_tile);  // [ECG_CH]
    float *sL = sphi + ECG_CH;                                // [ECG_CH][NL]
    const int tid = threadIdx.x;
    const int s_loc = tid % T_tile;
    const int g = tid / T_tile;
    const int64_t n0 = blockIdx.x * per_cta;
    const int64_t n1 = min(n0 + per_cta, n_v);
    for (int s_base = 0; s_base < T; s_base += T_tile) {
        const int s = s_base + s_loc;
        const float ts = fmaf((float)s, dt, t0);
        double accd[NL];
#pragma unroll
        for (int l = 0; l < NL; ++l) accd[l] = 0.0;
        for (int64_t c0 = n0; c0 < n1; c0 += ECG_CH) {
            const int cnt = (int)min((int64_t)ECG_CH, n1 - c0);
            __syncthreads();
            for (int q = tid; q < ECG_CH; q += blockDim.x) sphi[q] = q < cnt ? phi[c0 + q] : GBP_INF;
            for (int e = tid; e < NL * ECG_CH; e += blockDim.x) {
                const int l = e / ECG_CH, q = e - l * ECG_CH;
                sL[q * NL + l] = q < cnt ? __ldg(&L[(int64_t)l * n_v + c0 + q]) : 0.f;
            }
            __syncthreads();
            if (s < T) {
                float acc[NL];
#pragma unroll
                for (int l = 0; l < NL; ++l) acc[l] = 0.f;
                for (int q = g; q < cnt; q += G) {
                    const float sg = logistic((ts - sphi[q]) * c4);
                    const float *Lq = sL + q * NL;
#pragma unroll
                    for (int l = 0; l < NL; ++l) acc[l] = fmaf(Lq[l], sg, acc[l]);
                }
#pragma unroll
                for (int l = 0; l < NL; ++l) accd[l] += (double)acc[l];
            }
        }
        __syncthreads();
#pragma unroll
        for (int l = 0; l < NL; ++l) red[(g * NL + l) * T_tile + s_loc] = accd[l];
        __syncthreads();
        for (int e = tid; e < NL * T_tile; e += blockDim.x) {
            const int l = e / T_tile, sl = e - l * T_tile;
            if (s_base + sl >= T) continue;
            double v = 0.0;
            for (int gg = 0; gg < G; ++gg) v += red[(gg * NL + l) * T_tile + sl];
            part[((int64_t)blockIdx.x * NL + l) * T + s_base + sl] = v;
        }
    }
}

template <int NL>
static cudaError_t launch_fwd_n(int ncta, int nb, int threads, size_t smem, cudaStream_t st, int64_t n_v, int T,
                                const float *L, const float *phi, float t0, float dt, float c4, int T_tile, int G,
                                int64_t per, double *part, int64_t phi_stride, int64_t part_stride)
{
    cudaFuncSetAttribute(k_ecg_fwd_t<NL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_ecg_fwd_t<NL><<<dim3(ncta, nb), threads, smem, st>>>(n_v, T, L, phi, t0, dt, c4, T_tile, G, per, part,
                                                           phi_stride, part_stride);
    return cudaGetLastError();
}

// one instantiation per lead count 1..16; nb problems (grid y)
static cudaError_t launch_ecg_fwd_leads_b(int N, int ncta, int nb, int threads, size_t smem, cudaStream_t st,
                                          int64_t n_v, int T, const float *L, const float *phi, float t0, float dt,
                                          float c4, int T_tile, int G, int64_t per, double *part, int64_t phi_stride,
                                          int64_t part_stride)
{
    switch (N) {
#define GBP_ECG_CASE(n) \
    case n: return launch_fwd_n<n>(ncta, nb, threads, smem, st, n_v, T, L, phi, t0, dt, c4, T_tile, G, per, part, \
                                   phi_stride, part_stride);
        GBP_ECG_CASE(1) GBP_ECG_CASE(2) GBP_ECG_CASE(3) GBP_ECG_CASE(4) GBP_ECG_CASE(5) GBP_ECG_CASE(6)
        GBP_ECG_CASE(7) GBP_ECG_CASE(8) GBP_ECG_CASE(9) GBP_ECG_CASE(10) GBP_ECG_CASE(11) GBP_ECG_CASE(12)
        GBP_ECG_CASE(13) GBP_ECG_CASE(14) GBP_ECG_CASE(15) GBP_ECG_CASE(16)
#undef GBP_ECG_CASE
    }
    return cudaErrorInvalidValue;
}

// The forward kernel for N leads (1..16) as a function pointer, for callers
// that launch it with cudaLaunchKernel to get that launch's own status;
// nullptr for other N.
const void *ecg_fwd_kernel(int N)
{
    switch (N) {
#define GBP_ECG_PTR(n) \
    case n: return (const void *)k_ecg_fwd_t<n>;
        GBP_ECG_PTR(1) GBP_ECG_PTR(2) GBP_ECG_PTR(3) GBP_ECG_PTR(4) GBP_ECG_PTR(5) GBP_ECG_PTR(6)
        GBP_ECG_PTR(7) GBP_ECG_PTR(8) GBP_ECG_PTR(9) GBP_ECG_PTR(10) GBP_ECG_PTR(11) GBP_ECG_PTR(12)
        GBP_ECG_PTR(13) GBP_ECG_PTR(14) GBP_ECG_PTR(15) GBP_ECG_PTR(16)
#undef GBP_ECG_PTR
    }
    return nullptr;
}

// one problem
cudaError_t launch_ecg_fwd_leads(int N, int ncta, int threads, size_t smem, cudaStream_t st, int64_t n_v, int T,
                                 const float *L, const float *phi, float t0, float dt, float c4, int T_tile, int G,
                                 int64_t per, double *part)
{
    return launch_ecg_fwd_leads_b(N, ncta, 1, threads, smem, st, n_v, T, L, phi, t0, dt, c4, T_tile, G, per, part, 0,
                                  0);
}

// V[l][s] = K0 S_l + (K1 - K0) sum_cta part[cta][l][s]  (fixed order, FP64)
__global__ void k_ecg_reduce(int N, int T, int ncta, const double *__restrict__ part, const float *__restrict__ rowsum,
                             float K0, float dK, float *__restrict__ ecg)
{
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N * T) return;
    int l = e / T;
    double v = 0.0;
    for (int c = 0; c < ncta; ++c) v += part[(int64_t)c * N * T + e];
    ecg[e] = (float)((double)K0 * rowsum[l] + (double)dK * v);
}

// the same for nb problems: entry e of [nb][N][T], partials of problem b at
// part + b * part_stride
__global__ void k_ecg_reduce_b(int N, int T, int nb, int ncta, const double *__restrict__ part, int64_t part_stride,
                               const float *__restrict__ rowsum, float K0, float dK, float *__restrict__ ecg)
{
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int NT = N * T;
    if (e >= (int64_t)nb * NT) return;
    const int b = (int)(e / NT), en = (int)(e - (int64_t)b * NT);
    const int l = en / T;
    const double *pb = part + b * part_stride;
    double v = 0.0;
    for (int c = 0; c < ncta; ++c) v += pb[(int64_t)c * NT + en];
    ecg[e] = (float)((double)K0 * rowsum[l] + (double)dK * v);
}

// staging of the FP32 forward: FP64 partials of [ncta][N][T] plus the staged
// chunk, in bytes of dynamic shared memory
size_t ecg_fwd_smem(int N, int T_tile, int G)
{
    return sizeof(double) * (size_t)G * N * T_tile + sizeof(float) * (ECG_CH + (size_t)N * ECG_CH);
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

// nb problems: phi [b] at phi + b * phi_stride, ecg [nb][N][T]
cudaError_t launch_ecg_forward_fp32_batch(gbp_ctx *c, int nb, const float *phi, int64_t phi_stride,
                                          const gbp_template *t, float *ecg)
{
    const int N = c->N, T = t->T;
    int T_tile, G;
    ecg_fwd_shape(T, &T_tile, &G);
    int ncta = 2 * c->num_sms;
    int64_t per = (c->n_e + ncta - 1) / ncta;
    per = ((per + ECG_CH - 1) / ECG_CH) * ECG_CH;
    ncta = (int)((c->n_e + per - 1) / per);
    const int64_t part_stride = (int64_t)ncta * N * T;  // doubles per problem
    int64_t need = 2 * part_stride * nb;                // FP64 partials, counted in floats
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
    double *part = reinterpret_cast<double *>(c->ecg_part);
    size_t smem = ecg_fwd_smem(N, T_tile, G);
    float c4 = 4.f / t->tau;
    time_begin(c, 2);
    cudaError_t le = launch_ecg_fwd_leads_b(N, ncta, nb, T_tile * G, smem, c->stream, c->n_e, T, c->L, phi, t->t0,
                                            t->dt, c4, T_tile, G, per, part, phi_stride, part_stride);
    if (le) return le;
    const int64_t tot = (int64_t)nb * N * T;
    k_ecg_reduce_b<<<(unsigned)((tot + 255) / 256), 256, 0, c->stream>>>(N, T, nb, ncta, part, part_stride,
                                                                         c->Lrowsum, t->K0, t->K1 - t->K0, ecg);
    time_end(c, 2);
    c->launches += 2;
    return cudaGetLastError();
}

cudaError_t launch_ecg_forward_fp32(gbp_ctx *c, const float *phi, const gbp_template *t, float *ecg)
{
    return launch_ecg_forward_fp32_batch(c, 1, phi, 0, t, ecg);
}

// ---------------------------------------------------------------------------
// misfit and its derivative in phi
// ---------------------------------------------------------------------------
// r = ecg - target; loss = 1/(N T) sum r^2 (Eq. inverse_ecg, rectangle rule).
// One block per problem: block b reads [b][N][T] and writes loss[b].
__global__ void k_ecg_resid(int NT, const float *__restrict__ ecg, const float *__restrict__ target,
                            float *__restrict__ r, float inv_nt, float *__restrict__ loss)
{
    ecg += (int64_t)blockIdx.x * NT;
    target += (int64_t)blockIdx.x * NT;
    r += (int64_t)blockIdx.x * NT;
    loss += blockIdx.x;
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
// 2e-35 and are skipped (their terms vanish against the FP32 sum).  The
// residual is stored sample-major in shared memory (rT[s][l]) so one sample's
// leads are contiguous.  NL = number of leads (compile time).
// Problem blockIdx.y of a batch: phi and dphi at + blockIdx.y * phi_stride,
// r at + blockIdx.y * NL * T.
template <int NL>
__global__ void __launch_bounds__(256) k_ecg_bwd_t(int64_t n_v, int T, const float *__restrict__ L,
                                                   const float *__restrict__ phi, const float *__restrict__ r,
                                                   float t0, float dt, float tau, float scale,
                                                   float *__restrict__ dphi, int64_t phi_stride)
{
    phi += blockIdx.y * phi_stride;
    dphi += blockIdx.y * phi_stride;
    r += (int64_t)blockIdx.y * NL * T;
    extern __shared__ float rT[];  // [T][NL]
    for (int e = threadIdx.x; e < NL * T; e += blockDim.x) {
        const int l = e / T, s = e - l * T;
        rT[s * NL + l] = r[e];
    }
    __syncthreads();
    const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (n >= n_v) return;
    const float p = phi[n];
    if (!(p < GBP_INF)) {
        dphi[n] = 0.f;
        return;
    }
    float Ln[NL];
#pragma unroll
    for (int l = 0; l < NL; ++l) Ln[l] = __ldg(&L[(int64_t)l * n_v + n]);
    const float c4 = 4.f / tau;
    const float win = 20.f * tau;
    // clamp in float before converting, so huge phi cannot overflow the int
    const int s_lo = (int)fminf(fmaxf(ceilf((p - win - t0) / dt), 0.f), (float)T);
    const int s_hi = (int)fminf(fmaxf(floorf((p + win - t0) / dt), -1.f), (float)(T - 1));
    float acc = 0.f;
    for (int s = s_lo; s <= s_hi; ++s) {
        const float z = (fmaf((float)s, dt, t0) - p) * c4;
        const float e = expf(-fabsf(z));
        const float w = e / ((1.f + e) * (1.f + e));
        const float *rs = rT + s * NL;
        float cs = 0.f;
#pragma unroll
        for (int l = 0; l < NL; ++l) cs = fmaf(Ln[l], rs[l], cs);
        acc = fmaf(w, cs, acc);
    }
    dphi[n] = scale * acc;
}

template <int NL>
static cudaError_t launch_bwd_n(unsigned blocks, int nb, size_t smem, cudaStream_t st, int64_t n_v, int T,
                                const float *L, const float *phi, const float *r, float t0, float dt, float tau,
                                float scale, float *dphi, int64_t phi_stride)
{
    cudaFuncSetAttribute(k_ecg_bwd_t<NL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_ecg_bwd_t<NL><<<dim3(blocks, nb), 256, smem, st>>>(n_v, T, L, phi, r, t0, dt, tau, scale, dphi, phi_stride);
    return cudaGetLastError();
}

// nb problems: phi, dphi [b] at + b * phi_stride; ecg, target [nb][N][T]; loss [nb]
cudaError_t launch_ecg_backward_batch(gbp_ctx *c, int nb, const float *phi, int64_t phi_stride, const float *ecg,
                                      const float *target, const gbp_template *t, float *loss, float *dphi)
{
    const int N = c->N, T = t->T;
    int64_t NT = (int64_t)N * T;
    if (NT * nb > c->resid_cap) {
        if (c->resid) cudaFree(c->resid);
        cudaError_t err = cudaMalloc(&c->resid, sizeof(float) * NT * nb);
        if (err) {
            c->resid = nullptr;
            c->resid_cap = 0;
            return err;
        }
        c->resid_cap = NT * nb;
    }
    time_begin(c, 3);
    k_ecg_resid<<<nb, 1024, 0, c->stream>>>((int)NT, ecg, target, c->resid, 1.f / (float)NT, loss);
    size_t smem = sizeof(float) * NT;  // N * T <= 16 * 4096 floats = 256 KB at most
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    float scale = -2.f / (float)NT * (t->K1 - t->K0) * (4.f / t->tau);
    const unsigned blocks = (unsigned)((c->n_e + 255) / 256);
    cudaError_t le = cudaErrorInvalidValue;
    switch (N) {
#define GBP_BWD_CASE(n) \
    case n: le = launch_bwd_n<n>(blocks, nb, smem, c->stream, c->n_e, T, c->L, phi, c->resid, t->t0, t->dt, \
                                 t->tau, scale, dphi, phi_stride); break;
        GBP_BWD_CASE(1) GBP_BWD_CASE(2) GBP_BWD_CASE(3) GBP_BWD_CASE(4) GBP_BWD_CASE(5) GBP_BWD_CASE(6)
        GBP_BWD_CASE(7) GBP_BWD_CASE(8) GBP_BWD_CASE(9) GBP_BWD_CASE(10) GBP_BWD_CASE(11) GBP_BWD_CASE(12)
        GBP_BWD_CASE(13) GBP_BWD_CASE(14) GBP_BWD_CASE(15) GBP_BWD_CASE(16)
#undef GBP_BWD_CASE
    }
    if (le) return le;
    time_end(c, 3);
    c->launches += 2;
    return cudaGetLastError();
}

cudaError_t launch_ecg_backward(gbp_ctx *c, const float *phi, const float *ecg, const float *target,
                                const gbp_template *t, float *loss, float *dphi)
{
    return launch_ecg_backward_batch(c, 1, phi, 0, ecg, target, t, loss, dphi);
}

// dispatcher (the BF16 tensor-core path lives in ecg_bf16.cu)
cudaError_t launch_ecg_forward_bf16(gbp_ctx *c, const float *phi, const gbp_template *t, float *ecg);

cudaError_t launch_ecg_forward(gbp_ctx *c, const float *phi, const gbp_template *t, int prec, float *ecg)
{
    if (prec == GBP_PREC_BF16) return launch_ecg_forward_bf16(c, phi, t, ecg);
    return launch_ecg_forward_fp32(c, phi, t, ecg);
}

}  // namespace gbp
