// noalloc.cu -- an ECG forward pass for callers that must not allocate.
//
// Some callers cannot call cudaMalloc: code running under a fixed device
// memory budget, code inside a framework whose caching allocator owns the
// device heap (a direct cudaMalloc is invisible to it and cudaFree
// synchronises the whole device), or latency-critical loops that must never
// block on the allocator.  gbp_ecg_forward_noalloc serves them: it needs no
// context and allocates nothing.  Its scratch memory (the split-K partial
// sums and the lead-field row sums) is the file-scope device array below,
// which every GPU that loads the library holds until the process exits.
#include <mutex>

#include "gbp_internal.cuh"

namespace gbp {
// kernels shared with the context-based path (ecg.cu)
const void *ecg_fwd_kernel(int N);
__global__ void k_ecg_reduce(int N, int T, int ncta, const double *__restrict__ part, const float *__restrict__ rowsum,
                             float K0, float dK, float *__restrict__ ecg);
size_t ecg_fwd_smem(int N, int T_tile, int G);
}  // namespace gbp

namespace {

// 4 MiB of scratch per device: 16 row sums, then the FP64 partial sums.
constexpr int64_t NOALLOC_SCRATCH_FLOATS = (int64_t)1 << 20;
static __device__ __align__(256) float g_noalloc_scratch[NOALLOC_SCRATCH_FLOATS];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
float *g_scratch_ptr[MAX_DEVICES] = {nullptr};
int g_num_sms[MAX_DEVICES] = {0};

// Host code cannot use the array's name as a device address; look the
// address up once per device, with that device current.
cudaError_t scratch_for_device(int dev, float **ptr, int *sms)
{
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        float *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress((void **)&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        int n = 0;
        e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = p;
        g_num_sms[dev] = n;
    }
    *ptr = g_scratch_ptr[dev];
    *sms = g_num_sms[dev];
    return cudaSuccess;
}

__global__ void k_rowsum_noalloc(int64_t n_v, const float *__restrict__ L, float *__restrict__ rowsum)
{
    __shared__ double red[32];
    const float *Ll = L + (int64_t)blockIdx.x * n_v;
    double acc = 0.0;
    for (int64_t n = threadIdx.x; n < n_v; n += blockDim.x) acc += (double)Ll[n];
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (threadIdx.x == 0) rowsum[blockIdx.x] = (float)v;
    }
}

}  // namespace

// Every launch goes through cudaLaunchKernel, whose return value is that
// launch's own status: an error left pending by unrelated earlier work on the
// calling thread is neither reported here nor cleared.
extern "C" gbp_status gbp_ecg_forward_noalloc(const float *L, int32_t N, int64_t n_v, const float *phi,
                                             const gbp_template *tmpl, float *ecg, void *stream)
{
    if (!L || !phi || !ecg || !tmpl || N < 1 || N > 16 || n_v < 1) return GBP_ERR_INVALID_ARG;
    if (tmpl->T < 1 || tmpl->T > 4096 || !(tmpl->tau > 0.f) || !(tmpl->dt > 0.f)) return GBP_ERR_INVALID_ARG;
    const int T = tmpl->T;
    const int64_t per_cta_floats = 2 * (int64_t)N * T;  // FP64 partials
    // the scratch must hold the row sums and at least one CTA's partials
    if (16 + per_cta_floats > NOALLOC_SCRATCH_FLOATS) return GBP_ERR_INVALID_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return GBP_ERR_CUDA;
    float *scratch = nullptr;
    int sms = 0;
    if (scratch_for_device(dev, &scratch, &sms) != cudaSuccess) return GBP_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    float *rowsum = scratch;
    double *part = reinterpret_cast<double *>(scratch + 16);  // 64-byte offset: 8-byte aligned
    // same launch shape as the context path, with the CTA count capped by
    // the scratch size
    int tt = ((T + 31) / 32) * 32;
    if (tt > 512) tt = 512;
    int G = 512 / tt;
    if (G < 1) G = 1;
    int64_t ncta = 2 * (int64_t)sms;
    const int64_t cap_cta = (NOALLOC_SCRATCH_FLOATS - 16) / per_cta_floats;
    if (ncta > cap_cta) ncta = cap_cta;
    const int CH = 256;
    int64_t per = (n_v + ncta - 1) / ncta;
    per = ((per + CH - 1) / CH) * CH;
    ncta = (n_v + per - 1) / per;
    // every partial and row sum is overwritten below, so nothing is cleared
    {
        int64_t nv = n_v;
        const float *Lp = L;
        float *rs = rowsum;
        void *args[] = {&nv, &Lp, &rs};
        if (cudaLaunchKernel((const void *)k_rowsum_noalloc, dim3(N), dim3(256), args, 0, st) != cudaSuccess)
            return GBP_ERR_CUDA;
    }
    {
        const void *fn = gbp::ecg_fwd_kernel(N);
        const size_t smem = gbp::ecg_fwd_smem(N, tt, G);
        if (!fn || cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return GBP_ERR_CUDA;
        int64_t nv = n_v, phi_stride = 0, part_stride = 0;
        int TT = T, T_tile = tt, GG = G;
        float t0 = tmpl->t0, dt = tmpl->dt, c4 = 4.f / tmpl->tau;
        const float *Lp = L, *ph = phi;
        double *pp = part;
        // k_ecg_fwd_t<N>(n_v, T, L, phi, t0, dt, c4, T_tile, G, per_cta, part, phi_stride, part_stride)
        void *args[] = {&nv, &TT, &Lp, &ph, &t0, &dt, &c4, &T_tile, &GG, &per, &pp, &phi_stride, &part_stride};
        if (cudaLaunchKernel(fn, dim3((unsigned)ncta, 1), dim3(tt * G), args, smem, st) != cudaSuccess)
            return GBP_ERR_CUDA;
    }
    {
        int NN = N, TT = T, nc = (int)ncta;
        const double *pp = part;
        const float *rs = rowsum;
        float K0 = tmpl->K0, dK = tmpl->K1 - tmpl->K0;
        float *out = ecg;
        void *args[] = {&NN, &TT, &nc, &pp, &rs, &K0, &dK, &out};
        if (cudaLaunchKernel((const void *)gbp::k_ecg_reduce, dim3((N * T + 255) / 256), dim3(256), args, 0, st) !=
            cudaSuccess)
            return GBP_ERR_CUDA;
    }
    return GBP_OK;
}
