// ecg_bf16.cu -- lead-field ECG contraction on the 5th-generation tensor
// cores (tcgen05, accumulator in tensor memory), BF16 operands with FP32
// accumulation.
//
//   V_l(t_s) = K0 S_l + (K1 - K0) scale_l sum_n Bbf_ln sigma_bf(4 (t_s - phi_n)/tau)
//
// (Sec. II-D with the template of Eq. (tanh_waveform) in logistic form, see
// ecg.cu).  The constant part K0 S_l uses the FP32 row sums of B; only the
// activation part is quantised: sigma in [0, 1] to BF16 and each lead row of
// B scaled by its max |B_ln| before rounding to BF16.
//
// GEMM view: D[s][l] = sum_n A[s][n] Bt[l][n], M = 128 samples per tile,
// N = 16 leads (zero-padded), K = vertices (split across CTAs, partial sums
// reduced deterministically afterwards).  A (the template tile) is computed
// by the CTA's threads straight into shared memory in the no-swizzle K-major
// canonical layout; the B tile is copied there from the BF16 lead field.
// One thread issues tcgen05.mma (kind::f16, 128x16x16) per 16 vertices;
// tcgen05.commit on an mbarrier releases the stage; the accumulator is read
// back with tcgen05.ld.  Two pipeline stages overlap template generation with
// the tensor-core work.  Every wait is bounded; on a timeout the kernel
// records GBP_ERR_TIMEOUT, frees its tensor memory and returns.
#include "gbp_internal.cuh"

namespace gbp {

#ifndef GBP_BF16_CTAS_PER_SM
#define GBP_BF16_CTAS_PER_SM 6  // CTAs per SM of the split-K grid (128 threads, 36 KB of stages each)
#endif
constexpr int BF_M = 128;   // samples per tile (MMA M)
constexpr int BF_N = 16;    // leads (MMA N)
constexpr int BF_KT = 64;   // vertices per pipeline stage
// no-swizzle K-major canonical layout: 8-row x 16-byte core matrices stored
// as 128 contiguous bytes; element (r, k) at (r/8)*SBO + (k/8)*LBO + (r%8)*16 + (k%8)*2
constexpr uint32_t BF_LBO = 128;
constexpr uint32_t BF_SBO = (BF_KT / 8) * 128;
constexpr int A_BYTES = BF_M * BF_KT * 2;
constexpr int B_BYTES = BF_N * BF_KT * 2;
constexpr uint32_t TMEM_COLS = 32;

// tcgen05 shared-memory matrix descriptor (start, LBO, SBO in 16-byte units,
// descriptor version 1 at bit 46, base offset 0, no swizzle)
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((BF_LBO >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((BF_SBO >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor, kind::f16: D F32 (bits 4-5 = 1), A BF16 (bits 7-9 = 1),
// B BF16 (bits 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at bit 24
constexpr uint32_t BF_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BF_N >> 3) << 17) |
                              ((uint32_t)(BF_M >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity)
{
    for (uint32_t i = 0; i < (1u << 20); ++i) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}

__global__ void __launch_bounds__(128) k_ecg_bf16(int64_t n_v, int64_t n_pad, int N, int T,
                                                  const __nv_bfloat16 *__restrict__ Lbf,
                                                  const float *__restrict__ phi, float t0, float dt, float c4,
                                                  int64_t per_split, float *__restrict__ part, Control *ctl)
{
    __shared__ __align__(1024) uint8_t sA[2][A_BYTES];
    __shared__ __align__(1024) uint8_t sB[2][B_BYTES];
    __shared__ float sphi[2][BF_KT];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t s_tmem;

    const int tid = threadIdx.x, warp = tid >> 5;
    const int split = blockIdx.x, mt = blockIdx.y;
    const int s = mt * BF_M + tid;  // the sample (MMA row) this thread generates and reads back
    const float ts = fmaf((float)s, dt, t0);
    const int64_t n0 = (int64_t)split * per_split;
    const int64_t n1 = min(n0 + per_split, n_v);
    const int steps = n1 > n0 ? (int)((n1 - n0 + BF_KT - 1) / BF_KT) : 0;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;

    bool ok = true;
    for (int it = 0; it < steps; ++it) {
        const int st = it & 1;
        if (it >= 2) ok = mbar_wait(smem_u32(&mbar[st]), (uint32_t)(((it >> 1) - 1) & 1));
        const int64_t nb = n0 + (int64_t)it * BF_KT;
        if (tid < BF_KT) sphi[st][tid] = nb + tid < n1 ? phi[nb + tid] : GBP_INF;
        {
            // B tile: lead row l, 8-vertex chunk c (rows past N and vertices
            // past n_v are zero in the padded BF16 copy)
            const int l = tid >> 3, c = tid & 7;
            const uint4 v = __ldg(reinterpret_cast<const uint4 *>(Lbf + (int64_t)l * n_pad + nb + 8 * c));
            *reinterpret_cast<uint4 *>(&sB[st][(l >> 3) * BF_SBO + c * BF_LBO + (l & 7) * 16]) = v;
        }
        if (!__syncthreads_and(ok)) {
            ok = false;
            break;
        }
        // A tile: row = this thread's sample, 64 vertices in 8 chunks
#pragma unroll
        for (int c = 0; c < BF_KT / 8; ++c) {
            float v[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) v[e] = __fdividef(1.f, 1.f + __expf(-(ts - sphi[st][8 * c + e]) * c4));
            uint4 q = make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]),
                                 pack_bf16(v[6], v[7]));
            *reinterpret_cast<uint4 *>(&sA[st][(tid >> 3) * BF_SBO + c * BF_LBO + (tid & 7) * 16]) = q;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_u32(&sA[st][0]), b0 = smem_u32(&sB[st][0]);
#pragma unroll
            for (int kk = 0; kk < BF_KT / 16; ++kk) {
                // K = 16 per instruction = two core matrices along K
                const uint64_t ad = smem_desc(a0 + kk * 2 * BF_LBO);
                const uint64_t bd = smem_desc(b0 + kk * 2 * BF_LBO);
                const uint32_t acc = (it > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(BF_IDESC), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&mbar[st]))
                         : "memory");
        }
    }
    if (ok && steps > 0) ok = mbar_wait(smem_u32(&mbar[(steps - 1) & 1]), (uint32_t)(((steps - 1) >> 1) & 1));
    ok = __syncthreads_and(ok);
    if (ok) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        uint32_t r[16];
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
              "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(taddr)
            : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (s < T) {
#pragma unroll
            for (int l = 0; l < BF_N; ++l)
                if (l < N) part[((int64_t)split * BF_N + l) * T + s] = steps > 0 ? __uint_as_float(r[l]) : 0.f;
        }
    } else {
        if (tid == 0) atomicCAS(&ctl->status, 0, (int)GBP_ERR_TIMEOUT);
        // give any MMA still in flight a second bounded chance to finish
        // before the tensor memory is released
        if (steps > 0) mbar_wait(smem_u32(&mbar[(steps - 1) & 1]), (uint32_t)(((steps - 1) >> 1) & 1));
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
    }
}

// per-lead scale = max_n |B_ln| (block per lead)
__global__ void k_lead_scale(int64_t n_v, const float *__restrict__ L, float *__restrict__ scale)
{
    __shared__ float red[32];
    const float *Ll = L + (int64_t)blockIdx.x * n_v;
    float m = 0.f;
    for (int64_t n = threadIdx.x; n < n_v; n += blockDim.x) m = fmaxf(m, fabsf(Ll[n]));
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
        for (int off = 16; off > 0; off >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, off));
        if (threadIdx.x == 0) scale[blockIdx.x] = v > 0.f ? v : 1.f;
    }
}

__global__ void k_lead_bf16(int64_t n_v, int64_t n_pad, int N, const float *__restrict__ L,
                            const float *__restrict__ scale, __nv_bfloat16 *__restrict__ Lbf)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)BF_N * n_pad) return;
    int l = (int)(e / n_pad);
    int64_t n = e - (int64_t)l * n_pad;
    float v = (l < N && n < n_v) ? L[(int64_t)l * n_v + n] / scale[l] : 0.f;
    Lbf[e] = __float2bfloat16_rn(v);
}

cudaError_t prepare_leadfield_bf16(gbp_ctx *c)
{
    const int64_t n_pad = ((c->n_e + BF_KT - 1) / BF_KT) * BF_KT;
    cudaError_t e = cudaSuccess;
    if (c->Lbf) cudaFree(c->Lbf);
    c->Lbf = nullptr;
    e = cudaMalloc(&c->Lbf, sizeof(__nv_bfloat16) * BF_N * n_pad);
    if (!e && !c->Lscale) e = cudaMalloc(&c->Lscale, sizeof(float) * BF_N);
    if (e) return e;
    c->n_v_pad = n_pad;
    k_lead_scale<<<c->N, 256, 0, c->stream>>>(c->n_e, c->L, c->Lscale);
    int64_t tot = (int64_t)BF_N * n_pad;
    k_lead_bf16<<<(unsigned)((tot + 255) / 256), 256, 0, c->stream>>>(c->n_e, n_pad, c->N, c->L, c->Lscale,
                                                                      c->Lbf);
    c->launches += 2;
    return cudaGetLastError();
}

// V[l][s] = K0 S_l + (K1 - K0) scale_l sum_split part[split][l][s]
__global__ void k_ecg_reduce_bf16(int N, int T, int nsplit, const float *__restrict__ part,
                                  const float *__restrict__ rowsum, const float *__restrict__ scale, float K0,
                                  float dK, float *__restrict__ ecg)
{
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N * T) return;
    int l = e / T, s = e - l * T;
    float v = 0.f;
    for (int c = 0; c < nsplit; ++c) v += part[((int64_t)c * BF_N + l) * T + s];
    ecg[e] = fmaf(K0, rowsum[l], dK * scale[l] * v);
}

cudaError_t launch_ecg_forward_bf16(gbp_ctx *c, const float *phi, const gbp_template *t, float *ecg)
{
    const int N = c->N, T = t->T;
    const int mtiles = (T + BF_M - 1) / BF_M;
    int nsplit = (GBP_BF16_CTAS_PER_SM * c->num_sms + mtiles - 1) / mtiles;
    int64_t per = (c->n_e + nsplit - 1) / nsplit;
    per = ((per + BF_KT - 1) / BF_KT) * BF_KT;
    nsplit = (int)((c->n_e + per - 1) / per);
    int64_t need = (int64_t)nsplit * BF_N * T;
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
    time_begin(c, 2);
    k_ecg_bf16<<<dim3(nsplit, mtiles), 128, 0, c->stream>>>(c->n_e, c->n_v_pad, N, T, c->Lbf, phi, t->t0, t->dt,
                                                            4.f / t->tau, per, c->ecg_part, c->ctl);
    k_ecg_reduce_bf16<<<(N * T + 255) / 256, 256, 0, c->stream>>>(N, T, nsplit, c->ecg_part, c->Lrowsum, c->Lscale,
                                                                 t->K0, t->K1 - t->K0, ecg);
    time_end(c, 2);
    c->launches += 2;
    return cudaGetLastError();
}

}  // namespace gbp
