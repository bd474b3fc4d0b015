// nn.cu -- training and inference kernels of the learned initialiser: a small
// 1-D convolutional network + MLP that maps an ECG to initial onset sites,
// times and velocities.  Every layer is a BF16 tensor-core GEMM
// (tcgen05.mma, FP32 accumulator in tensor memory) around small elementwise
// kernels; weights are kept as FP32 masters updated by Adam and cast to BF16
// for the GEMMs.
//
// Layouts: activations are channels-last f32 [batch][length][channels];
// convolution weights are [C_out][ksize][C_in] (tap-major), so im2col rows
// are contiguous C_in-chunks.  GEMM operands are BF16 with the reduction
// dimension contiguous and padded with zeros to a multiple of 64.
#include <cuda.h>  // CUtensorMap and its encoder's types (the encoder is found at run time)

#include "gbp_internal.cuh"

namespace gbp {
namespace nn {

constexpr int GM = 128;  // rows of C per CTA (MMA M)
constexpr int GN = 64;   // columns of C per CTA (MMA N)
constexpr int GK = 64;   // reduction step per pipeline stage
// no-swizzle K-major canonical layout, 8-row x 16-byte core matrices
constexpr uint32_t G_LBO = 128;
constexpr uint32_t G_SBO = (GK / 8) * 128;
constexpr int GA_BYTES = GM * GK * 2;
constexpr int GB_BYTES = GN * GK * 2;
constexpr uint32_t G_TMEM_COLS = 64;
constexpr uint32_t G_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(GN >> 3) << 17) |
                             ((uint32_t)(GM >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t g_desc(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((G_LBO >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((G_SBO >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

__device__ __forceinline__ bool g_mbar_wait(uint32_t addr, uint32_t parity)
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

// C[m][n] = alpha * sum_k A[m][k] B[n][k] + beta * C[m][n]
// A bf16 [M][lda], B bf16 [N][ldb] (k contiguous, zero padded to Kp), C f32 [M][ldc].
// grid (ceil(M/128), ceil(N/64)), 128 threads; thread t owns row t of the tile.
__global__ void __launch_bounds__(128) k_gemm_tn(int M, int N, int Kp, const __nv_bfloat16 *__restrict__ A, int lda,
                                                 const __nv_bfloat16 *__restrict__ B, int ldb, float *__restrict__ C,
                                                 int ldc, float alpha, float beta, Control *ctl)
{
    // operand tiles in dynamic shared memory (the no-swizzle layout needs
    // 16-byte alignment only)
    extern __shared__ __align__(128) uint8_t g_smem[];
    uint8_t(*sA)[GA_BYTES] = reinterpret_cast<uint8_t(*)[GA_BYTES]>(g_smem);
    uint8_t(*sB)[GB_BYTES] = reinterpret_cast<uint8_t(*)[GB_BYTES]>(g_smem + 2 * GA_BYTES);
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t s_tmem;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int m0 = blockIdx.x * GM, n0 = blockIdx.y * GN;
    const int steps = Kp / GK;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(G_TMEM_COLS)
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
        if (it >= 2) ok = g_mbar_wait(smem_u32(&mbar[st]), (uint32_t)(((it >> 1) - 1) & 1));
        const int k0 = it * GK;
        // A tile: thread t copies row m0 + t (8 chunks of 8 bf16)
        {
            const int m = m0 + tid;
#pragma unroll
            for (int c = 0; c < GK / 8; ++c) {
                uint4 v = make_uint4(0u, 0u, 0u, 0u);
                if (m < M) v = __ldg(reinterpret_cast<const uint4 *>(A + (int64_t)m * lda + k0 + 8 * c));
                *reinterpret_cast<uint4 *>(&sA[st][(tid >> 3) * G_SBO + c * G_LBO + (tid & 7) * 16]) = v;
            }
        }
        // B tile: 64 rows x 8 chunks, 4 chunks per thread
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + 128 * q;  // 0..511
            const int r = e >> 3, c = e & 7;
            const int n = n0 + r;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (n < N) v = __ldg(reinterpret_cast<const uint4 *>(B + (int64_t)n * ldb + k0 + 8 * c));
            *reinterpret_cast<uint4 *>(&sB[st][(r >> 3) * G_SBO + c * G_LBO + (r & 7) * 16]) = v;
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (!__syncthreads_and(ok)) {
            ok = false;
            break;
        }
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a0 = smem_u32(&sA[st][0]), b0 = smem_u32(&sB[st][0]);
#pragma unroll
            for (int kk = 0; kk < GK / 16; ++kk) {
                const uint64_t ad = g_desc(a0 + kk * 2 * G_LBO);
                const uint64_t bd = g_desc(b0 + kk * 2 * G_LBO);
                const uint32_t acc = (it > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(G_IDESC), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&mbar[st]))
                         : "memory");
        }
    }
    if (ok && steps > 0) ok = g_mbar_wait(smem_u32(&mbar[(steps - 1) & 1]), (uint32_t)(((steps - 1) >> 1) & 1));
    ok = __syncthreads_and(ok);
    const int m = m0 + tid;
    if (ok) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            uint32_t r[32];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(32 * half);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                  "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                  "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                : "r"(taddr)
                : "memory");
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (m < M) {
#pragma unroll
                for (int q = 0; q < 32; ++q) {
                    const int n = n0 + 32 * half + q;
                    if (n < N) {
                        float v = alpha * (steps > 0 ? __uint_as_float(r[q]) : 0.f);
                        float *cp = C + (int64_t)m * ldc + n;
                        *cp = beta != 0.f ? fmaf(beta, *cp, v) : v;
                    }
                }
            }
        }
    } else {
        if (tid == 0) atomicCAS(&ctl->status, 0, (int)GBP_ERR_TIMEOUT);
        if (steps > 0) g_mbar_wait(smem_u32(&mbar[(steps - 1) & 1]), (uint32_t)(((steps - 1) >> 1) & 1));
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(G_TMEM_COLS)
                     : "memory");
    }
}

// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// The same product for shapes that fill 128 x 256 tiles exactly (M % 128 ==
// 0, N % 256 == 0), fed by the tensor memory accelerator: A and B tiles of 64
// K-columns land in shared memory by cp.async.bulk.tensor in the 128-byte
// swizzled K-major layout (8-row atoms of 1024 bytes), four stages deep, each
// stage's mbarrier counting the copies' bytes; tcgen05.mma with M = 128,
// N = 256, K = 16 per instruction and an FP32 accumulator in TMEM.
constexpr int TM = 128, TN = 256, TK = 64, TS = 4;
constexpr int TA_BYTES = TM * TK * 2;  // 16 KB
constexpr int TB_BYTES = TN * TK * 2;  // 32 KB
constexpr int T_STAGE = TA_BYTES + TB_BYTES;
constexpr int T_SMEM = TS * T_STAGE + 1024;  // + slack to align the tiles to 1024 bytes
constexpr uint32_t T_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) |
                             ((uint32_t)(TM >> 4) << 24);

// K-major, 128-byte swizzle: rows of 128 bytes, 8-row groups 1024 bytes apart
// (stride-dimension offset); the leading-dimension offset is not used when a
// row holds the whole K-step of one instruction
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t mbar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
            "r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(mbar)
        : "memory");
}

// One CTA per SM walks the tiles (t = blockIdx.x, + gridDim.x, ...;
// consecutive tiles share their B tile) with two 256-column accumulators in
// TMEM, so that a tile's epilogue overlaps the next tile's MMAs and the
// set-up is paid once per CTA.  Warp 0 (one lane) streams the copies through
// the four stages across tile boundaries, warp 1 (one lane) issues the MMAs
// into accumulator i & 1 and commits it to "acc full", warps 2-5 (TMEM lane
// quadrants 2, 3, 0, 1) read it, write C and release it on "acc empty"; the
// other lanes of warps 0 and 1 wait at __syncwarp (lanes of one warp that
// poll an mbarrier hold the warp in each try_wait window: with them polling,
// a first version ran at a quarter of this speed).  Every wait is bounded: a
// wait that runs out latches GBP_ERR_TIMEOUT, the copies in flight and the
// MMAs issued are waited for and TMEM is freed before the CTA leaves.
constexpr uint32_t TP_TMEM_COLS = 512;

__global__ void __launch_bounds__(192, 1) k_gemm_tma(int M, int N, int Kp, const __grid_constant__ CUtensorMap tA,
                                                   const __grid_constant__ CUtensorMap tB, float *__restrict__ C,
                                                   int ldc, float alpha, float beta, Control *ctl)
{
    extern __shared__ __align__(1024) uint8_t t_smem[];
    __shared__ __align__(8) uint64_t full[TS], empty[TS], accf[2], acce[2], done;
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tiles_m = M / TM, ntiles = tiles_m * (N / TN);
    const int steps = Kp / TK;
    const uint32_t base = (smem_u32(t_smem) + 1023u) & ~1023u;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(TP_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
    if (tid == 0) {
        for (int st = 0; st < TS; ++st) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[st])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[st])) : "memory");
        }
        for (int b = 0; b < 2; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&accf[b])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(smem_u32(&acce[b])) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&done)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_fail = 0;
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;
    int issued = 0;  // producer: stages issued (over all tiles)
    if (warp == 0) {
        if (lane == 0) {
            int g = 0;
            bool bad = false;
            for (int t = blockIdx.x; t < ntiles && !bad; t += gridDim.x) {
                const int m0 = (t % tiles_m) * TM, n0 = (t / tiles_m) * TN;
                for (int it = 0; it < steps; ++it, ++g) {
                    const int st = g % TS;
                    if (g >= TS && !g_mbar_wait(smem_u32(&empty[st]), (uint32_t)(((g / TS) & 1) ^ 1))) {
                        bad = true;
                        break;
                    }
                    const uint32_t fb = smem_u32(&full[st]);
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(T_STAGE)
                                 : "memory");
                    const uint32_t sa = base + (uint32_t)(st * T_STAGE);
                    tma_load_2d(sa, &tA, it * TK, m0, fb);
                    tma_load_2d(sa + TA_BYTES, &tB, it * TK, n0, fb);
                    issued = g + 1;
                }
            }
            if (bad) s_fail = 1;
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0) {
            int g = 0, i = 0;
            bool bad = false;
            for (int t = blockIdx.x; t < ntiles && !bad; t += gridDim.x, ++i) {
                const int buf = i & 1;
                if (i >= 2 && !g_mbar_wait(smem_u32(&acce[buf]), (uint32_t)(((i >> 1) - 1) & 1))) {
                    bad = true;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t acc = tmem + (uint32_t)(buf * 256);
                for (int it = 0; it < steps; ++it, ++g) {
                    const int st = g % TS;
                    if (!g_mbar_wait(smem_u32(&full[st]), (uint32_t)((g / TS) & 1))) {
                        bad = true;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t sa = base + (uint32_t)(st * T_STAGE);
#pragma unroll
                    for (int kk = 0; kk < TK / 16; ++kk) {
                        const uint64_t ad = sw128_desc(sa + 32u * kk);
                        const uint64_t bd = sw128_desc(sa + TA_BYTES + 32u * kk);
                        const uint32_t en = (it > 0 || kk > 0) ? 1u : 0u;
                        asm volatile(
                            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(acc),
                            "l"(ad), "l"(bd), "r"(T_IDESC), "r"(en)
                            : "memory");
                    }
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     smem_u32(&empty[st]))
                                 : "memory");
                }
                if (bad) break;
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(&accf[buf]))
                             : "memory");
            }
            if (bad) s_fail = 1;
            // every MMA issued completes before this arrives
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&done))
                         : "memory");
        }
        __syncwarp();
    } else {
        // epilogue: TMEM lanes 32 q .. 32 q + 31 (rows of the tile)
        const int q = warp & 3;
        int i = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
            const int buf = i & 1;
            if (!g_mbar_wait(smem_u32(&accf[buf]), (uint32_t)((i >> 1) & 1))) {
                if (lane == 0) s_fail = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int m = (t % tiles_m) * TM + q * 32 + lane, n0 = (t / tiles_m) * TN;
            float *crow = C + (int64_t)m * ldc + n0;
#pragma unroll 1
            for (int ch = 0; ch < TN / 32; ++ch) {
                uint32_t r[32];
                const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * 256 + 32 * ch);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                    "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                    : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                      "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                      "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
                      "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
                      "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                    : "r"(taddr)
                    : "memory");
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                float4 *cp = reinterpret_cast<float4 *>(crow + 32 * ch);
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    float4 v = make_float4(alpha * __uint_as_float(r[4 * e]), alpha * __uint_as_float(r[4 * e + 1]),
                                           alpha * __uint_as_float(r[4 * e + 2]),
                                           alpha * __uint_as_float(r[4 * e + 3]));
                    if (beta != 0.f) {
                        const float4 o = cp[e];
                        v.x = fmaf(beta, o.x, v.x);
                        v.y = fmaf(beta, o.y, v.y);
                        v.z = fmaf(beta, o.z, v.z);
                        v.w = fmaf(beta, o.w, v.w);
                    }
                    cp[e] = v;
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acce[buf])) : "memory");
        }
    }
    __syncthreads();
    if (s_fail && tid == 0) {
        atomicCAS(&ctl->status, 0, (int)GBP_ERR_TIMEOUT);
        // the copies still in flight land before the CTA's shared memory goes
        for (int g = max(0, issued - TS); g < issued; ++g)
            g_mbar_wait(smem_u32(&full[g % TS]), (uint32_t)((g / TS) & 1));
    }
    if (tid == 32) g_mbar_wait(smem_u32(&done), 0u);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TP_TMEM_COLS)
                     : "memory");
    }
}

// im2col of a channels-last activation for a 1-D convolution:
// col[b*Lo + l][k*Ci + c] = act[b][s*l + k - pad][c] (0 outside), bf16, row stride ldc (>= ks*Ci, zero padded)
__global__ void k_im2col(int Bn, int Li, int Ci, int Lo, int ks, int stride, int pad, const float *__restrict__ act,
                         __nv_bfloat16 *__restrict__ col, int ldc)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t tot = (int64_t)Bn * Lo * ldc;
    if (e >= tot) return;
    const int64_t row = e / ldc;
    const int kk = (int)(e - row * ldc);
    float v = 0.f;
    if (kk < ks * Ci) {
        const int k = kk / Ci, c = kk - k * Ci;
        const int b = (int)(row / Lo), l = (int)(row - (int64_t)b * Lo);
        const int j = stride * l + k - pad;
        if (j >= 0 && j < Li) v = act[((int64_t)b * Li + j) * Ci + c];
    }
    col[e] = __float2bfloat16_rn(v);
}

// transposed im2col: colT[k*Ci + c][b*Lo + l] (rows padded to Kp, row stride ldt >= B*Lo, zeros outside)
__global__ void k_im2col_t(int Bn, int Li, int Ci, int Lo, int ks, int stride, int pad, const float *__restrict__ act,
                           int Kp, __nv_bfloat16 *__restrict__ colT, int ldt)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t tot = (int64_t)Kp * ldt;
    if (e >= tot) return;
    const int kk = (int)(e / ldt);
    const int64_t row = e - (int64_t)kk * ldt;
    float v = 0.f;
    if (kk < ks * Ci && row < (int64_t)Bn * Lo) {
        const int k = kk / Ci, c = kk - k * Ci;
        const int b = (int)(row / Lo), l = (int)(row - (int64_t)b * Lo);
        const int j = stride * l + k - pad;
        if (j >= 0 && j < Li) v = act[((int64_t)b * Li + j) * Ci + c];
    }
    colT[e] = __float2bfloat16_rn(v);
}

// adjoint of im2col: dact[b][j][c] = sum over (k, l) with s*l + k - pad = j of dcol[b*Lo + l][k*Ci + c]
__global__ void k_col2im(int Bn, int Li, int Ci, int Lo, int ks, int stride, int pad, const float *__restrict__ dcol,
                         int ldc, float *__restrict__ dact)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t tot = (int64_t)Bn * Li * Ci;
    if (e >= tot) return;
    const int c = (int)(e % Ci);
    const int64_t bj = e / Ci;
    const int j = (int)(bj % Li), b = (int)(bj / Li);
    float acc = 0.f;
    for (int k = 0; k < ks; ++k) {
        const int t = j + pad - k;
        if (t < 0 || t % stride) continue;
        const int l = t / stride;
        if (l >= Lo) continue;
        acc += dcol[((int64_t)b * Lo + l) * ldc + k * Ci + c];
    }
    dact[e] = acc;
}

// y = act(z + bias) in place over rows of length N (row stride ld); pre keeps z + bias
__global__ void k_bias_act(int M, int N, float *__restrict__ y, int ld, const float *__restrict__ bias,
                           float *__restrict__ pre, int gelu)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)M * N) return;
    const int64_t m = e / N;
    const int n = (int)(e - m * N);
    float z = y[m * ld + n] + bias[n];
    if (pre) pre[e] = z;
    if (gelu) z = 0.5f * z * (1.f + erff(z * 0.70710678118654752f));
    y[m * ld + n] = z;
}

// d z = d y * GELU'(pre), GELU'(z) = Phi(z) + z phi(z)
__global__ void k_gelu_bwd(int M, int N, float *__restrict__ dy, int ld, const float *__restrict__ pre)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)M * N) return;
    const int64_t m = e / N;
    const int n = (int)(e - m * N);
    const float z = pre[e];
    const float d = 0.5f * (1.f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
    dy[m * ld + n] *= d;
}

// db[n] = sum_m dz[m][n]
__global__ void k_bias_grad(int M, int N, const float *__restrict__ dz, int ld, float *__restrict__ db)
{
    const int n = blockIdx.x;
    float acc = 0.f;
    for (int m = threadIdx.x; m < M; m += blockDim.x) acc += dz[(int64_t)m * ld + n];
    __shared__ float red[32];
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (threadIdx.x == 0) db[n] = v;
    }
}

// dst[r][c] = bf16(src[r][c]) for c < cols, zero for cols <= c < ldd
__global__ void k_cast_bf16(int rows, int cols, const float *__restrict__ src, int lds, __nv_bfloat16 *__restrict__ dst,
                            int ldd)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)rows * ldd) return;
    const int64_t r = e / ldd;
    const int c = (int)(e - r * ldd);
    dst[e] = __float2bfloat16_rn(c < cols ? src[r * lds + c] : 0.f);
}

// dst[c][r] = bf16(src[r][c]) for r < rows, zero for rows <= r < ldd  (dst has cols rows)
__global__ void k_transpose_bf16(int rows, int cols, const float *__restrict__ src, int lds,
                                 __nv_bfloat16 *__restrict__ dst, int ldd)
{
    __shared__ float tile[32][33];
    const int bx = blockIdx.x * 32, by = blockIdx.y * 32;  // bx over r (ldd), by over c
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int r = bx + threadIdx.x, c = by + i;
        tile[i][threadIdx.x] = (r < rows && c < cols) ? src[(int64_t)r * lds + c] : 0.f;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int c = by + i, r = bx + threadIdx.x;
        if (c < cols && r < ldd) dst[(int64_t)c * ldd + r] = __float2bfloat16_rn(tile[i][threadIdx.x]);
    }
}

// mean-squared error over n values and its gradient: loss = 1/n sum (y - t)^2
__global__ void k_mse(int n, const float *__restrict__ y, const float *__restrict__ t, float *__restrict__ dy,
                      float *__restrict__ loss)
{
    __shared__ double red[32];
    double acc = 0.0;
    const float s = 2.f / (float)n;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const float d = y[e] - t[e];
        dy[e] = s * d;
        acc += (double)d * d;
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
        if (threadIdx.x == 0) *loss = (float)(v / n);
    }
}

// Adam (Kingma & Ba) on FP32 masters, optional BF16 copy of the updated weights
__global__ void k_adam(int64_t n, float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m1,
                       float *__restrict__ m2, float lr, float b1, float b2, float eps, float c1, float c2,
                       __nv_bfloat16 *__restrict__ wb)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    const float gg = g[e];
    const float a = b1 * m1[e] + (1.f - b1) * gg;
    const float b = b2 * m2[e] + (1.f - b2) * gg * gg;
    m1[e] = a;
    m2[e] = b;
    const float w2 = w[e] - lr * (a / c1) / (sqrtf(b / c2) + eps);
    w[e] = w2;
    if (wb) wb[e] = __float2bfloat16_rn(w2);
}

}  // namespace nn
}  // namespace gbp

using namespace gbp::nn;

namespace {
inline unsigned nb(int64_t n, int th) { return (unsigned)((n + th - 1) / th); }
inline gbp_status st_of(cudaError_t e) { return e == cudaSuccess ? GBP_OK : GBP_ERR_CUDA; }
}  // namespace

extern "C" {

// The driver's tensor-map encoder, found through the runtime (the library
// does not link the driver API); null when the driver does not provide it.
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled()
{
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// Tiles of box_rows x 64 BF16 (K contiguous, row stride ld elements) of a
// rows x Kp operand, 128-byte swizzle (the layout sw128_desc describes).
static bool make_tile_map(CUtensorMap *map, const void *ptr, int rows, int Kp, int ld, int box_rows)
{
    const EncodeTiledFn enc = encode_tiled();
    if (!enc) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)TK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

gbp_status gbp_nn_gemm_bf16(gbp_ctx *c, int32_t M, int32_t N, int32_t Kp, const void *A, int32_t lda, const void *B,
                            int32_t ldb, float *C, int32_t ldc, float alpha, float beta)
{
    if (!c || !A || !B || !C || M < 1 || N < 1 || Kp < 0 || Kp % 64 || lda < Kp || ldb < Kp || lda % 8 ||
        ldb % 8 || ldc < N)
        return GBP_ERR_INVALID_ARG;
    // whole 128 x 256 tiles, 16-byte aligned operands, and enough tiles to
    // spread over the GPU (at a few tiles the 128 x 64 kernel, with four
    // times the CTAs, was as fast: 33 vs 35 us at 256 x 256 x 1216): the
    // TMA-fed kernel
    CUtensorMap ta, tb;
    if (M % TM == 0 && N % TN == 0 && (M / TM) * (N / TN) >= 64 && Kp >= TK && ldc % 4 == 0 &&
        ((uintptr_t)A & 15) == 0 &&
        ((uintptr_t)B & 15) == 0 && ((uintptr_t)C & 15) == 0 && make_tile_map(&ta, A, M, Kp, lda, TM) &&
        make_tile_map(&tb, B, N, Kp, ldb, TN)) {
        cudaFuncSetAttribute(k_gemm_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, T_SMEM);
        const int ntiles = (M / TM) * (N / TN);
        k_gemm_tma<<<min(ntiles, c->num_sms), 192, T_SMEM, c->stream>>>(M, N, Kp, ta, tb, C, ldc, alpha, beta,
                                                                         c->ctl);
        c->launches++;
        return st_of(cudaGetLastError());
    }
    dim3 grid((M + GM - 1) / GM, (N + GN - 1) / GN);
    const int smem = 2 * (GA_BYTES + GB_BYTES);
    cudaFuncSetAttribute(k_gemm_tn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    k_gemm_tn<<<grid, 128, smem, c->stream>>>(M, N, Kp, (const __nv_bfloat16 *)A, lda, (const __nv_bfloat16 *)B, ldb,
                                           C, ldc, alpha, beta, c->ctl);
    c->launches++;
    return st_of(cudaGetLastError());
}

gbp_status gbp_nn_im2col(gbp_ctx *c, int32_t Bn, int32_t Li, int32_t Ci, int32_t Lo, int32_t ks, int32_t stride,
                         int32_t pad, const float *act, void *col, int32_t ldc)
{
    if (!c || !act || !col || Bn < 1 || Li < 1 || Ci < 1 || Lo < 1 || ks < 1 || stride < 1 || pad < 0 ||
        ldc < ks * Ci)
        return GBP_ERR_INVALID_ARG;
    const int64_t tot = (int64_t)Bn * Lo * ldc;
    k_im2col<<<nb(tot, 256), 256, 0, c->stream>>>(Bn, Li, Ci, Lo, ks, stride, pad, act, (__nv_bfloat16 *)col, ldc);
    c->launches++;
    return st_of(cudaGetLastError());
}

gbp_status gbp_nn_im2col_t(gbp_ctx *c, int32_t Bn, int32_t Li, int32_t Ci, int32_t Lo, int32_t ks, int32_t stride,
                           int32_t pad, const float *act, int32_t Kp, void *colT, int32_t ldt)
{
    if (!c || !act || !colT || Bn < 1 || Li < 1 || Ci < 1 || Lo < 1 || ks < 1 || stride < 1 || pad < 0 ||
        Kp < ks * Ci || (int64_t)ldt < (int64_t)Bn * Lo)
        return GBP_ERR_INVALID_ARG;
    const int64_t tot = (int64_t)Kp * ldt;
    k_im2col_t<<<nb(tot, 256), 256, 0, c->stream>>>(Bn, Li, Ci, Lo, ks, stride, pad, act, Kp, (__nv_bfloat16 *)colT,
                                                     ldt);
    c->launches++;
    return st_of(cudaGetLastError());
}

gbp_status gbp_nn_col2im(gbp_ctx *c, int32_t Bn, int32_t Li, int32_t Ci, int32_t Lo, int32_t ks, int32_t stride,
                         int32_t pad, const float *dcol, int32_t ldc, float *dact)
{
    if (!c || !dcol || !dact || Bn < 1 || Li < 1 || Ci < 1 || Lo < 1 || ks < 1 || stride < 1 || pad < 0 ||
        ldc < ks * Ci)
        return GBP_ERR_INVALID_ARG;
    const int64_t tot = (int64_t)Bn * Li * Ci;
    k_col2im<<<nb(tot, 256), 256, 0, c->stream>>>(Bn, Li, Ci, Lo, ks, stride, pad, dcol, ldc, dact);
    c->launches++;
    return st_of(cudaGetLastError());
}

gbp_status gbp_nn_bias_act(gbp_ctx *c, int32_t M, int32_t N, float *y, int32_t ld, const float *bias, float *pre,
                           int32_t gelu)
{
    if (!c || !y || !bias || M < 1 || N < 1 || ld < N) return GBP_ERR_INVALID_ARG;
    k_bias_act<<<nb((int64_t)M * N, 256), 256, 0, c->stream>>>(M, N, y, ld, bias, pre, gelu);
    c->launches++;
    return st_of(cudaGetLastError());
}

gbp_status gbp_nn_gelu_backward(gbp_ctx *c, int32_t M, int32_t N, float *dy, int32_t ld, const float *pre)
{
    if (!c || !dy || !pre || M < 1 || N < 1 || ld < N) return GBP_ERR_INVALID_ARG;
    k_gelu_bwd<<<nb((int64_t)M * N, 256), 256, 0, c->stream>>>(M, N, dy, ld, pre);
    c->launches++;
    return st_of(cudaGetLastError());
}

gbp_status gbp_nn_bias_grad(gbp_ctx *c, int32_t M, int32_t N, const float *dz, int32_t ld, float *db)
{
    if (!c || !dz || !db || M < 1 || N < 1 || ld < N) return GBP_ERR_INVALID_ARG;
    k_bias_grad<<<N, 256, 0, c->stream>>>(M, N, dz, ld, db);
    c->launches++;
    return st_of(cudaGetLastError());
}

gbp_status gbp_nn_cast_bf16(gbp_ctx *c, int32_t rows, int32_t cols, const float *src, int32_t lds, void *dst,
                            int32_t ldd)
{
    if (!c || !src || !dst || rows < 1 || cols < 1 || lds < cols || ldd < cols) return GBP_ERR_INVALID_ARG;
    k_cast_bf16<<<nb((int64_t)rows * ldd, 256), 256, 0, c->stream>>>(rows, cols, src, lds, (__nv_bfloat16 *)dst,
                                                                      ldd);
    c->launches++;
    return st_of(cudaGetLastError());
}

gbp_status gbp_nn_transpose_bf16(gbp_ctx *c, int32_t rows, int32_t cols, const float *src, int32_t lds, void *dst,
                                 int32_t ldd)
{
    if (!c || !src || !dst || rows < 1 || cols < 1 || lds < cols || ldd < rows) return GBP_ERR_INVALID_ARG;
    dim3 grid((ldd + 31) / 32, (cols + 31) / 32);
    k_transpose_bf16<<<grid, dim3(32, 8), 0, c->stream>>>(rows, cols, src, lds, (__nv_bfloat16 *)dst, ldd);
    c->launches++;
    return st_of(cudaGetLastError());
}

gbp_status gbp_nn_mse(gbp_ctx *c, int32_t n, const float *y, const float *t, float *dy, float *loss)
{
    if (!c || !y || !t || !dy || !loss || n < 1) return GBP_ERR_INVALID_ARG;
    k_mse<<<1, 1024, 0, c->stream>>>(n, y, t, dy, loss);
    c->launches++;
    return st_of(cudaGetLastError());
}

gbp_status gbp_nn_adam(gbp_ctx *c, int64_t n, float *w, const float *g, float *m1, float *m2, float lr, float b1,
                       float b2, float eps, int32_t step, void *w_bf16)
{
    if (!c || !w || !g || !m1 || !m2 || n < 1 || step < 1) return GBP_ERR_INVALID_ARG;
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    k_adam<<<nb(n, 256), 256, 0, c->stream>>>(n, w, g, m1, m2, lr, b1, b2, eps, c1, c2, (__nv_bfloat16 *)w_bf16);
    c->launches++;
    return st_of(cudaGetLastError());
}

}  // extern "C"
