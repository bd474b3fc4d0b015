/*
 * gbp.h -- C ABI of the GB300 Geodesic-BP library (libgbp.so).
 *
 * One forward-plus-gradient evaluation of the eikonal ECG model of
 * Grandits et al., "Digital twinning of cardiac electrophysiology models from
 * the surface ECG: a geodesic backpropagation approach":
 *
 *   1. anisotropic eikonal solve on a P1 tetrahedral mesh (Eq. (1)) as the
 *      discrete Hopf-Lax fixed point (Eq. hopflax_global, Eq. hopflax_local,
 *      Algorithm 2), recording each vertex's minimising parent face and
 *      barycentric point;
 *   2. the lead-field ECG V = B U(t - phi) (Sec. II-D, Eq. tanh_waveform);
 *   3. the gradient of the ECG misfit (Eq. inverse_ecg) with respect to the
 *      conduction velocities and the onsets, taken along the frozen parent
 *      graph (Sec. II-C, Eq. dto_grad, Eq. upwind_xi).
 *
 * Conventions
 *   - Units: mm, ms, mm/ms.  Floating point is IEEE float32 unless stated.
 *   - Conduction tensor of element j (Eq. (1)): M_j = ct_j^2 I +
 *     (cf_j^2 - ct_j^2) f_j f_j^T with unit fibre f_j; the local metric is
 *     D_j = M_j^{-1} (Sec. II-A).
 *   - Parent code of vertex i: tet*4 + slot (slot = position of i in the tet);
 *     the face E_{j\i} is the tet's other three vertices in increasing slot
 *     order, and alpha[3] refers to that order.  A vertex holding its onset
 *     value has code -1-k (onset k); an unreached vertex INT32_MIN and
 *     phi = +inf.
 *   - Pointer kinds are stated per argument: "device" pointers are CUDA
 *     device memory of the context's device, "host" pointers are ordinary
 *     (pageable or pinned) host memory.  Arrays are caller-owned; the library
 *     never frees or retains them beyond the call unless stated.
 *   - Calls are stream-ordered on the context stream and asynchronous unless
 *     stated.  Errors: every call returns a gbp_status; argument errors are
 *     detected on the host before any launch.  Device-side failures (a
 *     bounded wait that ran out, an iteration limit) are latched into the
 *     context and reported by the next synchronising call
 *     (gbp_get_solve_stats, gbp_synchronize, the *_host calls).  The library
 *     never aborts the process and never traps on the device.
 *   - A context is not thread-safe; use one per host thread.
 */
#ifndef GBP_H
#define GBP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gbp_ctx gbp_ctx;

typedef enum {
    GBP_OK = 0,
    GBP_ERR_INVALID_ARG = 1,   /* bad size, NULL pointer, out-of-range index */
    GBP_ERR_BAD_MESH = 2,      /* inverted / degenerate tet, bad vertex id */
    GBP_ERR_NOT_SPD = 3,       /* velocity <= 0 or not finite, zero fibre */
    GBP_ERR_NOT_CONVERGED = 4, /* iteration limit reached */
    GBP_ERR_TIMEOUT = 5,       /* a bounded device-side wait ran out */
    GBP_ERR_UNREACHABLE = 6,   /* (informational) vertices left at +inf */
    GBP_ERR_CUDA = 7,          /* CUDA runtime error */
    GBP_ERR_STATE = 8,         /* call order violated (e.g. no mesh yet) */
    GBP_ERR_NO_MEMORY = 9
} gbp_status;

enum { GBP_LOCAL_EXACT = 0, GBP_LOCAL_FISTA = 1 };
enum { GBP_ONSET_NODAL = 0, GBP_ONSET_ELEMENT = 1 };
enum { GBP_PREC_FP32 = 0, GBP_PREC_BF16 = 1 };

/* Options of one eikonal solve (Algorithm 2). */
typedef struct {
    int32_t local_solver; /* GBP_LOCAL_EXACT: exact minimiser of Eq. (upwind_eq_lsqr);
                             GBP_LOCAL_FISTA: Algorithm 1 with n_f steps */
    int32_t n_f;          /* FISTA steps (ignored for EXACT); 1..256 */
    float eps;            /* Algorithm 2's epsilon: a vertex re-activates its
                             neighbours when it decreased by more than eps (ms);
                             0 = on any decrease */
    int32_t max_iters;    /* iteration limit; 0 = 8 * (cube root of n_v) + 64 + n_f */
} gbp_solve_opts;

/* Statistics of the last solve / backward pass (read by gbp_get_solve_stats). */
typedef struct {
    int64_t iterations;     /* FIM iterations (grid-wide steps) */
    int64_t candidates;     /* vertex updates attempted */
    int64_t face_updates;   /* local problems solved (faces with a changed vertex) */
    int64_t fp64_fallbacks; /* local problems redone in FP64 */
    int64_t unreached;      /* vertices left at +inf */
    int64_t adj_levels;     /* adjoint: vertices that seeded the dataflow (no children) */
    int64_t adj_cycle_nodes;/* adjoint: vertices solved by the cycle iteration */
    int64_t adj_cycle_iters;/* adjoint: iterations of the cycle iteration */
    int32_t status;         /* gbp_status of the last solve / backward */
    int32_t reserved;
    double adj_dataflow_ms; /* adjoint: device time of the dataflow phase */
    double adj_cycle_ms;    /* adjoint: device time of the cycle iteration */
    int64_t fim_deferred;   /* faces the FIM left to the FP64 repair (their interior step needs FP64) */
    int64_t fim_repaired;   /* vertices the repair lowered (the exact iteration resumed from them) */
} gbp_solve_stats;

/* Template action potential (Eq. tanh_waveform), read as
 * U(xi) = K0 + (K1 - K0)/2 (1 + tanh(2 xi / tau)), sampled at
 * t_s = t0 + s dt, s = 0..T-1. */
typedef struct {
    float K0, K1, tau, t0, dt;
    int32_t T;
} gbp_template;

/* ------------------------------------------------------------------ */
/* context                                                              */
/* ------------------------------------------------------------------ */

/* Create a context on CUDA device `device`.  `stream` is a cudaStream_t (or
 * NULL for the legacy default stream); every call of this context is ordered
 * on it.  *out receives the context (NULL on failure). */
gbp_status gbp_create(gbp_ctx **out, int device, void *stream);
void gbp_destroy(gbp_ctx *ctx);
gbp_status gbp_set_stream(gbp_ctx *ctx, void *stream);
const char *gbp_status_string(gbp_status s);
/* Synchronise the context stream and report any latched device error. */
gbp_status gbp_synchronize(gbp_ctx *ctx);

/* ------------------------------------------------------------------ */
/* problem set-up                                                       */
/* ------------------------------------------------------------------ */

/* Mesh of Sec. II-A: xyz host float32 [n_v][3], tets host int32 [n_t][4],
 * positively oriented.  Validates (vertex ids in range and distinct, volume
 * > 0), builds the vertex->tet and vertex->vertex adjacency on the host and
 * uploads it.  Synchronous.  Errors: GBP_ERR_BAD_MESH, GBP_ERR_INVALID_ARG.
 * Invalidates fibres, velocities, onsets, lead field and the last solve. */
gbp_status gbp_upload_mesh(gbp_ctx *ctx, const float *xyz, int64_t n_v, const int32_t *tets,
                           int64_t n_t);

/* Triangle mesh (d = 2; Sec. II states the method for any d, and in 2-D
 * the face opposite a vertex is an edge): xy host float32 [n_v][2], tris
 * host int32 [n_t][3], counter-clockwise.  Validates (ids in range and
 * distinct, signed area > 0) and sets the context to d = 2, in which the
 * other calls take their 2-D layouts:
 *   fibres [n_t][2]; element-onset barycentric coordinates [K][3] over the
 *   triangle; lead field [N][n_v]; phi, dphi [n_v]; parent code
 *   = triangle * 3 + slot with alpha [n_v][2], the weights of the
 *   triangle's other two vertices in slot order; d_x [K][2] (and
 *   [B][K][2] in the batched call).
 * Internally each triangle is solved as the tet (a, b, c, apex) with one
 * apex above the plane that no onset reaches: the face of a vertex then
 * holds one vertex at +inf and the local minimiser reduces exactly to the
 * edge problem.  Synchronous.  Errors: GBP_ERR_BAD_MESH, GBP_ERR_INVALID_ARG.
 * Invalidates what gbp_upload_mesh invalidates. */
gbp_status gbp_upload_mesh_2d(gbp_ctx *ctx, const float *xy, int64_t n_v, const int32_t *tris,
                              int64_t n_t);

/* Host-only validation (no context, no device, nothing allocated): the
 * checks gbp_upload_mesh / gbp_upload_mesh_2d make before they build
 * anything, on the same host arrays.  Tets: n_v >= 4, n_t >= 1, coordinates
 * finite, vertex ids in [0, n_v) and distinct within a tet, signed volume
 * above 1e-15 diag^3 (diag = bounding-box diagonal; right-handed).
 * Triangles: n_v >= 3, the same id checks, signed area above 1e-12 ext^2
 * (ext = larger bounding-box side; counter-clockwise).  Returns GBP_OK,
 * GBP_ERR_INVALID_ARG (NULL pointer, sizes out of range: n_v < 2^30 and
 * n_t < 2^29) or GBP_ERR_BAD_MESH. */
gbp_status gbp_check_mesh(const float *xyz, int64_t n_v, const int32_t *tets, int64_t n_t);
gbp_status gbp_check_mesh_2d(const float *xy, int64_t n_v, const int32_t *tris, int64_t n_t);

/* Host-only (no context, no device): the adjacency gbp_upload_mesh builds
 * for the FIM and the adjoint, on host arrays.  tets int32 [n_t][4] with ids
 * in [0, n_v).  Writes *n_faces (= 4 n_t entries of the vertex->tet lists)
 * and *n_nbr (entries of the vertex->vertex lists); when all five arrays are
 * non-NULL it also fills them (caller-owned host memory):
 *   n2t_ptr int32 [n_v + 1], n2t int32 [n_faces]: per vertex the codes
 *     tet * 4 + slot of its incident tets, in ascending code;
 *   n2n_ptr int32 [n_v + 1], n2n int32 [n_nbr]: per vertex its neighbours
 *     through a shared tet, sorted and unique;
 *   frec int32 [n_faces][4]: per vertex->tet entry, the tet's other three
 *     vertices in slot order and the code (the FIM's face records).
 * Call once with NULL arrays for the sizes, then with the arrays.  Errors:
 * GBP_ERR_INVALID_ARG (NULL tets or size pointers, sizes out of range),
 * GBP_ERR_BAD_MESH (an id out of range). */
gbp_status gbp_mesh_adjacency(const int32_t *tets, int64_t n_v, int64_t n_t, int64_t *n_faces,
                              int64_t *n_nbr, int32_t *n2t_ptr, int32_t *n2t, int32_t *n2n_ptr,
                              int32_t *n2n, int32_t *frec);

/* Fibre directions f_j: device float32 [n_t][3] (normalised here; a zero
 * vector is GBP_ERR_NOT_SPD at the next velocity update). Copied. */
gbp_status gbp_set_fibres(gbp_ctx *ctx, const float *fib);

/* Velocities cf_j, ct_j: device float32 [n_t] each.  Copied, and the
 * per-tet metric D_j = M_j^{-1} is precomputed on the device.  Invalid values
 * (<= 0, NaN) are latched as GBP_ERR_NOT_SPD and reported by the next
 * synchronising call.  Requires fibres. */
gbp_status gbp_set_velocities(gbp_ctx *ctx, const float *cf, const float *ct);

/* Lead-field operator B of Eq. (integral_potential_ecg), read as N x n_v
 * (one row per lead): device float32 [N][n_v], 1 <= N <= 16.  Copied; the
 * BF16 copy with per-lead scales is prepared here. */
gbp_status gbp_set_leadfield(gbp_ctx *ctx, const float *L, int32_t N);

/* Onsets X0 of Eq. (1).  kind GBP_ONSET_NODAL: idx = vertex ids, bary unused
 * (may be NULL); GBP_ONSET_ELEMENT: idx = tet ids and bary = barycentric
 * coordinates [K][4] of x_k in that tet (Eq. upwind_xi).  t = onset times.
 * All device pointers: idx int32 [K], bary float32 [K][4], t float32 [K].
 * 1 <= K <= 65536.  Copied.  Index range is checked on the device and
 * latched as GBP_ERR_INVALID_ARG. */
gbp_status gbp_set_onsets(gbp_ctx *ctx, int32_t kind, int32_t K, const int32_t *idx,
                          const float *bary, const float *t);

/* One set of onset sites per problem for gbp_forward_backward_batch with
 * the same B (multi-start over the sites themselves, Sec. IV: the paper
 * names batched optimisation as the way out of local minima of the site
 * fit).  Layouts as gbp_set_onsets with a leading B: idx int32 [B][K],
 * bary float32 [B][K][d + 1] (element onsets), t float32 [B][K] (the times
 * the batched call uses when its own t is NULL).  Device pointers, copied.
 * Grows the per-problem arrays to B problems like the batched call.  Until
 * the next gbp_set_onsets, a batched call with another B is GBP_ERR_STATE,
 * and single-problem calls use problem 0's sites.  Errors:
 * GBP_ERR_INVALID_ARG, GBP_ERR_STATE (no mesh), GBP_ERR_NO_MEMORY; ids out
 * of range are latched as in gbp_set_onsets. */
gbp_status gbp_set_onsets_batch(gbp_ctx *ctx, int32_t kind, int32_t B, int32_t K, const int32_t *idx,
                                const float *bary, const float *t);

/* ------------------------------------------------------------------ */
/* the hot path                                                         */
/* ------------------------------------------------------------------ */

/* Eikonal solve (Algorithm 2 with the local solver of Sec. II-B):
 * persistent active-list FIM, then the parent pass.  Outputs (device, any
 * may be NULL): phi float32 [n_v], parent int32 [n_v], alpha float32
 * [n_v][3].  The context keeps its own copy of the parent graph for
 * gbp_geodesic_backward.  Asynchronous; stats via gbp_get_solve_stats. */
gbp_status gbp_eikonal_solve(gbp_ctx *ctx, const gbp_solve_opts *opts, float *phi,
                             int32_t *parent, float *alpha);

/* The solution of problem b of the last solve: the activation map phi and
 * the parent record (Eq. dto_grad's frozen graph).  b = 0 after
 * gbp_eikonal_solve / gbp_forward_backward, 0 <= b < B after
 * gbp_forward_backward_batch.  phi float32 [n_v], parent int32 [n_v] and
 * alpha float32 [n_v][3] (d = 2: [n_v][2]) device pointers in the layouts of
 * gbp_eikonal_solve; any may be NULL.  Asynchronous.  Errors:
 * GBP_ERR_INVALID_ARG (b out of range, every output NULL), GBP_ERR_STATE (no
 * solve recorded since the mesh upload or the last growth of the batch). */
gbp_status gbp_get_solution(gbp_ctx *ctx, int32_t b, float *phi, int32_t *parent, float *alpha);

/* Synchronises and returns the statistics and status of the last solve and
 * backward pass. */
gbp_status gbp_get_solve_stats(gbp_ctx *ctx, gbp_solve_stats *stats);

/* ECG V[l][s] = sum_n B[l][n] U(t_s - phi_n) (Sec. II-D).  phi device float32
 * [n_v] (+inf allowed), ecg device float32 [N][T] (written).
 * precision GBP_PREC_FP32 (CUDA cores) or GBP_PREC_BF16 (tensor cores:
 * BF16 template values and per-lead-scaled BF16 lead field, FP32
 * accumulation; the constant part of U is applied exactly in FP32).
 * T <= 4096. */
gbp_status gbp_ecg_forward(gbp_ctx *ctx, const float *phi, const gbp_template *tmpl,
                           int32_t precision, float *ecg);

/* Misfit of Eq. (inverse_ecg) with the rectangle rule,
 * loss = 1/(N T) sum_{l,s} (ecg - target)^2, and its derivative with respect
 * to each phi_n (Sec. II-D: nabla V = -B^T U' nabla phi).  phi, ecg (from
 * gbp_ecg_forward), target device float32; loss device float32 [1];
 * dphi device float32 [n_v].  N * T <= 51200 (the residual is staged in
 * shared memory). */
gbp_status gbp_ecg_loss_backward(gbp_ctx *ctx, const float *phi, const float *ecg,
                                 const float *target, const gbp_template *tmpl, float *loss,
                                 float *dphi);

/* Frozen-graph adjoint of the last gbp_eikonal_solve (Sec. II-C, Eq.
 * dto_grad, Eq. upwind_xi; the conduction-tensor variant of Sec. IV):
 * mu = (I - P^T)^{-1} dphi, accumulated in reverse topological order of the
 * parent graph (short cycles are resolved by a bounded fixed-point
 * iteration).  dphi device float32 [n_v] (dLoss/dphi).  Outputs (device,
 * written, any may be NULL): d_cf, d_ct float32 [n_t], d_t float32 [K],
 * d_x float32 [K][3] (zero for nodal onsets).  GBP_ERR_STATE without a solve
 * or after the parameters changed since it. */
gbp_status gbp_geodesic_backward(gbp_ctx *ctx, const float *dphi, float *d_cf, float *d_ct,
                                 float *d_t, float *d_x);

/* One forward-plus-gradient evaluation: velocities -> eikonal -> ECG ->
 * misfit -> adjoint.  cf, ct device float32 [n_t]; t device float32 [K]
 * (NULL keeps the onset times of gbp_set_onsets); target device float32
 * [N][T]; outputs device: loss [1], ecg [N][T] (may be NULL), d_cf, d_ct
 * [n_t], d_t [K], d_x [K][3] (any may be NULL). */
gbp_status gbp_forward_backward(gbp_ctx *ctx, const gbp_solve_opts *opts,
                                const gbp_template *tmpl, int32_t precision, const float *cf,
                                const float *ct, const float *t, const float *target, float *loss,
                                float *ecg, float *d_cf, float *d_ct, float *d_t, float *d_x);

/* The same evaluation from HOST buffers: inputs are copied host->device and
 * outputs device->host inside the call, which synchronises.  cf, ct host
 * [n_t]; t host [K] (NULL keeps the current times); target host [N][T];
 * loss host [1]; d_cf, d_ct host [n_t]; d_t host [K]; d_x host [K][3]
 * (outputs may be NULL).  Uses staging buffers owned by the context. */
gbp_status gbp_forward_backward_host(gbp_ctx *ctx, const gbp_solve_opts *opts,
                                     const gbp_template *tmpl, int32_t precision,
                                     const float *cf, const float *ct, const float *t,
                                     const float *target, float *loss, float *d_cf,
                                     float *d_ct, float *d_t, float *d_x);

/* B independent evaluations on the same mesh, fibres and lead field in one
 * pass (multi-start: the paper suggests several starts against local minima
 * of the inverse problem, Sec. IV).  The onset sites are those of
 * gbp_set_onsets, shared by all problems, or one set per problem after
 * gbp_set_onsets_batch.  Each problem b has its own velocities, onset times
 * and target; the FIM, the parent pass and the
 * adjoint run all B problems in the same launches, so their per-iteration
 * latency is shared.  cf, ct device float32 [B][n_t]; t device float32
 * [B][K] (NULL: the times of gbp_set_onsets for every problem, or those of
 * gbp_set_onsets_batch); target device float32 [B][N][T]; outputs device:
 * loss [B], ecg [B][N][T] (may be NULL), d_cf, d_ct [B][n_t], d_t [B][K],
 * d_x [B][K][d] (any may be NULL).  Requires B * n_v < 2^31 / 3 and
 * N * T <= 51200; after gbp_set_onsets_batch, B equal to its B.  Grows the context's
 * per-problem arrays to B problems on first use (allocation, synchronises
 * once).  Afterwards the single-problem state is reset: the next
 * single-problem solve needs gbp_set_velocities first.  Statistics
 * (gbp_get_solve_stats) add up over the B problems.  Errors:
 * GBP_ERR_INVALID_ARG, GBP_ERR_STATE, GBP_ERR_CUDA and the device errors of
 * gbp_eikonal_solve / gbp_geodesic_backward. */
gbp_status gbp_forward_backward_batch(gbp_ctx *ctx, int32_t B, const gbp_solve_opts *opts,
                                      const gbp_template *tmpl, int32_t precision, const float *cf,
                                      const float *ct, const float *t, const float *target,
                                      float *loss, float *ecg, float *d_cf, float *d_ct, float *d_t,
                                      float *d_x);

/* gbp_forward_backward_batch from HOST buffers: the inputs are copied
 * host->device from the caller's arrays and the outputs device->host into
 * them inside the call, which synchronises.  cf, ct host [B][n_t]; t host
 * [B][K] (NULL: as in gbp_forward_backward_batch); target host [B][N][T];
 * loss host [B]; d_cf, d_ct host [B][n_t]; d_t host [B][K]; d_x host
 * [B][K][d] (outputs may be NULL).  The copies run straight from and to the
 * caller's memory: page-locked (pinned) host memory gives the full link
 * bandwidth, pageable memory works at the driver's staged rate.  Device
 * staging buffers are owned by the context.  Errors as the batched call. */
gbp_status gbp_forward_backward_batch_host(gbp_ctx *ctx, int32_t B, const gbp_solve_opts *opts,
                                           const gbp_template *tmpl, int32_t precision, const float *cf,
                                           const float *ct, const float *t, const float *target,
                                           float *loss, float *d_cf, float *d_ct, float *d_t, float *d_x);

/* ------------------------------------------------------------------ */
/* learned initialiser: network training and inference kernels          */
/* ------------------------------------------------------------------ */
/* A 1-D convolutional network + MLP maps an ECG to initial onset sites,
 * times and velocities, then Geodesic-BP refines them (not in the paper:
 * the initialiser of the inverse problem of Sec. II-D).  All calls are
 * stream-ordered on the context stream and take device pointers.  BF16
 * operands are raw 16-bit storage (void*).  Activations are channels-last
 * f32 [batch][length][channels]; convolution weights [C_out][ksize][C_in].
 * GEMM operands keep the reduction dimension contiguous, zero-padded to a
 * multiple of 64 (Kp). */

/* C[m][n] = alpha sum_k A[m][k] B[n][k] + beta C[m][n]: A bf16 [M][lda],
 * B bf16 [N][ldb] (k < Kp, Kp % 64 == 0, lda, ldb >= Kp and % 8 == 0),
 * C f32 [M][ldc].  Tensor cores (tcgen05, FP32 accumulation in TMEM). */
gbp_status gbp_nn_gemm_bf16(gbp_ctx *ctx, int32_t M, int32_t N, int32_t Kp, const void *A, int32_t lda,
                            const void *B, int32_t ldb, float *C, int32_t ldc, float alpha, float beta);
/* col[b*Lo + l][k*Ci + c] = act[b][stride*l + k - pad][c] (0 outside), bf16,
 * row stride ldc >= ks*Ci (padding zeroed). */
gbp_status gbp_nn_im2col(gbp_ctx *ctx, int32_t B, int32_t Li, int32_t Ci, int32_t Lo, int32_t ks,
                         int32_t stride, int32_t pad, const float *act, void *col, int32_t ldc);
/* the transpose colT[k*Ci + c][b*Lo + l], rows < Kp, row stride ldt >= B*Lo. */
gbp_status gbp_nn_im2col_t(gbp_ctx *ctx, int32_t B, int32_t Li, int32_t Ci, int32_t Lo, int32_t ks,
                           int32_t stride, int32_t pad, const float *act, int32_t Kp, void *colT,
                           int32_t ldt);
/* adjoint of im2col: dact[b][j][c] = sum of dcol entries that read act[b][j][c]. */
gbp_status gbp_nn_col2im(gbp_ctx *ctx, int32_t B, int32_t Li, int32_t Ci, int32_t Lo, int32_t ks,
                         int32_t stride, int32_t pad, const float *dcol, int32_t ldc, float *dact);
/* y[m][n] = act(y[m][n] + bias[n]) in place (row stride ld), act = GELU
 * (x Phi(x)) when gelu != 0; pre (may be NULL) keeps y + bias [M][N]. */
gbp_status gbp_nn_bias_act(gbp_ctx *ctx, int32_t M, int32_t N, float *y, int32_t ld, const float *bias,
                           float *pre, int32_t gelu);
/* dy[m][n] *= GELU'(pre[m][n]) in place. */
gbp_status gbp_nn_gelu_backward(gbp_ctx *ctx, int32_t M, int32_t N, float *dy, int32_t ld,
                                const float *pre);
/* db[n] = sum_m dz[m][n]. */
gbp_status gbp_nn_bias_grad(gbp_ctx *ctx, int32_t M, int32_t N, const float *dz, int32_t ld, float *db);
/* dst[r][c] = bf16(src[r][c]), zero for cols <= c < ldd. */
gbp_status gbp_nn_cast_bf16(gbp_ctx *ctx, int32_t rows, int32_t cols, const float *src, int32_t lds,
                            void *dst, int32_t ldd);
/* dst[c][r] = bf16(src[r][c]) (dst has cols rows of stride ldd >= rows, zero padded). */
gbp_status gbp_nn_transpose_bf16(gbp_ctx *ctx, int32_t rows, int32_t cols, const float *src, int32_t lds,
                                 void *dst, int32_t ldd);
/* loss = mean (y - t)^2 over n values (device scalar), dy = 2 (y - t) / n. */
gbp_status gbp_nn_mse(gbp_ctx *ctx, int32_t n, const float *y, const float *t, float *dy, float *loss);
/* Adam step `step` (>= 1) on FP32 master weights w with moments m1, m2;
 * w_bf16 (may be NULL) receives the updated weights in BF16. */
gbp_status gbp_nn_adam(gbp_ctx *ctx, int64_t n, float *w, const float *g, float *m1, float *m2, float lr,
                       float beta1, float beta2, float eps, int32_t step, void *w_bf16);

/* ------------------------------------------------------------------ */
/* allocation-free entry point                                          */
/* ------------------------------------------------------------------ */

/* The ECG forward pass of gbp_ecg_forward (FP32) for callers that must not
 * allocate device memory: code under a fixed memory budget, code inside a
 * framework whose caching allocator owns the device heap, and loops that must
 * never block on cudaMalloc / cudaFree.  It needs no context and calls no
 * allocating routine.  (The paper has no counterpart: this is a deployment
 * variant of the ECG contraction.)
 *
 * L device float32 [N][n_v] (1 <= N <= 16), phi device float32 [n_v],
 * ecg device float32 [N][T] (written), T <= 4096, stream a cudaStream_t or
 * NULL.  Runs on the calling thread's current CUDA device.
 * Scratch: a 4 MiB file-scope device array (partial sums and row sums) that
 * every GPU loading the library holds until the process exits.  The first
 * call on a device looks up that array's address (once per device); make
 * that first call before any stream capture.  All calls share the array and
 * every call overwrites what it reads, so nothing carries over between
 * calls; calls that overlap on the GPU (other streams, other threads) race
 * on it and must be serialised by the caller.
 * Errors: GBP_ERR_INVALID_ARG for a NULL pointer or N, T beyond the limits
 * above; GBP_ERR_CUDA for a CUDA runtime error. */
gbp_status gbp_ecg_forward_noalloc(const float *L, int32_t N, int64_t n_v, const float *phi,
                                   const gbp_template *tmpl, float *ecg, void *stream);

/* ------------------------------------------------------------------ */
/* diagnostics                                                          */
/* ------------------------------------------------------------------ */

/* The local problem of Eq. (upwind_eq_lsqr) on n independent faces (for
 * tests): e device float32 [n][3][3] (rows v_{j_m} - v_i), fib [n][3],
 * cf, ct [n], Phi [n][3] (+inf allowed); mode GBP_LOCAL_EXACT or
 * GBP_LOCAL_FISTA (Algorithm 1, n_f steps, Lipschitz constant of Eq.
 * (lipschitz_est) with h_ = h_min / 1.1).  Writes value [n], alpha [n][3]. */
gbp_status gbp_local_solve_batch(gbp_ctx *ctx, int64_t n, const float *e, const float *fib,
                                 const float *cf, const float *ct, const float *Phi,
                                 int32_t mode, int32_t n_f, float *value, float *alpha);

/* Failure detection on the device, exercised without a fault: one
 * cooperative launch of the grid barrier the FIM and the adjoint synchronise
 * with (one CTA per SM) in which the last absent_ctas CTAs never arrive, so
 * the other CTAs' bounded waits run out after max_spins polls (a short sleep
 * each) and latch GBP_ERR_TIMEOUT into the context, exactly as a stalled
 * solve would.  absent_ctas = 0 is the control case: the barrier completes
 * and nothing is latched.  The call resets the context's device status
 * first; the outcome is reported by the next synchronising call
 * (gbp_synchronize, gbp_get_solve_stats).  The context stays usable: the
 * next solve resets the status.  Errors: GBP_ERR_INVALID_ARG
 * (absent_ctas < 0 or >= the SM count, max_spins < 1), GBP_ERR_CUDA. */
gbp_status gbp_diag_barrier_timeout(gbp_ctx *ctx, int32_t absent_ctas, int32_t max_spins);

/* Kernel timing: when enabled, the library records CUDA events around its
 * main kernels on the context stream.  gbp_get_kernel_times synchronises and
 * returns, per kernel class (0 eikonal FIM, 1 parent pass, 2 ECG forward,
 * 3 ECG backward, 4 adjoint, 5 set-up/precompute), the summed milliseconds
 * and launch counts since the last reset.  n_classes <= 8. */
gbp_status gbp_enable_timing(gbp_ctx *ctx, int32_t on);
gbp_status gbp_get_kernel_times(gbp_ctx *ctx, int32_t n_classes, double *ms, int64_t *launches);
gbp_status gbp_reset_kernel_times(gbp_ctx *ctx);
/* Total kernels this context launched since creation. */
int64_t gbp_launch_count(gbp_ctx *ctx);

/* Per-iteration trace of the FIM: when enabled, each solve records, per
 * iteration, the number of active vertices and the GPU global timer (ns).
 * gbp_get_trace synchronises and copies up to max_rows rows (int64 pairs)
 * of the last solve into host memory `out`; returns the number of rows. */
gbp_status gbp_enable_trace(gbp_ctx *ctx, int32_t on);
int32_t gbp_get_trace(gbp_ctx *ctx, int64_t *out, int32_t max_rows);

#ifdef __cplusplus
}
#endif
#endif /* GBP_H */
