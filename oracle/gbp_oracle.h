/*
 * gbp_oracle.h -- plain FP64 CPU oracle for the Geodesic-BP hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA library; both read the same seeded
 * float32 input arrays.
 *
 * Conventions (identical on both sides because they are part of the problem
 * statement, not of the implementation):
 *   - xyz      float32 [n_v][3]
 *   - tets     int32   [n_t][4]
 *   - fib      float32 [n_t][3] fibre direction f (normalised here)
 *   - cf, ct   float32 [n_t] fibre / cross-fibre velocity.  The conduction
 *              tensor of Eq. (1) is M = ct^2 I + (cf^2 - ct^2) f f^T and the
 *              local metric is D = M^{-1} (Sec. II-A).
 *   - parent code of vertex i: tet*4 + slot, where slot is the position of i
 *     in tets[tet]; the face E_{j\i} is the tet's other three vertices in
 *     increasing slot order and alpha[3] refers to that order.  A vertex
 *     whose value is its onset value has code -1-k (onset k).  An unreached
 *     vertex has code INT32_MIN and phi = +inf.
 */
#ifndef GBP_ORACLE_H
#define GBP_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_EXACT = 0, ORC_FISTA = 1, ORC_FISTA_THEORY = 2 };
enum { ORC_ORDER_HEAP = 0, ORC_ORDER_FIFO = 1, ORC_ORDER_JACOBI = 2 };
enum { ORC_ONSET_NODAL = 0, ORC_ONSET_ELEMENT = 1 };

/* Local problem of Eq. (upwind_eq_lsqr) for n independent faces.
 * e[n][3][3]: rows are v_{j_m} - v_i.  Phi[n][3] may hold +inf.
 * mode ORC_EXACT: exact minimiser; ORC_FISTA: Algorithm 1 with n_f steps and
 * the Lipschitz constant of Eq. (lipschitz_est) (practical h_min/1.1 reading);
 * ORC_FISTA_THEORY: the same with the theoretical h_ = sigma_min(A)/(d sqrt d).
 * Writes value[n] and alpha[n][3]. */
void orc_local_batch(int64_t n, const float *e, const float *fib, const float *cf,
                     const float *ct, const float *Phi, int mode, int n_f,
                     double *value, double *alpha);

/* Lipschitz estimate of Eq. (lipschitz_est) per face, with the practical
 * lower bound h_min/1.1 (h_min = exact min of ||A alpha|| on the simplex)
 * and, in h_theory, the bound sigma_min(A)/(d sqrt d). */
void orc_lipschitz_batch(int64_t n, const float *e, const float *fib, const float *cf,
                         const float *ct, double *L, double *h_min, double *h_theory,
                         double *norm_G);

/* Discrete Hopf-Lax fixed point (Eq. hopflax_global / hopflax_local) by a
 * worklist (order HEAP or FIFO) or by the Jacobi sweeps of Algorithm 2
 * (order JACOBI), followed by a parent pass on the final values.
 * stats[0]=processed pops / sweeps, [1]=local solves, [2]=1e15*max fixed
 * point residual (relative), [3]=unreached vertices.  Returns 0 on success. */
int orc_eikonal(int64_t n_v, const float *xyz, int64_t n_t, const int32_t *tets,
                const float *cf, const float *ct, const float *fib,
                int onset_kind, int K, const int32_t *onset_idx,
                const float *onset_bary, const float *onset_t,
                int mode, int n_f, int order,
                double *phi, int32_t *parent, double *alpha, double *margin,
                int64_t *stats);

/* ECG of Sec. II-D: V[l][s] = sum_n L[l][n] U(t_s - phi_n),
 * U(xi) = K0 + (K1-K0)/2 (1 + tanh(2 xi / tau)),  t_s = t0 + s dt. */
void orc_ecg(int64_t n_v, int N, const float *L, const double *phi,
             double K0, double K1, double tau, double t0, double dt, int T,
             double *V);

/* Misfit of Eq. (inverse_ecg) (rectangle rule) and its derivative with
 * respect to every phi_n (Sec. II-D, nabla V = -B^T U' nabla phi).
 * Returns the loss; writes lam[n_v]. */
double orc_loss_grad_phi(int64_t n_v, int N, const float *L, const double *phi,
                         double K0, double K1, double tau, double t0, double dt, int T,
                         const double *V, const float *target, double *lam);

/* Frozen-graph adjoint (Eq. dto_grad, Eq. upwind_xi, conduction-tensor
 * variant of Sec. IV): mu = (I - P^T)^{-1} lam over the parent graph, solved
 * per strongly connected component in topological order (the graph can hold
 * short cycles).  Writes d_cf[n_t], d_ct[n_t], d_t[K], d_x[K][3] (element
 * onsets; zeros for nodal) and mu[n_v].  Returns the number of vertices whose
 * component could not be solved (0 in normal operation). */
int64_t orc_adjoint(int64_t n_v, const float *xyz, int64_t n_t, const int32_t *tets,
                    const float *cf, const float *ct, const float *fib,
                    int onset_kind, int K, const int32_t *onset_idx,
                    const float *onset_bary, const float *onset_t,
                    const int32_t *parent, const double *alpha, const double *lam,
                    double *d_cf, double *d_ct, double *d_t, double *d_x, double *mu);

int orc_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
