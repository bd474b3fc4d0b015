/*
 * gbp_oracle.c -- plain, slow, FP64 CPU oracle of the Geodesic-BP hot path
 * (Grandits et al., "Digital twinning of cardiac electrophysiology models
 * from the surface ECG: a geodesic backpropagation approach").
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg, never by the product path.  It shares no code
 * with the CUDA library.
 *
 * Every function states the passage it follows.  Readings of passages that are
 * silent or ambiguous are marked READING.  OpenMP is used only over
 * independent work (per vertex / per face / per lead).
 */
#include "gbp_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* small dense helpers                                                       */
/* ------------------------------------------------------------------------ */

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static void matvec3(double D[3][3], const double *w, double *out)
{
    for (int r = 0; r < 3; ++r) out[r] = D[r][0] * w[0] + D[r][1] * w[1] + D[r][2] * w[2];
}

/* ||w||_D = sqrt(<D w, w>)  (Sec. II-A). */
static double normD(double D[3][3], const double *w)
{
    double Dw[3];
    matvec3(D, w, Dw);
    double q = dot3(Dw, w);
    return sqrt(q > 0.0 ? q : 0.0);
}

/* Metric of element j: D_j = M_j^{-1} with the orthotropic conduction tensor
 * M = ct^2 I + (cf^2 - ct^2) f f^T for a unit fibre f (Eq. (1) and Sec. II-A:
 * "D = M^{-1}").  Its inverse is ct^-2 (I - f f^T) + cf^-2 f f^T. */
static void metric(double cf, double ct, const float *fibf, double D[3][3], double f[3])
{
    double n = sqrt((double)fibf[0] * fibf[0] + (double)fibf[1] * fibf[1] + (double)fibf[2] * fibf[2]);
    for (int r = 0; r < 3; ++r) f[r] = fibf[r] / n;
    double a = 1.0 / (ct * ct), b = 1.0 / (cf * cf) - 1.0 / (ct * ct);
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) D[r][c] = (r == c ? a : 0.0) + b * f[r] * f[c];
}

/* Objective of Eq. (upwind_eq_lsqr): <alpha, Phi> + ||sum_n alpha_n e_n||_D.
 * Terms with alpha_n == 0 are skipped so that Phi_n = +inf does not enter. */
static double objective(double e[3][3], double D[3][3], const double *Phi, const double *al)
{
    double w[3] = {0, 0, 0}, v = 0.0;
    for (int n = 0; n < 3; ++n) {
        if (al[n] == 0.0) continue;
        v += al[n] * Phi[n];
        for (int r = 0; r < 3; ++r) w[r] += al[n] * e[n][r];
    }
    return v + normD(D, w);
}

/* ------------------------------------------------------------------------ */
/* Local problem, exact (Sec. II-B, Eq. upwind_eq_lsqr)                      */
/* ------------------------------------------------------------------------ */
/*
 * The objective is convex on the simplex C_d (Sec. II-B: "each local problem
 * is convex"), so its minimum is attained at a KKT point: a stationary point
 * of the restriction to the relative interior of the whole face, of one of
 * its edges, or a vertex.  We enumerate all of them, keep the feasible ones
 * and evaluate the objective at each; the smallest value is the exact minimum.
 *
 * Edge (n,m), lambda = weight on n:  f = Phi_m + lambda delta + sqrt(q(lambda)),
 * q = A l^2 + 2 B l + C, A = |e_n - e_m|_D^2, B = <e_n-e_m, e_m>_D, C = |e_m|_D^2,
 * delta = Phi_n - Phi_m.  f' = 0 with S = C - B^2/A gives
 * sqrt(q) = sqrt(S A / (A - delta^2)) (needs A > delta^2) and
 * lambda = (-delta sqrt(q) - B) / A.
 *
 * Face: alpha_3 = 1 - b_1 - b_2, Q_ab = <e_a - e_3, e_b - e_3>_D,
 * q_a = <e_a - e_3, e_3>_D, r = |e_3|_D^2, Delta_a = Phi_a - Phi_3.
 * grad = 0 gives Q b + q = -h Delta with h = sqrt(S / (1 - Delta^T Q^-1 Delta)),
 * S = r - q^T Q^-1 q  (needs Delta^T Q^-1 Delta < 1), b = -Q^-1 (h Delta + q).
 */
static double local_exact(double e[3][3], double D[3][3], const double *Phi, double *alpha_out)
{
    double G[3][3];
    for (int a = 0; a < 3; ++a) {
        double De[3];
        matvec3(D, e[a], De);
        for (int b = 0; b < 3; ++b) G[a][b] = dot3(De, e[b]);
    }
    int fin[3];
    for (int n = 0; n < 3; ++n) fin[n] = isfinite(Phi[n]);

    double best = INFINITY, best_al[3] = {0, 0, 0};
    double al[3];
#define TRY_CANDIDATE()                                               \
    do {                                                              \
        double v_ = objective(e, D, Phi, al);                         \
        if (v_ < best) {                                              \
            best = v_;                                                \
            best_al[0] = al[0]; best_al[1] = al[1]; best_al[2] = al[2]; \
        }                                                             \
    } while (0)

    /* vertices */
    for (int n = 0; n < 3; ++n) {
        if (!fin[n]) continue;
        al[0] = al[1] = al[2] = 0.0;
        al[n] = 1.0;
        TRY_CANDIDATE();
    }
    /* edges */
    for (int n = 0; n < 3; ++n)
        for (int m = n + 1; m < 3; ++m) {
            if (!fin[n] || !fin[m]) continue;
            double A = G[n][n] - 2.0 * G[n][m] + G[m][m];
            double B = G[n][m] - G[m][m];
            double C = G[m][m];
            double delta = Phi[n] - Phi[m];
            if (!(A > delta * delta) || A <= 0.0) continue;
            double S = C - B * B / A;
            if (S < 0.0) S = 0.0;
            double h = sqrt(S * A / (A - delta * delta));
            double lam = (-delta * h - B) / A;
            if (!(lam > 0.0 && lam < 1.0)) continue;
            al[0] = al[1] = al[2] = 0.0;
            al[n] = lam;
            al[m] = 1.0 - lam;
            TRY_CANDIDATE();
        }
    /* interior of the face */
    if (fin[0] && fin[1] && fin[2]) {
        double d[2][3];
        for (int a = 0; a < 2; ++a)
            for (int r = 0; r < 3; ++r) d[a][r] = e[a][r] - e[2][r];
        double Q[2][2], q[2], r;
        for (int a = 0; a < 2; ++a) {
            double Dd[3];
            matvec3(D, d[a], Dd);
            for (int b = 0; b < 2; ++b) Q[a][b] = dot3(Dd, d[b]);
            q[a] = dot3(Dd, e[2]);
        }
        {
            double De3[3];
            matvec3(D, e[2], De3);
            r = dot3(De3, e[2]);
        }
        double det = Q[0][0] * Q[1][1] - Q[0][1] * Q[1][0];
        if (det > 0.0) {
            double Qi[2][2] = {{Q[1][1] / det, -Q[0][1] / det}, {-Q[1][0] / det, Q[0][0] / det}};
            double Dl[2] = {Phi[0] - Phi[2], Phi[1] - Phi[2]};
            double QiD[2] = {Qi[0][0] * Dl[0] + Qi[0][1] * Dl[1], Qi[1][0] * Dl[0] + Qi[1][1] * Dl[1]};
            double Qiq[2] = {Qi[0][0] * q[0] + Qi[0][1] * q[1], Qi[1][0] * q[0] + Qi[1][1] * q[1]};
            double k = Dl[0] * QiD[0] + Dl[1] * QiD[1];
            double S = r - (q[0] * Qiq[0] + q[1] * Qiq[1]);
            if (k < 1.0 && S > 0.0) {
                double h = sqrt(S / (1.0 - k));
                double b0 = -(h * QiD[0] + Qiq[0]);
                double b1 = -(h * QiD[1] + Qiq[1]);
                if (b0 > 0.0 && b1 > 0.0 && b0 + b1 < 1.0) {
                    al[0] = b0;
                    al[1] = b1;
                    al[2] = 1.0 - b0 - b1;
                    TRY_CANDIDATE();
                }
            }
        }
    }
#undef TRY_CANDIDATE
    if (alpha_out) {
        alpha_out[0] = best_al[0];
        alpha_out[1] = best_al[1];
        alpha_out[2] = best_al[2];
    }
    return best;
}

/* ------------------------------------------------------------------------ */
/* Local problem, FISTA (Algorithm 1) and the Lipschitz estimate             */
/* ------------------------------------------------------------------------ */

/* Euclidean projection onto the probability simplex of dimension k
 * (Duchi et al., Figure 1, the closed form cited after Eq. (fista_norm)):
 * sort descending, rho = max{j : u_j - (sum_{r<=j} u_r - 1)/j > 0},
 * theta = (sum_{r<=rho} u_r - 1)/rho, w = max(v - theta, 0). */
static void proj_simplex(int k, const double *v, double *w)
{
    double u[3];
    for (int i = 0; i < k; ++i) u[i] = v[i];
    for (int i = 0; i < k; ++i) /* insertion sort, descending */
        for (int j = i + 1; j < k; ++j)
            if (u[j] > u[i]) {
                double t = u[i];
                u[i] = u[j];
                u[j] = t;
            }
    double cs = 0.0, theta = 0.0;
    for (int j = 0; j < k; ++j) {
        cs += u[j];
        double t = (cs - 1.0) / (j + 1);
        if (u[j] - t > 0.0) theta = t;
    }
    for (int i = 0; i < k; ++i) w[i] = v[i] - theta > 0.0 ? v[i] - theta : 0.0;
}

/* Largest eigenvalue of a symmetric 3x3 matrix by cyclic Jacobi rotations. */
static double sym3_eig(double Ain[3][3], double *lmin)
{
    double A[3][3];
    memcpy(A, Ain, sizeof(A));
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
        if (off < 1e-300) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                if (fabs(A[p][q]) < 1e-300) continue;
                double th = 0.5 * (A[q][q] - A[p][p]) / A[p][q];
                double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < 3; ++k) { /* A <- A J */
                    double akp = A[k][p], akq = A[k][q];
                    A[k][p] = c * akp - s * akq;
                    A[k][q] = s * akp + c * akq;
                }
                for (int k = 0; k < 3; ++k) { /* A <- J^T A */
                    double apk = A[p][k], aqk = A[q][k];
                    A[p][k] = c * apk - s * aqk;
                    A[q][k] = s * apk + c * aqk;
                }
            }
    }
    double mx = A[0][0], mn = A[0][0];
    for (int i = 1; i < 3; ++i) {
        if (A[i][i] > mx) mx = A[i][i];
        if (A[i][i] < mn) mn = A[i][i];
    }
    if (lmin) *lmin = mn;
    return mx;
}

/* Eq. (lipschitz_est): L <= ||A^T A|| / h_ (1 + ||A|| / h_), with
 * ||A^T A|| = lambda_max(G), ||A|| = sqrt(lambda_max(G)), G = A^T A = E^T D E.
 * READING (Sec. II-E, "in practice"): h_ = h(alpha*)/1.1 with alpha* the
 * minimiser of ||A alpha|| over the simplex (Phi = 0); we take the exact
 * minimiser.  Also returns the theoretical h_ = sigma_min(A)/(d sqrt d). */
static double lipschitz(double e[3][3], double D[3][3], double *h_min, double *h_theory, double *normG)
{
    double G[3][3];
    for (int a = 0; a < 3; ++a) {
        double De[3];
        matvec3(D, e[a], De);
        for (int b = 0; b < 3; ++b) G[a][b] = dot3(De, e[b]);
    }
    double lmin;
    double lmax = sym3_eig(G, &lmin);
    double zero[3] = {0, 0, 0};
    double hm = local_exact(e, D, zero, NULL);
    double hlow = hm / 1.1;
    if (h_min) *h_min = hm;
    if (h_theory) *h_theory = sqrt(lmin > 0 ? lmin : 0) / (3.0 * sqrt(3.0));
    if (normG) *normG = lmax;
    return lmax / hlow * (1.0 + sqrt(lmax) / hlow);
}

/* Algorithm 1 (FISTA with beta_k = (k-1)/(k+1)) on the sub-face of finite
 * vertex values.  READINGS: alpha_0 = hat alpha_0 (Alg. 1 uses alpha_{k-1}
 * at k = 1); vertices with Phi = +inf are dropped (alpha = 0), since the
 * iteration is undefined with infinite entries. */
static double local_fista(double e[3][3], double D[3][3], const double *Phi, double L, int n_f,
                          double *alpha_out)
{
    int idx[3], k = 0;
    for (int n = 0; n < 3; ++n)
        if (isfinite(Phi[n])) idx[k++] = n;
    double al[3] = {0, 0, 0};
    if (k == 0) {
        if (alpha_out) alpha_out[0] = alpha_out[1] = alpha_out[2] = 0.0;
        return INFINITY;
    }
    if (k == 1) {
        al[idx[0]] = 1.0;
        if (alpha_out) memcpy(alpha_out, al, sizeof(al));
        return objective(e, D, Phi, al);
    }
    double G[3][3];
    for (int a = 0; a < 3; ++a) {
        double De[3];
        matvec3(D, e[a], De);
        for (int b = 0; b < 3; ++b) G[a][b] = dot3(De, e[b]);
    }
    double hat[3], prev[3], cur[3], ph[3];
    for (int i = 0; i < k; ++i) {
        hat[i] = 1.0 / k;
        prev[i] = hat[i];
        cur[i] = hat[i];
        ph[i] = Phi[idx[i]];
    }
    for (int it = 1; it <= n_f; ++it) {
        double y[3], h2 = 0.0;
        for (int a = 0; a < k; ++a) {
            y[a] = 0.0;
            for (int b = 0; b < k; ++b) y[a] += G[idx[a]][idx[b]] * hat[b];
            h2 += hat[a] * y[a];
        }
        double h = sqrt(h2); /* h = ||A hat alpha|| */
        double til[3];
        for (int a = 0; a < k; ++a) til[a] = (hat[a] - (y[a] / h) / L) - ph[a] / L;
        proj_simplex(k, til, cur);
        double beta = (double)(it - 1) / (double)(it + 1);
        for (int a = 0; a < k; ++a) {
            hat[a] = cur[a] + beta * (cur[a] - prev[a]);
            prev[a] = cur[a];
        }
    }
    for (int i = 0; i < k; ++i) al[idx[i]] = cur[i];
    if (alpha_out) memcpy(alpha_out, al, sizeof(al));
    return objective(e, D, Phi, al);
}

/* ------------------------------------------------------------------------ */
/* batch entry points for local-solver tests                                 */
/* ------------------------------------------------------------------------ */

static void load_face(const float *e, double E[3][3])
{
    for (int a = 0; a < 3; ++a)
        for (int r = 0; r < 3; ++r) E[a][r] = e[a * 3 + r];
}

void orc_local_batch(int64_t n, const float *e, const float *fib, const float *cf, const float *ct,
                     const float *Phi, int mode, int n_f, double *value, double *alpha)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double E[3][3], D[3][3], f[3], P[3];
        load_face(e + 9 * i, E);
        metric(cf[i], ct[i], fib + 3 * i, D, f);
        for (int a = 0; a < 3; ++a) P[a] = Phi[3 * i + a];
        if (mode == ORC_FISTA) {
            double L = lipschitz(E, D, NULL, NULL, NULL);
            value[i] = local_fista(E, D, P, L, n_f, alpha + 3 * i);
        } else if (mode == ORC_FISTA_THEORY) {
            /* Eq. (lipschitz_est) with the theoretical h_ = sigma_min(A)/(d sqrt d),
             * valid on the whole plane <alpha, 1> = 1 where the iterates live */
            double ht, nG;
            lipschitz(E, D, NULL, &ht, &nG);
            double L = nG / ht * (1.0 + sqrt(nG) / ht);
            value[i] = local_fista(E, D, P, L, n_f, alpha + 3 * i);
        } else {
            value[i] = local_exact(E, D, P, alpha + 3 * i);
        }
    }
}

void orc_lipschitz_batch(int64_t n, const float *e, const float *fib, const float *cf, const float *ct,
                         double *L, double *h_min, double *h_theory, double *norm_G)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double E[3][3], D[3][3], f[3];
        load_face(e + 9 * i, E);
        metric(cf[i], ct[i], fib + 3 * i, D, f);
        L[i] = lipschitz(E, D, h_min + i, h_theory + i, norm_G + i);
    }
}

/* ------------------------------------------------------------------------ */
/* Eikonal: discrete Hopf-Lax fixed point                                     */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t n_v, n_t;
    const float *xyz;
    const int32_t *tets;
    double (*D)[3][3];    /* per tet metric */
    double (*f)[3];       /* per tet unit fibre */
    int64_t *adj_ptr;     /* vertex -> (tet*4+slot) */
    int32_t *adj;
    int mode, n_f;
    double *Lf;           /* per tet*4+slot Lipschitz constant (FISTA) */
} mesh_t;

static int mesh_init(mesh_t *m, int64_t n_v, const float *xyz, int64_t n_t, const int32_t *tets,
                     const float *cf, const float *ct, const float *fib, int mode, int n_f)
{
    memset(m, 0, sizeof(*m));
    m->n_v = n_v;
    m->n_t = n_t;
    m->xyz = xyz;
    m->tets = tets;
    m->mode = mode;
    m->n_f = n_f;
    m->D = malloc(sizeof(double[3][3]) * (size_t)(n_t > 0 ? n_t : 1));
    m->f = malloc(sizeof(double[3]) * (size_t)(n_t > 0 ? n_t : 1));
    m->adj_ptr = calloc((size_t)n_v + 1, sizeof(int64_t));
    m->adj = malloc(sizeof(int32_t) * (size_t)(4 * n_t > 0 ? 4 * n_t : 1));
    if (!m->D || !m->f || !m->adj_ptr || !m->adj) return -1;
    for (int64_t j = 0; j < n_t; ++j) metric(cf[j], ct[j], fib + 3 * j, m->D[j], m->f[j]);
    for (int64_t j = 0; j < n_t; ++j)
        for (int s = 0; s < 4; ++s) m->adj_ptr[tets[4 * j + s] + 1]++;
    for (int64_t i = 0; i < n_v; ++i) m->adj_ptr[i + 1] += m->adj_ptr[i];
    int64_t *cur = malloc(sizeof(int64_t) * (size_t)(n_v > 0 ? n_v : 1));
    if (!cur) return -1;
    memcpy(cur, m->adj_ptr, sizeof(int64_t) * (size_t)n_v);
    for (int64_t j = 0; j < n_t; ++j)
        for (int s = 0; s < 4; ++s) m->adj[cur[tets[4 * j + s]]++] = (int32_t)(4 * j + s);
    free(cur);
    if (mode == ORC_FISTA) {
        m->Lf = malloc(sizeof(double) * (size_t)(4 * n_t > 0 ? 4 * n_t : 1));
        if (!m->Lf) return -1;
#pragma omp parallel for schedule(static)
        for (int64_t c = 0; c < 4 * n_t; ++c) {
            int64_t j = c >> 2;
            int s = (int)(c & 3);
            double E[3][3];
            int a = 0;
            const int32_t *t = tets + 4 * j;
            for (int q = 0; q < 4; ++q) {
                if (q == s) continue;
                for (int r = 0; r < 3; ++r) E[a][r] = (double)xyz[3 * t[q] + r] - (double)xyz[3 * t[s] + r];
                ++a;
            }
            m->Lf[c] = lipschitz(E, m->D[j], NULL, NULL, NULL);
        }
    }
    return 0;
}

static void mesh_free(mesh_t *m)
{
    free(m->D);
    free(m->f);
    free(m->adj_ptr);
    free(m->adj);
    free(m->Lf);
}

/* phi_{j\i} of Eq. (hopflax_local) for the face of tet j opposite slot s. */
static double face_value(const mesh_t *m, int64_t j, int s, const double *phi, double *alpha)
{
    const int32_t *t = m->tets + 4 * j;
    double E[3][3], P[3];
    int a = 0;
    for (int q = 0; q < 4; ++q) {
        if (q == s) continue;
        for (int r = 0; r < 3; ++r) E[a][r] = (double)m->xyz[3 * t[q] + r] - (double)m->xyz[3 * t[s] + r];
        P[a] = phi[t[q]];
        ++a;
    }
    if (!isfinite(P[0]) && !isfinite(P[1]) && !isfinite(P[2])) {
        if (alpha) alpha[0] = alpha[1] = alpha[2] = 0.0;
        return INFINITY;
    }
    if (m->mode == ORC_FISTA) return local_fista(E, m->D[j], P, m->Lf[4 * j + s], m->n_f, alpha);
    return local_exact(E, m->D[j], P, alpha);
}

/* Onset values (Alg. 2 initialisation and Eq. upwind_xi).  Nodal onsets set
 * phi(x_i) = t_i.  An element onset inside tet E sets, for each vertex v of
 * E, t_i + ||v - x_i||_{D_E}.  The smallest value wins, ties to the smaller
 * onset index. */
static void onset_values(const mesh_t *m, int kind, int K, const int32_t *idx, const float *bary,
                         const float *t, double *phi0, int32_t *root)
{
    for (int64_t i = 0; i < m->n_v; ++i) {
        phi0[i] = INFINITY;
        root[i] = -1;
    }
    for (int k = 0; k < K; ++k) {
        if (kind == ORC_ONSET_NODAL) {
            int64_t v = idx[k];
            if ((double)t[k] < phi0[v]) {
                phi0[v] = t[k];
                root[v] = k;
            }
        } else {
            const int32_t *tt = m->tets + 4 * (int64_t)idx[k];
            double x[3] = {0, 0, 0};
            for (int q = 0; q < 4; ++q)
                for (int r = 0; r < 3; ++r) x[r] += (double)bary[4 * k + q] * (double)m->xyz[3 * tt[q] + r];
            for (int q = 0; q < 4; ++q) {
                double w[3];
                for (int r = 0; r < 3; ++r) w[r] = (double)m->xyz[3 * tt[q] + r] - x[r];
                double val = (double)t[k] + normD(m->D[idx[k]], w);
                if (val < phi0[tt[q]]) {
                    phi0[tt[q]] = val;
                    root[tt[q]] = k;
                }
            }
        }
    }
}

/* binary min-heap of (value, vertex) with lazy deletion */
typedef struct {
    double *key;
    int64_t *val;
    int64_t n, cap;
} heap_t;

static int heap_push(heap_t *h, double k, int64_t v)
{
    if (h->n == h->cap) {
        int64_t nc = h->cap ? 2 * h->cap : 1024;
        double *nk = realloc(h->key, sizeof(double) * (size_t)nc);
        if (!nk) return -1;
        h->key = nk;
        int64_t *nv = realloc(h->val, sizeof(int64_t) * (size_t)nc);
        if (!nv) return -1;
        h->val = nv;
        h->cap = nc;
    }
    int64_t i = h->n++;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (h->key[p] <= k) break;
        h->key[i] = h->key[p];
        h->val[i] = h->val[p];
        i = p;
    }
    h->key[i] = k;
    h->val[i] = v;
    return 0;
}

static void heap_pop(heap_t *h, double *k, int64_t *v)
{
    *k = h->key[0];
    *v = h->val[0];
    double lk = h->key[--h->n];
    int64_t lv = h->val[h->n];
    int64_t i = 0;
    for (;;) {
        int64_t c = 2 * i + 1;
        if (c >= h->n) break;
        if (c + 1 < h->n && h->key[c + 1] < h->key[c]) c++;
        if (h->key[c] >= lk) break;
        h->key[i] = h->key[c];
        h->val[i] = h->val[c];
        i = c;
    }
    if (h->n > 0) {
        h->key[i] = lk;
        h->val[i] = lv;
    }
}

/* a decrease counts only beyond a relative 1e-13 (termination in FP64) */
static int improves(double val, double cur)
{
    if (!isfinite(cur)) return isfinite(val);
    return val < cur - 1e-13 * (fabs(cur) > 1.0 ? fabs(cur) : 1.0);
}

int orc_eikonal(int64_t n_v, const float *xyz, int64_t n_t, const int32_t *tets, const float *cf,
                const float *ct, const float *fib, int onset_kind, int K, const int32_t *onset_idx,
                const float *onset_bary, const float *onset_t, int mode, int n_f, int order,
                double *phi, int32_t *parent, double *alpha, double *margin, int64_t *stats)
{
    mesh_t m;
    if (mesh_init(&m, n_v, xyz, n_t, tets, cf, ct, fib, mode, n_f)) return -1;
    double *phi0 = malloc(sizeof(double) * (size_t)n_v);
    int32_t *root = malloc(sizeof(int32_t) * (size_t)n_v);
    if (!phi0 || !root) return -1;
    onset_values(&m, onset_kind, K, onset_idx, onset_bary, onset_t, phi0, root);
    for (int64_t i = 0; i < n_v; ++i) phi[i] = phi0[i];
    int64_t pops = 0, solves = 0;

    if (order == ORC_ORDER_HEAP || order == ORC_ORDER_FIFO) {
        /* Worklist Gauss-Seidel on Eq. (hopflax_global): when vertex c
         * changes, every face E_{j\i} containing c is re-solved and phi_i
         * lowered if the face value is smaller.  The operator is monotone,
         * so any order reaches the same (maximal) fixed point. */
        heap_t h = {0};
        int64_t *fifo = NULL, fhead = 0, ftail = 0, fcap = 0;
        char *inq = NULL;
        if (order == ORC_ORDER_FIFO) {
            fcap = n_v + 1;
            fifo = malloc(sizeof(int64_t) * (size_t)fcap);
            inq = calloc((size_t)n_v, 1);
            if (!fifo || !inq) return -1;
        }
        for (int64_t i = 0; i < n_v; ++i)
            if (isfinite(phi[i])) {
                if (order == ORC_ORDER_HEAP) {
                    if (heap_push(&h, phi[i], i)) return -1;
                } else {
                    fifo[ftail] = i;
                    ftail = (ftail + 1) % fcap;
                    inq[i] = 1;
                }
            }
        for (;;) {
            int64_t c;
            if (order == ORC_ORDER_HEAP) {
                if (h.n == 0) break;
                double kc;
                heap_pop(&h, &kc, &c);
                if (kc != phi[c]) continue; /* stale entry */
            } else {
                if (fhead == ftail) break;
                c = fifo[fhead];
                fhead = (fhead + 1) % fcap;
                inq[c] = 0;
            }
            ++pops;
            for (int64_t p = m.adj_ptr[c]; p < m.adj_ptr[c + 1]; ++p) {
                int64_t j = m.adj[p] >> 2;
                int sc = m.adj[p] & 3;
                for (int s = 0; s < 4; ++s) {
                    if (s == sc) continue;
                    int64_t i = tets[4 * j + s];
                    double val = face_value(&m, j, s, phi, NULL);
                    ++solves;
                    if (improves(val, phi[i])) {
                        phi[i] = val;
                        if (order == ORC_ORDER_HEAP) {
                            if (heap_push(&h, val, i)) return -1;
                        } else if (!inq[i]) {
                            fifo[ftail] = i;
                            ftail = (ftail + 1) % fcap;
                            inq[i] = 1;
                        }
                    }
                }
            }
        }
        free(h.key);
        free(h.val);
        free(fifo);
        free(inq);
    } else {
        /* Algorithm 2, literally: Jacobi sweeps reading phi_{k-1}, updating
         * every face that has a vertex changed in the previous sweep
         * (the optional mask), phi_k(v_i) = min(phi_{k-1}(v_i), min_j
         * phi_{j\i}) and stopping when no vertex changes.
         * READING: phi_{-1} = +inf everywhere, so the onsets form the first
         * changed set; the global update keeps the current value. */
        double *old = malloc(sizeof(double) * (size_t)n_v);
        char *chg = malloc((size_t)n_v), *nchg = malloc((size_t)n_v);
        if (!old || !chg || !nchg) return -1;
        for (int64_t i = 0; i < n_v; ++i) chg[i] = isfinite(phi[i]) ? 1 : 0;
        for (;;) {
            memcpy(old, phi, sizeof(double) * (size_t)n_v);
            memset(nchg, 0, (size_t)n_v);
            ++pops;
            int any = 0;
            for (int64_t j = 0; j < n_t; ++j)
                for (int s = 0; s < 4; ++s) {
                    int need = 0;
                    for (int q = 0; q < 4; ++q)
                        if (q != s && chg[tets[4 * j + q]]) need = 1;
                    if (!need) continue;
                    int64_t i = tets[4 * j + s];
                    double val = face_value(&m, j, s, old, NULL);
                    ++solves;
                    if (improves(val, phi[i])) {
                        phi[i] = val;
                        nchg[i] = 1;
                        any = 1;
                    }
                }
            memcpy(chg, nchg, (size_t)n_v);
            if (!any) break;
        }
        free(old);
        free(chg);
        free(nchg);
    }

    /* Parent pass: with the final values, the parent of vertex i is the face
     * (or onset) attaining the minimum of Eq. (hopflax_global); alpha is the
     * minimiser used by Eq. (dto_grad).  Ties within 1e-12 (relative) go to
     * the smallest code (onsets first).  margin = gap to the best candidate
     * with a different code. */
    double maxres = 0.0;
    int64_t unreached = 0;
    int64_t maxdeg = 0;
    for (int64_t i = 0; i < n_v; ++i)
        if (m.adj_ptr[i + 1] - m.adj_ptr[i] > maxdeg) maxdeg = m.adj_ptr[i + 1] - m.adj_ptr[i];
#pragma omp parallel reduction(max : maxres) reduction(+ : unreached)
    {
        double *cv = malloc(sizeof(double) * (size_t)(maxdeg + 1));
        double *ca = malloc(sizeof(double) * 3 * (size_t)(maxdeg + 1));
        int64_t *cc = malloc(sizeof(int64_t) * (size_t)(maxdeg + 1));
#pragma omp for schedule(dynamic, 256)
        for (int64_t i = 0; i < n_v; ++i) {
            /* candidates: the onset value (if any) and every face of i */
            int nc = 0;
            if (isfinite(phi0[i])) {
                cv[nc] = phi0[i];
                cc[nc] = -1 - root[i];
                ca[3 * nc] = ca[3 * nc + 1] = ca[3 * nc + 2] = 0.0;
                ++nc;
            }
            for (int64_t p = m.adj_ptr[i]; p < m.adj_ptr[i + 1]; ++p) {
                int64_t j = m.adj[p] >> 2;
                int s = m.adj[p] & 3;
                double val = face_value(&m, j, s, phi, ca + 3 * nc);
                if (!isfinite(val)) continue;
                cv[nc] = val;
                cc[nc] = 4 * j + s;
                ++nc;
            }
            if (nc == 0) {
                parent[i] = INT32_MIN;
                alpha[3 * i] = alpha[3 * i + 1] = alpha[3 * i + 2] = 0.0;
                margin[i] = INFINITY;
                phi[i] = INFINITY;
                unreached++;
                continue;
            }
            double bv = INFINITY;
            for (int q = 0; q < nc; ++q)
                if (cv[q] < bv) bv = cv[q];
            double tol = 1e-12 * (fabs(bv) > 1.0 ? fabs(bv) : 1.0);
            int bq = -1;
            for (int q = 0; q < nc; ++q)
                if (cv[q] <= bv + tol && (bq < 0 || cc[q] < cc[bq])) bq = q;
            double sv = INFINITY;
            for (int q = 0; q < nc; ++q)
                if (q != bq && cv[q] < sv) sv = cv[q];
            parent[i] = (int32_t)cc[bq];
            memcpy(alpha + 3 * i, ca + 3 * bq, 3 * sizeof(double));
            margin[i] = sv - cv[bq];
            double res = fabs(phi[i] - bv) / (fabs(bv) > 1.0 ? fabs(bv) : 1.0);
            if (res > maxres) maxres = res;
        }
        free(cv);
        free(ca);
        free(cc);
    }
    if (stats) {
        stats[0] = pops;
        stats[1] = solves;
        stats[2] = (int64_t)(maxres * 1e15);
        stats[3] = unreached;
    }
    free(phi0);
    free(root);
    mesh_free(&m);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* ECG and misfit (Sec. II-D)                                                */
/* ------------------------------------------------------------------------ */

/* Eq. (tanh_waveform).  READING: K0 + (K1-K0)/2 (1 + tanh(2 xi / tau)) so
 * that U spans [K0, K1] as the text says (minimum and maximum). */
static double U_tmpl(double xi, double K0, double K1, double tau)
{
    return K0 + 0.5 * (K1 - K0) * (1.0 + tanh(2.0 * xi / tau));
}

static double dU_tmpl(double xi, double K0, double K1, double tau)
{
    double th = tanh(2.0 * xi / tau);
    return 0.5 * (K1 - K0) * (2.0 / tau) * (1.0 - th * th);
}

void orc_ecg(int64_t n_v, int N, const float *L, const double *phi, double K0, double K1, double tau,
             double t0, double dt, int T, double *V)
{
    /* V_l(t) = (B U(t - phi))_l, B the lead-field operator (Sec. II-D).
     * READING: B is N x n_v (one row per lead). */
#pragma omp parallel for collapse(2) schedule(static)
    for (int l = 0; l < N; ++l)
        for (int s = 0; s < T; ++s) {
            double ts = t0 + s * dt, acc = 0.0;
            const float *Ll = L + (int64_t)l * n_v;
            for (int64_t n = 0; n < n_v; ++n) {
                double u = isfinite(phi[n]) ? U_tmpl(ts - phi[n], K0, K1, tau) : K0;
                acc += (double)Ll[n] * u;
            }
            V[(int64_t)l * T + s] = acc;
        }
}

double orc_loss_grad_phi(int64_t n_v, int N, const float *L, const double *phi, double K0, double K1,
                         double tau, double t0, double dt, int T, const double *V, const float *target,
                         double *lam)
{
    /* Eq. (inverse_ecg), READING: the time integral is the rectangle rule
     * over the T samples, loss = 1/(N T) sum_l sum_s r_l(s)^2. */
    double loss = 0.0;
    double *r = malloc(sizeof(double) * (size_t)N * (size_t)T);
    if (!r) return NAN;
    for (int64_t q = 0; q < (int64_t)N * T; ++q) {
        r[q] = V[q] - (double)target[q];
        loss += r[q] * r[q];
    }
    loss /= (double)N * (double)T;
    /* d loss / d phi_n = 2/(N T) sum_{l,s} r_l(s) L_ln dU(t_s - phi_n)/dphi_n
     *                  = -2/(N T) sum_s U'(t_s - phi_n) sum_l L_ln r_l(s). */
#pragma omp parallel for schedule(static)
    for (int64_t n = 0; n < n_v; ++n) {
        if (!isfinite(phi[n])) {
            lam[n] = 0.0;
            continue;
        }
        double acc = 0.0;
        for (int s = 0; s < T; ++s) {
            double c = 0.0;
            for (int l = 0; l < N; ++l) c += (double)L[(int64_t)l * n_v + n] * r[(int64_t)l * T + s];
            acc += dU_tmpl(t0 + s * dt - phi[n], K0, K1, tau) * c;
        }
        lam[n] = -2.0 / ((double)N * (double)T) * acc;
    }
    free(r);
    return loss;
}

/* ------------------------------------------------------------------------ */
/* Frozen-graph adjoint (Sec. II-C and the conduction-tensor remark, Sec. IV) */
/* ------------------------------------------------------------------------ */
/*
 * For a vertex with face parent (j, slot): phi_i = <alpha, Phi> + ||w||_{D_j},
 * w = v_i - sum_n alpha_n v_{j_n}, alpha frozen (first variation, Sec. II-C),
 * so d phi_i / d phi_{j_n} = alpha_n (Eq. dto_grad) and, with
 * ||w||_D^2 = ct^-2 (|w|^2 - (f.w)^2) + cf^-2 (f.w)^2,
 *   d phi_i / d cf_j = -(f.w)^2 / (cf^3 ||w||_D),
 *   d phi_i / d ct_j = -(|w|^2 - (f.w)^2) / (ct^3 ||w||_D).
 * For an onset vertex: d phi / d t_k = 1 and, for an element onset,
 * phi_v = t_k + ||v - x_k||_{D_E} (Eq. upwind_xi) gives
 * d phi_v / d x_k = -D_E (v - x_k) / ||v - x_k||_{D_E} and the two velocity
 * derivatives above with w = v - x_k, charged to E.
 *
 * With P[i][n] = d phi_i / d phi_n, the adjoint variable is
 * mu = (I - P^T)^{-1} lam.  The parent graph of the discrete fixed point can
 * contain short cycles (non-causal updates in anisotropic elements), so mu is
 * obtained per strongly connected component (Tarjan), components in
 * topological order (children before parents), each by a dense solve.
 */

/* per-vertex local sensitivities of phi_i with respect to its own parent's
 * parameters, accumulated with weight m into the gradients */
static void accumulate_local(int64_t i, double m, const float *xyz, const int32_t *tets,
                             const float *cf, const float *ct, const float *fib, int onset_kind,
                             const int32_t *onset_idx, const float *onset_bary, const int32_t *parent,
                             const double *alpha, double *d_cf, double *d_ct, double *d_t, double *d_x)
{
    int32_t c = parent[i];
    double vi[3] = {xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2]};
    if (c >= 0) {
        int64_t j = c >> 2;
        int s = c & 3, a = 0;
        double D[3][3], f[3], w[3] = {vi[0], vi[1], vi[2]};
        metric(cf[j], ct[j], fib + 3 * j, D, f);
        for (int q = 0; q < 4; ++q) {
            if (q == s) continue;
            int64_t v = tets[4 * j + q];
            for (int r = 0; r < 3; ++r) w[r] -= alpha[3 * i + a] * (double)xyz[3 * v + r];
            ++a;
        }
        double g = normD(D, w);
        if (g > 0.0) {
            double fw = dot3(f, w), ww = dot3(w, w);
            d_cf[j] += m * (-(fw * fw) / ((double)cf[j] * cf[j] * cf[j] * g));
            d_ct[j] += m * (-(ww - fw * fw) / ((double)ct[j] * ct[j] * ct[j] * g));
        }
    } else {
        int k = -1 - c;
        d_t[k] += m;
        if (onset_kind == ORC_ONSET_ELEMENT) {
            int64_t E = onset_idx[k];
            const int32_t *tt = tets + 4 * E;
            double x[3] = {0, 0, 0};
            for (int q = 0; q < 4; ++q)
                for (int r = 0; r < 3; ++r) x[r] += (double)onset_bary[4 * k + q] * (double)xyz[3 * tt[q] + r];
            double D[3][3], f[3], w[3];
            metric(cf[E], ct[E], fib + 3 * E, D, f);
            for (int r = 0; r < 3; ++r) w[r] = vi[r] - x[r];
            double g = normD(D, w);
            if (g > 0.0) {
                double Dw[3];
                matvec3(D, w, Dw);
                for (int r = 0; r < 3; ++r) d_x[3 * k + r] += m * (-Dw[r] / g);
                double fw = dot3(f, w), ww = dot3(w, w);
                d_cf[E] += m * (-(fw * fw) / ((double)cf[E] * cf[E] * cf[E] * g));
                d_ct[E] += m * (-(ww - fw * fw) / ((double)ct[E] * ct[E] * ct[E] * g));
            }
        }
    }
}

/* parent vertices of i with nonzero weight: returns count, fills out/w */
static int parent_edges(int64_t i, const int32_t *tets, const int32_t *parent, const double *alpha,
                        int64_t *out, double *w)
{
    int32_t c = parent[i];
    if (c < 0) return 0;
    int64_t j = c >> 2;
    int s = c & 3, a = 0, k = 0;
    for (int q = 0; q < 4; ++q) {
        if (q == s) continue;
        if (alpha[3 * i + a] != 0.0) {
            out[k] = tets[4 * j + q];
            w[k] = alpha[3 * i + a];
            ++k;
        }
        ++a;
    }
    return k;
}

/* dense Gaussian elimination with partial pivoting, A is k x k row-major */
static int dense_solve(int k, double *A, double *b)
{
    for (int c = 0; c < k; ++c) {
        int p = c;
        for (int r = c + 1; r < k; ++r)
            if (fabs(A[r * k + c]) > fabs(A[p * k + c])) p = r;
        if (A[p * k + c] == 0.0) return -1;
        if (p != c) {
            for (int q = 0; q < k; ++q) {
                double t = A[c * k + q];
                A[c * k + q] = A[p * k + q];
                A[p * k + q] = t;
            }
            double t = b[c];
            b[c] = b[p];
            b[p] = t;
        }
        for (int r = c + 1; r < k; ++r) {
            double f = A[r * k + c] / A[c * k + c];
            if (f == 0.0) continue;
            for (int q = c; q < k; ++q) A[r * k + q] -= f * A[c * k + q];
            b[r] -= f * b[c];
        }
    }
    for (int c = k - 1; c >= 0; --c) {
        double s = b[c];
        for (int q = c + 1; q < k; ++q) s -= A[c * k + q] * b[q];
        b[c] = s / A[c * k + c];
    }
    return 0;
}

int64_t orc_adjoint(int64_t n_v, const float *xyz, int64_t n_t, const int32_t *tets, const float *cf,
                    const float *ct, const float *fib, int onset_kind, int K, const int32_t *onset_idx,
                    const float *onset_bary, const float *onset_t, const int32_t *parent,
                    const double *alpha, const double *lam, double *d_cf, double *d_ct, double *d_t,
                    double *d_x, double *mu)
{
    (void)onset_t;
    for (int64_t j = 0; j < n_t; ++j) d_cf[j] = d_ct[j] = 0.0;
    for (int k = 0; k < K; ++k) {
        d_t[k] = 0.0;
        d_x[3 * k] = d_x[3 * k + 1] = d_x[3 * k + 2] = 0.0;
    }
    for (int64_t i = 0; i < n_v; ++i) mu[i] = lam[i];

    /* Tarjan's SCC algorithm (iterative) on edges child -> parent vertex.
     * Components are emitted sinks first; processing must go sources first
     * (a child is finished before any of its parents), so the emitted order
     * is stored and walked backwards. */
    int64_t *index = malloc(sizeof(int64_t) * (size_t)n_v);
    int64_t *low = malloc(sizeof(int64_t) * (size_t)n_v);
    char *onstack = calloc((size_t)n_v, 1);
    int64_t *stack = malloc(sizeof(int64_t) * (size_t)n_v);
    int64_t *cs_node = malloc(sizeof(int64_t) * (size_t)n_v);
    int *cs_edge = malloc(sizeof(int) * (size_t)n_v);
    int64_t *order = malloc(sizeof(int64_t) * (size_t)n_v);   /* vertices, by component */
    int64_t *comp_end = malloc(sizeof(int64_t) * (size_t)(n_v + 1));
    int64_t *comp_of = malloc(sizeof(int64_t) * (size_t)n_v);
    if (!index || !low || !onstack || !stack || !cs_node || !cs_edge || !order || !comp_end || !comp_of)
        return -1;
    for (int64_t i = 0; i < n_v; ++i) index[i] = -1;
    int64_t counter = 0, sp = 0, csp = 0, no = 0, ncomp = 0;
    for (int64_t r = 0; r < n_v; ++r) {
        if (index[r] >= 0 || parent[r] == INT32_MIN) continue;
        cs_node[csp] = r;
        cs_edge[csp] = 0;
        ++csp;
        index[r] = low[r] = counter++;
        stack[sp++] = r;
        onstack[r] = 1;
        while (csp > 0) {
            int64_t v = cs_node[csp - 1];
            int64_t nb[3];
            double wt[3];
            int ne = parent_edges(v, tets, parent, alpha, nb, wt);
            if (cs_edge[csp - 1] < ne) {
                int64_t u = nb[cs_edge[csp - 1]++];
                if (index[u] < 0) {
                    index[u] = low[u] = counter++;
                    stack[sp++] = u;
                    onstack[u] = 1;
                    cs_node[csp] = u;
                    cs_edge[csp] = 0;
                    ++csp;
                } else if (onstack[u] && index[u] < low[v]) {
                    low[v] = index[u];
                }
                continue;
            }
            /* v finished */
            --csp;
            if (csp > 0) {
                int64_t p = cs_node[csp - 1];
                if (low[v] < low[p]) low[p] = low[v];
            }
            if (low[v] == index[v]) {
                int64_t w;
                do {
                    w = stack[--sp];
                    onstack[w] = 0;
                    comp_of[w] = ncomp;
                    order[no++] = w;
                } while (w != v);
                comp_end[ncomp++] = no;
            }
        }
    }
    free(index);
    free(low);
    free(onstack);
    free(stack);
    free(cs_node);
    free(cs_edge);

    int64_t unsolved = 0;
    double *A = NULL, *b = NULL;
    int64_t acap = 0;
    for (int64_t c = ncomp - 1; c >= 0; --c) {
        int64_t beg = c > 0 ? comp_end[c - 1] : 0, end = comp_end[c];
        int64_t k = end - beg;
        if (k > 1) {
            /* (I - A_S) mu_S = r_S, A_S[i][c] = alpha_{c -> i} for c, i in S */
            if (k > 4096) {
                unsolved += k;
                continue;
            }
            if (k * k > acap) {
                acap = k * k;
                free(A);
                free(b);
                A = malloc(sizeof(double) * (size_t)acap);
                b = malloc(sizeof(double) * (size_t)k);
                if (!A || !b) return -1;
            }
            memset(A, 0, sizeof(double) * (size_t)(k * k));
            for (int64_t a = 0; a < k; ++a) {
                A[a * k + a] = 1.0;
                b[a] = mu[order[beg + a]];
            }
            for (int64_t a = 0; a < k; ++a) {
                int64_t v = order[beg + a];
                int64_t nb[3];
                double wt[3];
                int ne = parent_edges(v, tets, parent, alpha, nb, wt);
                for (int e = 0; e < ne; ++e) {
                    if (comp_of[nb[e]] != c) continue;
                    int64_t row = -1;
                    for (int64_t q = 0; q < k; ++q)
                        if (order[beg + q] == nb[e]) row = q;
                    A[row * k + a] -= wt[e];
                }
            }
            if (dense_solve((int)k, A, b)) {
                unsolved += k;
                continue;
            }
            for (int64_t a = 0; a < k; ++a) mu[order[beg + a]] = b[a];
        }
        for (int64_t a = beg; a < end; ++a) {
            int64_t v = order[a];
            accumulate_local(v, mu[v], xyz, tets, cf, ct, fib, onset_kind, onset_idx, onset_bary, parent,
                             alpha, d_cf, d_ct, d_t, d_x);
            int64_t nb[3];
            double wt[3];
            int ne = parent_edges(v, tets, parent, alpha, nb, wt);
            for (int e = 0; e < ne; ++e)
                if (comp_of[nb[e]] != c) mu[nb[e]] += wt[e] * mu[v];
        }
    }
    free(A);
    free(b);
    free(order);
    free(comp_end);
    free(comp_of);
    return unsolved;
}
