"""FP64 oracle of the method on triangle meshes (d = 2): the eikonal fixed
point with parent records, and the frozen-graph adjoint.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: plain NumPy / SciPy,
slow, for meshes of a few thousand vertices.  Shares nothing with the CUDA
path.

The paper states the method for any dimension (Sec. II: the local problem of
Eq. (upwind_eq_lsqr) is posed on the d-simplex opposite the vertex; Sec. III-A
runs it on 2-D triangle meshes of a torso slice).  In 2-D the face opposite a
vertex is an edge (v_1, v_2) and the local problem is

    min_{0 <= lam <= 1}  lam Phi_1 + (1 - lam) Phi_2 + || lam p_1 + (1 - lam) p_2 ||,

p_n = R (v_n - v_i) with R = D^{1/2}, D = M^{-1}, M = c_t^2 I + (c_f^2 - c_t^2) f f^T
(Sec. II-A).  The global update is Algorithm 2's min(phi_i, min_j phi_{j\\i}),
iterated here in label-correcting order until nothing changes (the fixed
point does not depend on the order).
"""
from __future__ import annotations

import heapq

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def metric_root(f, cf, ct):
    """R = (1/c_t)(I - f f^T) + (1/c_f) f f^T for a unit fibre f (2-vector)."""
    f = np.asarray(f, np.float64)
    f = f / np.linalg.norm(f)
    P = np.outer(f, f)
    return (np.eye(2) - P) / ct + P / cf


def local_edge(p1, p2, ph1, ph2):
    """Exact minimiser of the 2-D local problem.  Returns (value, lam).

    Candidates: the two end points, and the stationary point of the convex
    function g(lam) = Phi_2 + lam D + |p_2 + lam u| (D = Phi_1 - Phi_2,
    u = p_1 - p_2).  Writing x = x_0 + (lam - lam_0) u with x_0 the foot of the
    perpendicular from the origin (lam_0 = -u.p_2 / |u|^2, S = |x_0|^2),
    g'(lam) = 0 reads (lam - lam_0) |u|^2 = -D |x|, whose root is
    lam = lam_0 - D sqrt(S / (|u|^2 (|u|^2 - D^2))) when D^2 < |u|^2."""
    p1 = np.asarray(p1, np.float64)
    p2 = np.asarray(p2, np.float64)
    best = (np.inf, 0.0)
    if np.isfinite(ph1):
        best = min(best, (ph1 + np.linalg.norm(p1), 1.0))
    if np.isfinite(ph2):
        best = min(best, (ph2 + np.linalg.norm(p2), 0.0))
    if np.isfinite(ph1) and np.isfinite(ph2):
        u = p1 - p2
        A = u @ u
        D = ph1 - ph2
        if A > 0 and D * D < A:
            lam0 = -(u @ p2) / A
            S = max(p2 @ p2 - (u @ p2) ** 2 / A, 0.0)
            lam = lam0 - D * np.sqrt(S / (A * (A - D * D)))
            if 0.0 < lam < 1.0:
                v = ph2 + lam * D + np.linalg.norm(p2 + lam * u)
                best = min(best, (v, lam))
    return best


class Mesh2D:
    """xy [n_v, 2], tris [n_t, 3]."""

    def __init__(self, xy, tris):
        self.xy = np.asarray(xy, np.float64)
        self.tris = np.asarray(tris, np.int64)
        self.n_v, self.n_t = len(self.xy), len(self.tris)
        self.v2t = [[] for _ in range(self.n_v)]
        for j, t in enumerate(self.tris):
            for s in range(3):
                self.v2t[t[s]].append((j, s))


def onset_values(mesh: Mesh2D, fib, cf, ct, onset_idx, onset_t, onset_bary=None):
    """Initial values phi^0 (Sec. II, Eq. upwind_xi in 2-D): a nodal onset k
    (onset_bary None) sets phi^0 = t_k at vertex onset_idx[k]; an element
    onset at x_k = sum_q b_q v_q inside triangle E = onset_idx[k] sets
    phi^0_v = t_k + ||v - x_k||_{D_E} at the three vertices of E.  Minimum
    over onsets; returns (phi0, code) with code -1-k of the winning onset."""
    phi = np.full(mesh.n_v, np.inf)
    code = np.full(mesh.n_v, np.iinfo(np.int32).min, np.int64)
    for k, t in enumerate(onset_t):
        if onset_bary is None:
            pairs = [(int(onset_idx[k]), float(t))]
        else:
            E = int(onset_idx[k])
            tri = mesh.tris[E]
            x = np.asarray(onset_bary[k], np.float64) @ mesh.xy[tri]
            R = metric_root(fib[E], cf[E], ct[E])
            pairs = [(int(v), float(t) + np.linalg.norm(R @ (mesh.xy[v] - x))) for v in tri]
        for v, val in pairs:
            if val < phi[v]:
                phi[v], code[v] = val, -1 - k
    return phi, code


def eikonal(mesh: Mesh2D, fib, cf, ct, onset_idx, onset_t, onset_bary=None):
    """Fixed point of phi_i = min(phi_i^0, min over triangles of the local
    problem); parent code = tri * 3 + slot of i, alpha = weights of the two
    other vertices in slot order; onsets as in onset_values."""
    n = mesh.n_v
    R = [metric_root(fib[j], cf[j], ct[j]) for j in range(mesh.n_t)]
    phi, parent = onset_values(mesh, fib, cf, ct, onset_idx, onset_t, onset_bary)
    phi0 = phi.copy()
    alpha = np.zeros((n, 2))
    heap = [(phi[v], v) for v in np.nonzero(np.isfinite(phi))[0]]
    heapq.heapify(heap)

    def candidates(i):
        out = []
        for j, s in mesh.v2t[i]:
            t = mesh.tris[j]
            o = [t[q] for q in range(3) if q != s]
            v, _ = local_edge(R[j] @ (mesh.xy[o[0]] - mesh.xy[i]), R[j] @ (mesh.xy[o[1]] - mesh.xy[i]),
                              phi[o[0]], phi[o[1]])
            out.append(v)
        return out

    def solve_vertex(i):
        best = (phi[i], parent[i], alpha[i].copy())
        for j, s in mesh.v2t[i]:
            t = mesh.tris[j]
            o = [t[q] for q in range(3) if q != s]
            p1 = R[j] @ (mesh.xy[o[0]] - mesh.xy[i])
            p2 = R[j] @ (mesh.xy[o[1]] - mesh.xy[i])
            v, lam = local_edge(p1, p2, phi[o[0]], phi[o[1]])
            if not np.isfinite(v):
                continue
            code = 3 * j + s
            if v < best[0] - 1e-14 * max(1.0, abs(v)) or (abs(v - best[0]) <= 1e-14 * max(1.0, abs(v)) and 0 <= best[1] and code < best[1]):
                best = (v, code, np.array([lam, 1.0 - lam]))
        return best

    while heap:
        d, v = heapq.heappop(heap)
        if d > phi[v]:
            continue
        for j, s in mesh.v2t[v]:
            for q in range(3):
                i = mesh.tris[j][q]
                if i == v:
                    continue
                val, code, al = solve_vertex(i)
                if val < phi[i] * (1 - 1e-15) - 1e-300:
                    phi[i], parent[i], alpha[i] = val, code, al
                    heapq.heappush(heap, (val, i))
    # final parent records at the fixed point; margin = gap between the
    # winning value and the next candidate (another triangle, or the onset
    # value), which tells where the argmin is unambiguous
    margin = np.full(n, np.inf)
    for i in range(n):
        if parent[i] >= 0:
            val, code, al = solve_vertex(i)
            if code >= 0 and val <= phi[i] * (1 + 1e-12):
                parent[i], alpha[i] = code, al
        if np.isfinite(phi[i]):
            c = sorted(candidates(i) + ([phi0[i]] if np.isfinite(phi0[i]) else []))
            if len(c) > 1:
                margin[i] = c[1] - c[0]
    return dict(phi=phi, parent=parent, alpha=alpha, margin=margin)


def _velocity_terms(f, c_f, c_t, w):
    """(d/dc_f, d/dc_t) of ||w||_D for D = M^{-1}:
    ||w||_D^2 = |w_perp|^2 / c_t^2 + (f.w)^2 / c_f^2."""
    f = np.asarray(f, np.float64)
    f = f / np.linalg.norm(f)
    fw = f @ w
    wp = w - fw * f
    g = np.sqrt(wp @ wp / c_t ** 2 + fw * fw / c_f ** 2)
    if g == 0:
        return 0.0, 0.0
    return -fw * fw / (c_f ** 3 * g), -(wp @ wp) / (c_t ** 3 * g)


def adjoint(mesh: Mesh2D, fib, cf, ct, onset_idx, parent, alpha, lam, onset_t=None, onset_bary=None):
    """mu = (I - P^T)^{-1} lam along the frozen parent graph (P[c, n] = alpha of
    parent vertex n in child c's parent edge), then the per-triangle velocity
    derivatives and the onset derivatives (Sec. II-C):
        phi_i = sum_n alpha_n phi_n + ||w||_D,  w = v_i - sum_n alpha_n v_n,
        d phi_i / d c_f = -(f.w)^2 / (c_f^3 ||w||_D),
        d phi_i / d c_t = -|w_perp|^2 / (c_t^3 ||w||_D).
    An onset root v of onset k adds mu_v to d_t[k]; for an element onset
    (onset_bary given) phi_v = t_k + ||v - x_k||_{D_E} also adds
    mu_v * (-D_E (v - x_k) / ||v - x_k||_{D_E}) to d_x[k] and the velocity
    terms of E with w = v - x_k."""
    n = mesh.n_v
    rows, cols, vals = [], [], []
    for i in range(n):
        c = parent[i]
        if c < 0:
            continue
        j, s = divmod(int(c), 3)
        o = [mesh.tris[j][q] for q in range(3) if q != s]
        for q in range(2):
            if alpha[i][q] != 0.0:
                rows.append(i)
                cols.append(o[q])
                vals.append(alpha[i][q])
    P = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    mu = spla.spsolve((sp.identity(n, format="csc") - P.T.tocsc()), np.asarray(lam, np.float64))
    d_cf = np.zeros(mesh.n_t)
    d_ct = np.zeros(mesh.n_t)
    for i in range(n):
        c = parent[i]
        if c < 0:
            continue
        j, s = divmod(int(c), 3)
        o = [mesh.tris[j][q] for q in range(3) if q != s]
        w = mesh.xy[i] - alpha[i][0] * mesh.xy[o[0]] - alpha[i][1] * mesh.xy[o[1]]
        a_f, a_t = _velocity_terms(fib[j], cf[j], ct[j], w)
        d_cf[j] += mu[i] * a_f
        d_ct[j] += mu[i] * a_t
    K = len(onset_idx)
    d_t = np.zeros(K)
    d_x = np.zeros((K, 2))
    for i in range(n):
        c = parent[i]
        if not np.iinfo(np.int32).min < c < 0:
            continue
        k = -1 - int(c)
        d_t[k] += mu[i]
        if onset_bary is None:
            continue
        E = int(onset_idx[k])
        x = np.asarray(onset_bary[k], np.float64) @ mesh.xy[mesh.tris[E]]
        w = mesh.xy[i] - x
        R = metric_root(fib[E], cf[E], ct[E])
        D = R.T @ R
        g = np.sqrt(w @ D @ w)
        if g > 0:
            d_x[k] += mu[i] * (-(D @ w) / g)
            a_f, a_t = _velocity_terms(fib[E], cf[E], ct[E], w)
            d_cf[E] += mu[i] * a_f
            d_ct[E] += mu[i] * a_t
    return dict(mu=mu, d_cf=d_cf, d_ct=d_ct, d_t=d_t, d_x=d_x)
