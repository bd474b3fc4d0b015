"""Pins of the oracle's local solver (Sec. II-B, Eq. upwind_eq_lsqr,
Algorithm 1, Eq. fista_convergence, Eq. lipschitz_est).

The oracle enumerates KKT candidates of a convex problem; these tests pin it
to things that do not share that derivation: hand-derived closed forms,
brute-force minimisation over the simplex with an independently built metric
(np.linalg.inv of the conduction tensor), and the published FISTA rate.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2308_08410_gb300 import synth as S


def metric_inv(cf, ct, f):
    """D = M^{-1} with M = ct^2 I + (cf^2 - ct^2) f f^T, by numerical inverse."""
    f = np.asarray(f, float)
    f = f / np.linalg.norm(f)
    M = ct ** 2 * np.eye(3) + (cf ** 2 - ct ** 2) * np.outer(f, f)
    return np.linalg.inv(M)


def brute_min(e, D, phi, n=240):
    """Brute force over a barycentric grid of the finite sub-face, then a
    fine grid around the best point (step 1e-5)."""
    e = np.asarray(e, float)
    fin = np.isfinite(phi)
    idx = np.nonzero(fin)[0]

    def obj(al):  # al [m, 3]
        w = al @ e
        ph = np.where(fin, phi, 0.0)
        return al @ ph + np.sqrt(np.einsum("mi,ij,mj->m", w, D, w))

    k = len(idx)
    if k == 1:
        al = np.zeros((1, 3))
        al[0, idx[0]] = 1.0
        return obj(al)[0]
    g = np.arange(n + 1) / n
    if k == 2:
        al = np.zeros((n + 1, 3))
        al[:, idx[0]] = g
        al[:, idx[1]] = 1 - g
    else:
        a, b = np.meshgrid(g, g, indexing="ij")
        m = a + b <= 1 + 1e-12
        al = np.stack([a[m], b[m], np.clip(1 - a[m] - b[m], 0, 1)], axis=1)
    v = obj(al)
    best = al[np.argmin(v)]
    # refinement around the best grid point
    h = 1.0 / n
    fine = np.linspace(-h, h, 201)
    if k == 2:
        x0 = best[idx[0]]
        x = np.clip(x0 + fine, 0, 1)
        al = np.zeros((len(x), 3))
        al[:, idx[0]] = x
        al[:, idx[1]] = 1 - x
    else:
        A, B = np.meshgrid(best[0] + fine, best[1] + fine, indexing="ij")
        A, B = np.clip(A.ravel(), 0, 1), np.clip(B.ravel(), 0, 1)
        m = A + B <= 1
        al = np.stack([A[m], B[m], 1 - A[m] - B[m]], axis=1)
    return min(float(obj(al).min()), float(v.min()))


def test_closed_form_regular_corner():
    """Isotropic unit metric, v_i at the origin, face = unit simplex x+y+z=1.
    Phi = 0: the minimum is the distance to the plane, 1/sqrt(3), at the
    centroid.  Phi = (0, 5, 5): vertex 1 (value 1), since the directional
    derivative towards either other vertex is 5 - 1 > 0.  Phi = (0, .5, .5):
    by symmetry alpha_2 = alpha_3 = b with 30 b^2 - 20 b + 3 = 0, i.e.
    b = (10 - sqrt 10)/30 and value b + sqrt(6 b^2 - 4 b + 1)."""
    e = np.eye(3, dtype=np.float32)[None].repeat(3, 0)
    f = np.array([[1, 0, 0]] * 3, np.float32)
    c = np.ones(3, np.float32)
    phi = np.array([[0, 0, 0], [0, 5, 5], [0, 0.5, 0.5]], np.float32)
    v, al = O.local_batch(e, f, c, c, phi)
    b = (10 - math.sqrt(10)) / 30
    expect = [1 / math.sqrt(3), 1.0, b + math.sqrt(6 * b * b - 4 * b + 1)]
    np.testing.assert_allclose(v, expect, rtol=1e-14)
    np.testing.assert_allclose(al[0], [1 / 3] * 3, atol=1e-14)
    np.testing.assert_allclose(al[1], [1, 0, 0], atol=0)
    np.testing.assert_allclose(al[2], [1 - 2 * b, b, b], atol=1e-13)


def test_closed_form_edge_textbook():
    """Edge case with one infinite vertex: 1-D problem
    min_l  l*d + sqrt((1-l)^2 + l^2)  on e1=(1,0,0), e2=(0,1,0) (isotropic),
    Phi=(0, d, inf).  Stationary: u = 2l - 1 = -d/sqrt(2 - d^2), value
    (1+u)/2*d + sqrt((u^2+1)/2)."""
    for d in (0.1, 0.3, 0.7):
        e = np.eye(3, dtype=np.float32)[None]
        f = np.array([[0, 0, 1]], np.float32)
        c = np.ones(1, np.float32)
        phi = np.array([[0, d, np.inf]], np.float32)
        v, al = O.local_batch(e, f, c, c, phi)
        dd = float(np.float32(d))
        u = -dd / math.sqrt(2 - dd * dd)
        lam = (1 + u) / 2
        assert al[0, 2] == 0.0
        np.testing.assert_allclose(al[0, 1], lam, rtol=1e-12)
        np.testing.assert_allclose(v[0], lam * dd + math.sqrt((u * u + 1) / 2), rtol=1e-13)


def test_anisotropic_vertex_distance():
    """Single finite vertex: the value is Phi_n + ||e_n||_D with D = M^{-1};
    for e along the fibre ||e||_D = |e|/cf, across it |e|/ct (Sec. II-A)."""
    e = np.array([[[2, 0, 0], [0, 3, 0], [0, 0, 1]]], np.float32).repeat(2, 0)
    f = np.array([[1, 0, 0], [1, 0, 0]], np.float32)
    cf = np.array([0.6, 0.6], np.float32)
    ct = np.array([0.3, 0.3], np.float32)
    phi = np.array([[1.0, np.inf, np.inf], [np.inf, 1.0, np.inf]], np.float32)
    v, _ = O.local_batch(e, f, cf, ct, phi)
    np.testing.assert_allclose(v, [1 + 2 / np.float32(0.6), 1 + 3 / np.float32(0.3)], rtol=1e-7)


@pytest.mark.parametrize("skinny", [False, True])
def test_exact_vs_brute_force(skinny):
    e, f, cf, ct, phi = S.random_faces(160, seed=11 + skinny, skinny=skinny)
    v, al = O.local_batch(e, f, cf, ct, phi)
    classes = {"vertex": 0, "edge": 0, "interior": 0}
    for i in range(len(v)):
        D = metric_inv(float(cf[i]), float(ct[i]), f[i])
        ph = phi[i].astype(float)
        bf = brute_min(e[i], D, ph)
        # oracle value is attained at a feasible alpha, and matches brute force
        assert np.all(al[i] >= 0) and abs(al[i].sum() - 1) < 1e-12
        w = al[i] @ e[i].astype(float)
        val_at = float(np.sum(al[i] * np.where(al[i] > 0, ph, 0.0)) + math.sqrt(w @ D @ w))
        assert abs(val_at - v[i]) <= 1e-12 * max(1, abs(v[i]))
        assert v[i] <= bf + 1e-10 * max(1, abs(bf))
        assert v[i] >= bf - 2e-7 * max(1, abs(bf)), (i, v[i], bf)
        nz = int(np.sum(al[i] > 0))
        classes[{1: "vertex", 2: "edge", 3: "interior"}[nz]] += 1
    # every branch of the candidate enumeration is exercised (a nearly
    # collinear face has no interior minimiser)
    if not skinny:
        assert all(n > 5 for n in classes.values()), classes


def test_lipschitz_bounds():
    """h_theory = sigma_min(A)/(d sqrt d) <= h_min = min_simplex ||A alpha||
    (Eq. lipschitz_est), and the estimate bounds sampled difference quotients
    of grad h = G alpha / h on the simplex."""
    e, f, cf, ct, _ = S.random_faces(200, seed=5)
    out = O.lipschitz_batch(e, f, cf, ct)
    assert np.all(out["h_theory"] <= out["h_min"] * (1 + 1e-12))
    rng = np.random.default_rng(0)
    for i in range(200):
        D = metric_inv(float(cf[i]), float(ct[i]), f[i])
        E = e[i].astype(float)
        G = E @ D @ E.T
        a = rng.dirichlet(np.ones(3), size=64)
        b = rng.dirichlet(np.ones(3), size=64)

        def grad(x):
            y = x @ G
            return y / np.sqrt(np.sum(x * y, axis=1, keepdims=True))

        q = np.linalg.norm(grad(a) - grad(b), axis=1) / np.linalg.norm(a - b, axis=1)
        assert q.max() <= out["L"][i] * (1 + 1e-9)
        np.testing.assert_allclose(out["norm_G"][i], np.linalg.eigvalsh(G).max(), rtol=1e-10)
        np.testing.assert_allclose(out["h_theory"][i],
                                   np.sqrt(np.linalg.eigvalsh(G).min()) / (3 * math.sqrt(3)),
                                   rtol=1e-9)


def test_fista_rate_bound():
    """Eq. fista_convergence: F(alpha_k) - F* <= 2 L ||alpha_0 - alpha*||^2 / (k+1)^2
    with L from Eq. lipschitz_est (theoretical lower bound of h, valid on the
    whole plane the extrapolated iterates live on)."""
    e, f, cf, ct, phi = S.random_faces(200, seed=7, p_inf=0.0)
    v_ex, a_ex = O.local_batch(e, f, cf, ct, phi)
    lip = O.lipschitz_batch(e, f, cf, ct)
    h = lip["h_theory"]
    Lth = lip["norm_G"] / h * (1 + np.sqrt(lip["norm_G"]) / h)
    d0 = np.sum((a_ex - 1 / 3) ** 2, axis=1)
    for k in (1, 2, 4, 8, 16, 32, 64):
        v_k, a_k = O.local_batch(e, f, cf, ct, phi, mode=O.FISTA_THEORY, n_f=k)
        assert np.all(v_k >= v_ex - 1e-12 * np.maximum(1, np.abs(v_ex)))
        bound = 2 * Lth * d0 / (k + 1) ** 2
        assert np.all(v_k - v_ex <= bound + 1e-12), k


def test_fista_practical_converges_and_handles_inf():
    """With the practical constant (Sec. II-E: h_ = h(alpha*)/1.1) 64 steps land
    close to the exact minimum; +inf vertices get zero weight."""
    e, f, cf, ct, phi = S.random_faces(300, seed=9, p_inf=0.2)
    v_ex, _ = O.local_batch(e, f, cf, ct, phi)
    v_f, a_f = O.local_batch(e, f, cf, ct, phi, mode=O.FISTA, n_f=64)
    assert np.all(v_f >= v_ex - 1e-12 * np.maximum(1, np.abs(v_ex)))
    rel = (v_f - v_ex) / np.maximum(1, np.abs(v_ex))
    assert np.median(rel) < 1e-5
    assert np.all(a_f[~np.isfinite(phi)] == 0)
    assert np.all(np.isfinite(v_f))
