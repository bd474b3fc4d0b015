"""Pins of the oracle's frozen-graph gradient (Sec. II-C, Eq. dto_grad,
Eq. upwind_xi, the conduction-tensor remark of Sec. IV) against central
finite differences of full re-solves, an independent sparse direct solve of
mu = (I - P^T)^{-1} lam, and exact invariances of the model."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spl

from oracle import oracle as O
from paper_2308_08410_gb300 import synth as S


def small_problem(n=10, kind="element", seed=0, K=3):
    """c1 geometry with per-tet velocities jittered by 5 %: in the plain c1
    set-up tets of one depth share a metric exactly, so edge and vertex
    minimisers tie between tets and the loss has kinks along most
    directions; the jitter makes the problem generic for derivative checks."""
    p = S.make_c1(n=n, seed=seed)
    jr = np.random.default_rng(seed + 1234)
    p.cf = (p.cf * (1 + 0.05 * jr.standard_normal(p.mesh.n_t))).astype(np.float32)
    p.ct = (p.ct * (1 + 0.05 * jr.standard_normal(p.mesh.n_t))).astype(np.float32)
    if kind == "element":
        p.onsets = S.onsets_element(p.mesh, K, seed=seed + 7, tmin=0.0, tmax=6.0)
    rng = np.random.default_rng(seed + 99)
    # target: the ECG of perturbed velocities plus noise, so the residual is generic
    cf2 = (p.cf * (1 + 0.1 * rng.standard_normal(p.mesh.n_t))).astype(np.float32)
    ek = O.eikonal(p.mesh, p.fib, cf2, p.ct, p.onsets)
    V = O.ecg(p.L, ek["phi"], p.tmpl)
    p.extra["target"] = S.add_noise(V, 0.05, seed + 5)
    return p


def delaunay_small_problem(n_pts=800, seed=1):
    """synth.make_delaunay (jittered velocities, element onsets) with a target
    built as in small_problem."""
    p = S.make_delaunay(n_pts=n_pts, seed=seed)
    rng = np.random.default_rng(seed + 99)
    cf2 = (p.cf * (1 + 0.1 * rng.standard_normal(p.mesh.n_t))).astype(np.float32)
    ek = O.eikonal(p.mesh, p.fib, cf2, p.ct, p.onsets)
    p.extra["target"] = S.add_noise(O.ecg(p.L, ek["phi"], p.tmpl), 0.05, seed + 5)
    return p


def evaluate(p):
    return O.forward_backward(p.mesh, p.fib, p.cf, p.ct, p.onsets, p.L, p.tmpl, p.extra["target"])


def parent_matrix(mesh, parent, alpha):
    idx = np.nonzero(parent >= 0)[0]
    j, s = parent[idx] >> 2, parent[idx] & 3
    loc = np.array([[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]])
    fv = mesh.tets[j[:, None], loc[s]]
    n = mesh.n_v
    return sp.coo_matrix((alpha[idx].ravel(), (np.repeat(idx, 3), fv.ravel())), shape=(n, n)).tocsc()


@pytest.mark.parametrize("mesh", ["biv", "delaunay"])
def test_adjoint_matches_sparse_solve(mesh):
    """mu = (I - P^T)^{-1} lam with SuperLU, on meshes whose parent graph
    holds cycles (the oracle's SCC ordering must agree): the BiV-shaped mesh,
    and a 3,000-point Delaunay mesh with cycles of up to 15 vertices."""
    p = S.make_c2(h=1.6) if mesh == "biv" else S.make_delaunay(n_pts=3000, seed=2)
    ek = O.eikonal(p.mesh, p.fib, p.cf, p.ct, p.onsets)
    rng = np.random.default_rng(0)
    lam = rng.normal(size=p.mesh.n_v)
    g = O.adjoint(p.mesh, p.fib, p.cf, p.ct, p.onsets, ek["parent"], ek["alpha"], lam)
    P = parent_matrix(p.mesh, ek["parent"], ek["alpha"])
    if mesh == "delaunay":
        from scipy.sparse.csgraph import connected_components
        _, lab = connected_components((P != 0).astype(float), directed=True, connection="strong")
        assert np.bincount(lab).max() > 2
    mu = spl.spsolve((sp.eye(p.mesh.n_v) - P.T).tocsc(), lam)
    assert g["unprocessed"] == 0
    np.testing.assert_allclose(g["mu"], mu, rtol=1e-9, atol=1e-12 * np.abs(mu).max())


@pytest.mark.parametrize("mesh", ["kuhn", "delaunay"])
def test_fd_fifty_parameters(mesh):
    """Central differences (h = 1e-4) on 50 random parameters (per-tet c_f,
    c_t, onset times), on the jittered Kuhn cube and on an unstructured
    Delaunay mesh.  A probe whose +-h solves change a parent with margin
    below 1e-5 sits on a kink of the piecewise-smooth loss and is redrawn."""
    p = small_problem(n=9) if mesh == "kuhn" else delaunay_small_problem()
    r = evaluate(p)
    rng = np.random.default_rng(4)
    g = {"cf": r["d_cf"], "ct": r["d_ct"], "t": r["d_t"]}
    pools = {w: np.nonzero(np.abs(v) > 1e-3 * np.abs(v).max())[0] for w, v in g.items()}
    done, tried = 0, 0
    while done < 50 and tried < 400:
        tried += 1
        w = ["cf", "ct", "t"][rng.integers(3)]
        if w == "t" and done % 10:
            continue
        k = int(rng.choice(pools[w]))
        x = float({"cf": p.cf, "ct": p.ct, "t": p.onsets.t}[w][k])
        # the float32 inputs are widened by the oracle, so perturb in float64
        fd, ep, em = _fd_loss_f64(p, w, k, 1e-4)
        amb = r["margin"] < 1e-5 * np.maximum(1, r["phi"])
        if np.any((ep["parent"] != r["parent"]) & amb) or np.any((em["parent"] != r["parent"]) & amb):
            continue
        ad = g[w][k]
        assert abs(fd - ad) <= 1e-3 * abs(ad) + 1e-9 * np.abs(g[w]).max(), (w, k, x, fd, ad)
        done += 1
    assert done >= 50


def _fd_loss_f64(p, which, index, h):
    """Like _fd_loss but keeps the perturbation exact: the perturbed value is
    representable in float32 only approximately, so the step actually taken
    is measured and used."""
    arr = {"cf": p.cf, "ct": p.ct, "t": p.onsets.t}[which]
    x0 = float(arr[index])
    xp = np.float32(x0 + h)
    xm = np.float32(x0 - h)

    def run(xv):
        cf, ct, t = p.cf.copy(), p.ct.copy(), p.onsets.t.copy()
        {"cf": cf, "ct": ct, "t": t}[which][index] = xv
        ons = S.Onsets(p.onsets.kind, p.onsets.idx, t, p.onsets.bary)
        return O.loss_only(p.mesh, p.fib, cf, ct, ons, p.L, p.tmpl, p.extra["target"])

    lp, ep = run(xp)
    lm, em = run(xm)
    return (lp - lm) / (float(xp) - float(xm)), ep, em


def test_fd_onset_position():
    """d loss / d x_k (Eq. upwind_xi) against central differences of the
    onset position, moved along each axis inside its tet.  Barycentric
    coordinates are float32 inputs, so the displacement actually applied is
    recomputed from the rounded coordinates and the adjoint is contracted
    with it."""
    p = small_problem(n=9)
    r = evaluate(p)
    tets = p.mesh.tets
    checked = 0
    for k in range(p.onsets.K):
        if r["d_t"][k] == 0:
            continue
        v = p.mesh.xyz[tets[p.onsets.idx[k]]].astype(float)
        J = (v[1:] - v[0]).T  # x = v0 + J b[1:]
        for ax in range(3):
            d = np.zeros(3)
            d[ax] = 1.0
            db = np.linalg.solve(J, d)
            h = 1e-4

            def run(s):
                b = p.onsets.bary[k].astype(float).copy()
                b[1:] += s * db
                b[0] = 1 - b[1:].sum()
                bb = p.onsets.bary.copy()
                bb[k] = b.astype(np.float32)
                x = (bb[k].astype(float)[:, None] * v).sum(0)
                ons = S.Onsets(p.onsets.kind, p.onsets.idx, p.onsets.t, bb)
                loss, ek = O.loss_only(p.mesh, p.fib, p.cf, p.ct, ons, p.L, p.tmpl,
                                       p.extra["target"])
                return loss, x, ek["parent"]
            lp, xp, pp = run(+h)
            lm, xm, pm = run(-h)
            if np.any(pp != r["parent"]) or np.any(pm != r["parent"]):
                continue  # a kink of the piecewise-smooth loss lies inside the probe
            checked += 1
            fd = lp - lm
            ad = float(r["d_x"][k] @ (xp - xm))
            assert abs(fd - ad) <= 2e-3 * abs(ad) + 1e-6 * np.abs(r["d_x"]).max() * 2 * h, (k, ax, fd, ad)
    assert checked >= 6


def test_directional_derivatives():
    """Random directions in (c_f, c_t) and in the onset times.  The oracle
    reads float32 inputs, so the step actually taken per parameter is the
    difference of the rounded values; the adjoint is contracted with it."""
    p = small_problem(n=9)
    r = evaluate(p)
    rng = np.random.default_rng(8)
    for which in ("cf", "ct", "t"):
        base = {"cf": p.cf, "ct": p.ct, "t": p.onsets.t}[which].astype(np.float64)
        d = rng.normal(size=base.shape)
        grad = {"cf": r["d_cf"], "ct": r["d_ct"], "t": r["d_t"]}[which]
        h = 1e-5

        def run(s):
            cf, ct, t = p.cf.copy(), p.ct.copy(), p.onsets.t.copy()
            arr = {"cf": cf, "ct": ct, "t": t}[which]
            arr[:] = (base + s * d).astype(np.float32)
            ons = S.Onsets(p.onsets.kind, p.onsets.idx, t, p.onsets.bary)
            loss, ek = O.loss_only(p.mesh, p.fib, cf, ct, ons, p.L, p.tmpl, p.extra["target"])
            return loss, arr.astype(np.float64), ek["parent"]
        lp, xp, pp = run(+h)
        lm, xm, pm = run(-h)
        changed = int(np.sum(pp != r["parent"]) + np.sum(pm != r["parent"]))
        fd = lp - lm
        ad = float(grad @ (xp - xm))
        assert changed <= 2, changed
        assert abs(fd - ad) <= 2e-3 * abs(ad), (which, fd, ad)


def test_time_shift_invariance():
    """phi(t + c) = phi(t) + c for a common shift of all onsets, hence
    sum_k dL/dt_k = sum_n lam_n."""
    p = small_problem(n=10)
    r = evaluate(p)
    np.testing.assert_allclose(r["d_t"].sum(), r["lam"].sum(), rtol=1e-10)


def test_velocity_homogeneity():
    """With all t_k = 0, scaling every velocity by s scales phi by 1/s, hence
    sum_j (c_f dL/dc_f + c_t dL/dc_t) = -sum_n lam_n phi_n."""
    p = small_problem(n=10)
    p.onsets.t[:] = 0.0
    r = evaluate(p)
    lhs = np.dot(p.cf.astype(float), r["d_cf"]) + np.dot(p.ct.astype(float), r["d_ct"])
    rhs = -np.dot(r["lam"], r["phi"])
    np.testing.assert_allclose(lhs, rhs, rtol=1e-9)


def test_overshadowed_onset_has_zero_gradient():
    """Sec. II-E: an onset activated earlier by the surrounding front
    contributes nothing and gets a zero gradient."""
    p = small_problem(n=9, kind="nodal")
    n = 9
    a = 4 + n * (4 + n * 4)
    b = 5 + n * (4 + n * 4)  # x-neighbour of a
    p.onsets = S.Onsets(S.ONSET_NODAL, np.array([a, b], np.int32), np.array([0.0, 50.0], np.float32))
    r = evaluate(p)
    assert r["parent"][b] >= 0  # b took a face value, not its onset
    assert r["d_t"][1] == 0.0
    assert r["d_t"][0] != 0.0
