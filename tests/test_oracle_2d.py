"""Pins of the 2-D oracle (oracle/oracle2d.py): the edge local problem against
brute-force minimisation, planar fronts reproduced exactly, the point-source
lower bound with O(h) convergence, every parent edge reproducing its
vertex's value, and the frozen-graph adjoint against central finite
differences of the oracle's own loss."""
import numpy as np
import scipy.optimize

from oracle import oracle as O
from oracle import oracle2d as O2
from paper_2308_08410_gb300 import synth as S


def test_local_edge_vs_brute_force():
    rng = np.random.default_rng(0)
    for _ in range(300):
        p1, p2 = rng.standard_normal(2), rng.standard_normal(2)
        ph = rng.uniform(0, 2, 2)
        if rng.random() < 0.15:
            ph[rng.integers(2)] = np.inf
        v, lam = O2.local_edge(p1, p2, ph[0], ph[1])
        fin = np.isfinite(ph)
        if not fin.any():
            assert not np.isfinite(v)
            continue
        if not fin.all():
            n = int(np.argmax(fin))
            assert abs(v - (ph[n] + np.linalg.norm([p1, p2][n]))) < 1e-12
            continue
        g = lambda t: t * ph[0] + (1 - t) * ph[1] + np.linalg.norm(t * p1 + (1 - t) * p2)  # noqa: E731
        grid = np.linspace(0, 1, 20001)
        t0 = grid[np.argmin([g(t) for t in grid])]
        r = scipy.optimize.minimize_scalar(g, bounds=(max(0, t0 - 1e-4), min(1, t0 + 1e-4)), method="bounded",
                                           options={"xatol": 1e-12})
        ref = min(g(0.0), g(1.0), r.fun)
        assert abs(v - ref) <= 1e-10 * max(1.0, ref), (v, ref)
        assert abs(g(lam) - v) <= 1e-12 * max(1.0, v)


def planar_setup(n, fib_angle, cf, ct):
    m = S.tri_square(n, 10.0, jitter=0.3, seed=1)
    mesh = O2.Mesh2D(m.xy, m.tris)
    f = np.array([np.cos(fib_angle), np.sin(fib_angle)])
    fib = np.tile(f, (mesh.n_t, 1))
    return mesh, fib, np.full(mesh.n_t, cf), np.full(mesh.n_t, ct)


def test_planar_front_is_exact():
    """phi(x) = a . x with a^T M a = 1 (M the conduction tensor) is a solution
    of the continuous problem and, being linear, of every local problem whose
    edge the backward characteristic -M a crosses (Cauchy-Schwarz gives
    >= a . v_i for every other candidate).  Seeded on the inflow sides of the
    square it is reproduced at every vertex."""
    mesh, fib, cf, ct = planar_setup(15, 0.4, 0.6, 0.3)
    f = fib[0]
    M = ct[0] ** 2 * np.eye(2) + (cf[0] ** 2 - ct[0] ** 2) * np.outer(f, f)
    a = np.array([1.0, 0.35])
    a /= np.sqrt(a @ M @ a)
    x = mesh.xy
    ma = M @ a
    assert ma[0] > 0 and ma[1] > 0
    inflow = np.nonzero((x[:, 0] < 1e-9) | (x[:, 1] < 1e-9))[0]
    ek = O2.eikonal(mesh, fib, cf, ct, inflow, x[inflow] @ a)
    np.testing.assert_allclose(ek["phi"], x @ a, rtol=1e-11, atol=1e-11)


def test_point_source_bound_and_convergence():
    errs = []
    for n in (11, 21, 41):
        mesh, fib, cf, ct = planar_setup(n, 0.0, 0.6, 0.3)
        c = np.argmin(np.linalg.norm(mesh.xy - 5.0, axis=1))
        ek = O2.eikonal(mesh, fib, cf, ct, [c], [0.0])
        R = O2.metric_root(fib[0], cf[0], ct[0])
        exact = np.linalg.norm((mesh.xy - mesh.xy[c]) @ R.T, axis=1)
        assert np.all(ek["phi"] >= exact - 1e-12)  # linear interpolation of a convex distance
        errs.append(np.max(ek["phi"] - exact))
    assert errs[1] < 0.75 * errs[0] and errs[2] < 0.75 * errs[1], errs


def test_adjoint_vs_finite_differences():
    p = S.make_2d(12, seed=3)
    mesh = O2.Mesh2D(p.mesh.xy, p.mesh.tris)
    cf, ct = p.cf.astype(np.float64), p.ct.astype(np.float64)
    t = p.onset_t.astype(np.float64)

    def loss(cf_, ct_, t_):
        ek = O2.eikonal(mesh, p.fib, cf_, ct_, p.onset_nodes, t_)
        V = O.ecg(p.L, ek["phi"], p.tmpl)
        return O.loss_grad_phi(p.L, ek["phi"], p.tmpl, V, target), ek

    ek0 = O2.eikonal(mesh, p.fib, cf * 1.05, ct, p.onset_nodes, t)
    target = S.add_noise(O.ecg(p.L, ek0["phi"], p.tmpl), 0.05, 4)
    (l0, lam), ek = loss(cf, ct, t)
    g = O2.adjoint(mesh, p.fib, cf, ct, p.onset_nodes, ek["parent"], ek["alpha"], lam)
    rng = np.random.default_rng(5)
    h = 1e-6
    for j in rng.choice(mesh.n_t, 6, replace=False):
        for name, arr in (("d_cf", cf), ("d_ct", ct)):
            e = np.zeros_like(arr)
            e[j] = h
            a_p = (arr + e, ct) if name == "d_cf" else (cf, arr + e)
            a_m = (arr - e, ct) if name == "d_cf" else (cf, arr - e)
            fd = (loss(*a_p, t)[0][0] - loss(*a_m, t)[0][0]) / (2 * h)
            assert abs(fd - g[name][j]) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(g[name]).max()), (name, j, fd, g[name][j])
    for k in range(len(t)):
        e = np.zeros_like(t)
        e[k] = h
        fd = (loss(cf, ct, t + e)[0][0] - loss(cf, ct, t - e)[0][0]) / (2 * h)
        assert abs(fd - g["d_t"][k]) <= 1e-5 * max(abs(fd), 1e-8), (k, fd, g["d_t"][k])


def test_element_onset_at_a_vertex_is_nodal():
    p = S.make_2d(10, seed=2)
    mesh = O2.Mesh2D(p.mesh.xy, p.mesh.tris)
    E = 37
    for q in range(3):
        b = np.zeros((1, 3))
        b[0, q] = 1.0
        el = O2.eikonal(mesh, p.fib, p.cf, p.ct, [E], [2.0], b)
        nod = O2.eikonal(mesh, p.fib, p.cf, p.ct, [mesh.tris[E][q]], [2.0])
        np.testing.assert_allclose(el["phi"], nod["phi"], rtol=1e-13, atol=1e-13)


def test_element_onset_gradients_vs_finite_differences():
    p = S.make_2d(10, seed=6)
    mesh = O2.Mesh2D(p.mesh.xy, p.mesh.tris)
    cf, ct = p.cf.astype(np.float64), p.ct.astype(np.float64)
    rng = np.random.default_rng(8)
    tris = np.array([23, 101])
    bary = rng.dirichlet(np.ones(3), size=2)
    t = np.array([1.0, 4.0])

    def run(t_, bary_, cf_=cf):
        ek = O2.eikonal(mesh, p.fib, cf_, ct, tris, t_, bary_)
        return ek, O.ecg(p.L, ek["phi"], p.tmpl)

    target = S.add_noise(run(t + 0.5, bary)[1], 0.05, 9)

    def loss(t_, bary_, cf_=cf):
        ek, V = run(t_, bary_, cf_)
        return O.loss_grad_phi(p.L, ek["phi"], p.tmpl, V, target)[0]

    ek, V = run(t, bary)
    _, lam = O.loss_grad_phi(p.L, ek["phi"], p.tmpl, V, target)
    g = O2.adjoint(mesh, p.fib, cf, ct, tris, ek["parent"], ek["alpha"], lam, t, bary)
    h = 1e-6
    for k in range(2):
        e = np.zeros(2)
        e[k] = h
        fd = (loss(t + e, bary) - loss(t - e, bary)) / (2 * h)
        assert abs(fd - g["d_t"][k]) <= 1e-5 * max(abs(fd), 1e-8), (k, fd, g["d_t"][k])
        # moving x_k along a direction u inside the triangle: d bary = M^{-1} [u; 0]
        V3 = mesh.xy[mesh.tris[tris[k]]]
        Minv = np.linalg.inv(np.vstack([V3.T, np.ones(3)]))
        for u in (np.array([1.0, 0.0]), np.array([0.0, 1.0])):
            db = Minv @ np.append(u, 0.0)
            bp, bm = bary.copy(), bary.copy()
            bp[k] += h * db
            bm[k] -= h * db
            fd = (loss(t, bp) - loss(t, bm)) / (2 * h)
            assert abs(fd - g["d_x"][k] @ u) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(g["d_x"]).max()), (k, u, fd)
    # the onset triangle's velocity enters through the onset values too
    for E in tris:
        e = np.zeros_like(cf)
        e[E] = h
        fd = (loss(t, bary, cf + e) - loss(t, bary, cf - e)) / (2 * h)
        assert abs(fd - g["d_cf"][E]) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(g["d_cf"]).max()), (E, fd, g["d_cf"][E])


def test_parent_edge_reproduces_phi():
    """At the fixed point every vertex with a parent edge takes that edge's
    local value: phi_i equals the alpha-weighted edge values plus the metric
    length of v_i - sum alpha_n v_n, with the metric M^-1 built here from
    M = ct^2 I + (cf^2 - ct^2) f f^T (not the oracle's square root), alpha a
    point of the edge, and the edge value below phi_i."""
    p = S.make_2d(14, seed=8)
    mesh = O2.Mesh2D(p.mesh.xy, p.mesh.tris)
    ek = O2.eikonal(mesh, p.fib, p.cf, p.ct, p.onset_nodes, p.onset_t)
    checked = 0
    for i in range(mesh.n_v):
        code = int(ek["parent"][i])
        if code < 0:
            continue
        j, s = code // 3, code % 3
        assert mesh.tris[j][s] == i
        edge = [int(mesh.tris[j][q]) for q in range(3) if q != s]
        a = ek["alpha"][i]
        assert np.all(a >= -1e-15) and abs(a.sum() - 1.0) < 1e-12
        f = np.asarray(p.fib[j], float)
        f /= np.linalg.norm(f)
        M = float(p.ct[j]) ** 2 * np.eye(2) + (float(p.cf[j]) ** 2 - float(p.ct[j]) ** 2) * np.outer(f, f)
        w = mesh.xy[i] - a @ mesh.xy[edge]
        interp = float(a @ ek["phi"][edge])
        assert abs(ek["phi"][i] - (interp + np.sqrt(w @ np.linalg.solve(M, w)))) <= 1e-11 * max(1.0, ek["phi"][i])
        assert interp < ek["phi"][i]
        checked += 1
    assert checked > 0.9 * mesh.n_v
