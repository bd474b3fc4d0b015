"""The triangle-mesh (d = 2) path through the C ABI against the 2-D FP64
oracle (oracle/oracle2d.py) on the same seeded inputs.  The main case has
the size of the paper's 2-D torso-slice study (~2,700 vertices, 7 leads,
4 sites).  Tolerances as for tets: phi within 1e-4 relative, parents
bit-exact where the oracle's argmin is unambiguous (margin > 1e-5 phi), ECG
and gradients within 1e-3 relative L2."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from oracle import oracle2d as O2  # noqa: E402
from paper_2308_08410_gb300 import gbp  # noqa: E402
from paper_2308_08410_gb300 import synth as S  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = gbp.Context(0)
    yield c
    c.close()


def dev(a, dtype=np.float32):
    return torch.from_numpy(np.ascontiguousarray(a, dtype)).cuda()


def rel_l2(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def case(n=52, seed=0, K=4, kind="nodal"):
    """Problem2D with the onsets of the given kind and a noisy target from
    velocities 7 % faster along the fibres (oracle)."""
    p = S.make_2d(n, seed=seed, K=K)
    mesh = O2.Mesh2D(p.mesh.xy, p.mesh.tris)
    r = np.random.default_rng(seed + 11)
    if kind == "element":
        idx = r.choice(p.mesh.n_t, K, replace=False).astype(np.int32)
        bary = r.dirichlet(np.ones(3), size=K).astype(np.float32)
    else:
        idx, bary = p.onset_nodes, None
    ek = O2.eikonal(mesh, p.fib, p.cf * np.float32(1.07), p.ct, idx, p.onset_t, bary)
    target = S.add_noise(O.ecg(p.L, ek["phi"], p.tmpl), 0.05, seed + 5).astype(np.float32)
    return p, mesh, idx, bary, target


def upload(ctx, p, idx, bary):
    dp = gbp.setup_problem_2d(ctx, p)
    if bary is not None:
        ctx.set_onsets(gbp.ONSET_ELEMENT, dev(idx, np.int32), dev(p.onset_t), dev(bary))
    return dp


@pytest.mark.parametrize("kind", ["nodal", "element"])
def test_eikonal_2d(ctx, kind):
    p, mesh, idx, bary, _ = case(kind=kind)
    upload(ctx, p, idx, bary)
    phi, parent, alpha = ctx.eikonal_solve()
    st = ctx.stats()
    assert st["status"] == 0 and st["unreached"] == 0, st
    assert tuple(alpha.shape) == (p.mesh.n_v, 2)
    ref = O2.eikonal(mesh, p.fib, p.cf, p.ct, idx, p.onset_t, bary)
    g = phi.cpu().numpy().astype(float)
    rel = np.abs(g - ref["phi"]) / np.maximum(1.0, ref["phi"])
    assert rel.max() < 1e-4, rel.max()
    par, al = parent.cpu().numpy(), alpha.cpu().numpy()
    unamb = ref["margin"] > 1e-5 * np.maximum(1.0, ref["phi"])
    assert unamb.mean() > 0.95
    np.testing.assert_array_equal(par[unamb], ref["parent"][unamb])
    face = unamb & (ref["parent"] >= 0)
    da = np.abs(al[face] - ref["alpha"][face]).max(axis=1)
    assert np.median(da) < 1e-4 and np.quantile(da, 0.99) < 1e-2, (np.median(da), np.quantile(da, 0.99))
    np.testing.assert_allclose(al[face].sum(axis=1), 1.0, atol=1e-5)


def test_planar_front_2d(ctx):
    """phi = a . x with a^T M a = 1, seeded on the inflow sides, is reproduced
    at every vertex (the discrete scheme is exact for planar fronts)."""
    m = S.tri_square(31, 10.0, jitter=0.3, seed=4)
    n_t = m.n_t
    f = np.array([np.cos(0.4), np.sin(0.4)])
    cf, ct = 0.6, 0.3
    M = ct ** 2 * np.eye(2) + (cf ** 2 - ct ** 2) * np.outer(f, f)
    a = np.array([1.0, 0.35])
    a /= np.sqrt(a @ M @ a)
    x = m.xy.astype(np.float64)
    inflow = np.nonzero((x[:, 0] < 1e-9) | (x[:, 1] < 1e-9))[0].astype(np.int32)
    ctx.upload_mesh_2d(m.xy, m.tris)
    ctx.set_fibres(dev(np.tile(f, (n_t, 1))))
    ctx.set_velocities(dev(np.full(n_t, cf)), dev(np.full(n_t, ct)))
    ctx.set_leadfield(dev(np.ones((1, m.n_v))))
    ctx.set_onsets(gbp.ONSET_NODAL, dev(inflow, np.int32), dev(x[inflow] @ a))
    phi, _, _ = ctx.eikonal_solve()
    assert ctx.stats()["status"] == 0
    exact = x @ a
    assert np.max(np.abs(phi.cpu().numpy() - exact) / np.maximum(1.0, exact)) < 2e-6


@pytest.mark.parametrize("kind", ["nodal", "element"])
def test_gradient_2d(ctx, kind):
    p, mesh, idx, bary, target = case(kind=kind, seed=3)
    dp = upload(ctx, p, idx, bary)
    out = ctx.forward_backward(dp.cf, dp.ct, dev(target), p.tmpl)
    st = ctx.stats()
    assert st["status"] == 0, st
    g = {k: v.cpu().numpy() for k, v in out.items()}
    assert g["d_x"].shape == (len(idx), 2)
    ek = O2.eikonal(mesh, p.fib, p.cf, p.ct, idx, p.onset_t, bary)
    V = O.ecg(p.L, ek["phi"], p.tmpl)
    loss, lam = O.loss_grad_phi(p.L, ek["phi"], p.tmpl, V, target)
    ref = O2.adjoint(mesh, p.fib, p.cf, p.ct, idx, ek["parent"], ek["alpha"], lam, p.onset_t, bary)
    assert abs(g["loss"][0] - loss) / loss < 1e-4
    assert rel_l2(g["ecg"], V) < 1e-3
    for k in ("d_cf", "d_ct", "d_t"):
        assert rel_l2(g[k], ref[k]) < 1e-3, (k, rel_l2(g[k], ref[k]), st)
    if kind == "element":
        assert rel_l2(g["d_x"], ref["d_x"]) < 1e-3, rel_l2(g["d_x"], ref["d_x"])
    else:
        assert np.all(g["d_x"] == 0)


def test_ecg_bf16_2d(ctx):
    p, mesh, idx, bary, _ = case(n=40, seed=1)
    upload(ctx, p, idx, bary)
    ek = O2.eikonal(mesh, p.fib, p.cf, p.ct, idx, p.onset_t)
    phi32 = ek["phi"].astype(np.float32)
    Vr = O.ecg(p.L, phi32.astype(float), p.tmpl)
    V32 = ctx.ecg_forward(dev(phi32), p.tmpl).cpu().numpy()
    V16 = ctx.ecg_forward(dev(phi32), p.tmpl, precision=gbp.PREC_BF16).cpu().numpy()
    assert rel_l2(V32, Vr) < 1e-5
    assert rel_l2(V16, Vr) < 3e-2


def test_batch_and_host_2d(ctx):
    """Three starts in one batched call equal three single evaluations; the
    host entry point equals the device one."""
    p, mesh, idx, bary, target = case(n=30, seed=5, kind="element")
    dp = upload(ctx, p, idx, bary)
    r = np.random.default_rng(2)
    B = 3
    cf = (p.cf[None] * np.exp(0.1 * r.standard_normal((B, 1)))).astype(np.float32)
    ct = (p.ct[None] * np.exp(0.1 * r.standard_normal((B, 1)))).astype(np.float32)
    t = (p.onset_t[None] + r.uniform(-1, 1, (B, len(idx)))).astype(np.float32)
    tgt = np.repeat(target[None], B, axis=0)
    ob = ctx.forward_backward_batch(dev(cf), dev(ct), dev(tgt), p.tmpl, t=dev(t))
    assert ctx.stats()["status"] == 0
    ob = {k: v.cpu().numpy() for k, v in ob.items()}
    assert ob["d_x"].shape == (B, len(idx), 2)
    for b in range(B):
        ctx.set_velocities(dev(cf[b]), dev(ct[b]))
        o = ctx.forward_backward(dev(cf[b]), dev(ct[b]), dev(target), p.tmpl, t=dev(t[b]))
        o = {k: v.cpu().numpy() for k, v in o.items()}
        assert abs(o["loss"][0] - ob["loss"][b]) <= 1e-6 * abs(o["loss"][0])
        for k in ("d_cf", "d_ct", "d_t", "d_x"):
            assert rel_l2(ob[k][b], o[k]) < 1e-4, (b, k)
    d = ctx.forward_backward(dp.cf, dp.ct, dev(target), p.tmpl, t=dev(p.onset_t))
    d = {k: v.cpu().numpy() for k, v in d.items()}
    h = ctx.forward_backward_host(p.cf, p.ct, target, p.tmpl, t=p.onset_t)
    assert abs(h["loss"][0] - d["loss"][0]) <= 1e-6 * abs(d["loss"][0])
    for k in ("d_cf", "d_ct", "d_t", "d_x"):
        assert rel_l2(h[k], d[k]) < 1e-5, k


def test_tiny_meshes_2d(ctx):
    """One triangle, and two triangles sharing an edge (ragged: far below a
    warp), against the oracle."""
    xy = np.array([[0, 0], [1, 0], [0.3, 0.8], [1.2, 0.9]], np.float32)
    for tris in (np.array([[0, 1, 2]], np.int32), np.array([[0, 1, 2], [1, 3, 2]], np.int32)):
        nv = int(tris.max()) + 1
        n_t = len(tris)
        fib = np.tile(np.array([[0.8, 0.6]], np.float32), (n_t, 1))
        cf, ct = np.full(n_t, 0.6, np.float32), np.full(n_t, 0.3, np.float32)
        ctx.upload_mesh_2d(xy[:nv], tris)
        ctx.set_fibres(dev(fib))
        ctx.set_velocities(dev(cf), dev(ct))
        ctx.set_leadfield(dev(np.ones((1, nv))))
        ctx.set_onsets(gbp.ONSET_NODAL, dev(np.array([0], np.int32), np.int32), dev(np.array([1.5])))
        phi, par, al = ctx.eikonal_solve()
        assert ctx.stats()["status"] == 0
        ref = O2.eikonal(O2.Mesh2D(xy[:nv], tris), fib, cf, ct, [0], [1.5])
        np.testing.assert_allclose(phi.cpu().numpy(), ref["phi"], rtol=1e-6)
        np.testing.assert_array_equal(par.cpu().numpy(), ref["parent"])


def test_errors_2d(ctx):
    xy = np.array([[0, 0], [1, 0], [0, 1]], np.float32)
    with pytest.raises(gbp.GbpError):
        ctx.upload_mesh_2d(xy, np.array([[0, 2, 1]], np.int32))  # clockwise
    with pytest.raises(gbp.GbpError):
        ctx.upload_mesh_2d(xy, np.array([[0, 1, 3]], np.int32))  # bad id
    ctx.upload_mesh_2d(xy, np.array([[0, 1, 2]], np.int32))
    ctx.set_fibres(dev(np.array([[1.0, 0.0]])))
    ctx.set_velocities(dev(np.array([0.6])), dev(np.array([0.3])))
    ctx.set_leadfield(dev(np.ones((1, 3))))
    # vertex id 3 would be the internal apex: out of range for the caller
    ctx.set_onsets(gbp.ONSET_NODAL, dev(np.array([3], np.int32), np.int32), dev(np.array([0.0])))
    ctx.eikonal_solve()
    assert ctx.stats()["status"] == 1  # GBP_ERR_INVALID_ARG
