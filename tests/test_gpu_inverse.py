"""The differentiable wrapper (torch.autograd.Function over the C ABI) and the
Adam inverse loop on a reduced version of the c3 problem.

Gradient check: central finite differences (h = 1e-4) of the FP64 oracle's
loss on 50 random parameters (per-vertex log c_f / log c_t, onset times).  The
oracle reads float32 velocities, so each probe's actual per-tet steps are the
differences of the rounded velocities; the GPU's per-tet gradient is
contracted with exactly those steps (the vertex-to-tet map itself is checked
separately against its closed-form Jacobian)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2308_08410_gb300 import gbp  # noqa: E402
from paper_2308_08410_gb300 import synth as S  # noqa: E402
from paper_2308_08410_gb300.inverse import InverseProblem  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = gbp.Context(0)
    yield c
    c.close()


def reduced_c3(n=14, seed=0):
    p = S.make_c3(n=n, seed=seed)
    ek = O.eikonal(p.mesh, p.fib, p.cf, p.ct, p.onsets)
    target = S.add_noise(O.ecg(p.L, ek["phi"], p.tmpl), 0.05, seed + 11)
    return p, target, ek["phi"]


def tet_velocity(mesh, log_nodal):
    return np.exp(np.asarray(log_nodal, np.float64)[mesh.tets].mean(axis=1))


def test_autograd_gradient_vs_oracle_fd(ctx):
    p, target, _ = reduced_c3()
    rng = np.random.default_rng(5)
    lcf = np.log(0.6) + 0.1 * rng.standard_normal(p.mesh.n_v)
    lct = np.log(0.3) + 0.1 * rng.standard_normal(p.mesh.n_v)
    t0 = (p.onsets.t + rng.uniform(-2, 2, p.onsets.K)).astype(np.float32)
    inv = InverseProblem(ctx, p, target, init_log_cf=lcf, init_log_ct=lct, init_t=t0,
                         optimise_positions=False)
    # one evaluation; nodal and per-tet gradients both come from it (the
    # chaotic-relaxation FIM may pick another parent at FP32 near-ties on a
    # second run)
    from paper_2308_08410_gb300.inverse import GeodesicEcgLoss
    cf_t, ct_t = inv.tet_velocities()
    loss = GeodesicEcgLoss.apply(cf_t, ct_t, inv.t, inv.x, inv.bary(), inv.op)
    g = torch.autograd.grad(loss, [cf_t, ct_t, inv.log_cf, inv.log_ct, inv.t])
    d_cf, d_ct, g_lcf, g_lct, g_t = [x.detach().cpu().numpy().astype(float) for x in g]
    cf_np = cf_t.detach().cpu().numpy()
    ct_np = ct_t.detach().cpu().numpy()
    ons = S.Onsets(p.onsets.kind, p.onsets.idx, t0, p.onsets.bary)
    ref = O.forward_backward(p.mesh, p.fib, cf_np, ct_np, ons, p.L, p.tmpl, target)
    assert abs(loss.item() - ref["loss"]) <= 1e-4 * ref["loss"]

    # the vertex -> tet map: d L / d log c_v = sum_{j ∋ v} c_j / 4 * dL/dc_j
    chain = np.zeros(p.mesh.n_v)
    np.add.at(chain, p.mesh.tets.ravel(), np.repeat(cf_np.astype(float) * d_cf / 4.0, 4))
    np.testing.assert_allclose(g_lcf, chain, rtol=1e-4, atol=1e-6 * np.abs(chain).max())

    h = 1e-4
    done = tried = 0
    amb = ref["margin"] < 1e-5 * np.maximum(1.0, ref["phi"])
    while done < 50 and tried < 300:
        tried += 1
        kind = ["cf", "ct", "t"][rng.integers(3)]
        if kind == "t":
            k = int(rng.integers(p.onsets.K))
            if ref["d_t"][k] == 0:
                continue
            tp, tm = t0.copy(), t0.copy()
            tp[k] = np.float32(t0[k] + h)
            tm[k] = np.float32(t0[k] - h)
            lp, ep = O.loss_only(p.mesh, p.fib, cf_np, ct_np, S.Onsets(ons.kind, ons.idx, tp, ons.bary),
                                 p.L, p.tmpl, target)
            lm, em = O.loss_only(p.mesh, p.fib, cf_np, ct_np, S.Onsets(ons.kind, ons.idx, tm, ons.bary),
                                 p.L, p.tmpl, target)
            ad = g_t[k] * (float(tp[k]) - float(tm[k]))
        else:
            v = int(rng.integers(p.mesh.n_v))
            base = lcf if kind == "cf" else lct
            gvec = g_lcf if kind == "cf" else g_lct
            if abs(gvec[v]) < 1e-3 * np.abs(gvec).max():
                continue
            bp, bm = base.copy(), base.copy()
            bp[v] += h
            bm[v] -= h
            cp = tet_velocity(p.mesh, bp).astype(np.float32)
            cm = tet_velocity(p.mesh, bm).astype(np.float32)
            if kind == "cf":
                lp, ep = O.loss_only(p.mesh, p.fib, cp, ct_np, ons, p.L, p.tmpl, target)
                lm, em = O.loss_only(p.mesh, p.fib, cm, ct_np, ons, p.L, p.tmpl, target)
                ad = float(d_cf @ (cp.astype(float) - cm.astype(float)))
            else:
                lp, ep = O.loss_only(p.mesh, p.fib, cf_np, cp, ons, p.L, p.tmpl, target)
                lm, em = O.loss_only(p.mesh, p.fib, cf_np, cm, ons, p.L, p.tmpl, target)
                ad = float(d_ct @ (cp.astype(float) - cm.astype(float)))
        if np.any((ep["parent"] != ref["parent"]) & amb) or np.any((em["parent"] != ref["parent"]) & amb):
            continue
        fd = lp - lm
        assert abs(fd - ad) <= 1e-3 * abs(ad) + 1e-12, (kind, fd, ad)
        done += 1
    assert done >= 50


def test_adam_inverse_reduces_misfit(ctx):
    """Adam on the per-vertex log-velocity fields, onset times and positions
    (Sec. II-D) from the prior-mean start: the misfit drops several fold and
    the activation map moves towards the ground truth."""
    p, target, phi_true = reduced_c3(n=16, seed=2)
    inv = InverseProblem(ctx, p, target, init_t=np.full(p.onsets.K, 10.0, np.float32))
    l0 = inv.loss().item()
    rmse0 = float(np.sqrt(np.mean((inv.op.phi.cpu().numpy() - phi_true) ** 2)))
    hist, secs = inv.run_adam(iters=120, lr=2e-2, log_every=20)
    l1 = inv.loss().item()
    rmse1 = float(np.sqrt(np.mean((inv.op.phi.cpu().numpy() - phi_true) ** 2)))
    assert l1 < 0.3 * l0, (l0, l1, hist)
    assert rmse1 < rmse0, (rmse0, rmse1)


def test_onset_relocation_across_elements(ctx):
    """Element onsets started 1.2 mm from the truth, in other tets: with
    relocation (relocate.py) Adam moves them through the mesh, reaching a
    lower misfit than onsets confined to their initial tets and ending
    closer to the true sites than they started (position and onset time
    partly trade off, so the sites need not reach the truth)."""
    from paper_2308_08410_gb300.relocate import SimplexLocator
    p, target, _ = reduced_c3(n=14, seed=3)
    ons = p.onsets
    V = p.mesh.xyz.astype(np.float64)[p.mesh.tets[ons.idx]]
    x_true = np.einsum("kq,kqr->kr", ons.bary.astype(np.float64), V)
    rng = np.random.default_rng(5)
    d = rng.standard_normal((ons.K, 3))
    x0 = np.clip(x_true + 1.2 * d / np.linalg.norm(d, axis=1, keepdims=True), 0.3, 9.7)
    loc = SimplexLocator(p.mesh.xyz, p.mesh.tets)
    idx0, bary0 = [], []
    for k in range(ons.K):
        j, b, inside = loc.walk(int(ons.idx[k]), x0[k])
        assert inside
        idx0.append(j)
        bary0.append(b)
    start = S.Onsets(ons.kind, np.array(idx0, np.int32), ons.t.copy(), np.array(bary0, np.float32))
    p0 = S.Problem(p.name, p.mesh, p.fib, p.cf, p.ct, start, p.L, p.tmpl, p.extra)
    err, final = {}, {}
    for relocate in (True, False):
        inv = InverseProblem(ctx, p0, target, init_log_cf=p.extra["log_cf_nodal"],
                             init_log_ct=p.extra["log_ct_nodal"], relocate=relocate)
        # positions and times only
        inv.log_cf.requires_grad_(False)
        inv.log_ct.requires_grad_(False)
        opt = torch.optim.Adam([inv.t, inv.x], lr=2e-2)
        for _ in range(150):
            opt.zero_grad(set_to_none=True)
            inv.loss().backward()
            opt.step()
            inv.project_positions()
        final[relocate] = float(inv.loss().item())
        err[relocate] = float(np.linalg.norm(inv.x.detach().cpu().numpy() - x_true, axis=1).mean())
        if relocate:
            assert np.any(inv.op.on_idx.cpu().numpy() != np.array(idx0))
    e0 = float(np.linalg.norm(x0 - x_true, axis=1).mean())
    assert final[True] < final[False], (final, err, e0)
    assert err[True] < e0, (final, err, e0)


def test_2d_study_recovers_the_activation():
    """The paper's 2-D study on the synthetic LV slice (Sec. III-A set-up:
    2,700 vertices, 7 leads, 8 sites at 0 ms refined by 400 Adam epochs at
    lr 0.5 against the ECG of a 4-site truth on a mesh of half the spacing):
    the misfit falls by more than an order of magnitude, the activation-time
    RMSE against the truth ends below a quarter of its start, and an epoch
    costs milliseconds.  (A single start can stop in a local minimum; where
    it ends varies from run to run with the FIM's rounding.)"""
    from paper_2308_08410_gb300.inverse import run_2d
    r = run_2d(log=lambda *_: None)
    assert r["loss_final"] < 0.1 * r["loss0"], r
    rmse0, rmse1 = r["act_rmse_ms"]
    assert rmse1 < 0.25 * rmse0, r
    assert r["ms_per_epoch"] < 50.0, r["ms_per_epoch"]


def test_2d_study_multi_start():
    """Eight starts of the 2-D study in one batch: the best start's misfit is
    no worse than start 0's (the single-start protocol), and an epoch of all
    eight costs well under eight single-start epochs."""
    from paper_2308_08410_gb300.inverse import run_2d
    r = run_2d(starts=8, log=lambda *_: None)
    assert r["loss_final"] <= r["start0_loss"] + 1e-12, r
    assert r["loss_final"] < 0.1 * r["loss0"], r
    assert r["act_rmse_ms"][1] < 0.25 * r["act_rmse_ms"][0], r
    assert r["ms_per_epoch"] < 50.0, r["ms_per_epoch"]


def test_c3_loop_from_random_surface_sites():
    """The c3 inverse loop at reduced size (16^3 cube) from 10 random surface
    sites at 10 ms and the prior-mean velocities: relocation lets the sites
    walk into the mesh, the misfit falls several fold and the activation map
    moves towards the ground truth."""
    from paper_2308_08410_gb300.inverse import run_c3
    r = run_c3(n=16, iters=150, lr_sites=5e-2, log=lambda *_: None)
    assert r["loss_final"] < 0.3 * r["loss0"], r
    assert r["act_rmse_ms"][1] < r["act_rmse_ms"][0], r


def test_c3_loop_multi_start():
    """Four surface draws of the reduced c3 loop in one batch, velocity fields
    included: the kept start's misfit is the lowest of the four and no worse
    than start 0's."""
    from paper_2308_08410_gb300.inverse import run_c3
    r = run_c3(n=16, iters=100, starts=4, lr_sites=5e-2, log=lambda *_: None)
    assert r["loss_final"] == min(r["start_losses"]) and r["loss_final"] <= r["start0_loss"], r
    assert r["loss_final"] < 0.3 * r["loss0"], r
