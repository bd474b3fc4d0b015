"""Parity at the benchmark's exact workload, point and launch configuration:
the 72^3 Kuhn cube (373,248 vertices, 2,147,466 tets, 10 element onsets, 8
leads, T = 150) with the 16 starts the benchmark times (synth.c3_starts:
prior-mean velocities with a global scale exp(N(0, 0.1)) per start and 5 %
per-vertex log-velocity noise, onset times 10 ms (+ U(-2, 2) ms)) through
gbp_forward_backward_batch in FP32 with the exact local solver, the call the
benchmark times.  Three problems of the batch (the first, a middle one and
the last) are compared with the FP64 oracle element by element.

Inputs: the target is the oracle's ECG of the seeded ground truth plus 5 %
noise per lead (the benchmark computes the same target with the GPU's ECG;
the two agree to the ECG tolerance, far below the noise).

Tolerances (parity_helpers.py): phi 2e-6 relative per vertex; parents
bit-exact where the oracle's margin exceeds 1e-5 phi; alpha within
2e-5 + 4x the oracle's own sensitivity; loss 1e-4 relative; ECG, d_t and d_x
1e-3 relative L2; d_cf and d_ct per tet within 1e-3 |r| + 1e-6 max |r| on every
tet no tie touched.  Over all tets, d_cf and d_ct are held to 1e-2 relative L2:
about 2 % of the vertices lie within 1e-5 phi of a tie, where the gradient is
only a subgradient and an FP32 solve may take the other face; a vertex high
in the tree then moves a large adjoint weight to a neighbouring tet.  The sum
of c_f d_cf + c_t d_ct over all tets is the derivative of the loss under a
common scaling of every velocity; it does not depend on which face of a tie
is taken and is held to 1e-3."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import parity_helpers as PH  # noqa: E402
from oracle import oracle as O  # noqa: E402
from paper_2308_08410_gb300 import gbp  # noqa: E402
from paper_2308_08410_gb300 import synth as S  # noqa: E402

pytestmark = pytest.mark.gpu

B = 16
COMPARED = (0, 7, 15)


def dev(a, dtype=np.float32):
    return torch.from_numpy(np.ascontiguousarray(a, dtype)).cuda()


def rel_l2(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def workload():
    p = S.make_c3(n=72, seed=0)
    ek = O.eikonal(p.mesh, p.fib, p.cf, p.ct, p.onsets)
    target = S.add_noise(O.ecg(p.L, ek["phi"], p.tmpl), 0.05, 4242).astype(np.float32)
    cf, ct, t = S.c3_starts(p, B)
    return p, cf, ct, t, target


def test_batch_of_16_at_full_size(workload):
    p, cf, ct, t, target = workload
    assert (p.mesh.n_v, p.mesh.n_t, p.onsets.K, p.L.shape[0], p.tmpl.T) == (373248, 2147466, 10, 8, 150)
    ctx = gbp.Context(0)
    try:
        gbp.setup_problem(ctx, p)
        opts = gbp.make_opts(local_solver=gbp.LOCAL_EXACT, n_f=32)
        tg = np.repeat(target[None], B, axis=0)
        out = ctx.forward_backward_batch(dev(cf), dev(ct), dev(tg), p.tmpl, t=dev(t), opts=opts)
        st = ctx.stats()
        assert st["status"] == 0 and st["unreached"] == 0, st
        g = {k: v.cpu().numpy() for k, v in out.items()}
        assert np.all(np.isfinite(g["loss"])) and np.all(np.isfinite(g["d_cf"]))
        for b in COMPARED:
            ons = S.Onsets(p.onsets.kind, p.onsets.idx, t[b], p.onsets.bary)
            ref = O.forward_backward(p.mesh, p.fib, cf[b], ct[b], ons, p.L, p.tmpl, target)
            phi, par, al = (x.cpu().numpy() for x in ctx.solution(b))
            PH.check_phi(phi, ref)
            PH.check_parents(par, ref, min_unambiguous=0.95)
            PH.check_alpha(al, par, p.mesh, p.fib, cf[b], ct[b], ref)
            assert abs(g["loss"][b] - ref["loss"]) / ref["loss"] < 1e-4, (b, g["loss"][b], ref["loss"])
            assert rel_l2(g["ecg"][b], ref["V"]) < 1e-3, b
            for k in ("d_t", "d_x"):
                assert rel_l2(g[k][b], ref[k]) < 1e-3, (b, k, rel_l2(g[k][b], ref[k]))
            for k in ("d_cf", "d_ct"):
                assert rel_l2(g[k][b], ref[k]) < 1e-2, (b, k, rel_l2(g[k][b], ref[k]))
            gb = {"d_cf": g["d_cf"][b], "d_ct": g["d_ct"][b]}
            PH.check_tet_gradients(gb, ref, par, p.mesh, ons)
            hom = float(np.dot(cf[b], g["d_cf"][b].astype(float)) + np.dot(ct[b], g["d_ct"][b].astype(float)))
            hom_ref = float(np.dot(cf[b], ref["d_cf"]) + np.dot(ct[b], ref["d_ct"]))
            assert abs(hom - hom_ref) <= 1e-3 * abs(hom_ref), (b, hom, hom_ref)
    finally:
        ctx.close()


def test_single_evaluation_at_the_benchmarked_point(workload):
    """gbp_forward_backward on start 0 (the benchmark's one-evaluation leg)
    against the oracle: loss, ECG, per-vertex phi and parents, alpha and
    per-tet gradients."""
    p, cf, ct, t, target = workload
    ctx = gbp.Context(0)
    try:
        gbp.setup_problem(ctx, p)
        ctx.set_onsets(p.onsets.kind, dev(p.onsets.idx, np.int32), dev(t[0]), dev(p.onsets.bary))
        out = ctx.forward_backward(dev(cf[0]), dev(ct[0]), dev(target), p.tmpl)
        assert ctx.stats()["status"] == 0
        g = {k: v.cpu().numpy() for k, v in out.items()}
        ons = S.Onsets(p.onsets.kind, p.onsets.idx, t[0], p.onsets.bary)
        ref = O.forward_backward(p.mesh, p.fib, cf[0], ct[0], ons, p.L, p.tmpl, target)
        phi, par, al = (x.cpu().numpy() for x in ctx.solution(0))
        PH.check_phi(phi, ref)
        PH.check_parents(par, ref, min_unambiguous=0.95)
        PH.check_alpha(al, par, p.mesh, p.fib, cf[0], ct[0], ref)
        assert abs(g["loss"][0] - ref["loss"]) / ref["loss"] < 1e-4
        assert rel_l2(g["ecg"], ref["V"]) < 1e-3
        PH.check_tet_gradients(g, ref, par, p.mesh, ons)
    finally:
        ctx.close()


def test_biv_batch_at_the_benchmarked_point():
    """The biventricular shell of `bench.py --workload biv` (h = 1 mm: 95,199
    vertices, 472,692 tets, 5 element onsets, 12 leads, T = 300) with the 16
    starts that benchmark times (synth.c2_starts: a tissue velocity scale
    exp(N(0, 0.1)) per start, 5 % per-tet log-velocity noise, onset times
    +U(-2, 2) ms) through gbp_forward_backward_batch; three problems of the
    batch against the oracle element by element, with the tolerances of the
    cube test above (d_cf and d_ct as whole vectors at 1e-3 where no parent
    differs from the oracle's)."""
    p = S.make_c2(h=1.0, seed=0)
    assert (p.mesh.n_v, p.mesh.n_t, p.onsets.K, p.L.shape[0], p.tmpl.T) == (95199, 472692, 5, 12, 300)
    ek = O.eikonal(p.mesh, p.fib, p.cf, p.ct, p.onsets)
    target = S.add_noise(O.ecg(p.L, ek["phi"], p.tmpl), 0.05, 4242).astype(np.float32)
    cf, ct, t = S.c2_starts(p, B)
    ctx = gbp.Context(0)
    try:
        gbp.setup_problem(ctx, p)
        tg = np.repeat(target[None], B, axis=0)
        out = ctx.forward_backward_batch(dev(cf), dev(ct), dev(tg), p.tmpl, t=dev(t))
        st = ctx.stats()
        assert st["status"] == 0 and st["unreached"] == 0, st
        g = {k: v.cpu().numpy() for k, v in out.items()}
        for b in COMPARED:
            ons = S.Onsets(p.onsets.kind, p.onsets.idx, t[b], p.onsets.bary)
            ref = O.forward_backward(p.mesh, p.fib, cf[b], ct[b], ons, p.L, p.tmpl, target)
            phi, par, al = (x.cpu().numpy() for x in ctx.solution(b))
            PH.check_phi(phi, ref)
            PH.check_parents(par, ref, min_unambiguous=0.95)
            PH.check_alpha(al, par, p.mesh, p.fib, cf[b], ct[b], ref)
            assert abs(g["loss"][b] - ref["loss"]) / ref["loss"] < 1e-4, (b, g["loss"][b], ref["loss"])
            assert rel_l2(g["ecg"][b], ref["V"]) < 1e-3, b
            for k in ("d_t", "d_x"):
                assert rel_l2(g[k][b], ref[k]) < 1e-3, (b, k, rel_l2(g[k][b], ref[k]))
            tol = 1e-2 if PH.parents_differ(par, ref) else 1e-3
            for k in ("d_cf", "d_ct"):
                assert rel_l2(g[k][b], ref[k]) < tol, (b, k, rel_l2(g[k][b], ref[k]))
            PH.check_tet_gradients({"d_cf": g["d_cf"][b], "d_ct": g["d_ct"][b]}, ref, par, p.mesh, ons)
    finally:
        ctx.close()
