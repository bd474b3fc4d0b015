"""Failure detection on the GPU without a fault: the two device-side failure
paths of the hot path are made to trigger on purpose from the host, and the
context must report them as status codes and stay usable.

1. Iteration limit: an eikonal solve (Algorithm 2) stopped after two
   iterations (opts.max_iters = 2) reports GBP_ERR_NOT_CONVERGED with
   iterations == 2; the next solve on the same context converges and matches
   the oracle.
2. Bounded wait: the grid barrier the persistent FIM and the adjoint use,
   launched with one CTA that never arrives (a flag nothing sets), so every
   other CTA's wait runs out after a short poll limit and latches
   GBP_ERR_TIMEOUT; the control launch with every CTA present latches
   nothing; afterwards a full forward-plus-gradient evaluation on the same
   context matches the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2308_08410_gb300 import gbp  # noqa: E402
from paper_2308_08410_gb300 import synth as S  # noqa: E402

pytestmark = pytest.mark.gpu

NOT_CONVERGED, TIMEOUT = 4, 5


def dev(a, dtype=np.float32):
    return torch.from_numpy(np.ascontiguousarray(a, dtype)).cuda()


def phi_ok(phi, ref):
    rel = np.abs(phi.cpu().numpy() - ref["phi"]) / np.maximum(1.0, ref["phi"])
    return float(rel.max())


def test_iteration_limit_is_reported_and_the_context_recovers():
    p = S.make_c1(n=14)
    ctx = gbp.Context(0)
    try:
        gbp.setup_problem(ctx, p)
        ctx.eikonal_solve(gbp.make_opts(max_iters=2))
        st = ctx.stats()
        assert st["status_code"] == NOT_CONVERGED and st["status"] == NOT_CONVERGED, st
        assert st["iterations"] == 2, st
        phi, _, _ = ctx.eikonal_solve()
        st = ctx.stats()
        assert st["status"] == 0 and st["iterations"] > 2, st
        ref = O.eikonal(p.mesh, p.fib, p.cf, p.ct, p.onsets)
        assert phi_ok(phi, ref) < 1e-4
    finally:
        ctx.close()


def test_bounded_barrier_wait_times_out_and_the_context_recovers():
    p = S.make_c1(n=12)
    r = np.random.default_rng(0)
    p.cf = (p.cf * (1 + 0.05 * r.standard_normal(p.mesh.n_t))).astype(np.float32)
    ek = O.eikonal(p.mesh, p.fib, (p.cf * 1.05).astype(np.float32), p.ct, p.onsets)
    target = S.add_noise(O.ecg(p.L, ek["phi"], p.tmpl), 0.05, 2)
    ctx = gbp.Context(0)
    try:
        dp = gbp.setup_problem(ctx, p)
        # control: every CTA arrives, the barrier completes
        ctx.diag_barrier_timeout(0, 1 << 16)
        ctx.synchronize()
        # one CTA never arrives: the others' waits run out
        ctx.diag_barrier_timeout(1, 1 << 16)
        with pytest.raises(gbp.GbpError) as ei:
            ctx.synchronize()
        assert ei.value.status == TIMEOUT
        assert ctx.stats()["status_code"] == TIMEOUT
        # invalid arguments are refused on the host
        with pytest.raises(gbp.GbpError) as ei:
            ctx.diag_barrier_timeout(-1, 10)
        assert ei.value.status == 1
        # the same context evaluates correctly afterwards
        out = ctx.forward_backward(dp.cf, dp.ct, dev(target), p.tmpl)
        st = ctx.stats()
        assert st["status"] == 0, st
        ref = O.forward_backward(p.mesh, p.fib, p.cf, p.ct, p.onsets, p.L, p.tmpl, target)
        assert abs(out["loss"].item() - ref["loss"]) <= 1e-4 * ref["loss"]
        for k in ("d_cf", "d_ct", "d_t"):
            g = out[k].cpu().numpy().astype(float)
            assert np.linalg.norm(g - ref[k]) <= 1e-3 * np.linalg.norm(ref[k]), k
    finally:
        ctx.close()
