"""ECG precision at the 1M-vertex workload (100^3 cube, 12 standard leads,
T = 500 at 1 ms, phi uniform in [0, 120] ms plus smooth seeded noise): the
FP32 CUDA-core contraction and the BF16 tensor-core contraction (FP32
accumulation, per-lead scaling) against the FP64 oracle.

This workload is ill-conditioned on purpose: phi is independent from vertex
to vertex and the lead-field rows sum to zero, so every V_l(t) is a sum of
10^6 terms L_ln U(t - phi_n) that cancel to a small fraction of their
magnitudes.  The FP32 error is then set by the rounding of each term, about
eps * (K1 - K0) * sum_n |L_ln| sigma_n(t) with eps = 2^-24; the test measures
that sum with the oracle (an ECG of |L| with the template 0 .. 1) and holds
the FP32 error to a small multiple of it.  BF16 (8-bit significands) is not
a parity claim; its error is bounded and reported."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2308_08410_gb300 import gbp  # noqa: E402
from paper_2308_08410_gb300 import synth as S  # noqa: E402

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_ecg_precision_1m_vertices():
    mesh, L, phi, tmpl = S.make_c4()
    ctx = gbp.Context(0)
    try:
        ctx.upload_mesh(mesh.xyz, mesh.tets)
        ctx.set_leadfield(torch.from_numpy(np.ascontiguousarray(L, np.float32)).cuda())
        phid = torch.from_numpy(phi).cuda()
        V32 = ctx.ecg_forward(phid, tmpl, precision=gbp.PREC_FP32).cpu().numpy()
        V16 = ctx.ecg_forward(phid, tmpl, precision=gbp.PREC_BF16).cpu().numpy()
    finally:
        ctx.close()
    phi64 = phi.astype(np.float64)
    Vr = O.ecg(L, phi64, tmpl)
    # sum_n |L_ln| sigma_n(t): the oracle's ECG of |L| with U = sigma
    unit = S.Template(0.0, 1.0, tmpl.tau, tmpl.t0, tmpl.dt, tmpl.T)
    Sabs = O.ecg(np.abs(L), phi64, unit)
    cond = (tmpl.K1 - tmpl.K0) * np.linalg.norm(Sabs) / np.linalg.norm(Vr)
    e32, e16 = rel_l2(V32, Vr), rel_l2(V16, Vr)
    print(f"ECG at {mesh.n_v} vertices: condition (K1-K0) |sum |L| sigma| / |V| = {cond:.3e}; "
          f"relative L2 vs FP64 oracle: FP32 {e32:.3e} (eps * condition {cond * 2.0 ** -24:.3e}), BF16 {e16:.3e}")
    assert e32 < 16.0 * cond * 2.0 ** -24, (e32, cond)
    assert e16 < 5e-2, e16
