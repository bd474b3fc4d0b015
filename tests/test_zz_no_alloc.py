"""The allocation-free ECG entry point (gbp_ecg_forward_noalloc).

It exists for callers that cannot allocate device memory (a fixed memory
budget, a framework's caching allocator owning the heap, loops that must not
block on cudaMalloc / cudaFree).  These tests call it through the C ABI:

- against the context-based gbp_ecg_forward, twice in a row with different
  activation maps, so that nothing left in the shared scratch array by the
  first call leaks into the second, with the device's free memory unchanged
  across the calls that follow a first warm-up call (the property the entry
  point exists for);
- against the FP64 oracle at the limits of its scratch array: 16 leads and
  T = 4096 samples on 10^6 vertices, where the 4 MiB array caps the split-K
  grid at 7 CTAs (sampled time columns, which the oracle computes alone), and
  T = 1.

This file is collected last; it passes alone in a fresh process and after
the other tests."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2308_08410_gb300 import gbp  # noqa: E402
from paper_2308_08410_gb300 import synth as S  # noqa: E402

pytestmark = pytest.mark.gpu

SCRATCH_FLOATS = 1 << 20  # the entry point's fixed scratch (include/gbp.h)


def rel_l2(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def call(lib, L, phi, tmpl, out, stream):
    tm = gbp.make_template(tmpl)
    return lib.gbp_ecg_forward_noalloc(C.c_void_p(L.data_ptr()), L.shape[0], L.shape[1],
                                       C.c_void_p(phi.data_ptr()), C.byref(tm),
                                       C.c_void_p(out.data_ptr()), stream)


def test_noalloc_ecg_matches_context_path_twice():
    lib = gbp.load()
    ctx = gbp.Context(0)
    p = S.make_c1(T=150)
    gbp.setup_problem(ctx, p)
    L = torch.from_numpy(np.ascontiguousarray(p.L, np.float32)).cuda()
    phi_a = O.eikonal(p.mesh, p.fib, p.cf, p.ct, p.onsets)["phi"].astype(np.float32)
    phi_b = (phi_a * np.float32(1.3) + np.float32(4.0)).astype(np.float32)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    phis = [torch.from_numpy(x).cuda() for x in (phi_a, phi_b)]
    refs = [ctx.ecg_forward(ph, p.tmpl) for ph in phis]
    outs = [torch.full_like(r, float("nan")) for r in refs]
    # the first call on this device looks up the scratch array's address
    assert call(lib, L, phis[0], p.tmpl, outs[0], stream) == 0
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for ph, ref, out in zip(phis, refs, outs):
        out.fill_(float("nan"))
        assert call(lib, L, ph, p.tmpl, out, stream) == 0
        torch.cuda.synchronize()
        assert rel_l2(out.cpu().numpy(), ref.cpu().numpy()) < 1e-5
    assert torch.cuda.mem_get_info()[0] == free0
    # sizes beyond the stated limits are rejected before any launch
    bad = S.Template(T=5000)
    assert call(lib, L, phis[0], bad, outs[0], stream) == 1
    ctx.close()


def test_noalloc_ecg_at_its_limits_against_the_oracle():
    """16 leads, T = 4096 on 10^6 vertices (the 100^3 cube, 16 electrodes on
    a 30 mm sphere, P1 lead field): 2 * 16 * 4096 floats of partial sums per
    CTA leave room for 7 CTAs in the scratch array.  The samples span the
    activation window (dt = 150 ms / 4096); 7 time columns are compared with
    the oracle, which computes them alone (an ECG sample depends only on its
    own time).  Then T = 1 on the c1 workload."""
    lib = gbp.load()
    N, T = 16, 4096
    assert (SCRATCH_FLOATS - 16) // (2 * N * T) == 7
    mesh = S.kuhn_cube(100, 10.0)
    Lnp = S.lead_field(mesh, S.fibonacci_sphere(N, 30.0, (5.0, 5.0, 5.0)))
    phi_np = S.make_c4_phi(mesh.xyz, seed=3)
    tm = S.Template(-80.0, 20.0, 1.0, 0.0, 150.0 / T, T)
    L = torch.from_numpy(np.ascontiguousarray(Lnp, np.float32)).cuda()
    phi = torch.from_numpy(phi_np).cuda()
    out = torch.full((N, T), float("nan"), dtype=torch.float32, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        out.fill_(float("nan"))
        assert call(lib, L, phi, tm, out, stream) == 0
        torch.cuda.synchronize()
        V = out.cpu().numpy()
        assert np.all(np.isfinite(V))
        stride = 587
        cols = np.arange(0, T, stride)
        sub = S.Template(tm.K0, tm.K1, tm.tau, tm.t0, tm.dt * stride, len(cols))
        Vr = O.ecg(Lnp, phi_np.astype(np.float64), sub)
        assert rel_l2(V[:, cols], Vr) < 1e-3, rel_l2(V[:, cols], Vr)
    # T = 1 (one sample at t0 = 15 ms: c1 activates between 0.2 and 30 ms)
    p = S.make_c1(T=1)
    ph1 = O.eikonal(p.mesh, p.fib, p.cf, p.ct, p.onsets)["phi"]
    t1 = S.Template(-80.0, 20.0, 1.0, 15.0, 1.0, 1)
    L1 = torch.from_numpy(np.ascontiguousarray(p.L, np.float32)).cuda()
    phid = torch.from_numpy(ph1.astype(np.float32)).cuda()
    o1 = torch.full((p.L.shape[0], 1), float("nan"), dtype=torch.float32, device="cuda")
    assert call(lib, L1, phid, t1, o1, stream) == 0
    torch.cuda.synchronize()
    Vr1 = O.ecg(p.L, ph1.astype(np.float32).astype(np.float64), t1)
    assert rel_l2(o1.cpu().numpy(), Vr1) < 1e-3, rel_l2(o1.cpu().numpy(), Vr1)
