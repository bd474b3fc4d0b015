"""The allocation-free ECG entry point (gbp_ecg_forward_noalloc).

It exists for callers that cannot allocate device memory (a fixed memory
budget, a framework's caching allocator owning the heap, loops that must not
block on cudaMalloc / cudaFree).  This test calls it through the C ABI and
checks it against the context-based gbp_ecg_forward, twice in a row with
different activation maps, so that nothing left in the shared scratch array
by the first call leaks into the second.  This file is collected last; it
passes alone in a fresh process and after the other tests."""
import ctypes as C

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


def test_noalloc_ecg_matches_context_path_twice():
    lib = gbp.load()
    ctx = gbp.Context(0)
    p = S.make_c1(T=150)
    gbp.setup_problem(ctx, p)
    L = torch.from_numpy(np.ascontiguousarray(p.L, np.float32)).cuda()
    phi_a = O.eikonal(p.mesh, p.fib, p.cf, p.ct, p.onsets)["phi"].astype(np.float32)
    phi_b = (phi_a * np.float32(1.3) + np.float32(4.0)).astype(np.float32)
    tm = gbp.make_template(p.tmpl)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for phi_np in (phi_a, phi_b):
        phi = torch.from_numpy(phi_np).cuda()
        ref = ctx.ecg_forward(phi, p.tmpl)
        out = torch.full_like(ref, float("nan"))
        st = lib.gbp_ecg_forward_noalloc(C.c_void_p(L.data_ptr()), L.shape[0], L.shape[1],
                                         C.c_void_p(phi.data_ptr()), C.byref(tm),
                                         C.c_void_p(out.data_ptr()), stream)
        assert st == 0
        torch.cuda.synchronize()
        assert rel_l2(out.cpu().numpy(), ref.cpu().numpy()) < 1e-3
        assert rel_l2(out.cpu().numpy(), ref.cpu().numpy()) < 1e-5
    # sizes beyond the stated limits are rejected before any launch
    bad = gbp.make_template(S.Template(T=5000))
    assert lib.gbp_ecg_forward_noalloc(C.c_void_p(L.data_ptr()), L.shape[0], L.shape[1],
                                       C.c_void_p(phi.data_ptr()), C.byref(bad),
                                       C.c_void_p(out.data_ptr()), stream) == 1
    ctx.close()
