"""The parameter map of the inverse loops (inverse.VertexLogToTet: per-vertex
log velocity -> per-element velocity exp(mean of the element's vertex
values)), single and batched, against torch autograd through the plain
gather on the CPU."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2308_08410_gb300 import synth as S  # noqa: E402
from paper_2308_08410_gb300.inverse import VertexLogToTet  # noqa: E402


@pytest.mark.parametrize("batched", [False, True])
@pytest.mark.parametrize("dim", [2, 3])
def test_vertex_log_to_element(batched, dim):
    m = S.kuhn_cube(4, 1.0) if dim == 3 else S.lv_slice(4, 12)
    cells = torch.from_numpy((m.tets if dim == 3 else m.tris).astype(np.int64))
    g = torch.Generator().manual_seed(0)
    shape = (3, m.n_v) if batched else (m.n_v,)
    logc = torch.randn(shape, generator=g, dtype=torch.float64)
    w = torch.randn(shape[:-1] + (cells.shape[0],), generator=g, dtype=torch.float64)
    a = logc.clone().requires_grad_(True)
    c = VertexLogToTet.apply(a, cells)
    (c * w).sum().backward()
    b = logc.clone().requires_grad_(True)
    c_ref = torch.exp(b[..., cells].mean(dim=-1))
    (c_ref * w).sum().backward()
    torch.testing.assert_close(c, c_ref, rtol=1e-14, atol=0)
    torch.testing.assert_close(a.grad, b.grad, rtol=1e-12, atol=1e-14)
