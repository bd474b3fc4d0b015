"""The frozen-parent-graph adjoint (oracle.adjoint, Sec. II-C) against
automatic differentiation through the unrolled iterations of Algorithm 2
(oracle/unrolled.py, written separately in PyTorch from the same equations).
On meshes without exact ties between faces both are the derivative of the
same piecewise-smooth function, so they agree to rounding; that includes
meshes whose parent graph has cycles (the adjoint solves (I - P^T) mu = lam
exactly there, the unrolled gradient is the converged Neumann series).  At
exact ties (uniform velocities on the Kuhn cube) the loss has a kink and the
two pick different subgradients, so the inputs here are jittered."""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from oracle import unrolled as UR  # noqa: E402
from paper_2308_08410_gb300 import synth as S  # noqa: E402


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def cycle_vertices(mesh, parent, alpha):
    rows, cols = [], []
    for i in np.nonzero(parent >= 0)[0]:
        j, s = parent[i] >> 2, parent[i] & 3
        f = [mesh.tets[j][q] for q in range(4) if q != s]
        for q in range(3):
            if alpha[i][q] != 0:
                rows.append(i)
                cols.append(f[q])
    G = sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(mesh.n_v, mesh.n_v))
    _, lab = connected_components(G, directed=True, connection="strong")
    return int((np.bincount(lab)[lab] > 1).sum()), int(np.bincount(lab).max())


def compare(p, cf, ct, onsets, tol=1e-10):
    ek = O.eikonal(p.mesh, p.fib, (cf * 1.07).astype(np.float32), ct, onsets)
    target = S.add_noise(O.ecg(p.L, ek["phi"], p.tmpl), 0.05, 3)
    ref = O.forward_backward(p.mesh, p.fib, cf, ct, onsets, p.L, p.tmpl, target)
    g = UR.gradients(p.mesh, p.fib, cf, ct, onsets, p.L, p.tmpl, target)
    np.testing.assert_allclose(g["phi"], ref["phi"], rtol=1e-12, atol=1e-12)
    assert abs(g["loss"] - ref["loss"]) <= 1e-12 * ref["loss"]
    for k in ("d_cf", "d_ct", "d_t"):
        assert rel_l2(g[k], ref[k]) < tol, (k, rel_l2(g[k], ref[k]))
    if onsets.kind == O.ONSET_ELEMENT:
        assert rel_l2(g["d_x"], ref["d_x"]) < tol
    return ref


def jitter(n_t, seed):
    r = np.random.default_rng(seed)
    return (1 + 0.05 * r.standard_normal(n_t)).astype(np.float32)


def test_unrolled_matches_adjoint_element_onsets():
    p = S.make_c1(n=6, seed=1)
    cf, ct = (p.cf * jitter(p.mesh.n_t, 5)).astype(np.float32), (p.ct * jitter(p.mesh.n_t, 6)).astype(np.float32)
    compare(p, cf, ct, S.onsets_element(p.mesh, 3, seed=9, tmin=0.0, tmax=3.0))


def test_unrolled_matches_adjoint_nodal_onsets():
    p = S.make_c1(n=7, seed=1)
    cf, ct = (p.cf * jitter(p.mesh.n_t, 7)).astype(np.float32), (p.ct * jitter(p.mesh.n_t, 8)).astype(np.float32)
    compare(p, cf, ct, p.onsets)


def test_unrolled_matches_adjoint_with_parent_cycles():
    """10^3 cube, per-tet velocities jittered by 5 %: the discrete fixed
    point's parent graph has a 5-vertex strongly connected component."""
    p = S.make_c3(n=10, seed=2)
    r = np.random.default_rng(102)
    cf = (0.6 * (1 + 0.05 * r.standard_normal(p.mesh.n_t))).astype(np.float32)
    ct = (0.3 * (1 + 0.05 * r.standard_normal(p.mesh.n_t))).astype(np.float32)
    ons = S.Onsets(p.onsets.kind, p.onsets.idx, (10 + r.uniform(-2, 2, p.onsets.K)).astype(np.float32),
                   p.onsets.bary)
    ref = compare(p, cf, ct, ons)
    assert cycle_vertices(p.mesh, ref["parent"], ref["alpha"])[0] > 0


def test_unrolled_matches_adjoint_on_an_unstructured_mesh():
    """A 500-point Delaunay mesh (synth.make_delaunay: jittered velocities,
    element onsets) whose parent graph holds a 5-vertex cycle: the
    differentiated Jacobi iterations and the frozen-graph adjoint agree."""
    p = S.make_delaunay(n_pts=500, seed=1)
    ref = compare(p, p.cf, p.ct, p.onsets)
    assert cycle_vertices(p.mesh, ref["parent"], ref["alpha"])[1] > 2
