"""The library's host-side mesh validation (gbp_check_mesh / _2d, the checks
gbp_upload_mesh and gbp_upload_mesh_2d make before building anything) on
CPU: valid seeded meshes pass, each kind of defect is refused, and on random
meshes the verdict equals an independent orientation test in NumPy."""
import numpy as np

from paper_2308_08410_gb300 import gbp
from paper_2308_08410_gb300 import synth as S

OK, INVALID, BAD = 0, 1, 2


def test_valid_meshes_pass():
    m = S.kuhn_cube(5, 10.0)
    assert gbp.check_mesh(m.xyz, m.tets) == OK
    t = S.tri_square(9, 10.0, jitter=0.3, seed=2)
    assert gbp.check_mesh_2d(t.xy, t.tris) == OK
    xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], np.float32)
    assert gbp.check_mesh(xyz, np.array([[0, 1, 2, 3]])) == OK


def test_tet_defects_are_refused():
    m = S.kuhn_cube(4, 10.0)
    xyz, tets = m.xyz.copy(), m.tets.copy()
    for j in (0, len(tets) // 2, len(tets) - 1):
        t = tets.copy()
        t[j, [1, 2]] = t[j, [2, 1]]                       # inverted
        assert gbp.check_mesh(xyz, t) == BAD
        t = tets.copy()
        t[j, 3] = t[j, 0]                                  # repeated vertex
        assert gbp.check_mesh(xyz, t) == BAD
        t = tets.copy()
        t[j, 2] = m.n_v                                    # id out of range
        assert gbp.check_mesh(xyz, t) == BAD
        t = tets.copy()
        t[j, 1] = -1
        assert gbp.check_mesh(xyz, t) == BAD
    x = xyz.copy()
    x[7, 1] = np.nan
    assert gbp.check_mesh(x, tets) == BAD
    x = xyz.copy()
    x[3, 2] = np.inf
    assert gbp.check_mesh(x, tets) == BAD
    flat = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [1, 1, 0]], np.float32)   # zero volume
    assert gbp.check_mesh(flat, np.array([[0, 1, 2, 3]])) == BAD
    assert gbp.check_mesh(xyz[:3], np.array([[0, 1, 2, 0]])) == INVALID         # fewer than 4 vertices
    assert gbp.check_mesh(xyz, np.zeros((0, 4), np.int32)) == INVALID             # no tets


def test_triangle_defects_are_refused():
    t = S.tri_square(7, 10.0, jitter=0.2, seed=5)
    xy, tris = t.xy.copy(), t.tris.copy()
    for j in (0, len(tris) - 1):
        c = tris.copy()
        c[j, [1, 2]] = c[j, [2, 1]]                        # clockwise
        assert gbp.check_mesh_2d(xy, c) == BAD
        c = tris.copy()
        c[j, 2] = c[j, 0]
        assert gbp.check_mesh_2d(xy, c) == BAD
        c = tris.copy()
        c[j, 0] = t.n_v
        assert gbp.check_mesh_2d(xy, c) == BAD
    x = xy.copy()
    x[4, 0] = np.nan
    assert gbp.check_mesh_2d(x, tris) == BAD
    line = np.array([[0, 0], [1, 0], [2, 0]], np.float32)                        # zero area
    assert gbp.check_mesh_2d(line, np.array([[0, 1, 2]])) == BAD
    assert gbp.check_mesh_2d(xy[:2], np.array([[0, 1, 0]])) == INVALID
    assert gbp.check_mesh_2d(xy, np.zeros((0, 3), np.int32)) == INVALID


def test_orientation_verdict_matches_numpy_on_random_meshes():
    """Random tets / triangles over random points: refused exactly when some
    element has a non-positive orientation determinant (float64 NumPy
    determinant of the edge matrix; random points keep every determinant
    far from the tolerance)."""
    r = np.random.default_rng(11)
    for trial in range(40):
        xyz = r.uniform(-5, 5, (30, 3)).astype(np.float32)
        tets = np.stack([r.choice(30, 4, replace=False) for _ in range(12)]).astype(np.int32)
        e = xyz[tets[:, 1:]].astype(np.float64) - xyz[tets[:, :1]].astype(np.float64)
        det = np.linalg.det(e)
        if trial % 2 == 0:                                 # every other trial: flip the negative ones
            neg = det < 0
            tets[neg] = tets[neg][:, [0, 2, 1, 3]]
            det = np.abs(det)
        expect = OK if np.all(det > 0) else BAD
        assert gbp.check_mesh(xyz, tets) == expect, trial
        xy = r.uniform(-5, 5, (20, 2)).astype(np.float32)
        tris = np.stack([r.choice(20, 3, replace=False) for _ in range(10)]).astype(np.int32)
        a = xy[tris[:, 1]].astype(np.float64) - xy[tris[:, 0]]
        b = xy[tris[:, 2]].astype(np.float64) - xy[tris[:, 0]]
        cross = a[:, 0] * b[:, 1] - a[:, 1] * b[:, 0]
        if trial % 2 == 0:
            neg = cross < 0
            tris[neg] = tris[neg][:, [0, 2, 1]]
            cross = np.abs(cross)
        expect = OK if np.all(cross > 0) else BAD
        assert gbp.check_mesh_2d(xy, tris) == expect, trial
