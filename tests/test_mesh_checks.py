"""The library's host-side mesh logic on CPU: the validation the uploads
make before building anything (gbp_check_mesh / _2d: valid seeded meshes
pass, each kind of defect is refused, and on random meshes the verdict
equals an independent orientation test in NumPy) and the adjacency they
build for the FIM and the adjoint (gbp_mesh_adjacency against a brute-force
construction)."""
import numpy as np
import pytest

from paper_2308_08410_gb300 import gbp
from paper_2308_08410_gb300 import synth as S

OK, INVALID, BAD = 0, 1, 2


def test_valid_meshes_pass():
    m = S.kuhn_cube(5, 10.0)
    assert gbp.check_mesh(m.xyz, m.tets) == OK
    m = S.delaunay_cloud(800, 5)
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


def brute_adjacency(tets, n_v):
    """Vertex->tet codes, neighbour sets and face records by definition."""
    n2t = [[] for _ in range(n_v)]
    nbr = [set() for _ in range(n_v)]
    for j, t in enumerate(tets):
        for q, v in enumerate(t):
            n2t[v].append(4 * j + q)
            nbr[v].update(int(u) for u in t if u != v)
    return n2t, [sorted(s) for s in nbr]


def check_adjacency(tets, n_v):
    a = gbp.mesh_adjacency(tets, n_v)
    n2t, nbr = brute_adjacency(tets, n_v)
    assert a["n2t_ptr"][0] == 0 and a["n2n_ptr"][0] == 0
    assert len(a["n2t"]) == 4 * len(tets)
    for i in range(n_v):
        row = a["n2t"][a["n2t_ptr"][i]:a["n2t_ptr"][i + 1]]
        assert list(row) == sorted(n2t[i]), i
        assert list(a["n2n"][a["n2n_ptr"][i]:a["n2n_ptr"][i + 1]]) == nbr[i], i
        for e in range(a["n2t_ptr"][i], a["n2t_ptr"][i + 1]):
            code = int(a["frec"][e, 3])
            j, s = code >> 2, code & 3
            assert code == a["n2t"][e] and tets[j][s] == i
            assert list(a["frec"][e, :3]) == [int(tets[j][q]) for q in range(4) if q != s]


def test_adjacency_matches_its_definition():
    """The vertex->tet lists (ascending tet * 4 + slot), the neighbour lists
    (sorted, unique) and the FIM's face records (the other three vertices in
    slot order) equal a brute-force construction: on a Kuhn cube, on random
    tets over a few vertex ids (shared faces, isolated vertices), on a
    single tet; and on an unstructured Delaunay mesh, whose vertices have up
    to 40 incident tets."""
    m = S.kuhn_cube(4, 10.0)
    check_adjacency(m.tets, m.n_v)
    m = S.delaunay_cloud(300, 6)
    check_adjacency(m.tets, m.n_v)
    r = np.random.default_rng(3)
    for _ in range(10):
        n_v = int(r.integers(5, 40))
        tets = np.stack([r.choice(n_v, 4, replace=False) for _ in range(int(r.integers(1, 30)))]).astype(np.int32)
        check_adjacency(tets, n_v)
    check_adjacency(np.array([[0, 1, 2, 3]], np.int32), 4)


def test_adjacency_errors():
    with pytest.raises(gbp.GbpError) as ei:
        gbp.mesh_adjacency(np.array([[0, 1, 2, 4]], np.int32), 4)
    assert ei.value.status == BAD
    with pytest.raises(gbp.GbpError) as ei:
        gbp.mesh_adjacency(np.zeros((0, 4), np.int32), 4)
    assert ei.value.status == INVALID
