"""Onset relocation (paper_2308_08410_gb300/relocate.py): tet adjacency and
walking point location on the Kuhn cube, checked against brute force."""
import numpy as np

from paper_2308_08410_gb300 import relocate as R
from paper_2308_08410_gb300 import synth as S


def test_neighbours_share_a_face_both_ways():
    m = S.kuhn_cube(5, 1.0)
    nbr = R.tet_neighbours(m.tets)
    n_bnd = 0
    for j in range(m.n_t):
        for s in range(4):
            k = nbr[j, s]
            face = set(np.delete(m.tets[j], s))
            if k < 0:
                n_bnd += 1
                continue
            assert face <= set(m.tets[k]) and k != j
            assert j in nbr[k]
    # boundary faces of a Kuhn cube: 6 sides x (n-1)^2 squares x 2 triangles
    assert n_bnd == 6 * 4 * 4 * 2


def test_walk_finds_the_containing_tet():
    m = S.kuhn_cube(7, 2.0)
    loc = R.TetLocator(m.xyz, m.tets)
    rng = np.random.default_rng(0)
    V = m.xyz.astype(np.float64)[m.tets]
    for _ in range(200):
        x = rng.uniform(0.0, 2.0, 3)
        j, b, inside = loc.walk(int(rng.integers(m.n_t)), x)
        assert inside
        assert b.min() >= -1e-9 and abs(b.sum() - 1) < 1e-9
        np.testing.assert_allclose(b @ V[j], x, atol=1e-9)


def test_walk_outside_stops_on_the_boundary():
    m = S.kuhn_cube(5, 1.0)
    loc = R.TetLocator(m.xyz, m.tets)
    j, b, inside = loc.walk(0, np.array([1.5, 0.5, 0.5]))
    assert not inside
    assert np.any(loc.nbr[j] < 0)
    c = R.TetLocator.clamp(b)
    assert c.min() > 0 and abs(c.sum() - 1) < 1e-12
