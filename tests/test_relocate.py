"""Onset relocation (paper_2308_08410_gb300/relocate.py): simplex adjacency
and walking point location on the Kuhn cube (tets) and the LV slice
(triangles), checked against brute force."""
import numpy as np

from paper_2308_08410_gb300 import relocate as R
from paper_2308_08410_gb300 import synth as S


def test_neighbours_share_a_face_both_ways():
    m = S.kuhn_cube(5, 1.0)
    nbr = R.simplex_neighbours(m.tets)
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
    loc = R.SimplexLocator(m.xyz, m.tets)
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
    loc = R.SimplexLocator(m.xyz, m.tets)
    j, b, inside = loc.walk(0, np.array([1.5, 0.5, 0.5]))
    assert not inside
    assert np.any(loc.nbr[j] < 0)
    c = R.SimplexLocator.clamp(b)
    assert c.min() > 0 and abs(c.sum() - 1) < 1e-12


def test_triangles_walk_and_adjacency():
    """The annular LV slice: every interior edge is shared by exactly two
    triangles (no boundary but the two circles), walks from random triangles
    land in a triangle that contains the point, and a point in the cavity
    stops on the inner boundary."""
    m = S.lv_slice()
    nbr = R.simplex_neighbours(m.tris)
    assert np.sum(nbr < 0) == 2 * 180  # inner and outer circle edges
    loc = R.SimplexLocator(m.xy, m.tris)
    rng = np.random.default_rng(1)
    V = m.xy.astype(np.float64)[m.tris]
    for _ in range(100):
        r, th = rng.uniform(18.5, 30.5), rng.uniform(0, 2 * np.pi)
        x = np.array([r * np.cos(th), r * np.sin(th)])
        j, b, inside = loc.walk(int(rng.integers(m.n_t)), x)
        if not inside:  # a walk may stop on the inner circle when the cavity is in the way
            assert np.any(loc.nbr[j] < 0)
            continue
        assert b.min() >= -1e-9
        np.testing.assert_allclose(b @ V[j], x, atol=1e-9)
    j, b, inside = loc.walk(0, np.array([0.0, 1.0]))
    assert not inside and np.any(loc.nbr[j] < 0)
