"""Host logic of the learned initialiser on CPU: the c5 surface (every
boundary triangle of the Kuhn cube, each owned by one tet), draws of the
prior (sites on the surface with barycentric coordinates of the owning
tet), the network target's encoding and its decoding back to parameters,
and the projection of a point onto a surface triangle."""
import numpy as np
import pytest

from paper_2308_08410_gb300 import learned_init as LI


@pytest.fixture(scope="module")
def c5():
    return LI.make_c5(n=8)


def test_surface_is_the_cube_boundary(c5):
    m = c5.problem.mesh
    n = 8
    assert len(c5.surf_tet) == 6 * 2 * (n - 1) ** 2
    X = m.xyz.astype(np.float64)
    for f, (j, s) in enumerate(zip(c5.surf_tet, c5.surf_opp)):
        tri = c5.surf_tri[f]
        assert sorted(tri) == sorted(int(v) for q, v in enumerate(m.tets[j]) if q != s)
        P = X[tri]
        on_face = [(np.allclose(P[:, r], 0.0) or np.allclose(P[:, r], c5.side)) for r in range(3)]
        assert any(on_face), f
    # each boundary triangle appears once
    assert len({tuple(sorted(t)) for t in c5.surf_tri}) == len(c5.surf_tri)


def test_prior_draws_lie_on_the_surface(c5):
    r = np.random.default_rng(1)
    for _ in range(5):
        prm = LI.sample_params(c5, r)
        assert LI.CF_RANGE[0] <= prm.cf <= LI.CF_RANGE[1] and LI.CT_RANGE[0] <= prm.ct <= LI.CT_RANGE[1]
        assert LI.CE_RANGE[0] <= prm.ce <= LI.CE_RANGE[1]
        assert np.all((prm.t >= LI.T_RANGE[0]) & (prm.t <= LI.T_RANGE[1]))
        np.testing.assert_allclose(prm.bary.sum(axis=1), 1.0, atol=1e-6)
        assert np.all(prm.bary >= 0)
        x = LI.site_xyz(c5, prm)
        d = np.minimum(np.abs(x), np.abs(x - c5.side)).min(axis=1)
        assert np.all(d < 1e-5)                             # a coordinate at 0 or side: on the boundary


def test_encode_then_decode_recovers_the_parameters(c5):
    r = np.random.default_rng(2)
    for _ in range(5):
        prm = LI.sample_params(c5, r)
        y = LI.encode(c5, prm)
        assert y.shape == (4 * LI.N_SITES + 3,)
        back = LI.decode(c5, y)
        assert abs(back.cf - prm.cf) < 1e-5 and abs(back.ct - prm.ct) < 1e-5 and abs(back.ce - prm.ce) < 1e-5
        # sites come back sorted by onset time, on the surface, near where they were
        o = np.argsort(prm.t, kind="stable")
        np.testing.assert_allclose(back.t, prm.t[o], atol=1e-4)
        x0, x1 = LI.site_xyz(c5, prm)[o], LI.site_xyz(c5, back)
        h = c5.side / 7                                    # edge length of the 8^3 cube
        assert np.all(np.linalg.norm(x1 - x0, axis=1) < 0.5 * h)


def test_plane_projection_onto_a_triangle():
    """Points whose plane projection falls inside the triangle map to their
    closest point (checked against dense sampling of the triangle); any
    point maps to a point of the triangle, on its boundary when the
    projection falls outside."""
    r = np.random.default_rng(3)
    u = np.linspace(0, 1, 301)
    U, V = np.meshgrid(u, u)
    keep = U + V <= 1
    B = np.stack([1 - U[keep] - V[keep], U[keep], V[keep]], axis=1)
    for _ in range(20):
        tri = r.normal(size=(3, 3))
        n = np.cross(tri[1] - tri[0], tri[2] - tri[0])
        n /= np.linalg.norm(n)
        inside = r.dirichlet(np.ones(3)) @ tri + r.normal() * n       # projects inside
        w = LI._closest_bary(tri, inside)
        d = np.linalg.norm(w @ tri - inside)
        assert d <= np.linalg.norm(B @ tri - inside, axis=1).min() + 1e-9
        a = r.uniform(0.1, 1.2)
        outside = np.array([-0.3, a, 1.3 - a]) @ tri + r.normal() * n      # beyond the edge opposite vertex 0
        w = LI._closest_bary(tri, outside)
        assert np.all(w >= 0) and abs(w.sum() - 1) < 1e-12 and w[0] == 0.0
