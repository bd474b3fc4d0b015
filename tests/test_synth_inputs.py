"""Pins of the seeded input generators (paper_2308_08410_gb300/synth.py)
against what geometry and the lead definitions fix: the Kuhn cube and the
triangulated square fill their domains with positively oriented elements,
the annular slice's area is that of the inscribed polygons, P1 lead-field rows sum
to zero (constant potentials carry no current), the 12-lead combination
obeys Einthoven's and Goldberger's identities and references V1-V6 to
Wilson's central terminal, fibres are unit vectors rotating with depth, and
onsets and noise follow their recipes."""
import numpy as np

from paper_2308_08410_gb300 import gbp
from paper_2308_08410_gb300 import synth as S


def cross2(u, v):
    return u[:, 0] * v[:, 1] - u[:, 1] * v[:, 0]


def tet_volumes(m):
    X = m.xyz.astype(np.float64)[m.tets]
    return np.linalg.det(X[:, 1:] - X[:, :1]) / 6.0


def test_kuhn_cube_fills_the_cube():
    for n in (2, 5, 9):
        m = S.kuhn_cube(n, 10.0)
        assert m.n_v == n ** 3 and m.n_t == 6 * (n - 1) ** 3
        v = tet_volumes(m)
        assert np.all(v > 0)
        np.testing.assert_allclose(v.sum(), 1000.0, rtol=1e-9)
        np.testing.assert_allclose(v, 1000.0 / m.n_t, rtol=1e-5)   # Kuhn: six equal tets per cell
        assert gbp.check_mesh(m.xyz, m.tets) == 0


def test_triangulated_square_and_annulus():
    t = S.tri_square(11, 10.0, jitter=0.3, seed=1)
    P = t.xy.astype(np.float64)[t.tris]
    a = 0.5 * cross2(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
    assert np.all(a > 0)
    np.testing.assert_allclose(a.sum(), 100.0, rtol=1e-6)
    for n_theta in (90, 180, 360):
        s = S.lv_slice(15, n_theta)
        P = s.xy.astype(np.float64)[s.tris]
        a = 0.5 * cross2(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
        assert np.all(a > 0) and gbp.check_mesh_2d(s.xy, s.tris) == 0
        # the annulus between two inscribed regular n-gons
        polygon = 0.5 * n_theta * np.sin(2 * np.pi / n_theta) * (31.0 ** 2 - 18.0 ** 2)
        np.testing.assert_allclose(a.sum(), polygon, rtol=1e-6)


def test_lead_field_rows_sum_to_zero():
    m = S.kuhn_cube(6, 10.0)
    el = S.fibonacci_sphere(8, 30.0, (5.0, 5.0, 5.0))
    L = S.lead_field(m, el).astype(np.float64)
    scale = np.abs(L).sum(axis=1)
    assert np.all(np.abs(L.sum(axis=1)) <= 1e-5 * scale)
    t = S.tri_square(9, 10.0, jitter=0.2, seed=3)
    L2 = S.lead_field_2d(t, np.array([[30.0, 0.0], [0.0, 30.0], [-30.0, -5.0]])).astype(np.float64)
    assert np.all(np.abs(L2.sum(axis=1)) <= 1e-5 * np.abs(L2).sum(axis=1))


def test_twelve_lead_identities():
    C = S.twelve_lead_matrix()
    I, II, III, aVR, aVL, aVF = C[:6]
    np.testing.assert_allclose(II, I + III, atol=1e-15)              # Einthoven
    np.testing.assert_allclose(aVR + aVL + aVF, 0.0, atol=1e-15)      # Goldberger
    np.testing.assert_allclose(C.sum(axis=1), 0.0, atol=1e-15)        # a common potential cancels
    wct = np.zeros(10)
    wct[:3] = 1.0 / 3.0
    for v in range(6):
        e = np.zeros(10)
        e[4 + v] = 1.0
        np.testing.assert_allclose(C[6 + v], e - wct, atol=1e-15)
    assert np.all(C[:, 3] == 0)                                       # RL is ground


def test_fibres_are_unit_and_rotate_with_depth():
    m = S.kuhn_cube(7, 10.0)
    f = S.fibres_cube(m, 10.0).astype(np.float64)
    np.testing.assert_allclose(np.linalg.norm(f, axis=1), 1.0, atol=1e-6)
    assert np.all(f[:, 2] == 0)
    zc = m.xyz.astype(np.float64)[m.tets][:, :, 2].mean(axis=1)
    ang = np.rad2deg(np.arctan2(f[:, 1], f[:, 0]))
    np.testing.assert_allclose(ang, -60.0 + 12.0 * zc, atol=1e-4)


def test_onsets_and_noise_follow_their_recipes():
    m = S.kuhn_cube(6, 10.0)
    ons = S.onsets_element(m, 7, seed=2, tmin=1.0, tmax=4.0)
    assert ons.kind == S.ONSET_ELEMENT and len(set(ons.idx.tolist())) == 7
    assert np.all((ons.idx >= 0) & (ons.idx < m.n_t))
    np.testing.assert_allclose(ons.bary.sum(axis=1), 1.0, atol=1e-6)
    assert np.all(ons.bary >= 0) and np.all((ons.t >= 1.0) & (ons.t <= 4.0))
    V = np.stack([np.sin(np.linspace(0, 20, 20000)) * (l + 1) for l in range(3)])
    noisy = S.add_noise(V, 0.05, seed=7).astype(np.float64)
    rms = np.sqrt((V ** 2).mean(axis=1))
    np.testing.assert_allclose((noisy - V).std(axis=1) / rms, 0.05, rtol=0.03)
    assert np.array_equal(S.add_noise(V, 0.05, seed=7), S.add_noise(V, 0.05, seed=7))   # seeded
