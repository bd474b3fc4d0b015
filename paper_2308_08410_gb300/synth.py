"""Seeded synthetic inputs for the Geodesic-BP hot path.

This module is shared by the CUDA path and by the FP64 oracle's tests, so it
holds NO arithmetic of the method itself (no metric tensor, no local solver,
no eikonal iteration, no ECG contraction, no gradient).  It only produces the
*inputs* the paper's method consumes:

* P1 simplicial meshes (Sec. II-A: "simplicial triangulation", one metric per
  element): Kuhn-split cubes, voxel-Kuhn biventricular shells and
  Delaunay tetrahedralisations of random points;
* fibre directions and the two conduction velocities per element (the
  orthotropic conduction tensor of Eq. (1) is built from them by each side on
  its own);
* onset sites X0 = {(x_i, t_i)} (Eq. (1)), nodal or inside an element
  (Eq. upwind_xi);
* the discretised lead-field operator B of Eq. (integral_potential_ecg)
  (Sec. II-D), assembled here with first-order elements and an
  infinite-medium lead field Z = 1/(4 pi |x - e|) because the torso solve of
  Eq. (lead_field) needs torso meshes the paper does not provide;
* activation maps for the ECG precision study and 12-lead combinations
  (Wilson's central terminal, Sec. II-D).

All float outputs are float32: both the CUDA path and the oracle read the same
float32 arrays (the oracle widens them to float64), so the geometry is
identical on both sides.
"""
from __future__ import annotations

import dataclasses
import itertools
import math

import numpy as np

__all__ = [
    "Mesh", "Onsets", "Template", "Problem", "TriMesh", "Problem2D", "make_2d",
    "lv_slice", "lead_field_2d", "locate_2d", "make_2d_torso",
    "kuhn_cube", "voxel_kuhn", "biv_shell_mask", "delaunay_cloud",
    "fibres_cube", "fibres_biv", "smooth_field", "nodal_to_tet_mean",
    "fibonacci_sphere", "torso_electrodes", "lead_field", "twelve_lead_matrix",
    "onsets_nodal", "onsets_element", "onsets_surface",
    "add_noise", "boundary_faces",
    "make_c1", "make_c2", "make_c3", "make_c4_phi", "make_c4", "make_delaunay",
    "c5_sample_params", "random_faces",
]

# ----------------------------------------------------------------------------
# containers
# ----------------------------------------------------------------------------

ONSET_NODAL = 0
ONSET_ELEMENT = 1


@dataclasses.dataclass
class Mesh:
    xyz: np.ndarray   # float32 [n_v, 3], mm
    tets: np.ndarray  # int32 [n_t, 4], positively oriented

    @property
    def n_v(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def n_t(self) -> int:
        return int(self.tets.shape[0])


@dataclasses.dataclass
class Onsets:
    """Activation sites X0 (Eq. (1)).

    kind == ONSET_NODAL: ``idx`` are vertex ids, ``bary`` is unused.
    kind == ONSET_ELEMENT: ``idx`` are tet ids and ``bary`` [K,4] the
    barycentric coordinates of x_i inside that tet (Eq. upwind_xi).
    """
    kind: int
    idx: np.ndarray   # int32 [K]
    t: np.ndarray     # float32 [K], ms
    bary: np.ndarray | None = None  # float32 [K, 4]

    @property
    def K(self) -> int:
        return int(self.idx.shape[0])


@dataclasses.dataclass
class Template:
    """Template action potential of Eq. (tanh_waveform), sampled at
    t_s = t0 + s*dt, s = 0..T-1."""
    K0: float = -80.0
    K1: float = 20.0
    tau: float = 1.0
    t0: float = 0.0
    dt: float = 1.0
    T: int = 150


@dataclasses.dataclass
class Problem:
    name: str
    mesh: Mesh
    fib: np.ndarray   # float32 [n_t, 3], unit
    cf: np.ndarray    # float32 [n_t], mm/ms
    ct: np.ndarray    # float32 [n_t], mm/ms
    onsets: Onsets
    L: np.ndarray     # float32 [N, n_v]
    tmpl: Template
    extra: dict = dataclasses.field(default_factory=dict)


# ----------------------------------------------------------------------------
# meshes
# ----------------------------------------------------------------------------

# The six Kuhn (path) simplices of the unit cube share the main diagonal
# (0,0,0)-(1,1,1); using the same split in every cell gives a conforming mesh.
_KUHN = []
for _perm in itertools.permutations(range(3)):
    _c = [np.zeros(3, dtype=np.int64)]
    for _ax in _perm:
        _n = _c[-1].copy()
        _n[_ax] = 1
        _c.append(_n)
    _c = np.array(_c)
    _sgn = np.linalg.det((_c[1:] - _c[0]).astype(float))
    if _sgn < 0:
        _c[[1, 2]] = _c[[2, 1]]
    _KUHN.append(_c)
_KUHN = np.array(_KUHN)  # [6, 4, 3] corner offsets


def kuhn_cube(n: int, side: float = 10.0) -> Mesh:
    """n x n x n vertex grid on [0, side]^3, 6 Kuhn tets per cell."""
    h = side / (n - 1)
    g = np.arange(n)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")  # node (i,j,k)
    # node id = i + n*(j + n*k)  (x fastest)
    xyz = np.stack([X.transpose(2, 1, 0).ravel(), Y.transpose(2, 1, 0).ravel(),
                    Z.transpose(2, 1, 0).ravel()], axis=1).astype(np.float64) * h
    c = np.arange(n - 1)
    CI, CJ, CK = np.meshgrid(c, c, c, indexing="ij")
    base = np.stack([CI.transpose(2, 1, 0).ravel(), CJ.transpose(2, 1, 0).ravel(),
                     CK.transpose(2, 1, 0).ravel()], axis=1)  # [n_cells,3]
    corners = base[:, None, None, :] + _KUHN[None]  # [cells, 6, 4, 3]
    ids = corners[..., 0] + n * (corners[..., 1] + n * corners[..., 2])
    tets = ids.reshape(-1, 4).astype(np.int32)
    return Mesh(xyz.astype(np.float32), tets)


def kuhn_slab(n: int, layers: int, hz: float, side: float = 10.0) -> Mesh:
    """The bottom `layers` vertex layers of the n^3 Kuhn cube on [0, side]^3,
    with the layer spacing squashed to hz (mm): a slab of sliver tets whose
    vertices lie close to the planes of their opposite faces."""
    m = kuhn_cube(n, side)
    xyz = m.xyz.astype(np.float64)
    h = side / (n - 1)
    keep_v = xyz[:, 2] <= (layers - 1) * h + 1e-9
    keep_t = keep_v[m.tets].all(axis=1)
    idx = -np.ones(len(xyz), np.int64)
    idx[keep_v] = np.arange(int(keep_v.sum()))
    tets = idx[m.tets[keep_t]].astype(np.int32)
    xyz = xyz[keep_v]
    xyz[:, 2] *= hz / h
    return Mesh(xyz.astype(np.float32), tets)


def delaunay_cloud(n_pts: int, seed: int, side: float = 10.0, sliver: float = 0.02) -> Mesh:
    """Unstructured mesh: the Delaunay tetrahedralisation (scipy) of n_pts
    uniform random points in [0, side]^3, each tet oriented positively, tets
    below `sliver` x the mean volume dropped, unused points removed.  About
    26 incident tets and 15 neighbours per vertex on average, up to ~80 and
    ~45 at 20,000 points (a Kuhn lattice: at most 24 and 14)."""
    from scipy.spatial import Delaunay
    r = np.random.default_rng(seed)
    pts = r.uniform(0.0, side, (n_pts, 3))
    t = Delaunay(pts).simplices.astype(np.int64)
    det = np.linalg.det(pts[t[:, 1:]] - pts[t[:, :1]])
    neg = det < 0
    t[neg] = t[neg][:, [0, 2, 1, 3]]
    vol = np.abs(det) / 6.0
    t = t[vol > sliver * vol.mean()]
    used = np.unique(t)
    remap = np.full(n_pts, -1, np.int64)
    remap[used] = np.arange(used.size)
    return Mesh(pts[used].astype(np.float32), remap[t].astype(np.int32))


def voxel_kuhn(mask: np.ndarray, h: float, origin) -> Mesh:
    """Kuhn-split every voxel cell with mask[i,j,k] True (cell spans
    origin + h*[i,i+1] x ...).  Unused grid nodes are dropped."""
    nx, ny, nz = mask.shape
    cells = np.argwhere(mask)  # [c, 3]
    corners = cells[:, None, None, :] + _KUHN[None]  # [c, 6, 4, 3]
    gid = corners[..., 0] + (nx + 1) * (corners[..., 1] + (ny + 1) * corners[..., 2])
    gid = gid.reshape(-1, 4)
    used, inv = np.unique(gid.ravel(), return_inverse=True)
    tets = inv.reshape(-1, 4).astype(np.int32)
    gi = used % (nx + 1)
    gj = (used // (nx + 1)) % (ny + 1)
    gk = used // ((nx + 1) * (ny + 1))
    xyz = np.stack([gi, gj, gk], axis=1).astype(np.float64) * h + np.asarray(origin, float)
    return Mesh(xyz.astype(np.float32), tets)


def _tet_centroids(mesh: Mesh) -> np.ndarray:
    return mesh.xyz.astype(np.float64)[mesh.tets].mean(axis=1)


def boundary_faces(mesh: Mesh) -> np.ndarray:
    """Triangles [F,3] that belong to exactly one tet (the mesh surface)."""
    loc = np.array([[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]])
    f = mesh.tets[:, loc].reshape(-1, 3)
    fs = np.sort(f, axis=1)
    _, inv, cnt = np.unique(fs, axis=0, return_inverse=True, return_counts=True)
    keep = cnt[inv.ravel()] == 1
    return f[keep].astype(np.int32)


# --- biventricular shell ------------------------------------------------------

# Geometry (mm).  LV: truncated prolate spheroid shell, long axis z, apex at
# negative z, 10 mm wall.  RV: thinner (4 mm) shell wrapped around the septal
# (negative x) side; its cavity is bounded by the LV wall (the septum).
_LV_OUT = (25.0, 25.0, 45.0)
_LV_IN = (15.0, 15.0, 35.0)
_RV_C = (-14.0, 0.0, -4.0)
_RV_OUT = (32.0, 27.0, 41.0)
_RV_IN = (28.0, 23.0, 37.0)
_Z_BASE = 12.0


def _ell(p, c, a):
    return (((p[..., 0] - c[0]) / a[0]) ** 2 + ((p[..., 1] - c[1]) / a[1]) ** 2
            + ((p[..., 2] - c[2]) / a[2]) ** 2)


def biv_shell_mask(p: np.ndarray):
    """Region labels for points p[...,3]: 0 outside, 1 LV wall, 2 RV wall."""
    lv_out = _ell(p, (0, 0, 0), _LV_OUT) <= 1.0
    lv_in = _ell(p, (0, 0, 0), _LV_IN) < 1.0
    rv_out = _ell(p, _RV_C, _RV_OUT) <= 1.0
    rv_in = _ell(p, _RV_C, _RV_IN) < 1.0
    base = p[..., 2] <= _Z_BASE
    lv = lv_out & ~lv_in & base
    rv = rv_out & ~rv_in & ~lv_out & base
    lab = np.zeros(p.shape[:-1], dtype=np.int8)
    lab[lv] = 1
    lab[rv] = 2
    return lab


def _transmural_lv(p):
    """0 at the LV endocardium, 1 at the epicardium (radial spheroid param)."""
    r_in = np.sqrt(_ell(p, (0, 0, 0), _LV_IN))
    r_out = np.sqrt(_ell(p, (0, 0, 0), _LV_OUT))
    # r_in = 1 on the inner surface, r_out = 1 on the outer surface
    a = r_in - 1.0
    b = 1.0 - r_out
    return np.clip(a / np.maximum(a + b, 1e-12), 0.0, 1.0)


def _transmural_rv(p):
    r_in = np.sqrt(_ell(p, _RV_C, _RV_IN))
    r_out = np.sqrt(_ell(p, _RV_C, _RV_OUT))
    a = r_in - 1.0
    b = 1.0 - r_out
    return np.clip(a / np.maximum(a + b, 1e-12), 0.0, 1.0)


# ----------------------------------------------------------------------------
# fibres, fields
# ----------------------------------------------------------------------------

def fibres_cube(mesh: Mesh, side: float = 10.0) -> np.ndarray:
    """Fibres in the xy-plane rotating linearly with depth: angle -60 deg at
    z=0 to +60 deg at z=side, evaluated at each tet centroid."""
    zc = _tet_centroids(mesh)[:, 2]
    th = np.deg2rad(-60.0 + 120.0 * zc / side)
    f = np.stack([np.cos(th), np.sin(th), np.zeros_like(th)], axis=1)
    return f.astype(np.float32)


def fibres_biv(mesh: Mesh, labels: np.ndarray, tm: np.ndarray) -> np.ndarray:
    """Rule-based fibres: helix angle -60 deg (epicardium, tm=1) to +60 deg
    (endocardium, tm=0) in the local circumferential/longitudinal plane."""
    pc = _tet_centroids(mesh)
    cen = np.where(labels[:, None] == 2, np.asarray(_RV_C, float)[None], 0.0)
    d = pc - cen
    circ = np.stack([-d[:, 1], d[:, 0], np.zeros(len(d))], axis=1)
    nrm = np.linalg.norm(circ, axis=1, keepdims=True)
    circ = np.where(nrm > 1e-9, circ / np.maximum(nrm, 1e-12), np.array([[1.0, 0.0, 0.0]]))
    lon = np.array([0.0, 0.0, 1.0])
    # make the longitudinal direction orthogonal to the radial direction
    rad = d / np.maximum(np.linalg.norm(d, axis=1, keepdims=True), 1e-12)
    lon = lon[None] - (rad @ lon)[:, None] * rad
    lon = lon - np.sum(lon * circ, axis=1, keepdims=True) * circ
    lon /= np.maximum(np.linalg.norm(lon, axis=1, keepdims=True), 1e-12)
    helix = np.deg2rad(60.0 - 120.0 * tm)
    f = np.cos(helix)[:, None] * circ + np.sin(helix)[:, None] * lon
    f /= np.linalg.norm(f, axis=1, keepdims=True)
    return f.astype(np.float32)


def smooth_field(xyz: np.ndarray, n_bumps: int, seed: int, width=(1.5, 3.0),
                 lo=None, hi=None) -> np.ndarray:
    """Sum of seeded Gaussian bumps, scaled to max |value| = 1."""
    rng = np.random.default_rng(seed)
    x = xyz.astype(np.float64)
    lo = x.min(axis=0) if lo is None else np.asarray(lo, float)
    hi = x.max(axis=0) if hi is None else np.asarray(hi, float)
    out = np.zeros(len(x))
    for _ in range(n_bumps):
        c = rng.uniform(lo, hi)
        w = rng.uniform(*width)
        a = rng.uniform(-1.0, 1.0)
        out += a * np.exp(-np.sum((x - c) ** 2, axis=1) / (2 * w * w))
    m = np.max(np.abs(out))
    return out / m if m > 0 else out


def nodal_to_tet_mean(mesh: Mesh, nodal: np.ndarray) -> np.ndarray:
    """Mean of the four vertex values per tet (float64)."""
    return np.asarray(nodal, float)[mesh.tets].mean(axis=1)


# ----------------------------------------------------------------------------
# electrodes, lead fields
# ----------------------------------------------------------------------------

def fibonacci_sphere(k: int, radius: float, centre) -> np.ndarray:
    i = np.arange(k) + 0.5
    phi = np.arccos(1 - 2 * i / k)
    th = np.pi * (1 + 5 ** 0.5) * i
    p = np.stack([np.cos(th) * np.sin(phi), np.sin(th) * np.sin(phi), np.cos(phi)], axis=1)
    return p * radius + np.asarray(centre, float)


# Standard electrode order for 12-lead ECGs: RA, LA, LL, RL, V1..V6
_TORSO_AX = np.array([75.0, 50.0, 125.0])  # semi-axes of a 150x100x250 mm ellipsoid


def torso_electrodes(centre=(-10.0, 15.0, 20.0)) -> np.ndarray:
    """10 electrodes on an ellipsoidal torso (150x100x250 mm) around the
    heart: RA, LA, LL, RL and the precordial V1..V6 (front = -y)."""
    c = np.asarray(centre, float)
    dirs = [(-0.75, 0.0, 0.65), (0.75, 0.0, 0.65), (0.45, 0.0, -0.85), (-0.45, 0.0, -0.85)]
    for ang in (-100.0, -80.0, -62.0, -45.0, -25.0, 0.0):  # around the chest at heart level
        a = np.deg2rad(ang)
        dirs.append((np.cos(a), np.sin(a), -0.12))
    out = []
    for d in dirs:
        d = np.asarray(d, float)
        # ray from torso centre, scaled onto the ellipsoid surface
        s = 1.0 / math.sqrt(np.sum((d / _TORSO_AX) ** 2))
        out.append(c + s * d)
    return np.array(out)


def twelve_lead_matrix() -> np.ndarray:
    """12x10 combination of electrode potentials (RA,LA,LL,RL,V1..V6) into
    I, II, III, aVR, aVL, aVF, V1..V6 referenced to Wilson's central terminal."""
    C = np.zeros((12, 10))
    RA, LA, LL = 0, 1, 2
    C[0, LA], C[0, RA] = 1, -1
    C[1, LL], C[1, RA] = 1, -1
    C[2, LL], C[2, LA] = 1, -1
    C[3, RA], C[3, LA], C[3, LL] = 1, -0.5, -0.5
    C[4, LA], C[4, RA], C[4, LL] = 1, -0.5, -0.5
    C[5, LL], C[5, RA], C[5, LA] = 1, -0.5, -0.5
    for v in range(6):
        C[6 + v, 4 + v] = 1.0
        C[6 + v, [RA, LA, LL]] -= 1.0 / 3.0
    return C


def lead_field(mesh: Mesh, electrodes: np.ndarray, combos: np.ndarray | None = None,
               chunk: int = 1 << 19) -> np.ndarray:
    """Discrete lead-field operator L [N, n_v] of Eq. (integral_potential_ecg)
    with unit isotropic intracellular conductivity: L_l = K Z_l with K the P1
    stiffness matrix and Z_l(x) = 1/(4 pi |x - e_l|) the infinite-medium lead
    field.  Assembled element by element as
    L_l[a] += vol_t * grad(lambda_a) . grad(Z_h)|_t  (no global K needed)."""
    x = mesh.xyz.astype(np.float64)
    E = np.asarray(electrodes, float)
    Z = 1.0 / (4.0 * np.pi * np.linalg.norm(x[None, :, :] - E[:, None, :], axis=2))  # [ne, n_v]
    ne = E.shape[0]
    L = np.zeros((ne, mesh.n_v))
    for s in range(0, mesh.n_t, chunk):
        t = mesh.tets[s:s + chunk]
        v = x[t]  # [c,4,3]
        J = (v[:, 1:] - v[:, :1]).transpose(0, 2, 1)  # columns = edges
        det = np.linalg.det(J)
        Jinv = np.linalg.inv(J)  # rows: grad lambda_1..3
        g = np.concatenate([-Jinv.sum(axis=1, keepdims=True), Jinv], axis=1)  # [c,4,3]
        vol = det / 6.0
        for e in range(ne):
            gz = np.einsum("cai,ca->ci", g, Z[e][t])  # grad Z_h per tet
            contrib = vol[:, None] * np.einsum("cai,ci->ca", g, gz)
            L[e] += np.bincount(t.ravel(), weights=contrib.ravel(), minlength=mesh.n_v)
    if combos is not None:
        L = np.asarray(combos, float) @ L
    return L.astype(np.float32)


# ----------------------------------------------------------------------------
# onsets
# ----------------------------------------------------------------------------

def onsets_nodal(n_v: int, K: int, seed: int, tmax: float, candidates=None) -> Onsets:
    rng = np.random.default_rng(seed)
    pool = np.arange(n_v) if candidates is None else np.asarray(candidates)
    idx = rng.choice(pool, size=K, replace=False).astype(np.int32)
    t = rng.uniform(0.0, tmax, size=K).astype(np.float32)
    return Onsets(ONSET_NODAL, idx, t)


def onsets_element(mesh: Mesh, K: int, seed: int, tmin: float, tmax: float,
                   tets=None, bary_floor: float = 0.05) -> Onsets:
    """K sites at random points strictly inside random tets."""
    rng = np.random.default_rng(seed)
    pool = np.arange(mesh.n_t) if tets is None else np.asarray(tets)
    idx = rng.choice(pool, size=K, replace=False).astype(np.int32)
    b = rng.dirichlet(np.ones(4), size=K)
    b = bary_floor + (1 - 4 * bary_floor) * b
    t = rng.uniform(tmin, tmax, size=K).astype(np.float32)
    return Onsets(ONSET_ELEMENT, idx, t, b.astype(np.float32))


def onsets_surface(mesh: Mesh, K: int, seed: int, tmin: float, tmax: float) -> Onsets:
    """K sites on boundary triangles, represented as element onsets in the tet
    owning the triangle (barycentric weight 0 on the opposite vertex)."""
    rng = np.random.default_rng(seed)
    loc = np.array([[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]])
    f = mesh.tets[:, loc].reshape(-1, 3)
    fs = np.sort(f, axis=1)
    _, inv, cnt = np.unique(fs, axis=0, return_inverse=True, return_counts=True)
    surf = np.nonzero(cnt[inv.ravel()] == 1)[0]  # flat index tet*4 + opposite slot
    pick = rng.choice(surf, size=K, replace=False)
    tet = (pick // 4).astype(np.int32)
    opp = pick % 4
    b3 = rng.dirichlet(np.ones(3), size=K)
    b3 = 0.05 + 0.85 * b3
    b = np.zeros((K, 4))
    for k in range(K):
        b[k, loc[opp[k]]] = b3[k]
    t = rng.uniform(tmin, tmax, size=K).astype(np.float32)
    return Onsets(ONSET_ELEMENT, tet, t, b.astype(np.float32))


def add_noise(V: np.ndarray, rel: float, seed: int) -> np.ndarray:
    """Per-lead Gaussian noise with sigma_l = rel * RMS_t(V_l)."""
    rng = np.random.default_rng(seed)
    V = np.asarray(V, float)
    sig = rel * np.sqrt(np.mean(V * V, axis=1, keepdims=True))
    return (V + sig * rng.standard_normal(V.shape)).astype(np.float32)


# ----------------------------------------------------------------------------
# configurations
# ----------------------------------------------------------------------------

def make_c1(n: int = 20, seed: int = 0, side: float = 10.0, n_leads: int = 8,
            T: int = 150) -> Problem:
    """Plain method, small: n^3-vertex Kuhn cube (10 mm), fibres -60..+60 deg
    with depth, c_f=0.6 / c_t=0.3 mm/ms, 3 nodal onsets t~U[0,10] ms,
    8 electrodes on a 30 mm sphere, 50 tanh(2(t-phi)) - 30 mV, T=150 @ 1 ms."""
    mesh = kuhn_cube(n, side)
    fib = fibres_cube(mesh, side)
    cf = np.full(mesh.n_t, 0.6, np.float32)
    ct = np.full(mesh.n_t, 0.3, np.float32)
    ons = onsets_nodal(mesh.n_v, 3, seed, 10.0)
    el = fibonacci_sphere(n_leads, 30.0, (side / 2,) * 3)
    L = lead_field(mesh, el)
    return Problem("c1", mesh, fib, cf, ct, ons, L, Template(-80.0, 20.0, 1.0, 0.0, 1.0, T))


def make_delaunay(n_pts: int = 1500, seed: int = 0, side: float = 10.0, n_leads: int = 8,
                  T: int = 150) -> Problem:
    """The c1 set-up on an unstructured mesh (delaunay_cloud): fibres rotating
    with depth, c_f = 0.6 / c_t = 0.3 mm/ms with 5 % per-tet jitter, 3
    element onsets t ~ U[0, 6] ms, 8 electrodes on a 30 mm sphere."""
    mesh = delaunay_cloud(n_pts, seed, side)
    fib = fibres_cube(mesh, side)
    r = np.random.default_rng(seed + 1234)
    cf = (0.6 * (1 + 0.05 * r.standard_normal(mesh.n_t))).astype(np.float32)
    ct = (0.3 * (1 + 0.05 * r.standard_normal(mesh.n_t))).astype(np.float32)
    ons = onsets_element(mesh, 3, seed=seed + 7, tmin=0.0, tmax=6.0)
    el = fibonacci_sphere(n_leads, 30.0, (side / 2,) * 3)
    L = lead_field(mesh, el)
    return Problem("delaunay", mesh, fib, cf, ct, ons, L, Template(-80.0, 20.0, 1.0, 0.0, 1.0, T))


def make_c2(h: float = 1.0, seed: int = 0, T: int = 300, fast_layer_mm: float = 1.0) -> Problem:
    """Biventricular-shaped voxel-Kuhn mesh (~100k nodes at h=1.0 mm), rule
    based fibres, c_f=0.6 / c_t=0.3 with a 1 mm fast endocardial layer at
    2.0 mm/ms, 12 leads from 10 torso electrodes, T=300 @ 1 ms."""
    lo = np.array([-48.0, -30.0, -48.0])
    hi = np.array([28.0, 30.0, _Z_BASE + h])
    shape = np.ceil((hi - lo) / h).astype(int)
    gi = [lo[d] + h * (np.arange(shape[d]) + 0.5) for d in range(3)]
    P = np.stack(np.meshgrid(*gi, indexing="ij"), axis=-1)
    lab_cell = biv_shell_mask(P)
    mesh = voxel_kuhn(lab_cell > 0, h, lo)
    pc = _tet_centroids(mesh)
    labels = biv_shell_mask(pc)
    # centroids of Kuhn tets lie inside their (tissue) cell; a few may test
    # outside the analytic region on the boundary: give them the cell's label
    cell_lab = lab_cell[tuple(np.floor((pc - lo) / h).astype(int).T)]
    labels = np.where(labels == 0, cell_lab, labels)
    tm = np.where(labels == 2, _transmural_rv(pc), _transmural_lv(pc))
    fib = fibres_biv(mesh, labels, tm)
    cf = np.full(mesh.n_t, 0.6, np.float32)
    ct = np.full(mesh.n_t, 0.3, np.float32)
    # fast endocardial layer: within fast_layer_mm of the cavity surface
    wall = np.where(labels == 2, 4.0, 10.0)
    fast = tm * wall <= fast_layer_mm
    cf[fast] = 2.0
    ct[fast] = 2.0
    ons = onsets_element(mesh, 5, seed, 0.0, 10.0,
                         tets=np.nonzero(fast)[0])
    el = torso_electrodes()
    L = lead_field(mesh, el, twelve_lead_matrix())
    return Problem("c2", mesh, fib, cf, ct, ons, L, Template(-80.0, 20.0, 1.0, 0.0, 1.0, T),
                   extra={"labels": labels, "fast": fast})


def make_c3(n: int = 72, seed: int = 0, side: float = 10.0, n_sites: int = 10,
            n_leads: int = 8, T: int = 150, noise: float = 0.05) -> Problem:
    """Inverse-loop workload on the config-1 geometry refined to n^3 vertices
    (72^3: 373,248 nodes / 2,147,346 tets).  Ground truth: per-node log c
    fields (log 0.6 / log 0.3 +- 0.2 from 8 seeded bumps each), 10 element
    onsets with t~U[0,20] ms.  The per-tet velocity is exp(mean of the four
    nodal logs).  Stored in ``extra``: the ground-truth nodal log fields."""
    mesh = kuhn_cube(n, side)
    fib = fibres_cube(mesh, side)
    lcf = np.log(0.6) + 0.2 * smooth_field(mesh.xyz, 8, seed + 101)
    lct = np.log(0.3) + 0.2 * smooth_field(mesh.xyz, 8, seed + 202)
    cf = np.exp(nodal_to_tet_mean(mesh, lcf)).astype(np.float32)
    ct = np.exp(nodal_to_tet_mean(mesh, lct)).astype(np.float32)
    ons = onsets_element(mesh, n_sites, seed + 303, 0.0, 20.0)
    el = fibonacci_sphere(n_leads, 30.0, (side / 2,) * 3)
    L = lead_field(mesh, el)
    return Problem("c3", mesh, fib, cf, ct, ons, L, Template(-80.0, 20.0, 1.0, 0.0, 1.0, T),
                   extra={"log_cf_nodal": lcf.astype(np.float32),
                          "log_ct_nodal": lct.astype(np.float32),
                          "noise": noise})


def c3_starts(p: Problem, B: int, seed: int = 1234, log_noise: float = 0.05):
    """B starting points of the c3 inverse problem (the multi-start batch the
    benchmark times): per start a global velocity scale exp(N(0, 0.1)) on the
    prior means c_f = 0.6 / c_t = 0.3 mm/ms (start 0 unscaled), per-vertex
    log-velocity noise of std log_noise mapped to tets by the exponential of
    the vertex mean (the inverse problem's parameterisation), and onset times
    10 ms (start 0) or 10 ms + U(-2, 2) at the true sites.  The noise keeps
    exact ties out of the Kuhn cube's faces.  Start b draws from its own
    generator (seed, b), so a start does not depend on B.  Returns cf, ct
    float32 [B, n_t] and t float32 [B, K]."""
    n_v, K = p.mesh.n_v, p.onsets.K
    cf, ct, t = [], [], []
    for b in range(B):
        r = np.random.default_rng([seed, b])
        sf, st = (1.0, 1.0) if b == 0 else tuple(np.exp(r.normal(0, 0.1, 2)))
        lcf = np.log(0.6 * sf) + log_noise * r.standard_normal(n_v)
        lct = np.log(0.3 * st) + log_noise * r.standard_normal(n_v)
        cf.append(np.exp(nodal_to_tet_mean(p.mesh, lcf)).astype(np.float32))
        ct.append(np.exp(nodal_to_tet_mean(p.mesh, lct)).astype(np.float32))
        t.append(np.full(K, 10.0, np.float32) if b == 0 else (10.0 + r.uniform(-2, 2, K)).astype(np.float32))
    return np.stack(cf), np.stack(ct), np.stack(t)


def c2_starts(p: Problem, B: int, seed: int = 4321, log_noise: float = 0.05):
    """B starting points on the biventricular mesh (the BiV benchmark batch):
    per start a global scale exp(N(0, 0.1)) on the tissue velocities c_f, c_t
    (the fast endocardial layer keeps its 2.0 mm/ms), per-tet log-velocity
    noise of std log_noise on every tet, and the true onset sites with their
    times (start 0) or those times + U(-2, 2) ms.  Start b draws from its own
    generator (seed, b).  Returns cf, ct float32 [B, n_t] and t float32
    [B, K]."""
    fast = p.extra["fast"]
    n_t, K = p.mesh.n_t, p.onsets.K
    cf, ct, t = [], [], []
    for b in range(B):
        r = np.random.default_rng([seed, b])
        sf, st = (1.0, 1.0) if b == 0 else tuple(np.exp(r.normal(0, 0.1, 2)))
        base_f = np.where(fast, p.cf, p.cf * sf)
        base_t = np.where(fast, p.ct, p.ct * st)
        cf.append((base_f * np.exp(log_noise * r.standard_normal(n_t))).astype(np.float32))
        ct.append((base_t * np.exp(log_noise * r.standard_normal(n_t))).astype(np.float32))
        t.append(p.onsets.t.astype(np.float32) if b == 0 else (p.onsets.t + r.uniform(-2, 2, K)).astype(np.float32))
    return np.stack(cf), np.stack(ct), np.stack(t)


def make_c4_phi(xyz: np.ndarray, seed: int, tmax: float = 120.0, amp: float = 5.0,
                n_modes: int = 16) -> np.ndarray:
    """Activation map for the ECG precision study: i.i.d. U[0, tmax] plus a
    smooth field of n_modes random Fourier modes (amplitude amp ms), >= 0."""
    rng = np.random.default_rng(seed)
    x = xyz.astype(np.float64)
    span = x.max(axis=0) - x.min(axis=0)
    phi = rng.uniform(0.0, tmax, size=len(x))
    s = np.zeros(len(x))
    for _ in range(n_modes):
        k = rng.integers(1, 4, size=3) * 2 * np.pi / np.maximum(span, 1e-9)
        s += np.cos(x @ k + rng.uniform(0, 2 * np.pi))
    s *= amp / max(np.max(np.abs(s)), 1e-12)
    return np.maximum(phi + s, 0.0).astype(np.float32)


def make_c4(n: int = 100, seed: int = 0, side: float = 10.0, T: int = 500):
    """ECG precision workload: n^3-vertex cube (1M nodes at n=100), 12 leads
    (10 torso electrodes scaled to the cube), T=500 @ 1 ms.  Returns
    (mesh, L, phi, template)."""
    mesh = kuhn_cube(n, side)
    el = torso_electrodes(centre=(side / 2, side / 2, side / 2)) * 0.4 + 0.6 * side / 2
    L = lead_field(mesh, el, twelve_lead_matrix())
    phi = make_c4_phi(mesh.xyz, seed)
    return mesh, L, phi, Template(-80.0, 20.0, 1.0, 0.0, 1.0, T)


def c5_sample_params(rng: np.random.Generator, mesh: Mesh, surf_faces: np.ndarray,
                     n_sites: int = 10):
    """One draw of the learned-initialiser prior: c_f~U[0.4,0.8],
    c_t~U[0.2,0.4], c_endo~U[1,3], n_sites surface sites with t~U[0,20]."""
    cf = rng.uniform(0.4, 0.8)
    ct = rng.uniform(0.2, 0.4)
    ce = rng.uniform(1.0, 3.0)
    fi = rng.choice(len(surf_faces), size=n_sites, replace=False)
    b3 = rng.dirichlet(np.ones(3), size=n_sites)
    t = rng.uniform(0.0, 20.0, size=n_sites)
    return dict(cf=cf, ct=ct, ce=ce, face=fi, b3=b3, t=t)


def random_faces(n: int, seed: int, aniso: float = 2.0, spread: float = 4.0,
                 p_inf: float = 0.1, skinny: bool = False):
    """Random local problems (Eq. upwind_eq_lsqr) for solver tests: edge
    vectors e [n,3,3] (rows v_jn - v_i), fibre f [n,3], velocities cf/ct [n],
    vertex values Phi [n,3] (some +inf)."""
    rng = np.random.default_rng(seed)
    e = rng.normal(size=(n, 3, 3))
    if skinny:
        e[:, 2] = e[:, 0] * 0.5 + e[:, 1] * 0.5 + 0.02 * rng.normal(size=(n, 3))
    # positively oriented: det[e1,e2,e3] > 0 means v_i sees the face from one side
    det = np.linalg.det(e)
    e[det < 0, 0] *= -1
    f = rng.normal(size=(n, 3))
    f /= np.linalg.norm(f, axis=1, keepdims=True)
    ct = rng.uniform(0.2, 0.5, size=n)
    cf = ct * rng.uniform(1.0, aniso, size=n)
    phi = rng.uniform(0.0, spread, size=(n, 3))
    if p_inf > 0:
        m = rng.uniform(size=(n, 3)) < p_inf
        m[np.all(m, axis=1), 0] = False
        phi[m] = np.inf
    return (e.astype(np.float32), f.astype(np.float32), cf.astype(np.float32),
            ct.astype(np.float32), phi.astype(np.float32))


# ----------------------------------------------------------------------------
# 2-D triangle meshes (the paper's d = 2 setting)
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class TriMesh:
    xy: np.ndarray    # float32 [n_v, 2], mm
    tris: np.ndarray  # int32 [n_t, 3], counter-clockwise

    @property
    def n_v(self) -> int:
        return int(self.xy.shape[0])

    @property
    def n_t(self) -> int:
        return int(self.tris.shape[0])


@dataclasses.dataclass
class Problem2D:
    name: str
    mesh: TriMesh
    fib: np.ndarray   # float32 [n_t, 2], unit
    cf: np.ndarray    # float32 [n_t]
    ct: np.ndarray    # float32 [n_t]
    onset_nodes: np.ndarray  # int32 [K]
    onset_t: np.ndarray      # float32 [K]
    L: np.ndarray     # float32 [N, n_v]
    tmpl: Template
    onsets: Onsets | None = None  # element onsets (idx = triangles, bary [K, 3]); None: the nodal ones above
    extra: dict = dataclasses.field(default_factory=dict)


def tri_square(n: int, side: float = 10.0, jitter: float = 0.0, seed: int = 0) -> TriMesh:
    """n x n vertex grid on [0, side]^2 split into 2 counter-clockwise
    triangles per cell (alternating diagonals); interior vertices jittered by
    up to jitter * h."""
    h = side / (n - 1)
    g = np.arange(n)
    X, Y = np.meshgrid(g, g, indexing="xy")
    xy = np.stack([X.ravel(), Y.ravel()], axis=1).astype(np.float64) * h
    if jitter > 0:
        r = np.random.default_rng(seed)
        inner = (X.ravel() > 0) & (X.ravel() < n - 1) & (Y.ravel() > 0) & (Y.ravel() < n - 1)
        xy[inner] += r.uniform(-jitter * h, jitter * h, size=(int(inner.sum()), 2))
    tris = []
    for j in range(n - 1):
        for i in range(n - 1):
            a, b, c, d = j * n + i, j * n + i + 1, (j + 1) * n + i + 1, (j + 1) * n + i
            if (i + j) % 2 == 0:
                tris += [(a, b, c), (a, c, d)]
            else:
                tris += [(a, b, d), (b, c, d)]
    return TriMesh(xy.astype(np.float32), np.asarray(tris, np.int32))


def make_2d(n: int = 40, seed: int = 0, side: float = 10.0, n_leads: int = 7, K: int = 2, T: int = 120,
            jitter: float = 0.25) -> Problem2D:
    """2-D workload in the spirit of the paper's torso-slice study: a
    jittered triangulated square, fibres in the plane rotating -60 .. +60 deg
    across it, c_f = 0.6 / c_t = 0.3 mm/ms with 5 % per-triangle jitter, K
    nodal onsets with t ~ U[0, 10] ms, n_leads electrodes on a circle of
    radius 2 * side around the centre with a 1 / r lead field whose rows are
    centred to sum to zero, T samples at 1 ms."""
    r = np.random.default_rng(seed)
    mesh = tri_square(n, side, jitter, seed)
    cen = mesh.xy.astype(np.float64)[mesh.tris].mean(axis=1)
    ang = np.deg2rad(-60.0 + 120.0 * cen[:, 1] / side)
    fib = np.stack([np.cos(ang), np.sin(ang)], axis=1).astype(np.float32)
    cf = (0.6 * (1 + 0.05 * r.standard_normal(mesh.n_t))).astype(np.float32)
    ct = (0.3 * (1 + 0.05 * r.standard_normal(mesh.n_t))).astype(np.float32)
    nodes = r.choice(mesh.n_v, size=K, replace=False).astype(np.int32)
    t = r.uniform(0.0, 10.0, size=K).astype(np.float32)
    th = 2 * np.pi * (np.arange(n_leads) + 0.5) / n_leads
    el = side / 2 + 2 * side * np.stack([np.cos(th), np.sin(th)], axis=1)
    d = np.linalg.norm(mesh.xy.astype(np.float64)[None, :, :] - el[:, None, :], axis=2)
    L = 1.0 / d
    L -= L.mean(axis=1, keepdims=True)
    L *= 100.0 / mesh.n_v
    return Problem2D("2d", mesh, fib, cf, ct, nodes, t, L.astype(np.float32), Template(-80.0, 20.0, 1.0, 0.0, 1.0, T))


def lv_slice(n_r: int = 15, n_theta: int = 180, r_in: float = 18.0, r_out: float = 31.0) -> TriMesh:
    """Annular left-ventricular slice: n_r rings from r_in to r_out (mm),
    n_theta vertices per ring, each cell split into two counter-clockwise
    triangles (alternating diagonals).  The default has 2,700 vertices and a
    spacing of about 0.9 mm, the size of the paper's 2-D study; (2 n_r - 1,
    2 n_theta) gives the half-spacing mesh whose even vertices coincide with
    these."""
    r = np.linspace(r_in, r_out, n_r)
    th = 2 * np.pi * np.arange(n_theta) / n_theta
    R, TH = np.meshgrid(r, th, indexing="ij")  # [n_r, n_theta]
    xy = np.stack([R * np.cos(TH), R * np.sin(TH)], axis=-1).reshape(-1, 2)
    tris = []
    for i in range(n_r - 1):
        for j in range(n_theta):
            a, b = i * n_theta + j, i * n_theta + (j + 1) % n_theta
            c, d = (i + 1) * n_theta + (j + 1) % n_theta, (i + 1) * n_theta + j
            # (radius, angle) is positively oriented: a -> d -> c is counter-clockwise
            if (i + j) % 2 == 0:
                tris += [(a, c, b), (a, d, c)]
            else:
                tris += [(a, d, b), (b, d, c)]
    return TriMesh(xy.astype(np.float32), np.asarray(tris, np.int32))


def lead_field_2d(mesh: TriMesh, electrodes: np.ndarray, combos: np.ndarray | None = None) -> np.ndarray:
    """2-D counterpart of lead_field: L_l = K Z_l with K the P1 stiffness
    matrix of the triangle mesh (unit conductivity) and Z_l(x) =
    -ln|x - e_l| / (2 pi) the infinite-plane lead field, assembled per
    triangle as L_l[a] += area * grad(lambda_a) . grad(Z_h)."""
    x = mesh.xy.astype(np.float64)
    E = np.asarray(electrodes, float)
    Z = -np.log(np.linalg.norm(x[None, :, :] - E[:, None, :], axis=2)) / (2 * np.pi)
    t = mesh.tris
    v = x[t]  # [n_t, 3, 2]
    J = (v[:, 1:] - v[:, :1]).transpose(0, 2, 1)
    area = 0.5 * np.linalg.det(J)
    Jinv = np.linalg.inv(J)
    g = np.concatenate([-Jinv.sum(axis=1, keepdims=True), Jinv], axis=1)  # [n_t, 3, 2]
    L = np.zeros((E.shape[0], mesh.n_v))
    for e in range(E.shape[0]):
        gz = np.einsum("cai,ca->ci", g, Z[e][t])
        contrib = area[:, None] * np.einsum("cai,ci->ca", g, gz)
        L[e] = np.bincount(t.ravel(), weights=contrib.ravel(), minlength=mesh.n_v)
    if combos is not None:
        L = np.asarray(combos, float) @ L
    return L.astype(np.float32)


def locate_2d(mesh: TriMesh, pts: np.ndarray):
    """(triangle, barycentric coordinates) of each point, by brute force."""
    v = mesh.xy.astype(np.float64)[mesh.tris]
    J = (v[:, 1:] - v[:, :1]).transpose(0, 2, 1)
    idx, bary = [], []
    for p in np.asarray(pts, float):
        lam = np.linalg.solve(J, (p - v[:, 0])[..., None])[..., 0]
        b = np.concatenate([1 - lam.sum(axis=1, keepdims=True), lam], axis=1)
        j = int(np.argmax(b.min(axis=1)))
        bj = np.clip(b[j], 0, 1)
        idx.append(j)
        bary.append(bj / bj.sum())
    return np.asarray(idx), np.asarray(bary)


def make_2d_torso(fine: bool = False, seed: int = 0, K: int = 4, T: int = 200, perturb: float = 0.0,
                  onsets: Onsets | None = None) -> Problem2D:
    """The paper's 2-D simulation study, synthetic (its torso geometry and
    conductivities are not given): the LV slice of lv_slice (0.9 mm, 2,700
    vertices; fine=True: 0.45 mm, 10,440 vertices), fibres along the local
    circumferential direction turned from -60 deg (epicardium) to +60 deg
    (endocardium), c_f = 0.6 / c_t = 0.3 mm/ms (times a smooth factor
    exp(+-perturb) around the ring when perturb > 0), 8 electrodes on a
    60 mm circle around a torso centre 10 mm left of the slice, electrodes 0
    and 1 (the arms) forming Wilson's central terminal, 7 leads (the 6 others
    against it, and lead I = e1 - e0), T samples at 1 ms.  Sites: K element
    onsets in the half y > 2 mm with times U[2.5, 10] ms, drawn on the coarse
    mesh and located on the fine one, unless given."""
    coarse = lv_slice()
    mesh = lv_slice(29, 360) if fine else coarse
    xy = mesh.xy.astype(np.float64)
    cen = xy[mesh.tris].mean(axis=1)
    rad = np.linalg.norm(cen, axis=1)
    tang = np.stack([-cen[:, 1], cen[:, 0]], axis=1) / rad[:, None]
    ang = np.deg2rad(-60.0 + 120.0 * (31.0 - rad) / (31.0 - 18.0))
    c, s_ = np.cos(ang), np.sin(ang)
    fib = np.stack([c * tang[:, 0] - s_ * tang[:, 1], s_ * tang[:, 0] + c * tang[:, 1]], axis=1)
    cf = np.full(mesh.n_t, 0.6)
    ct = np.full(mesh.n_t, 0.3)
    if perturb > 0:
        r = np.random.default_rng(seed + 99)
        ph = r.uniform(0, 2 * np.pi, 4)
        th = np.arctan2(cen[:, 1], cen[:, 0])
        cf *= np.exp(perturb * (0.6 * np.sin(2 * th + ph[0]) + 0.4 * np.sin(3 * th + ph[1])))
        ct *= np.exp(perturb * (0.6 * np.sin(2 * th + ph[2]) + 0.4 * np.cos(3 * th + ph[3])))
    if onsets is None:
        rng = np.random.default_rng(seed)
        ccen = coarse.xy.astype(np.float64)[coarse.tris].mean(axis=1)
        pool = np.nonzero(ccen[:, 1] > 2.0)[0]
        idx = rng.choice(pool, size=K, replace=False)
        b = 0.1 + 0.7 * rng.dirichlet(np.ones(3), size=K)
        t = rng.uniform(2.5, 10.0, size=K)
        if fine:
            pts = np.einsum("kq,kqr->kr", b, coarse.xy.astype(np.float64)[coarse.tris[idx]])
            idx, b = locate_2d(mesh, pts)
        onsets = Onsets(ONSET_ELEMENT, idx.astype(np.int32), t.astype(np.float32), b.astype(np.float32))
    th = 2 * np.pi * (np.arange(8) + 0.5) / 8 + np.pi / 2
    el = np.array([-10.0, 0.0]) + 60.0 * np.stack([np.cos(th), np.sin(th)], axis=1)
    combos = np.zeros((7, 8))
    for q in range(6):
        combos[q, q + 2] = 1.0
        combos[q, :2] = -0.5
    combos[6, 1], combos[6, 0] = 1.0, -1.0
    L = lead_field_2d(mesh, el, combos)
    return Problem2D("2d_torso_fine" if fine else "2d_torso", mesh, fib.astype(np.float32),
                     cf.astype(np.float32), ct.astype(np.float32), np.zeros(0, np.int32), onsets.t, L,
                     Template(-80.0, 20.0, 1.0, 0.0, 1.0, T), onsets=onsets)
