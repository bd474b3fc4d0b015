"""Onset relocation across elements for the inverse problem.

An element onset (Eq. upwind_xi) lives in a simplex E (a tet, or a triangle
for d = 2) at barycentric coordinates b.  When Adam moves its position x out
of E (some b_q < 0), the onset is handed to the neighbouring simplex across
the facet opposite the most negative coordinate, and so on until x is
inside a simplex ("walking" point location); at the mesh boundary x is
clamped back into the last simplex.  This lets sites migrate through the
mesh during the fit instead of being confined to their initial element.
Host-side bookkeeping on a handful of sites: the adjacency is built once
with NumPy, the per-simplex inverse vertex matrices on demand.
"""
from __future__ import annotations

import numpy as np


def simplex_neighbours(cells: np.ndarray) -> np.ndarray:
    """nbr[j, s] = the simplex sharing the facet of simplex j opposite slot s,
    or -1 (cells [n, d + 1])."""
    cells = np.asarray(cells, np.int64)
    n, w = cells.shape
    facets = np.concatenate([np.sort(np.delete(cells, s, axis=1), axis=1) for s in range(w)])  # [w n, d]
    owner = np.concatenate([np.arange(n)] * w)
    slot = np.repeat(np.arange(w), n)
    order = np.lexsort(facets.T[::-1])
    fs = facets[order]
    nbr = np.full((n, w), -1, np.int64)
    same = np.nonzero(np.all(fs[1:] == fs[:-1], axis=1))[0]
    a, b = order[same], order[same + 1]
    nbr[owner[a], slot[a]] = owner[b]
    nbr[owner[b], slot[b]] = owner[a]
    return nbr


class SimplexLocator:
    """Walking point location on a tet (d = 3) or triangle (d = 2) mesh:
    xyz [n_v, d], cells [n, d + 1]."""

    def __init__(self, xyz: np.ndarray, cells: np.ndarray):
        self.xyz = np.asarray(xyz, np.float64)
        self.cells = np.asarray(cells, np.int64)
        self.nbr = simplex_neighbours(self.cells)
        self._inv = {}

    def inverse(self, j: int) -> np.ndarray:
        """M^{-1} with M = [[v_0 .. v_d], [1 .. 1]], so b = M^{-1} [x; 1]."""
        m = self._inv.get(j)
        if m is None:
            V = self.xyz[self.cells[j]]
            M = np.vstack([V.T, np.ones(V.shape[0])])
            m = np.linalg.inv(M)
            self._inv[j] = m
        return m

    def bary(self, j: int, x) -> np.ndarray:
        return self.inverse(j) @ np.append(np.asarray(x, np.float64), 1.0)

    def walk(self, j: int, x, max_steps: int = 1000, tol: float = 1e-12):
        """Simplex containing x reached by walking from simplex j.  Returns
        (simplex, barycentric coordinates, inside).  When the walk leaves the
        mesh (or does not settle within max_steps) the last simplex is
        returned with inside = False."""
        j = int(j)
        for _ in range(max_steps):
            b = self.bary(j, x)
            q = int(np.argmin(b))
            if b[q] >= -tol:
                return j, b, True
            nxt = int(self.nbr[j, q])
            if nxt < 0:
                return j, b, False
            j = nxt
        return j, self.bary(j, x), False

    @staticmethod
    def clamp(b: np.ndarray, floor: float = 1e-3) -> np.ndarray:
        """Barycentric coordinates pulled inside the simplex (each >= floor, sum 1)."""
        b = np.maximum(np.asarray(b, np.float64), floor)
        return b / b.sum()


def relocate_onsets(loc: SimplexLocator, x, on_idx, Vt_inv, Vt=None, floor: float = 1e-3) -> int:
    """After an optimiser step: hand every onset whose position x[k] left its
    simplex on_idx[k] to the simplex that contains it (walking from the old
    one), or clamp it back inside the last simplex at the mesh boundary.
    Updates the torch tensors x [K, d], on_idx [K] (int32), Vt_inv
    [K, d + 1, d + 1] (barycentric map) and Vt [K, d + 1, d] (simplex
    vertices, if given) in place.  Returns the number of onsets that changed
    simplex."""
    import torch

    xs = x.detach().cpu().numpy().astype(np.float64)
    idx = on_idx.cpu().numpy().astype(np.int64)
    moved, clamped = 0, False
    inv = Vt_inv.cpu().numpy()
    for k in range(len(idx)):
        j, b, inside = loc.walk(idx[k], xs[k])
        if not inside:
            b = SimplexLocator.clamp(b, floor)
            xs[k] = b @ loc.xyz[loc.cells[j]]
            clamped = True
        if j != idx[k]:
            idx[k] = j
            inv[k] = loc.inverse(j)
            moved += 1
    with torch.no_grad():
        if moved:
            on_idx.copy_(torch.from_numpy(idx.astype(np.int32)))
            Vt_inv.copy_(torch.from_numpy(inv.astype(np.float32)))
            if Vt is not None:
                Vt.copy_(torch.from_numpy(loc.xyz[loc.cells[idx]].astype(np.float32)))
        if moved or clamped:
            x.copy_(torch.from_numpy(xs.astype(np.float32)))
    return moved
