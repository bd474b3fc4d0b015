"""Onset relocation across elements for the inverse problem.

An element onset (Eq. upwind_xi) lives in a tet E at barycentric coordinates
b.  When Adam moves its position x out of E (some b_q < 0), the onset is
handed to the neighbouring tet across the face opposite the most negative
coordinate, and so on until x is inside a tet ("walking" point location); at
the mesh boundary x is clamped back into the last tet.  This lets sites
migrate through the mesh during the fit instead of being confined to their
initial tet.  Host-side bookkeeping on a handful of sites: the tet adjacency
is built once with NumPy, the per-tet inverse vertex matrices on demand.
"""
from __future__ import annotations

import numpy as np


def tet_neighbours(tets: np.ndarray) -> np.ndarray:
    """nbr[j, s] = the tet sharing the face of tet j opposite slot s, or -1."""
    tets = np.asarray(tets, np.int64)
    n_t = tets.shape[0]
    faces = np.concatenate([np.sort(np.delete(tets, s, axis=1), axis=1) for s in range(4)])  # [4 n_t, 3]
    owner = np.concatenate([np.arange(n_t)] * 4)
    slot = np.repeat(np.arange(4), n_t)
    order = np.lexsort((faces[:, 2], faces[:, 1], faces[:, 0]))
    fs = faces[order]
    nbr = np.full((n_t, 4), -1, np.int64)
    same = np.nonzero(np.all(fs[1:] == fs[:-1], axis=1))[0]
    a, b = order[same], order[same + 1]
    nbr[owner[a], slot[a]] = owner[b]
    nbr[owner[b], slot[b]] = owner[a]
    return nbr


class TetLocator:
    """Walking point location on a tet mesh."""

    def __init__(self, xyz: np.ndarray, tets: np.ndarray):
        self.xyz = np.asarray(xyz, np.float64)
        self.tets = np.asarray(tets, np.int64)
        self.nbr = tet_neighbours(self.tets)
        self._inv = {}

    def inverse(self, j: int) -> np.ndarray:
        """M^{-1} with M = [[v_0 .. v_3], [1 1 1 1]], so b = M^{-1} [x; 1]."""
        m = self._inv.get(j)
        if m is None:
            V = self.xyz[self.tets[j]]
            M = np.vstack([V.T, np.ones(4)])
            m = np.linalg.inv(M)
            self._inv[j] = m
        return m

    def bary(self, j: int, x) -> np.ndarray:
        return self.inverse(j) @ np.append(np.asarray(x, np.float64), 1.0)

    def walk(self, j: int, x, max_steps: int = 1000, tol: float = 1e-12):
        """Tet containing x reached by walking from tet j.  Returns
        (tet, barycentric coordinates, inside).  When the walk leaves the mesh
        (or does not settle within max_steps) the last tet is returned with
        inside = False."""
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
        """Barycentric coordinates pulled inside the tet (each >= floor, sum 1)."""
        b = np.maximum(np.asarray(b, np.float64), floor)
        return b / b.sum()


def relocate_onsets(loc: TetLocator, x, on_idx, Vt_inv, Vt=None, floor: float = 1e-3) -> int:
    """After an optimiser step: hand every onset whose position x[k] left its
    tet on_idx[k] to the tet that contains it (walking from the old one), or
    clamp it back inside the last tet at the mesh boundary.  Updates the torch
    tensors x [K, 3], on_idx [K] (int32), Vt_inv [K, 4, 4] (barycentric map)
    and Vt [K, 4, 3] (tet vertices, if given) in place.  Returns the number of
    onsets that changed tet."""
    import torch

    xs = x.detach().cpu().numpy().astype(np.float64)
    idx = on_idx.cpu().numpy().astype(np.int64)
    moved, clamped = 0, False
    inv = Vt_inv.cpu().numpy()
    for k in range(len(idx)):
        j, b, inside = loc.walk(idx[k], xs[k])
        if not inside:
            b = TetLocator.clamp(b, floor)
            xs[k] = b @ loc.xyz[loc.tets[j]]
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
                Vt.copy_(torch.from_numpy(loc.xyz[loc.tets[idx]].astype(np.float32)))
        if moved or clamped:
            x.copy_(torch.from_numpy(xs.astype(np.float32)))
    return moved
