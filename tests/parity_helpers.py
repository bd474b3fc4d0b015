"""Shared checks of the GPU parity tests, computed from the FP64 oracle alone.

Tolerances (written here once, used by every parity test):

- phi: within PHI_RTOL = 2e-6 relative (max(1, phi)) of the oracle at every
  vertex; the acceptance bound of the method is 1e-4, and FP32 reaches about
  4e-7.  The tighter bound is what makes the parent check consistent: a face
  value is a convex combination of three vertex values plus an FP32 length,
  so it is within about 3e-6 phi of the oracle's, and two faces can only
  trade places when the oracle's gap between them is below about 6e-6 phi.
- parents: bit-exact wherever the oracle's margin (its gap between the best
  and the second-best candidate) exceeds MARGIN = 1e-5 phi.
- alpha (the barycentric point of the parent face, Eq. dto_grad): where the
  parent agrees, within 2e-5 + 4 s_i (max norm), s_i being the oracle's own
  sensitivity: how far its minimiser moves when one face value moves by
  1e-6 relative (the local problem is flat near a minimiser close to an edge
  or vertex, and there the location is only as good as the values).
- per-tet velocity gradients: on the tets no tie can have touched (below),
  |g - r| <= 1e-3 |r| + 1e-6 max_j |r_j|.  The absolute term is the FP32
  ECG's own relative error (about 1e-6, measured against the oracle): every
  dL/dphi_n is a sum of U' B r over samples and leads whose residuals r can
  cancel to zero, so the chain dL/dphi -> mu -> gradient resolves a tet's
  gradient only to about that fraction of the largest one.

A tet is "touched by a tie" when it is the parent tet (oracle's or GPU's) of
a vertex whose mu can differ: the vertices where the GPU took the other face
of a tie, the vertices of both faces they chose from, and every ancestor of
those in the parent graph; element-onset tets of such onset vertices too."""
from __future__ import annotations

import numpy as np

from oracle import oracle as O

MARGIN = 1e-5
PHI_RTOL = 2e-6
_OTHER = np.array([[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]])


def face_vertices(tets, code):
    """The three vertices (slot order) of face codes tet * 4 + slot."""
    code = np.asarray(code, np.int64)
    tets = np.asarray(tets, np.int64)
    return tets[code >> 2][np.arange(len(code))[:, None], _OTHER[code & 3]]


def unambiguous(ref):
    phi = ref["phi"]
    return np.isfinite(phi) & (ref["margin"] > MARGIN * np.maximum(1.0, phi))


def check_phi(phi_gpu, ref):
    phi_gpu = np.asarray(phi_gpu, float)
    fin = np.isfinite(ref["phi"])
    np.testing.assert_array_equal(np.isfinite(phi_gpu), fin)
    rel = np.abs(phi_gpu[fin] - ref["phi"][fin]) / np.maximum(1.0, np.abs(ref["phi"][fin]))
    assert rel.max() <= PHI_RTOL, rel.max()
    return float(rel.max())


def check_parents(par_gpu, ref, min_unambiguous=0.9):
    un = unambiguous(ref)
    assert un.mean() >= min_unambiguous, un.mean()
    np.testing.assert_array_equal(np.asarray(par_gpu)[un], ref["parent"][un])
    return float(un.mean())


def alpha_sensitivity(mesh, fib, cf, ct, ref, idx, rel=1e-6):
    """max over the six one-sided moves of one face value by rel * max(1, value)
    of the change of the oracle's minimiser (max norm), per vertex idx."""
    code = ref["parent"][idx]
    fv = face_vertices(mesh.tets, code)
    xyz = np.asarray(mesh.xyz, np.float32)
    e = xyz[fv] - xyz[idx][:, None, :]
    j = code >> 2
    Phi = ref["phi"][fv]
    _, a0 = O.local_batch(e, fib[j], cf[j], ct[j], Phi)
    s = np.zeros(len(idx))
    for n in range(3):
        for sg in (-1.0, 1.0):
            Q = Phi.copy()
            Q[:, n] += sg * rel * np.maximum(1.0, Q[:, n])
            _, a = O.local_batch(e, fib[j], cf[j], ct[j], Q)
            s = np.maximum(s, np.abs(a - a0).max(axis=1))
    return s


def check_alpha(al_gpu, par_gpu, mesh, fib, cf, ct, ref):
    """alpha where the oracle is unambiguous and the parents agree."""
    idx = np.nonzero(unambiguous(ref) & (ref["parent"] >= 0) & (np.asarray(par_gpu) == ref["parent"]))[0]
    s = alpha_sensitivity(mesh, fib, cf, ct, ref, idx)
    da = np.abs(np.asarray(al_gpu, float)[idx] - ref["alpha"][idx]).max(axis=1)
    tol = 2e-5 + 4.0 * s
    bad = np.nonzero(da > tol)[0]
    assert len(bad) == 0, [(int(idx[k]), float(da[k]), float(s[k])) for k in bad[:10]]
    return {"n": int(len(idx)), "max": float(da.max()), "median": float(np.median(da))}


def touched_tets(mesh, onsets, ref, par_gpu):
    """Tets whose gradient a tie choice of the GPU can have changed (module
    docstring).  par_gpu must equal the oracle's parent wherever it is
    unambiguous (check_parents)."""
    n_v = mesh.n_v
    tets = np.asarray(mesh.tets, np.int64)
    par_o = ref["parent"]
    par_g = np.asarray(par_gpu)
    diff = np.nonzero(par_g != par_o)[0]
    seed = np.zeros(n_v, bool)
    seed[diff] = True
    for par in (par_o, par_g):
        f = diff[par[diff] >= 0]
        seed[face_vertices(tets, par[f]).ravel()] = True
    # ancestors through the oracle's parent edges (alpha > 0)
    ch = np.nonzero(par_o >= 0)[0]
    fv = face_vertices(tets, par_o[ch])
    al = ref["alpha"][ch]
    cs = np.concatenate([ch[al[:, k] > 0] for k in range(3)])
    ps = np.concatenate([fv[al[:, k] > 0, k] for k in range(3)])
    aff = seed.copy()
    front = seed.copy()
    while front.any():
        nxt = np.zeros(n_v, bool)
        nxt[ps[front[cs]]] = True
        nxt &= ~aff
        aff |= nxt
        front = nxt
    bad = np.zeros(len(tets), bool)
    for par in (par_o, par_g):
        bad[par[aff & (par >= 0)] >> 2] = True
    if onsets.kind == O.ONSET_ELEMENT:
        for par in (par_o, par_g):
            on = aff & (par < 0) & (par != O.UNREACHED)
            bad[np.asarray(onsets.idx)[-1 - par[on]]] = True
    return bad


def check_tet_gradients(g, ref, par_gpu, mesh, onsets, min_clean=0.3):
    """Per-tet d_cf, d_ct on the tets no tie touched (module docstring)."""
    bad = touched_tets(mesh, onsets, ref, par_gpu)
    out = {}
    for k in ("d_cf", "d_ct"):
        r = ref[k]
        nz = r != 0
        clean = ~bad
        assert (clean & nz).sum() >= min_clean * nz.sum(), ((clean & nz).sum(), nz.sum())
        e = np.abs(np.asarray(g[k], float) - r)
        lim = 1e-3 * np.abs(r) + 1e-6 * np.abs(r).max()
        over = np.nonzero(clean & (e > lim))[0]
        assert len(over) == 0, (k, [(int(j), float(g[k][j]), float(r[j])) for j in over[:10]])
        cn = clean & nz
        out[k] = {"clean_nonzero": int(cn.sum()), "nonzero": int(nz.sum()),
                  "within_1e-3_relative": float(np.mean(e[cn] <= 1e-3 * np.abs(r[cn]))) if cn.any() else 1.0}
    return out


def parents_differ(par_gpu, ref) -> bool:
    """True when the GPU took another face than the oracle anywhere (only
    possible at ties, check_parents)."""
    return bool(np.any(np.asarray(par_gpu) != ref["parent"]))
