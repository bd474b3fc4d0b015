"""Python driver of the FP64 CPU oracle (ctypes over ``libgbp_oracle.so``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by the smoke check and by
the benchmark's CPU-baseline leg; never by the product path.  It imports
nothing from the CUDA package.  Inputs are the float32 arrays of the seeded
generators; results are float64.

Functions follow the paper's sections as cited in ``gbp_oracle.c``; this file
only marshals arrays and drives finite differences (central, Sec. II-C is
checked against them).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

EXACT, FISTA, FISTA_THEORY = 0, 1, 2
ORDER_HEAP, ORDER_FIFO, ORDER_JACOBI = 0, 1, 2
ONSET_NODAL, ONSET_ELEMENT = 0, 1
UNREACHED = np.iinfo(np.int32).min

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        P = C.c_void_p
        i64, i32, dbl = C.c_int64, C.c_int, C.c_double
        L.orc_local_batch.argtypes = [i64, P, P, P, P, P, i32, i32, P, P]
        L.orc_local_batch.restype = None
        L.orc_lipschitz_batch.argtypes = [i64, P, P, P, P, P, P, P, P]
        L.orc_lipschitz_batch.restype = None
        L.orc_eikonal.argtypes = [i64, P, i64, P, P, P, P, i32, i32, P, P, P, i32, i32, i32,
                                  P, P, P, P, P]
        L.orc_eikonal.restype = i32
        L.orc_ecg.argtypes = [i64, i32, P, P, dbl, dbl, dbl, dbl, dbl, i32, P]
        L.orc_ecg.restype = None
        L.orc_loss_grad_phi.argtypes = [i64, i32, P, P, dbl, dbl, dbl, dbl, dbl, i32, P, P, P]
        L.orc_loss_grad_phi.restype = dbl
        L.orc_adjoint.argtypes = [i64, P, i64, P, P, P, P, i32, i32, P, P, P, P, P, P, P, P, P, P, P]
        L.orc_adjoint.restype = i64
        L.orc_num_threads.argtypes = []
        L.orc_num_threads.restype = i32
        _lib = L
    return _lib


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def num_threads() -> int:
    return int(lib().orc_num_threads())


# ---------------------------------------------------------------------------
# local problem
# ---------------------------------------------------------------------------

def local_batch(e, fib, cf, ct, phi, mode=EXACT, n_f=64):
    """Eq. (upwind_eq_lsqr) for n faces: returns (value [n], alpha [n,3])."""
    e, fib, cf, ct, phi = _f32(e), _f32(fib), _f32(cf), _f32(ct), _f32(phi)
    n = e.shape[0]
    val = np.empty(n)
    al = np.empty((n, 3))
    lib().orc_local_batch(n, _p(e), _p(fib), _p(cf), _p(ct), _p(phi), int(mode), int(n_f),
                          _p(val), _p(al))
    return val, al


def lipschitz_batch(e, fib, cf, ct):
    """Eq. (lipschitz_est): returns dict(L, h_min, h_theory, norm_G)."""
    e, fib, cf, ct = _f32(e), _f32(fib), _f32(cf), _f32(ct)
    n = e.shape[0]
    out = {k: np.empty(n) for k in ("L", "h_min", "h_theory", "norm_G")}
    lib().orc_lipschitz_batch(n, _p(e), _p(fib), _p(cf), _p(ct), _p(out["L"]), _p(out["h_min"]),
                              _p(out["h_theory"]), _p(out["norm_G"]))
    return out


# ---------------------------------------------------------------------------
# eikonal / ECG / loss / adjoint
# ---------------------------------------------------------------------------

def _onset_arrays(onsets):
    kind = int(onsets.kind)
    idx = _i32(onsets.idx)
    t = _f32(onsets.t)
    bary = _f32(onsets.bary) if onsets.bary is not None else np.zeros((len(idx), 4), np.float32)
    return kind, idx, t, bary


def eikonal(mesh, fib, cf, ct, onsets, mode=EXACT, n_f=64, order=ORDER_HEAP):
    """Discrete Hopf-Lax fixed point + parent pass.  Returns dict with
    phi [n_v], parent [n_v] (tet*4+slot, -1-k onset, UNREACHED),
    alpha [n_v,3], margin [n_v], stats."""
    xyz, tets = _f32(mesh.xyz), _i32(mesh.tets)
    fib, cf, ct = _f32(fib), _f32(cf), _f32(ct)
    kind, idx, t, bary = _onset_arrays(onsets)
    n_v, n_t = xyz.shape[0], tets.shape[0]
    phi = np.empty(n_v)
    parent = np.empty(n_v, np.int32)
    alpha = np.empty((n_v, 3))
    margin = np.empty(n_v)
    stats = np.zeros(4, np.int64)
    rc = lib().orc_eikonal(n_v, _p(xyz), n_t, _p(tets), _p(cf), _p(ct), _p(fib), kind, len(idx),
                           _p(idx), _p(bary), _p(t), int(mode), int(n_f), int(order), _p(phi),
                           _p(parent), _p(alpha), _p(margin), _p(stats))
    if rc != 0:
        raise RuntimeError(f"orc_eikonal failed ({rc})")
    return dict(phi=phi, parent=parent, alpha=alpha, margin=margin,
                stats=dict(pops=int(stats[0]), solves=int(stats[1]),
                           max_fixed_point_residual=stats[2] * 1e-15, unreached=int(stats[3])))


def ecg(L, phi, tmpl):
    L = _f32(L)
    phi = _f64(phi)
    N, n_v = L.shape
    V = np.empty((N, tmpl.T))
    lib().orc_ecg(n_v, N, _p(L), _p(phi), tmpl.K0, tmpl.K1, tmpl.tau, tmpl.t0, tmpl.dt, tmpl.T,
                  _p(V))
    return V


def loss_grad_phi(L, phi, tmpl, V, target):
    """Eq. (inverse_ecg) and d loss / d phi.  Returns (loss, lam [n_v])."""
    L, phi, V, target = _f32(L), _f64(phi), _f64(V), _f32(target)
    N, n_v = L.shape
    lam = np.empty(n_v)
    loss = lib().orc_loss_grad_phi(n_v, N, _p(L), _p(phi), tmpl.K0, tmpl.K1, tmpl.tau, tmpl.t0,
                                   tmpl.dt, tmpl.T, _p(V), _p(target), _p(lam))
    return float(loss), lam


def adjoint(mesh, fib, cf, ct, onsets, parent, alpha, lam):
    """Frozen-graph adjoint.  Returns dict(d_cf, d_ct, d_t, d_x, mu, unprocessed)."""
    xyz, tets = _f32(mesh.xyz), _i32(mesh.tets)
    fib, cf, ct = _f32(fib), _f32(cf), _f32(ct)
    kind, idx, t, bary = _onset_arrays(onsets)
    parent, alpha, lam = _i32(parent), _f64(alpha), _f64(lam)
    n_v, n_t, K = xyz.shape[0], tets.shape[0], len(idx)
    d_cf, d_ct = np.empty(n_t), np.empty(n_t)
    d_t, d_x = np.empty(K), np.empty((K, 3))
    mu = np.empty(n_v)
    left = lib().orc_adjoint(n_v, _p(xyz), n_t, _p(tets), _p(cf), _p(ct), _p(fib), kind, K,
                             _p(idx), _p(bary), _p(t), _p(parent), _p(alpha), _p(lam), _p(d_cf),
                             _p(d_ct), _p(d_t), _p(d_x), _p(mu))
    return dict(d_cf=d_cf, d_ct=d_ct, d_t=d_t, d_x=d_x, mu=mu, unprocessed=int(left))


def forward_backward(mesh, fib, cf, ct, onsets, L, tmpl, target, mode=EXACT, n_f=64):
    """One forward + gradient evaluation: eikonal -> ECG -> misfit -> adjoint."""
    ek = eikonal(mesh, fib, cf, ct, onsets, mode=mode, n_f=n_f)
    V = ecg(L, ek["phi"], tmpl)
    loss, lam = loss_grad_phi(L, ek["phi"], tmpl, V, target)
    g = adjoint(mesh, fib, cf, ct, onsets, ek["parent"], ek["alpha"], lam)
    return dict(loss=loss, V=V, lam=lam, **ek, **g)


def loss_only(mesh, fib, cf, ct, onsets, L, tmpl, target, mode=EXACT, n_f=64):
    ek = eikonal(mesh, fib, cf, ct, onsets, mode=mode, n_f=n_f)
    V = ecg(L, ek["phi"], tmpl)
    r = V - np.asarray(target, float)
    return float(np.mean(r * r)), ek


# ---------------------------------------------------------------------------
# finite differences
# ---------------------------------------------------------------------------

def fd_probe(fun, h: float):
    """Central difference (fun(+h) - fun(-h)) / 2h of a scalar function of a
    scalar offset."""
    return (fun(+h) - fun(-h)) / (2.0 * h)


def ensure_built() -> str:
    return _build.build()


def library_path() -> str:
    return os.path.abspath(_build.LIB)
