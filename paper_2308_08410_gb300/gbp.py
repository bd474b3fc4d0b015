"""Thin Python binding of libgbp.so (include/gbp.h): argument marshalling only.

Every step of the computation runs in the library's CUDA kernels; this module
passes device pointers of torch tensors (PyTorch is used for device memory and
streams).  There is no CPU fallback: if the library cannot be loaded, or no
CUDA device is present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os

import numpy as np

from . import build as _build

LOCAL_EXACT, LOCAL_FISTA = 0, 1
ONSET_NODAL, ONSET_ELEMENT = 0, 1
PREC_FP32, PREC_BF16 = 0, 1
UNREACHED = -(2 ** 31)

_STATUS = {
    0: "ok", 1: "invalid argument", 2: "bad mesh", 3: "conduction tensor not SPD",
    4: "iteration limit reached", 5: "bounded device wait ran out", 6: "unreachable vertices",
    7: "CUDA runtime error", 8: "call order violated", 9: "out of device memory",
}


class GbpError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {_STATUS.get(status, 'unknown')} (status {status})")
        self.status = status


class SolveOpts(C.Structure):
    _fields_ = [("local_solver", C.c_int32), ("n_f", C.c_int32), ("eps", C.c_float),
                ("max_iters", C.c_int32)]


class SolveStats(C.Structure):
    _fields_ = [("iterations", C.c_int64), ("candidates", C.c_int64), ("face_updates", C.c_int64),
                ("fp64_fallbacks", C.c_int64), ("unreached", C.c_int64), ("adj_levels", C.c_int64),
                ("adj_cycle_nodes", C.c_int64), ("adj_cycle_iters", C.c_int64),
                ("status", C.c_int32), ("reserved", C.c_int32), ("adj_dataflow_ms", C.c_double),
                ("adj_cycle_ms", C.c_double), ("fim_deferred", C.c_int64), ("fim_repaired", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class Template(C.Structure):
    _fields_ = [("K0", C.c_float), ("K1", C.c_float), ("tau", C.c_float), ("t0", C.c_float),
                ("dt", C.c_float), ("T", C.c_int32)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load():
    """Load libgbp.so, building it in place when missing or stale.  The
    environment variable GBP_LIBRARY selects another prebuilt copy of the
    library (for example one compiled with different kernel shapes)."""
    global _lib
    if _lib is not None:
        return _lib
    path = os.environ.get("GBP_LIBRARY") or _build.build()
    L = C.CDLL(path)
    P, i32, i64, f32 = C.c_void_p, C.c_int32, C.c_int64, C.c_float
    sig = {
        "gbp_create": ([C.POINTER(P), C.c_int, P], i32),
        "gbp_destroy": ([P], None),
        "gbp_set_stream": ([P, P], i32),
        "gbp_status_string": ([i32], C.c_char_p),
        "gbp_synchronize": ([P], i32),
        "gbp_upload_mesh": ([P, P, i64, P, i64], i32),
        "gbp_upload_mesh_2d": ([P, P, i64, P, i64], i32),
        "gbp_check_mesh": ([P, i64, P, i64], i32),
        "gbp_check_mesh_2d": ([P, i64, P, i64], i32),
        "gbp_mesh_adjacency": ([P, i64, i64, P, P, P, P, P, P, P], i32),
        "gbp_set_fibres": ([P, P], i32),
        "gbp_set_velocities": ([P, P, P], i32),
        "gbp_set_leadfield": ([P, P, i32], i32),
        "gbp_set_onsets": ([P, i32, i32, P, P, P], i32),
        "gbp_set_onsets_batch": ([P, i32, i32, i32, P, P, P], i32),
        "gbp_eikonal_solve": ([P, C.POINTER(SolveOpts), P, P, P], i32),
        "gbp_get_solve_stats": ([P, C.POINTER(SolveStats)], i32),
        "gbp_get_solution": ([P, i32, P, P, P], i32),
        "gbp_ecg_forward": ([P, P, C.POINTER(Template), i32, P], i32),
        "gbp_ecg_loss_backward": ([P, P, P, P, C.POINTER(Template), P, P], i32),
        "gbp_geodesic_backward": ([P, P, P, P, P, P], i32),
        "gbp_forward_backward": ([P, C.POINTER(SolveOpts), C.POINTER(Template), i32, P, P, P, P, P, P, P, P,
                                  P, P], i32),
        "gbp_forward_backward_host": ([P, C.POINTER(SolveOpts), C.POINTER(Template), i32, P, P, P, P, P, P,
                                       P, P, P], i32),
        "gbp_forward_backward_batch": ([P, i32, C.POINTER(SolveOpts), C.POINTER(Template), i32, P, P, P, P, P,
                                        P, P, P, P, P], i32),
        "gbp_forward_backward_batch_host": ([P, i32, C.POINTER(SolveOpts), C.POINTER(Template), i32, P, P, P, P,
                                             P, P, P, P, P], i32),
        "gbp_local_solve_batch": ([P, i64, P, P, P, P, P, i32, i32, P, P], i32),
        "gbp_diag_barrier_timeout": ([P, i32, i32], i32),
        "gbp_enable_timing": ([P, i32], i32),
        "gbp_get_kernel_times": ([P, i32, P, P], i32),
        "gbp_reset_kernel_times": ([P], i32),
        "gbp_launch_count": ([P], i64),
        "gbp_ecg_forward_noalloc": ([P, i32, i64, P, C.POINTER(Template), P, P], i32),
        "gbp_enable_trace": ([P, i32], i32),
        "gbp_get_trace": ([P, P, i32], i32),
        "gbp_nn_gemm_bf16": ([P, i32, i32, i32, P, i32, P, i32, P, i32, f32, f32], i32),
        "gbp_nn_im2col": ([P, i32, i32, i32, i32, i32, i32, i32, P, P, i32], i32),
        "gbp_nn_im2col_t": ([P, i32, i32, i32, i32, i32, i32, i32, P, i32, P, i32], i32),
        "gbp_nn_col2im": ([P, i32, i32, i32, i32, i32, i32, i32, P, i32, P], i32),
        "gbp_nn_bias_act": ([P, i32, i32, P, i32, P, P, i32], i32),
        "gbp_nn_gelu_backward": ([P, i32, i32, P, i32, P], i32),
        "gbp_nn_bias_grad": ([P, i32, i32, P, i32, P], i32),
        "gbp_nn_cast_bf16": ([P, i32, i32, P, i32, P, i32], i32),
        "gbp_nn_transpose_bf16": ([P, i32, i32, P, i32, P, i32], i32),
        "gbp_nn_mse": ([P, i32, P, P, P, P], i32),
        "gbp_nn_adam": ([P, i64, P, P, P, P, f32, f32, f32, f32, i32, P], i32),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def exported_symbols():
    """Names of the entry points this binding expects the library to export."""
    return [
        "gbp_create", "gbp_destroy", "gbp_set_stream", "gbp_status_string", "gbp_synchronize",
        "gbp_upload_mesh", "gbp_upload_mesh_2d", "gbp_check_mesh", "gbp_check_mesh_2d", "gbp_mesh_adjacency",
        "gbp_set_fibres", "gbp_set_velocities", "gbp_set_leadfield",
        "gbp_set_onsets", "gbp_set_onsets_batch", "gbp_eikonal_solve", "gbp_get_solve_stats",
        "gbp_get_solution", "gbp_ecg_forward",
        "gbp_ecg_loss_backward", "gbp_geodesic_backward", "gbp_forward_backward",
        "gbp_forward_backward_host", "gbp_forward_backward_batch", "gbp_forward_backward_batch_host", "gbp_local_solve_batch", "gbp_diag_barrier_timeout",
        "gbp_enable_timing",
        "gbp_get_kernel_times", "gbp_reset_kernel_times", "gbp_launch_count",
        "gbp_ecg_forward_noalloc", "gbp_enable_trace", "gbp_get_trace",
        "gbp_nn_gemm_bf16", "gbp_nn_im2col", "gbp_nn_im2col_t", "gbp_nn_col2im", "gbp_nn_bias_act",
        "gbp_nn_gelu_backward", "gbp_nn_bias_grad", "gbp_nn_cast_bf16", "gbp_nn_transpose_bf16",
        "gbp_nn_mse", "gbp_nn_adam",
    ]


def _check(st, where):
    if st != 0:
        raise GbpError(int(st), where)


def _ptr(t):
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def _hptr(a, dtype=None):
    if a is None:
        return None
    if not (isinstance(a, np.ndarray) and a.flags["C_CONTIGUOUS"]):
        raise ValueError("expected a C-contiguous numpy array")
    if dtype is not None and a.dtype != dtype:
        raise ValueError(f"expected a {np.dtype(dtype).name} array, got {a.dtype.name}")
    return a.ctypes.data_as(C.c_void_p)


def _f32(a):
    """Host pointer of a float32 array (the host entry points read float32)."""
    return _hptr(a, np.float32)


def check_mesh(xyz: np.ndarray, tets: np.ndarray) -> int:
    """Host-only validation of a tet mesh (gbp_check_mesh): the status
    gbp_upload_mesh would return for it before building anything."""
    xyz = np.ascontiguousarray(xyz, np.float32)
    tets = np.ascontiguousarray(tets, np.int32)
    return int(load().gbp_check_mesh(_hptr(xyz), xyz.shape[0], _hptr(tets), tets.shape[0]))


def check_mesh_2d(xy: np.ndarray, tris: np.ndarray) -> int:
    """Host-only validation of a triangle mesh (gbp_check_mesh_2d)."""
    xy = np.ascontiguousarray(xy, np.float32)
    tris = np.ascontiguousarray(tris, np.int32)
    return int(load().gbp_check_mesh_2d(_hptr(xy), xy.shape[0], _hptr(tris), tris.shape[0]))


def mesh_adjacency(tets: np.ndarray, n_v: int) -> dict:
    """The host adjacency the upload builds (gbp_mesh_adjacency): n2t_ptr,
    n2t (tet * 4 + slot per vertex), n2n_ptr, n2n (neighbours) and frec
    [n_faces, 4] (the other three vertices in slot order, code)."""
    tets = np.ascontiguousarray(tets, np.int32)
    L = load()
    nf, nn = C.c_int64(0), C.c_int64(0)
    _check(L.gbp_mesh_adjacency(_hptr(tets), int(n_v), tets.shape[0], C.byref(nf), C.byref(nn),
                                None, None, None, None, None), "gbp_mesh_adjacency")
    out = dict(n2t_ptr=np.zeros(n_v + 1, np.int32), n2t=np.zeros(nf.value, np.int32),
               n2n_ptr=np.zeros(n_v + 1, np.int32), n2n=np.zeros(nn.value, np.int32),
               frec=np.zeros((nf.value, 4), np.int32))
    _check(L.gbp_mesh_adjacency(_hptr(tets), int(n_v), tets.shape[0], C.byref(nf), C.byref(nn),
                                _hptr(out["n2t_ptr"]), _hptr(out["n2t"]), _hptr(out["n2n_ptr"]),
                                _hptr(out["n2n"]), _hptr(out["frec"])), "gbp_mesh_adjacency")
    return out


def make_opts(local_solver=LOCAL_EXACT, n_f=32, eps=0.0, max_iters=0) -> SolveOpts:
    return SolveOpts(int(local_solver), int(n_f), float(eps), int(max_iters))


def make_template(tm) -> Template:
    return Template(float(tm.K0), float(tm.K1), float(tm.tau), float(tm.t0), float(tm.dt), int(tm.T))


class Context:
    """One libgbp context on one CUDA device, ordered on a torch stream."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libgbp needs a CUDA device; none is available")
        self.lib = load()
        self.device = int(device)
        self.torch_device = torch.device("cuda", self.device)
        if stream is None:
            stream = torch.cuda.current_stream(self.torch_device)
        self.stream = stream
        h = C.c_void_p()
        _check(self.lib.gbp_create(C.byref(h), self.device, C.c_void_p(stream.cuda_stream)), "gbp_create")
        self.h = h
        self.n_v = self.n_t = self.N = self.K = 0
        self.dim = 3

    def close(self):
        if getattr(self, "h", None):
            self.lib.gbp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        self.stream = stream
        _check(self.lib.gbp_set_stream(self.h, C.c_void_p(stream.cuda_stream)), "gbp_set_stream")

    # ---- set-up -----------------------------------------------------------
    def upload_mesh(self, xyz: np.ndarray, tets: np.ndarray):
        xyz = np.ascontiguousarray(xyz, np.float32)
        tets = np.ascontiguousarray(tets, np.int32)
        _check(self.lib.gbp_upload_mesh(self.h, _hptr(xyz), xyz.shape[0], _hptr(tets), tets.shape[0]),
               "gbp_upload_mesh")
        self.n_v, self.n_t = xyz.shape[0], tets.shape[0]
        self.dim = 3

    def upload_mesh_2d(self, xy: np.ndarray, tris: np.ndarray):
        """Triangle mesh (d = 2): xy [n_v, 2], tris [n_t, 3] counter-clockwise.
        From here on fibres are [n_t, 2], alpha [n_v, 2], d_x [K, 2]."""
        xy = np.ascontiguousarray(xy, np.float32)
        tris = np.ascontiguousarray(tris, np.int32)
        _check(self.lib.gbp_upload_mesh_2d(self.h, _hptr(xy), xy.shape[0], _hptr(tris), tris.shape[0]),
               "gbp_upload_mesh_2d")
        self.n_v, self.n_t = xy.shape[0], tris.shape[0]
        self.dim = 2

    def set_fibres(self, fib):
        _check(self.lib.gbp_set_fibres(self.h, _ptr(fib)), "gbp_set_fibres")

    def set_velocities(self, cf, ct):
        _check(self.lib.gbp_set_velocities(self.h, _ptr(cf), _ptr(ct)), "gbp_set_velocities")

    def set_leadfield(self, L):
        _check(self.lib.gbp_set_leadfield(self.h, _ptr(L), L.shape[0]), "gbp_set_leadfield")
        self.N = L.shape[0]

    def set_onsets(self, kind, idx, t, bary=None):
        _check(self.lib.gbp_set_onsets(self.h, int(kind), idx.shape[0], _ptr(idx), _ptr(bary), _ptr(t)),
               "gbp_set_onsets")
        self.K = idx.shape[0]

    def set_onsets_batch(self, kind, idx, t, bary=None):
        """One site set per problem of the next batched calls: idx [B, K],
        t [B, K], bary [B, K, d + 1] (element onsets)."""
        B, K = int(idx.shape[0]), int(idx.shape[1])
        _check(self.lib.gbp_set_onsets_batch(self.h, int(kind), B, K, _ptr(idx), _ptr(bary), _ptr(t)),
               "gbp_set_onsets_batch")
        self.K = K

    # ---- hot path -----------------------------------------------------------
    def eikonal_solve(self, opts: SolveOpts | None = None, phi=None, parent=None, alpha=None):
        import torch
        dev = self.torch_device
        phi = torch.empty(self.n_v, dtype=torch.float32, device=dev) if phi is None else phi
        parent = torch.empty(self.n_v, dtype=torch.int32, device=dev) if parent is None else parent
        alpha = torch.empty(self.n_v, self.dim, dtype=torch.float32, device=dev) if alpha is None else alpha
        o = opts if opts is not None else make_opts()
        _check(self.lib.gbp_eikonal_solve(self.h, C.byref(o), _ptr(phi), _ptr(parent), _ptr(alpha)),
               "gbp_eikonal_solve")
        return phi, parent, alpha

    def solution(self, b: int = 0):
        """phi [n_v], parent codes [n_v] and alpha [n_v, d] of problem b of
        the last solve (a batched call keeps all B)."""
        import torch
        dev = self.torch_device
        phi = torch.empty(self.n_v, dtype=torch.float32, device=dev)
        parent = torch.empty(self.n_v, dtype=torch.int32, device=dev)
        alpha = torch.empty(self.n_v, self.dim, dtype=torch.float32, device=dev)
        _check(self.lib.gbp_get_solution(self.h, int(b), _ptr(phi), _ptr(parent), _ptr(alpha)), "gbp_get_solution")
        return phi, parent, alpha

    def stats(self) -> dict:
        s = SolveStats()
        st = self.lib.gbp_get_solve_stats(self.h, C.byref(s))
        d = s.as_dict()
        d["status_code"] = int(st)
        return d

    def synchronize(self):
        _check(self.lib.gbp_synchronize(self.h), "gbp_synchronize")

    def ecg_forward(self, phi, tmpl, precision=PREC_FP32, out=None):
        import torch
        t = make_template(tmpl)
        out = torch.empty(self.N, t.T, dtype=torch.float32, device=self.torch_device) if out is None else out
        _check(self.lib.gbp_ecg_forward(self.h, _ptr(phi), C.byref(t), int(precision), _ptr(out)),
               "gbp_ecg_forward")
        return out

    def ecg_loss_backward(self, phi, ecg, target, tmpl):
        import torch
        t = make_template(tmpl)
        loss = torch.empty(1, dtype=torch.float32, device=self.torch_device)
        dphi = torch.empty(self.n_v, dtype=torch.float32, device=self.torch_device)
        _check(self.lib.gbp_ecg_loss_backward(self.h, _ptr(phi), _ptr(ecg), _ptr(target), C.byref(t),
                                              _ptr(loss), _ptr(dphi)), "gbp_ecg_loss_backward")
        return loss, dphi

    def geodesic_backward(self, dphi):
        import torch
        dev = self.torch_device
        d_cf = torch.empty(self.n_t, dtype=torch.float32, device=dev)
        d_ct = torch.empty(self.n_t, dtype=torch.float32, device=dev)
        d_t = torch.empty(self.K, dtype=torch.float32, device=dev)
        d_x = torch.empty(self.K, self.dim, dtype=torch.float32, device=dev)
        _check(self.lib.gbp_geodesic_backward(self.h, _ptr(dphi), _ptr(d_cf), _ptr(d_ct), _ptr(d_t),
                                              _ptr(d_x)), "gbp_geodesic_backward")
        return d_cf, d_ct, d_t, d_x

    def forward_backward(self, cf, ct, target, tmpl, t=None, opts=None, precision=PREC_FP32,
                         out=None):
        """One fused evaluation; returns dict of device tensors."""
        import torch
        dev = self.torch_device
        if out is None:
            out = dict(loss=torch.empty(1, dtype=torch.float32, device=dev),
                       ecg=torch.empty(self.N, tmpl.T, dtype=torch.float32, device=dev),
                       d_cf=torch.empty(self.n_t, dtype=torch.float32, device=dev),
                       d_ct=torch.empty(self.n_t, dtype=torch.float32, device=dev),
                       d_t=torch.empty(self.K, dtype=torch.float32, device=dev),
                       d_x=torch.empty(self.K, self.dim, dtype=torch.float32, device=dev))
        tm = make_template(tmpl)
        o = opts if opts is not None else make_opts()
        _check(self.lib.gbp_forward_backward(self.h, C.byref(o), C.byref(tm), int(precision), _ptr(cf),
                                             _ptr(ct), _ptr(t), _ptr(target), _ptr(out["loss"]),
                                             _ptr(out.get("ecg")), _ptr(out["d_cf"]), _ptr(out["d_ct"]),
                                             _ptr(out["d_t"]), _ptr(out["d_x"])), "gbp_forward_backward")
        return out

    def forward_backward_batch(self, cf, ct, target, tmpl, t=None, opts=None, precision=PREC_FP32, out=None):
        """B evaluations in one pass: cf, ct [B, n_t]; target [B, N, T];
        t [B, K] or None.  Returns dict of device tensors with a leading B."""
        import torch
        B = int(cf.shape[0])
        dev = self.torch_device
        if out is None:
            f32 = dict(dtype=torch.float32, device=dev)
            out = dict(loss=torch.empty(B, **f32), ecg=torch.empty(B, self.N, tmpl.T, **f32),
                       d_cf=torch.empty(B, self.n_t, **f32), d_ct=torch.empty(B, self.n_t, **f32),
                       d_t=torch.empty(B, self.K, **f32), d_x=torch.empty(B, self.K, self.dim, **f32))
        tm = make_template(tmpl)
        o = opts if opts is not None else make_opts()
        _check(self.lib.gbp_forward_backward_batch(self.h, B, C.byref(o), C.byref(tm), int(precision), _ptr(cf),
                                                   _ptr(ct), _ptr(t), _ptr(target), _ptr(out["loss"]),
                                                   _ptr(out.get("ecg")), _ptr(out["d_cf"]), _ptr(out["d_ct"]),
                                                   _ptr(out["d_t"]), _ptr(out["d_x"])),
               "gbp_forward_backward_batch")
        return out

    def forward_backward_host(self, cf: np.ndarray, ct: np.ndarray, target: np.ndarray, tmpl,
                              t: np.ndarray | None = None, opts=None, precision=PREC_FP32, out=None):
        """The same evaluation from host arrays (copies inside the call)."""
        if out is None:
            out = dict(loss=np.zeros(1, np.float32), d_cf=np.empty(self.n_t, np.float32),
                       d_ct=np.empty(self.n_t, np.float32), d_t=np.empty(self.K, np.float32),
                       d_x=np.empty((self.K, self.dim), np.float32))
        tm = make_template(tmpl)
        o = opts if opts is not None else make_opts()
        _check(self.lib.gbp_forward_backward_host(self.h, C.byref(o), C.byref(tm), int(precision),
                                                  _f32(cf), _f32(ct), _f32(t), _f32(target),
                                                  _f32(out["loss"]), _f32(out["d_cf"]),
                                                  _f32(out["d_ct"]), _f32(out["d_t"]),
                                                  _f32(out["d_x"])), "gbp_forward_backward_host")
        return out

    def forward_backward_batch_host(self, cf: np.ndarray, ct: np.ndarray, target: np.ndarray, tmpl,
                                    t: np.ndarray | None = None, opts=None, precision=PREC_FP32, out=None):
        """The batched evaluation from host arrays (cf, ct [B, n_t], target
        [B, N, T], t [B, K] or None); outputs into host arrays.  Pinned
        arrays (e.g. numpy views of pinned torch tensors) copy fastest."""
        B = int(cf.shape[0])
        if out is None:
            out = dict(loss=np.zeros(B, np.float32), d_cf=np.empty((B, self.n_t), np.float32),
                       d_ct=np.empty((B, self.n_t), np.float32), d_t=np.empty((B, self.K), np.float32),
                       d_x=np.empty((B, self.K, self.dim), np.float32))
        tm = make_template(tmpl)
        o = opts if opts is not None else make_opts()
        _check(self.lib.gbp_forward_backward_batch_host(self.h, B, C.byref(o), C.byref(tm), int(precision),
                                                        _f32(cf), _f32(ct), _f32(t), _f32(target),
                                                        _f32(out["loss"]), _f32(out["d_cf"]),
                                                        _f32(out["d_ct"]), _f32(out["d_t"]),
                                                        _f32(out["d_x"])), "gbp_forward_backward_batch_host")
        return out

    def local_solve_batch(self, e, fib, cf, ct, phi, mode=LOCAL_EXACT, n_f=32):
        import torch
        n = e.shape[0]
        val = torch.empty(n, dtype=torch.float32, device=self.torch_device)
        al = torch.empty(n, 3, dtype=torch.float32, device=self.torch_device)
        _check(self.lib.gbp_local_solve_batch(self.h, n, _ptr(e), _ptr(fib), _ptr(cf), _ptr(ct), _ptr(phi),
                                              int(mode), int(n_f), _ptr(val), _ptr(al)),
               "gbp_local_solve_batch")
        return val, al

    def diag_barrier_timeout(self, absent_ctas: int, max_spins: int):
        """Grid barrier with absent_ctas CTAs that never arrive (bounded
        waits of max_spins polls); the outcome is latched in the context."""
        _check(self.lib.gbp_diag_barrier_timeout(self.h, int(absent_ctas), int(max_spins)),
               "gbp_diag_barrier_timeout")

    # ---- timing ---------------------------------------------------------------
    def enable_timing(self, on=True):
        _check(self.lib.gbp_enable_timing(self.h, int(bool(on))), "gbp_enable_timing")

    def kernel_times(self, n=6):
        ms = np.zeros(n, np.float64)
        ln = np.zeros(n, np.int64)
        _check(self.lib.gbp_get_kernel_times(self.h, n, _hptr(ms), _hptr(ln)), "gbp_get_kernel_times")
        return ms, ln

    def reset_kernel_times(self):
        _check(self.lib.gbp_reset_kernel_times(self.h), "gbp_reset_kernel_times")

    def launch_count(self) -> int:
        return int(self.lib.gbp_launch_count(self.h))

    def enable_trace(self, on=True):
        _check(self.lib.gbp_enable_trace(self.h, int(bool(on))), "gbp_enable_trace")

    def trace(self, max_rows=4096):
        """(active vertices, global-timer ns) per FIM iteration of the last solve."""
        buf = np.zeros((max_rows, 2), np.int64)
        n = int(self.lib.gbp_get_trace(self.h, _hptr(buf), max_rows))
        return buf[:n]


@dataclasses.dataclass
class DeviceProblem:
    """A problem uploaded to a context (device tensors kept alive here)."""
    ctx: Context
    fib: object
    cf: object
    ct: object
    L: object
    on_idx: object
    on_t: object
    on_bary: object
    kind: int


def setup_problem(ctx: Context, problem) -> DeviceProblem:
    """Upload a seeded problem (mesh, fibres, velocities, lead field, onsets)."""
    import torch
    dev = ctx.torch_device
    ctx.upload_mesh(problem.mesh.xyz, problem.mesh.tets)
    fib = torch.from_numpy(np.ascontiguousarray(problem.fib, np.float32)).to(dev)
    cf = torch.from_numpy(np.ascontiguousarray(problem.cf, np.float32)).to(dev)
    ct = torch.from_numpy(np.ascontiguousarray(problem.ct, np.float32)).to(dev)
    L = torch.from_numpy(np.ascontiguousarray(problem.L, np.float32)).to(dev)
    ons = problem.onsets
    idx = torch.from_numpy(np.ascontiguousarray(ons.idx, np.int32)).to(dev)
    t = torch.from_numpy(np.ascontiguousarray(ons.t, np.float32)).to(dev)
    bary = None
    if ons.bary is not None:
        bary = torch.from_numpy(np.ascontiguousarray(ons.bary, np.float32)).to(dev)
    ctx.set_fibres(fib)
    ctx.set_velocities(cf, ct)
    ctx.set_leadfield(L)
    ctx.set_onsets(ons.kind, idx, t, bary)
    return DeviceProblem(ctx, fib, cf, ct, L, idx, t, bary, ons.kind)


def setup_problem_2d(ctx: Context, problem) -> DeviceProblem:
    """Upload a seeded triangle-mesh problem (synth.Problem2D): its element
    onsets when it has them (problem.onsets), else its nodal ones."""
    import torch
    dev = ctx.torch_device
    ctx.upload_mesh_2d(problem.mesh.xy, problem.mesh.tris)

    def up(a, dt=np.float32):
        return torch.from_numpy(np.ascontiguousarray(a, dt)).to(dev)

    fib, cf, ct, L = up(problem.fib), up(problem.cf), up(problem.ct), up(problem.L)
    ons = getattr(problem, "onsets", None)
    if ons is None:
        kind, idx, t, bary = ONSET_NODAL, up(problem.onset_nodes, np.int32), up(problem.onset_t), None
    else:
        kind, idx, t = ons.kind, up(ons.idx, np.int32), up(ons.t)
        bary = up(ons.bary) if ons.bary is not None else None
    ctx.set_fibres(fib)
    ctx.set_velocities(cf, ct)
    ctx.set_leadfield(L)
    ctx.set_onsets(kind, idx, t, bary)
    return DeviceProblem(ctx, fib, cf, ct, L, idx, t, bary, kind)


def library_exists() -> bool:
    return os.path.exists(_build.LIB)
