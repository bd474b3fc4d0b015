"""Learned initialiser for Geodesic-BP: a 1-D convolutional network + MLP that
maps a 12-lead ECG to initial onset sites, onset times and velocities.

Not in the paper: it initialises the inverse problem of Sec. II-D, which
Geodesic-BP then refines.  The network is trained in BF16 with FP32 master
weights by the library's own kernels (include/gbp.h, gbp_nn_*: tcgen05 GEMMs,
im2col / col2im, bias + GELU, Adam); this module only owns device buffers and
sequences the calls.  Training pairs come from the forward model itself
(gbp_eikonal_solve + gbp_ecg_forward).
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import math
import time

import numpy as np
import torch

from . import gbp
from . import synth as S


def _p(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _r64(n):
    return ((n + 63) // 64) * 64


@dataclasses.dataclass
class NetConfig:
    C_in: int = 12
    L_in: int = 300
    channels: int = 64
    n_conv: int = 4
    ksize: int = 5
    stride: int = 2
    pad: int = 2
    hidden: int = 256
    n_out: int = 43

    def lens(self):
        ls = [self.L_in]
        for _ in range(self.n_conv):
            ls.append((ls[-1] + 2 * self.pad - self.ksize) // self.stride + 1)
        return ls


class ConvMLP:
    """Parameters in FP32 masters (+ BF16 copies, Adam moments); activations
    for a fixed maximum batch.  Parameter order matches the FP64 reference:
    [W_conv0 (Co, ks, Ci), b_conv0, ..., W_fc1 (hidden, flat), b_fc1,
     W_fc2 (n_out, hidden), b_fc2]."""

    def __init__(self, ctx: gbp.Context, cfg: NetConfig, params: list[np.ndarray], max_batch: int):
        self.ctx, self.lib, self.cfg = ctx, ctx.lib, cfg
        dev = ctx.torch_device
        self.dev = dev
        self.B = max_batch
        L = cfg.lens()
        self.L = L
        self.flat = L[-1] * cfg.channels
        # layer GEMM shapes: K (reduction, unpadded) and N (outputs)
        self.Kc = [cfg.ksize * (cfg.C_in if i == 0 else cfg.channels) for i in range(cfg.n_conv)]
        f32 = dict(dtype=torch.float32, device=dev)
        bf = dict(dtype=torch.bfloat16, device=dev)
        self.W, self.Wb, self.Wp, self.g, self.m1, self.m2 = [], [], [], [], [], []
        for i, p in enumerate(params):
            t = torch.tensor(np.asarray(p, np.float32), **f32)
            if t.dim() == 3:  # conv weight [Co, ks, Ci] -> [Co, Kp] zero padded
                Co, ks, Ci = t.shape
                K = ks * Ci
                w = torch.zeros(Co, _r64(K), **f32)
                w[:, :K] = t.reshape(Co, K)
            elif t.dim() == 2:
                No, K = t.shape
                w = torch.zeros(No, _r64(K), **f32)
                w[:, :K] = t
            else:
                w = t.clone()
            self.W.append(w)
            self.Wb.append(w.to(torch.bfloat16) if w.dim() == 2 else None)
            self.g.append(torch.zeros_like(w))
            self.m1.append(torch.zeros_like(w))
            self.m2.append(torch.zeros_like(w))
        B = max_batch
        ch = cfg.channels
        # forward buffers
        self.act = [torch.empty(B, L[0], cfg.C_in, **f32)]
        self.pre = []
        self.col = []
        for i in range(cfg.n_conv):
            self.col.append(torch.empty(B * L[i + 1], _r64(self.Kc[i]), **bf))
            self.act.append(torch.empty(B, L[i + 1], ch, **f32))
            self.pre.append(torch.empty(B * L[i + 1], ch, **f32))
        self.flat_bf = torch.empty(B, _r64(self.flat), **bf)
        self.h = torch.empty(B, cfg.hidden, **f32)
        self.h_pre = torch.empty(B, cfg.hidden, **f32)
        self.h_bf = torch.empty(B, _r64(cfg.hidden), **bf)
        self.y = torch.empty(B, cfg.n_out, **f32)
        # backward buffers
        self.dy = torch.empty(B, cfg.n_out, **f32)
        self.loss = torch.empty(1, **f32)
        self.dh = torch.empty(B, cfg.hidden, **f32)
        self.dflat = torch.empty(B, self.flat, **f32)
        self.dact = [torch.empty_like(a) for a in self.act]
        self.dcol = [torch.empty(B * L[i + 1], _r64(self.Kc[i]), **f32) for i in range(cfg.n_conv)]
        mp = _r64(B * max(L[1:]))
        self.tA = torch.empty(max(ch, cfg.hidden, cfg.n_out), mp, **bf)  # dZ^T
        self.tB = torch.empty(max(_r64(max(self.Kc)), self.flat, cfg.hidden), mp, **bf)  # X^T
        self.dz_bf = torch.empty(B * max(L[1:]), _r64(max(ch, cfg.hidden, cfg.n_out)), **bf)
        self.wt_bf = torch.empty(max(_r64(max(self.Kc)), self.flat, cfg.hidden),
                                 _r64(max(ch, cfg.hidden, cfg.n_out)), **bf)
        self.step_count = 0

    # -- helpers ---------------------------------------------------------------
    def _ck(self, st, where):
        gbp._check(st, where)

    def _gemm(self, M, N, Kp, A, lda, Bm, ldb, Cm, ldc, alpha=1.0, beta=0.0):
        self._ck(self.lib.gbp_nn_gemm_bf16(self.ctx.h, M, N, Kp, _p(A), lda, _p(Bm), ldb, _p(Cm), ldc,
                                           alpha, beta), "gbp_nn_gemm_bf16")

    # -- forward ------------------------------------------------------------------
    def forward(self, x: torch.Tensor, batch: int):
        """x: f32 [batch, L_in, C_in] (channels-last).  Returns y [batch, n_out]."""
        cfg, lib, h = self.cfg, self.lib, self.ctx.h
        B = batch
        self.act[0][:B].copy_(x)
        for i in range(cfg.n_conv):
            Ci = cfg.C_in if i == 0 else cfg.channels
            Li, Lo = self.L[i], self.L[i + 1]
            Kp = _r64(self.Kc[i])
            self._ck(lib.gbp_nn_im2col(h, B, Li, Ci, Lo, cfg.ksize, cfg.stride, cfg.pad, _p(self.act[i]),
                                       _p(self.col[i]), Kp), "im2col")
            out = self.act[i + 1]
            self._gemm(B * Lo, cfg.channels, Kp, self.col[i], Kp, self.Wb[2 * i], Kp, out, cfg.channels)
            self._ck(lib.gbp_nn_bias_act(h, B * Lo, cfg.channels, _p(out), cfg.channels, _p(self.W[2 * i + 1]),
                                         _p(self.pre[i]), 1), "bias_act")
        nc = 2 * cfg.n_conv
        Fp = _r64(self.flat)
        self._ck(lib.gbp_nn_cast_bf16(h, B, self.flat, _p(self.act[-1]), self.flat, _p(self.flat_bf), Fp), "cast")
        self._gemm(B, cfg.hidden, Fp, self.flat_bf, Fp, self.Wb[nc], Fp, self.h, cfg.hidden)
        self._ck(lib.gbp_nn_bias_act(h, B, cfg.hidden, _p(self.h), cfg.hidden, _p(self.W[nc + 1]),
                                     _p(self.h_pre), 1), "bias_act")
        Hp = _r64(cfg.hidden)
        self._ck(lib.gbp_nn_cast_bf16(h, B, cfg.hidden, _p(self.h), cfg.hidden, _p(self.h_bf), Hp), "cast")
        self._gemm(B, cfg.n_out, Hp, self.h_bf, Hp, self.Wb[nc + 2], Hp, self.y, cfg.n_out)
        self._ck(lib.gbp_nn_bias_act(h, B, cfg.n_out, _p(self.y), cfg.n_out, _p(self.W[nc + 3]), None, 0),
                 "bias_act")
        return self.y[:B]

    # -- backward -----------------------------------------------------------------
    def _dense_backward(self, B, dz, N, X, K, W, gW, gb, dX):
        """dz f32 [B, N] (already through the activation), X f32 [B, K]: writes
        gW [N, Kp] (first K columns), gb [N], and dX [B, K] if dX is given."""
        lib, h = self.lib, self.ctx.h
        Bp = _r64(B)
        self._ck(lib.gbp_nn_bias_grad(h, B, N, _p(dz), N, _p(gb)), "bias_grad")
        self._ck(lib.gbp_nn_transpose_bf16(h, B, N, _p(dz), N, _p(self.tA), Bp), "transpose")
        self._ck(lib.gbp_nn_transpose_bf16(h, B, K, _p(X), K, _p(self.tB), Bp), "transpose")
        Kp = _r64(K)
        gW.zero_()
        self._gemm(N, K, Bp, self.tA, Bp, self.tB, Bp, gW, Kp)
        if dX is not None:
            Np = _r64(N)
            self._ck(lib.gbp_nn_cast_bf16(h, B, N, _p(dz), N, _p(self.dz_bf), Np), "cast")
            self._ck(lib.gbp_nn_transpose_bf16(h, N, K, _p(W), Kp, _p(self.wt_bf), Np), "transpose")
            self._gemm(B, K, Np, self.dz_bf, Np, self.wt_bf, Np, dX, K)

    def backward(self, dy: torch.Tensor, batch: int):
        """dy f32 [batch, n_out] = dLoss/dy; fills self.g (FP32 gradients)."""
        cfg, lib, h = self.cfg, self.lib, self.ctx.h
        B = batch
        nc = 2 * cfg.n_conv
        dyc = self.dy[:B]
        if dyc.data_ptr() != dy.data_ptr():
            dyc.copy_(dy)
        # output layer (no activation)
        self._dense_backward(B, dyc, cfg.n_out, self.h, cfg.hidden, self.W[nc + 2], self.g[nc + 2],
                             self.g[nc + 3], self.dh)
        self._ck(lib.gbp_nn_gelu_backward(h, B, cfg.hidden, _p(self.dh), cfg.hidden, _p(self.h_pre)), "gelu_bwd")
        self._dense_backward(B, self.dh, cfg.hidden, self.act[-1], self.flat, self.W[nc], self.g[nc],
                             self.g[nc + 1], self.dflat)
        da = self.dflat  # [B, L_last * ch] == [B, L_last, ch]
        for i in reversed(range(cfg.n_conv)):
            Ci = cfg.C_in if i == 0 else cfg.channels
            Li, Lo = self.L[i], self.L[i + 1]
            M = B * Lo
            ch = cfg.channels
            Kp = _r64(self.Kc[i])
            self._ck(lib.gbp_nn_gelu_backward(h, M, ch, _p(da), ch, _p(self.pre[i])), "gelu_bwd")
            self._ck(lib.gbp_nn_bias_grad(h, M, ch, _p(da), ch, _p(self.g[2 * i + 1])), "bias_grad")
            Mp = _r64(M)
            self._ck(lib.gbp_nn_transpose_bf16(h, M, ch, _p(da), ch, _p(self.tA), Mp), "transpose")
            self._ck(lib.gbp_nn_im2col_t(h, B, Li, Ci, Lo, cfg.ksize, cfg.stride, cfg.pad, _p(self.act[i]), Kp,
                                         _p(self.tB), Mp), "im2col_t")
            self.g[2 * i].zero_()
            self._gemm(ch, self.Kc[i], Mp, self.tA, Mp, self.tB, Mp, self.g[2 * i], Kp)
            if i > 0:
                chp = _r64(ch)
                self._ck(lib.gbp_nn_cast_bf16(h, M, ch, _p(da), ch, _p(self.dz_bf), chp), "cast")
                self._ck(lib.gbp_nn_transpose_bf16(h, ch, self.Kc[i], _p(self.W[2 * i]), Kp, _p(self.wt_bf),
                                                   chp), "transpose")
                dcol = self.dcol[i]
                self._gemm(M, Kp, chp, self.dz_bf, chp, self.wt_bf, chp, dcol, Kp)
                self._ck(lib.gbp_nn_col2im(h, B, Li, Ci, Lo, cfg.ksize, cfg.stride, cfg.pad, _p(dcol), Kp,
                                           _p(self.dact[i])), "col2im")
                da = self.dact[i]

    def mse(self, target: torch.Tensor, batch: int):
        n = batch * self.cfg.n_out
        self._ck(self.lib.gbp_nn_mse(self.ctx.h, n, _p(self.y), _p(target), _p(self.dy), _p(self.loss)), "mse")
        return self.loss

    def adam_step(self, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.step_count += 1
        for w, wb, g, m1, m2 in zip(self.W, self.Wb, self.g, self.m1, self.m2):
            self._ck(self.lib.gbp_nn_adam(self.ctx.h, w.numel(), _p(w), _p(g), _p(m1), _p(m2), lr, b1, b2, eps,
                                          self.step_count, _p(wb)), "adam")

    def params_numpy(self):
        """Current FP32 masters in the reference layout."""
        out = []
        cfg = self.cfg
        for i, w in enumerate(self.W):
            a = w.detach().cpu().numpy()
            if i < 2 * cfg.n_conv and i % 2 == 0:
                Ci = cfg.C_in if i == 0 else cfg.channels
                out.append(a[:, :cfg.ksize * Ci].reshape(cfg.channels, cfg.ksize, Ci))
            elif a.ndim == 2:
                K = self.flat if i == 2 * cfg.n_conv else cfg.hidden
                out.append(a[:, :K])
            else:
                out.append(a)
        return out

    def grads_numpy(self):
        out = []
        cfg = self.cfg
        for i, g in enumerate(self.g):
            a = g.detach().cpu().numpy()
            if i < 2 * cfg.n_conv and i % 2 == 0:
                Ci = cfg.C_in if i == 0 else cfg.channels
                out.append(a[:, :cfg.ksize * Ci].reshape(cfg.channels, cfg.ksize, Ci))
            elif a.ndim == 2:
                K = self.flat if i == 2 * cfg.n_conv else cfg.hidden
                out.append(a[:, :K])
            else:
                out.append(a)
        return out
