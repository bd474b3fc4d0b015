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


# ---------------------------------------------------------------------------
# the c5 problem: cube mesh with a fast endocardial layer, surface sites
# ---------------------------------------------------------------------------

N_SITES = 10
CF_RANGE, CT_RANGE, CE_RANGE, T_RANGE = (0.4, 0.8), (0.2, 0.4), (1.0, 3.0), (0.0, 20.0)


@dataclasses.dataclass
class C5:
    """Cube mesh (c1 geometry) with a 1 mm fast layer on the z = 0 face whose
    isotropic velocity c_endo is the third global velocity, 12 standard leads
    from 10 electrodes on a 30 mm sphere, T = 300 @ 1 ms."""
    problem: S.Problem
    layer: np.ndarray        # bool [n_t]
    surf_tet: np.ndarray     # int32 [F] tet owning each boundary triangle
    surf_opp: np.ndarray     # int32 [F] slot of the tet vertex opposite the triangle
    surf_tri: np.ndarray     # int32 [F, 3] vertex ids
    side: float = 10.0


def make_c5(n=20, side=10.0, T=300) -> C5:
    mesh = S.kuhn_cube(n, side)
    fib = S.fibres_cube(mesh, side)
    zc = mesh.xyz.astype(np.float64)[mesh.tets][:, :, 2].mean(axis=1)
    layer = zc < 1.0
    el = S.fibonacci_sphere(10, 30.0, (side / 2,) * 3)
    L = S.lead_field(mesh, el, S.twelve_lead_matrix())
    loc = np.array([[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]])
    f = mesh.tets[:, loc].reshape(-1, 3)
    fs = np.sort(f, axis=1)
    _, inv, cnt = np.unique(fs, axis=0, return_inverse=True, return_counts=True)
    surf = np.nonzero(cnt[inv.ravel()] == 1)[0]
    p = S.Problem("c5", mesh, fib, np.full(mesh.n_t, 0.6, np.float32), np.full(mesh.n_t, 0.3, np.float32),
                  S.Onsets(S.ONSET_ELEMENT, np.zeros(N_SITES, np.int32), np.zeros(N_SITES, np.float32),
                           np.full((N_SITES, 4), 0.25, np.float32)), L, S.Template(-80.0, 20.0, 1.0, 0.0, 1.0, T))
    return C5(p, layer, (surf // 4).astype(np.int32), (surf % 4).astype(np.int32), f[surf].astype(np.int32), side)


@dataclasses.dataclass
class Params:
    cf: float
    ct: float
    ce: float
    tet: np.ndarray   # int32 [K]
    bary: np.ndarray  # float32 [K, 4]
    t: np.ndarray     # float32 [K]


def sample_params(c5: C5, rng: np.random.Generator) -> Params:
    """One draw of the prior: c_f ~ U[0.4,0.8], c_t ~ U[0.2,0.4],
    c_endo ~ U[1,3], 10 surface sites, t ~ U[0,20]."""
    fi = rng.choice(len(c5.surf_tet), size=N_SITES, replace=False)
    b3 = 0.05 + 0.85 * rng.dirichlet(np.ones(3), size=N_SITES)
    return Params(float(rng.uniform(*CF_RANGE)), float(rng.uniform(*CT_RANGE)), float(rng.uniform(*CE_RANGE)),
                  c5.surf_tet[fi], _surface_bary(c5, fi, b3), rng.uniform(*T_RANGE, size=N_SITES).astype(np.float32))


def _surface_bary(c5: C5, fi, b3):
    loc = np.array([[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]])
    b = np.zeros((len(fi), 4))
    for k, f in enumerate(fi):
        b[k, loc[c5.surf_opp[f]]] = b3[k]
    return b.astype(np.float32)


def site_xyz(c5: C5, prm: Params) -> np.ndarray:
    V = c5.problem.mesh.xyz.astype(np.float64)[c5.problem.mesh.tets[prm.tet]]
    return np.einsum("kq,kqr->kr", prm.bary.astype(np.float64), V)


# Loss weights of the target blocks (the MSE sees weight w as a sqrt(w) scale
# of target and output): the ECG constrains the earliest activations and the
# velocities best; late sites are often overshadowed (inactive).
SITE_SCALE = np.sqrt(1.0 / (1.0 + np.arange(N_SITES) / 3.0))
VEL_SCALE = 2.0


def encode(c5: C5, prm: Params) -> np.ndarray:
    """Network target: sites sorted by onset time as (x, y, z)/side and
    t / 20 (site k scaled by SITE_SCALE[k]), then the three velocities mapped
    to [0, 1] by their priors (scaled by VEL_SCALE)."""
    x = site_xyz(c5, prm)
    o = np.argsort(prm.t, kind="stable")
    sites = np.concatenate([x[o] / c5.side, (prm.t[o] / T_RANGE[1])[:, None]], axis=1) * SITE_SCALE[:, None]
    vel = np.array([(prm.cf - CF_RANGE[0]) / (CF_RANGE[1] - CF_RANGE[0]),
                    (prm.ct - CT_RANGE[0]) / (CT_RANGE[1] - CT_RANGE[0]),
                    (prm.ce - CE_RANGE[0]) / (CE_RANGE[1] - CE_RANGE[0])]) * VEL_SCALE
    return np.concatenate([sites.ravel(), vel]).astype(np.float32)


def decode(c5: C5, y: np.ndarray) -> Params:
    """Network output -> parameters: each site is moved to the closest point
    of the mesh surface (nearest boundary triangle, clamped barycentric
    coordinates); velocities clipped to their prior ranges."""
    y = np.asarray(y, np.float64)
    sites = y[:4 * N_SITES].reshape(N_SITES, 4) / SITE_SCALE[:, None]
    y = np.concatenate([y[:4 * N_SITES], y[4 * N_SITES:] / VEL_SCALE])
    xyz = np.clip(sites[:, :3] * c5.side, 0.0, c5.side)
    t = np.clip(sites[:, 3] * T_RANGE[1], -5.0, 40.0).astype(np.float32)
    X = c5.problem.mesh.xyz.astype(np.float64)
    tri = X[c5.surf_tri]  # [F, 3, 3]
    cen = tri.mean(axis=1)
    fi = np.argmin(((xyz[:, None, :] - cen[None]) ** 2).sum(-1), axis=1)
    b3 = np.zeros((N_SITES, 3))
    for k in range(N_SITES):
        b3[k] = _closest_bary(tri[fi[k]], xyz[k])
    b3 = 0.02 + 0.94 * b3
    cf = float(np.clip(CF_RANGE[0] + y[40] * (CF_RANGE[1] - CF_RANGE[0]), 0.3, 1.0))
    ct = float(np.clip(CT_RANGE[0] + y[41] * (CT_RANGE[1] - CT_RANGE[0]), 0.15, 0.6))
    ce = float(np.clip(CE_RANGE[0] + y[42] * (CE_RANGE[1] - CE_RANGE[0]), 0.5, 4.0))
    return Params(cf, ct, ce, c5.surf_tet[fi], _surface_bary(c5, fi, b3), t)


def _closest_bary(tri, p):
    """Barycentric coordinates of a point of triangle tri near p: those of
    p's projection onto the triangle's plane, negative ones set to zero and
    the rest renormalised.  This is the closest point of the triangle when
    the projection falls inside it; outside it is a point of the triangle's
    boundary, not necessarily the nearest one."""
    a, b, c = tri
    v0, v1, v2 = b - a, c - a, p - a
    G = np.array([[v0 @ v0, v0 @ v1], [v0 @ v1, v1 @ v1]])
    rhs = np.array([v2 @ v0, v2 @ v1])
    try:
        s, u = np.linalg.solve(G, rhs)
    except np.linalg.LinAlgError:
        s, u = 1 / 3, 1 / 3
    w = np.array([1 - s - u, s, u])
    w = np.clip(w, 0, None)
    return w / w.sum() if w.sum() > 0 else np.full(3, 1 / 3)


def default_params(c5: C5, rng: np.random.Generator) -> Params:
    """Plain Geodesic-BP start: prior-mean velocities, 10 random surface sites
    at t = 10 ms."""
    fi = rng.choice(len(c5.surf_tet), size=N_SITES, replace=False)
    b3 = np.full((N_SITES, 3), 1 / 3)
    return Params(0.6, 0.3, 2.0, c5.surf_tet[fi], _surface_bary(c5, fi, b3), np.full(N_SITES, 10.0, np.float32))


class C5Device:
    """The c5 problem uploaded to a context, with helpers to run the forward
    model for one parameter set."""

    def __init__(self, ctx: gbp.Context, c5: C5):
        self.ctx, self.c5 = ctx, c5
        self.dp = gbp.setup_problem(ctx, c5.problem)
        dev = ctx.torch_device
        self.layer = torch.from_numpy(c5.layer).to(dev)
        self.n_t = c5.problem.mesh.n_t
        self.phi = torch.empty(c5.problem.mesh.n_v, device=dev)
        self.ecg = torch.empty(c5.problem.L.shape[0], c5.problem.tmpl.T, device=dev)

    def velocities(self, cf, ct, ce):
        """Per-tet velocities (torch, differentiable in the three globals)."""
        one = torch.ones(self.n_t, device=self.ctx.torch_device)
        cft = torch.where(self.layer, ce * one, cf * one)
        ctt = torch.where(self.layer, ce * one, ct * one)
        return cft.contiguous(), ctt.contiguous()

    def simulate(self, prm: Params, precision=gbp.PREC_FP32):
        dev = self.ctx.torch_device
        cf, ct = self.velocities(torch.tensor(prm.cf, device=dev), torch.tensor(prm.ct, device=dev),
                                 torch.tensor(prm.ce, device=dev))
        self.ctx.set_velocities(cf, ct)
        self.ctx.set_onsets(gbp.ONSET_ELEMENT, torch.from_numpy(prm.tet).to(dev), torch.from_numpy(prm.t).to(dev),
                            torch.from_numpy(prm.bary).to(dev))
        self.ctx.eikonal_solve(phi=self.phi)
        return self.ctx.ecg_forward(self.phi, self.c5.problem.tmpl, precision=precision, out=self.ecg)


def generate(dev_c5: C5Device, n: int, seed: int):
    """n (ECG, target) pairs from the forward model: ECG [n, T, 12]
    (channels-last), targets [n, 43], and the parameter sets."""
    rng = np.random.default_rng(seed)
    T = dev_c5.c5.problem.tmpl.T
    X = np.empty((n, T, 12), np.float32)
    Y = np.empty((n, 43), np.float32)
    P = []
    for i in range(n):
        prm = sample_params(dev_c5.c5, rng)
        V = dev_c5.simulate(prm)
        X[i] = V.t().cpu().numpy()
        Y[i] = encode(dev_c5.c5, prm)
        P.append(prm)
    return X, Y, P


def he_init(cfg: NetConfig, seed: int):
    """Seeded He-normal weights, zero biases, in the reference layout."""
    rng = np.random.default_rng(seed)
    ps = []
    cin = cfg.C_in
    flat = cfg.lens()[-1] * cfg.channels
    shapes = []
    for _ in range(cfg.n_conv):
        shapes += [(cfg.channels, cfg.ksize, cin), (cfg.channels,)]
        cin = cfg.channels
    shapes += [(cfg.hidden, flat), (cfg.hidden,), (cfg.n_out, cfg.hidden), (cfg.n_out,)]
    for shp in shapes:
        if len(shp) == 1:
            ps.append(np.zeros(shp, np.float32))
        else:
            fan_in = int(np.prod(shp[1:]))
            ps.append((rng.standard_normal(shp) * math.sqrt(2.0 / fan_in)).astype(np.float32))
    return ps


def train(ctx: gbp.Context, X: np.ndarray, Y: np.ndarray, epochs=30, batch=256, lr=1e-3, seed=0, x_scale=None,
          X_val=None, Y_val=None, log=None):
    """Adam on the MSE with the project's kernels only.  Returns
    (net, x_scale, history) with history rows (epoch, train loss, val loss, s)."""
    cfg = NetConfig(C_in=X.shape[2], L_in=X.shape[1], n_out=Y.shape[1])
    if x_scale is None:
        x_scale = float(1.0 / max(np.sqrt(np.mean(X.astype(np.float64) ** 2)), 1e-12))
    net = ConvMLP(ctx, cfg, he_init(cfg, seed), max_batch=batch)
    dev = ctx.torch_device
    Xd = torch.from_numpy(X).to(dev) * x_scale
    Yd = torch.from_numpy(Y).to(dev)
    rng = np.random.default_rng(seed + 1)
    n = X.shape[0]
    hist = []
    t0 = time.perf_counter()
    steps_per_epoch = max(1, n // batch)
    total = epochs * steps_per_epoch
    step = 0
    for ep in range(epochs):
        perm = torch.from_numpy(rng.permutation(n)).to(dev)
        acc = torch.zeros(1, device=dev)
        for s in range(steps_per_epoch):
            idx = perm[s * batch:(s + 1) * batch]
            net.forward(Xd[idx], batch)
            acc += net.mse(Yd[idx].contiguous(), batch)
            net.backward(net.dy[:batch], batch)
            # cosine decay of the learning rate
            lr_s = lr * 0.5 * (1.0 + math.cos(math.pi * step / total))
            net.adam_step(lr=lr_s)
            step += 1
        vl = evaluate_loss(net, X_val, Y_val, x_scale, batch) if X_val is not None else float("nan")
        hist.append((ep, float(acc.item()) / steps_per_epoch, vl, time.perf_counter() - t0))
        if log:
            log(hist[-1])
    torch.cuda.synchronize()
    return net, x_scale, hist


def predict(net: ConvMLP, X: np.ndarray, x_scale: float, batch: int = 256) -> np.ndarray:
    dev = net.ctx.torch_device
    out = np.empty((X.shape[0], net.cfg.n_out), np.float32)
    for s in range(0, X.shape[0], batch):
        xb = torch.from_numpy(X[s:s + batch]).to(dev) * x_scale
        out[s:s + len(xb)] = net.forward(xb.contiguous(), len(xb)).cpu().numpy()
    return out


def evaluate_loss(net: ConvMLP, X, Y, x_scale, batch=256):
    if X is None:
        return float("nan")
    P = predict(net, X, x_scale, batch)
    return float(np.mean((P.astype(np.float64) - Y) ** 2))


# ---------------------------------------------------------------------------
# Geodesic-BP refinement with three global velocities and the onsets
# ---------------------------------------------------------------------------

class C5Inverse:
    """Adam over (c_f, c_t, c_endo, onset times, onset positions inside their
    tets) with the loss and gradient of the C ABI (GeodesicEcgLoss)."""

    def __init__(self, dev_c5: C5Device, target_ecg: np.ndarray, init: Params, precision=gbp.PREC_FP32,
                 opts=None, locator=None):
        from .inverse import EvalOp
        self.d = dev_c5
        ctx = dev_c5.ctx
        dv = ctx.torch_device
        c5 = dev_c5.c5
        self.log_c = torch.tensor(np.log([init.cf, init.ct, init.ce]), dtype=torch.float32, device=dv,
                                  requires_grad=True)
        self.t = torch.tensor(init.t, dtype=torch.float32, device=dv, requires_grad=True)
        V = c5.problem.mesh.xyz.astype(np.float64)[c5.problem.mesh.tets[init.tet]]
        x0 = np.einsum("kq,kqr->kr", init.bary.astype(np.float64), V)
        M = np.concatenate([V.transpose(0, 2, 1), np.ones((N_SITES, 1, 4))], axis=1)
        self.Vt_inv = torch.tensor(np.linalg.inv(M), dtype=torch.float32, device=dv)
        self.Vt = torch.tensor(V, dtype=torch.float32, device=dv)
        self.x = torch.tensor(x0.astype(np.float32), device=dv, requires_grad=True)
        n_v = c5.problem.mesh.n_v
        self.op = EvalOp(ctx=ctx, kind=gbp.ONSET_ELEMENT,
                         on_idx=torch.from_numpy(np.asarray(init.tet, np.int32)).to(dv),
                         target=torch.from_numpy(np.ascontiguousarray(target_ecg, np.float32)).to(dv),
                         tmpl=c5.problem.tmpl, opts=opts if opts is not None else gbp.make_opts(),
                         precision=precision, phi=torch.empty(n_v, device=dv),
                         parent=torch.empty(n_v, dtype=torch.int32, device=dv),
                         alpha=torch.empty(n_v, 3, device=dv),
                         ecg=torch.empty(c5.problem.L.shape[0], c5.problem.tmpl.T, device=dv))
        self.locator = locator

    def bary(self):
        xh = torch.cat([self.x.detach(), torch.ones_like(self.x[:, :1])], dim=1)
        return torch.einsum("kij,kj->ki", self.Vt_inv, xh).contiguous()

    def loss(self):
        from .inverse import GeodesicEcgLoss
        c = torch.exp(self.log_c)
        cf, ct = self.d.velocities(c[0], c[1], c[2])
        return GeodesicEcgLoss.apply(cf, ct, self.t, self.x, self.bary(), self.op)

    @torch.no_grad()
    def project(self, floor=1e-3):
        """Onsets that left their tet move to the tet containing them (with a
        locator, relocate.py); otherwise they are clamped into their tet."""
        if self.locator is not None:
            from .relocate import relocate_onsets
            relocate_onsets(self.locator, self.x, self.op.on_idx, self.Vt_inv, self.Vt, floor=floor)
            return
        b = self.bary().clamp_min(floor)
        b = b / b.sum(dim=1, keepdim=True)
        self.x.copy_(torch.einsum("kq,kqr->kr", b, self.Vt))

    def fp32_loss(self):
        """The misfit of the current iterate with the FP32 ECG: the activation
        map of the last forward solve (op.phi) through the FP32 contraction
        and the misfit kernel; the parent graph and the pending gradient are
        untouched."""
        ctx, op = self.d.ctx, self.op
        ecg = ctx.ecg_forward(op.phi, op.tmpl, precision=gbp.PREC_FP32)
        loss, _ = ctx.ecg_loss_backward(op.phi, ecg, op.target, op.tmpl)
        return float(loss.item())

    def run(self, iters, lr=2e-2, stop_at=None, time_budget=None, check_fp32=False):
        """Adam; returns [(iteration, loss, seconds, fp32 loss or None)],
        stopping early once the loss is <= stop_at or after time_budget
        seconds.  With check_fp32 (an arm whose ECG is not FP32), an iterate
        whose loss is <= stop_at is re-evaluated with the FP32 ECG, and the
        run stops only once that FP32 misfit is <= stop_at as well; the time
        of an iteration includes its check."""
        opt = torch.optim.Adam([self.log_c, self.t, self.x], lr=lr)
        hist = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for it in range(iters):
            opt.zero_grad(set_to_none=True)
            loss = self.loss()
            loss.backward()
            lv = float(loss.item())
            l32 = None
            if check_fp32 and stop_at is not None and lv <= stop_at:
                l32 = self.fp32_loss()
            opt.step()
            self.project()
            hist.append((it, lv, time.perf_counter() - t0, l32))
            if stop_at is not None and (l32 if check_fp32 else lv) is not None and \
                    (l32 if check_fp32 else lv) <= stop_at:
                break
            if time_budget is not None and hist[-1][2] > time_budget:
                break
        return hist


# ---------------------------------------------------------------------------
# the experiment: learned init + BF16 ECG vs default-init plain Geodesic-BP
# ---------------------------------------------------------------------------

def run_experiment(n_train=20000, n_test=2000, epochs=60, n_eval=20, iters=300, lr_refine=2e-2, seed=0,
                   noise=0.05, lr_train=2e-3, relocate=True, log=print):
    """Generate the data with the forward model, train the network, then for
    n_eval held-out noisy ECGs run (a) plain Geodesic-BP from the default
    start with the FP32 ECG and (b) Geodesic-BP from the network's prediction
    with the BF16 tensor-core ECG until it reaches (a)'s best misfit, judged
    on the FP32 misfit of (b)'s iterate (re-evaluated with the FP32 ECG
    whenever its BF16 misfit is at or below the target), so both arms are
    held to the same error.  Returns a dict of timings, losses (BF16 and FP32
    at arrival) and activation errors."""
    ctx = gbp.Context(0)
    c5 = make_c5()
    d = C5Device(ctx, c5)
    t0 = time.perf_counter()
    X, Y, _ = generate(d, n_train, seed + 1)
    Xv, Yv, Pv = generate(d, n_test, seed + 2)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    log(f"generated {n_train}+{n_test} pairs in {t_gen:.1f} s")
    net, xs, hist = train(ctx, X, Y, epochs=epochs, lr=lr_train, X_val=Xv, Y_val=Yv,
                          log=lambda h: log(f"epoch {h[0]} train {h[1]:.4e} val {h[2]:.4e} {h[3]:.1f}s"))
    t_train = hist[-1][3]
    rng = np.random.default_rng(seed + 3)
    loc = None
    if relocate:
        from .relocate import SimplexLocator
        loc = SimplexLocator(c5.problem.mesh.xyz, c5.problem.mesh.tets)
    rows = []
    for i in range(n_eval):
        truth = Pv[i]
        clean = d.simulate(truth).cpu().numpy()
        phi_true = d.phi.cpu().numpy().copy()
        target = S.add_noise(clean, noise, seed + 100 + i)
        # (a) plain
        inv_p = C5Inverse(d, target, default_params(c5, rng), precision=gbp.PREC_FP32, locator=loc)
        hp = inv_p.run(iters, lr=lr_refine)
        best = min(range(len(hp)), key=lambda k: hp[k][1])
        m_plain, t_plain = hp[best][1], hp[best][2]
        phi_p = inv_p.op.phi.cpu().numpy().copy()
        # (b) learned init + BF16 ECG
        torch.cuda.synchronize()
        ti = time.perf_counter()
        xin = np.ascontiguousarray(target.T[None].astype(np.float32))
        init = decode(c5, predict(net, xin, xs)[0])
        t_inf = time.perf_counter() - ti
        inv_l = C5Inverse(d, target, init, precision=gbp.PREC_BF16, locator=loc)
        hl = inv_l.run(iters, lr=lr_refine, stop_at=m_plain, check_fp32=True)
        reached = [h for h in hl if h[3] is not None and h[3] <= m_plain]
        t_learned = (reached[0][2] if reached else float("inf")) + t_inf
        phi_l = inv_l.op.phi.cpu().numpy().copy()
        rmse = lambda a: float(np.sqrt(np.mean((a - phi_true) ** 2)))  # noqa: E731
        rows.append(dict(case=i, plain_loss0=hp[0][1], learned_loss0=hl[0][1], plain_best=m_plain,
                         plain_iters=best + 1, plain_time=t_plain, learned_iters=len(hl), learned_time=t_learned,
                         learned_final=hl[-1][1],
                         learned_bf16_at_arrival=reached[0][1] if reached else None,
                         learned_fp32_at_arrival=reached[0][3] if reached else None,
                         plain_rmse=rmse(phi_p), learned_rmse=rmse(phi_l)))
        log(rows[-1])
    med = lambda k: float(np.median([r[k] for r in rows]))  # noqa: E731
    return dict(n_train=n_train, n_test=n_test, epochs=epochs, gen_s=t_gen, train_s=t_train, relocate=relocate,
                val_mse=float(hist[-1][2]), cases=rows,
                median=dict(plain_time=med("plain_time"), learned_time=med("learned_time"),
                            plain_loss0=med("plain_loss0"), learned_loss0=med("learned_loss0"),
                            plain_best=med("plain_best"),
                            plain_rmse=med("plain_rmse"), learned_rmse=med("learned_rmse")),
                reached=int(sum(bool(np.isfinite(r["learned_time"])) for r in rows)))


# The network's GEMM shapes at the training minibatch of 256 (M, N, K): the
# first convolution (256 x 150 output positions, 64 channels, 12 leads x 5
# taps padded to 64), a later convolution (64 channels x 5 taps), the hidden
# layer; and two larger products (the TMA-fed kernel) that show the kernels
# themselves.
GEMM_SHAPES = ((38400, 64, 64), (19200, 64, 320), (256, 256, 1216), (2048, 2048, 2048), (8192, 8192, 4096))


def gemm_rates(ctx: gbp.Context, shapes=GEMM_SHAPES, reps: int = 20) -> list:
    """Achieved TFLOP/s of the tcgen05 BF16 GEMM (gbp_nn_gemm_bf16) per shape:
    CUDA events on the context stream around `reps` calls after 3 warm-up
    calls; 2 M N K flops per call."""
    lib, dev, st = ctx.lib, ctx.torch_device, ctx.stream
    out = []
    for M, N, K in shapes:
        Kp = _r64(K)
        g = torch.Generator(device=dev).manual_seed(0)
        A = torch.randn(M, Kp, device=dev, generator=g).to(torch.bfloat16)
        Bm = torch.randn(N, Kp, device=dev, generator=g).to(torch.bfloat16)
        Cm = torch.empty(M, N, device=dev, dtype=torch.float32)

        def call():
            gbp._check(lib.gbp_nn_gemm_bf16(ctx.h, M, N, Kp, _p(A), Kp, _p(Bm), Kp, _p(Cm), N, 1.0, 0.0),
                       "gbp_nn_gemm_bf16")
        for _ in range(3):
            call()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        e0.record(st)
        for _ in range(reps):
            call()
        e1.record(st)
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / reps
        out.append({"M": M, "N": N, "K": K, "us": ms * 1e3, "tflops": 2.0 * M * N * Kp / (ms * 1e-3) / 1e12})
    return out


def summary(res) -> dict:
    """One JSON record of the experiment: time to the plain FP32 arm's best
    misfit for learned init + BF16 ECG (misses count as never), the misfits
    at arrival, and the configuration."""
    rows = res["cases"]
    arr = [r for r in rows if np.isfinite(r["learned_time"])]
    return {
        "metric": "time to the plain FP32 Geodesic-BP best misfit: learned init + BF16 ECG vs default init FP32",
        "cases": len(rows), "reached": len(arr),
        "faster": int(sum(r["learned_time"] < r["plain_time"] for r in rows)),
        "median_s": {"plain_fp32": res["median"]["plain_time"], "learned_bf16": res["median"]["learned_time"]},
        "median_misfit": {"plain_fp32_best": res["median"]["plain_best"],
                          "learned_fp32_at_arrival": float(np.median([r["learned_fp32_at_arrival"] for r in arr]))
                          if arr else None,
                          "learned_bf16_at_arrival": float(np.median([r["learned_bf16_at_arrival"] for r in arr]))
                          if arr else None},
        "median_loss0": {"plain": res["median"]["plain_loss0"], "learned": res["median"]["learned_loss0"]},
        "median_activation_rmse_ms": {"plain": res["median"]["plain_rmse"], "learned": res["median"]["learned_rmse"]},
        "config": {"n_train": res["n_train"], "n_test": res["n_test"], "epochs": res["epochs"],
                   "relocate": res["relocate"], "val_mse": res["val_mse"], "gen_s": res["gen_s"],
                   "train_s": res["train_s"]},
    }


if __name__ == "__main__":
    import argparse
    import json

    ap = argparse.ArgumentParser(description="learned initialiser + BF16 ECG vs plain Geodesic-BP (c5)")
    ap.add_argument("--train", type=int, default=20000)
    ap.add_argument("--test", type=int, default=2000)
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--eval", type=int, default=20)
    ap.add_argument("--iters", type=int, default=300)
    ap.add_argument("--out", default=None)
    ap.add_argument("--no-relocate", action="store_true", help="keep every onset inside its initial tet")
    ap.add_argument("--json", action="store_true",
                    help="print one JSON summary line (cases reached, median seconds, misfits at arrival)")
    ap.add_argument("--gemm", action="store_true",
                    help="only time the BF16 GEMM at the network's shapes and one large square shape (JSON)")
    a = ap.parse_args()
    if a.gemm:
        import os
        peak = None
        mp = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "MEASURED_PEAKS.json")
        if os.path.exists(mp):
            with open(mp) as f:
                peak = json.load(f).get("bf16_tflops")
        rows = gemm_rates(gbp.Context(0))
        for r in rows:
            r["frac_of_measured_bf16"] = r["tflops"] / peak if peak else None
        print(json.dumps({"kernel": "k_gemm_tn", "peak_bf16_tflops_measured": peak, "shapes": rows}))
        raise SystemExit(0)
    res = run_experiment(a.train, a.test, a.epochs, a.eval, a.iters, relocate=not a.no_relocate,
                         log=(lambda *_: None) if a.json else print)
    s = json.dumps(summary(res) if a.json else res)
    print(s)
    if a.out:
        with open(a.out, "w") as f:
            f.write(json.dumps(res))
