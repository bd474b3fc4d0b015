"""Backpropagation through the unrolled iterations of Algorithm 2, in plain
PyTorch (CPU, float64): the paper's own way of differentiating the eikonal
solve (Sec. II-C: the solver is written with differentiable operations and
the gradient is taken by automatic differentiation through every iteration).

TEST INFRASTRUCTURE ONLY (like the rest of ``oracle/``): it cross-checks the
frozen-parent-graph adjoint of ``oracle.adjoint`` and of the CUDA path on
small meshes.  It shares nothing with either: the local problem of
Eq. (upwind_eq_lsqr) is written out again below as closed-form candidates
(vertices, edges, face interior) whose minimum is taken with ``torch``
operations, and the global update is the Jacobi form of Algorithm 2,
phi_i <- min(phi_i, min_j phi_{j\\i}), repeated until nothing changes and then
a fixed number of times more (so that short cycles of the parent graph,
where the unrolled gradient is a truncated Neumann series, converge).

Parameters are per-tet velocities c_f, c_t (Sec. II-A: D = M^{-1},
M = c_t^2 I + (c_f^2 - c_t^2) f f^T), onset times t and, for element onsets
(Eq. upwind_xi), onset positions x.  The loss is Eq. (inverse_ecg) with the
template of Sec. II-D, U = K0 + (K1 - K0) / 2 (1 + tanh(2 xi / tau)).
"""
from __future__ import annotations

import numpy as np
import torch

BIG = 1e6  # stands for +inf in the iterate (kept finite so that gradients stay finite)


def _metric_apply(e, f, cf, ct):
    """R e with R = D^{1/2} = (1/c_t)(I - f f^T) + (1/c_f) f f^T (f unit):
    ||e||_D = |R e|."""
    fe = (e * f).sum(-1, keepdim=True)
    return e / ct + (1.0 / cf - 1.0 / ct) * fe * f


def _norm(v):
    return torch.sqrt((v * v).sum(-1))


def _safe(cond, x, fill=1.0):
    return torch.where(cond, x, torch.full_like(x, fill))


def local_values(p, ph, fin):
    """Minimum of Eq. (upwind_eq_lsqr) over the simplex for a batch of faces.

    p [F, 3, 3]: rows p_n = R (v_{j_n} - v_i); ph [F, 3] vertex values;
    fin [F, 3] which values are finite.  The objective
    sum_n a_n ph_n + |sum_n a_n p_n| is convex, so its minimum is at one of
    the candidates below (each kept only where it is feasible)."""
    cands = []
    # vertices: a = e_n
    for n in range(3):
        v = ph[:, n] + _norm(p[:, n])
        cands.append(torch.where(fin[:, n], v, torch.full_like(v, 2 * BIG)))
    # edges (n, m): a = lam e_n + (1 - lam) e_m, stationary in lam
    for n, m in ((0, 1), (0, 2), (1, 2)):
        ok = fin[:, n] & fin[:, m]
        u = p[:, n] - p[:, m]
        A = (u * u).sum(-1)
        dl = ph[:, n] - ph[:, m]
        g = dl * dl / A
        ok = ok & (g < 1.0)
        cr = torch.cross(u, p[:, m], dim=-1)
        S = (cr * cr).sum(-1) / A
        h = torch.sqrt(_safe(ok, S / _safe(ok, 1.0 - g)))
        lam = (-dl * h - (u * p[:, m]).sum(-1)) / A
        ok = ok & (lam > 0.0) & (lam < 1.0)
        lam = _safe(ok, lam, 0.5)
        x = lam[:, None] * p[:, n] + (1.0 - lam[:, None]) * p[:, m]
        v = lam * ph[:, n] + (1.0 - lam) * ph[:, m] + _norm(x)
        cands.append(torch.where(ok, v, torch.full_like(v, 2 * BIG)))
    # face interior: a = (b0, b1, 1 - b0 - b1), stationary in (b0, b1)
    ok = fin.all(-1)
    d1 = p[:, 0] - p[:, 2]
    d2 = p[:, 1] - p[:, 2]
    Q00, Q01, Q11 = (d1 * d1).sum(-1), (d1 * d2).sum(-1), (d2 * d2).sum(-1)
    nrm = torch.cross(d1, d2, dim=-1)
    det = (nrm * nrm).sum(-1)
    ok = ok & (det > 1e-14 * Q00 * Q11)
    det = _safe(ok, det)
    D0, D1 = ph[:, 0] - ph[:, 2], ph[:, 1] - ph[:, 2]
    k = (Q11 * D0 * D0 - 2.0 * Q01 * D0 * D1 + Q00 * D1 * D1) / det
    ok = ok & (k < 1.0)
    S = (nrm * p[:, 2]).sum(-1) ** 2 / det
    h = torch.sqrt(_safe(ok, S / _safe(ok, 1.0 - k)))
    y0 = h * D0 + (d1 * p[:, 2]).sum(-1)
    y1 = h * D1 + (d2 * p[:, 2]).sum(-1)
    b0 = -(Q11 * y0 - Q01 * y1) / det
    b1 = -(Q00 * y1 - Q01 * y0) / det
    ok = ok & (b0 > 0.0) & (b1 > 0.0) & (b0 + b1 < 1.0)
    b0, b1 = _safe(ok, b0, 1 / 3), _safe(ok, b1, 1 / 3)
    b2 = 1.0 - b0 - b1
    x = b0[:, None] * p[:, 0] + b1[:, None] * p[:, 1] + b2[:, None] * p[:, 2]
    v = b0 * ph[:, 0] + b1 * ph[:, 1] + b2 * ph[:, 2] + _norm(x)
    cands.append(torch.where(ok, v, torch.full_like(v, 2 * BIG)))
    return torch.stack(cands, -1).min(-1).values


class Unrolled:
    """Faces of every (tet, vertex) pair of a mesh, for the Jacobi form of
    Algorithm 2."""

    def __init__(self, mesh, fib):
        xyz = torch.tensor(np.asarray(mesh.xyz, np.float64))
        tets = torch.tensor(np.asarray(mesh.tets, np.int64))
        f = torch.tensor(np.asarray(fib, np.float64))
        f = f / _norm(f)[:, None]
        self.n_v = xyz.shape[0]
        self.xyz, self.tets, self.f = xyz, tets, f
        owner, others, tet = [], [], []
        for s in range(4):
            owner.append(tets[:, s])
            others.append(tets[:, [q for q in range(4) if q != s]])
            tet.append(torch.arange(tets.shape[0]))
        self.owner = torch.cat(owner)          # [F] target vertex i
        self.others = torch.cat(others)        # [F, 3] face vertices j_n
        self.tet = torch.cat(tet)              # [F]
        self.e = xyz[self.others] - xyz[self.owner][:, None, :]  # [F, 3, 3] v_{j_n} - v_i

    def initial(self, kind, idx, t, x, cf, ct):
        """Onset values (Algorithm 2's initialisation): nodal onsets
        phi_v = t_k; element onsets (Eq. upwind_xi) phi_v = t_k + ||v - x_k||_{D_E}
        for the four vertices v of tet E.  Minimum over onsets."""
        phi = torch.full((self.n_v,), BIG, dtype=torch.float64)
        idx = torch.as_tensor(np.asarray(idx, np.int64))
        if kind == 0:
            phi = phi.scatter_reduce(0, idx, t, reduce="amin", include_self=True)
        else:
            verts = self.tets[idx]                                     # [K, 4]
            w = self.xyz[verts] - x[:, None, :]                        # [K, 4, 3]
            ff = self.f[idx][:, None, :].expand_as(w)
            cfe = cf[idx][:, None, None]
            cte = ct[idx][:, None, None]
            d = _norm(_metric_apply(w, ff, cfe, cte))                  # [K, 4]
            vals = t[:, None] + d
            phi = phi.scatter_reduce(0, verts.reshape(-1), vals.reshape(-1), reduce="amin", include_self=True)
        return phi

    def solve(self, phi0, cf, ct, max_iters=2000, extra=60):
        p = _metric_apply(self.e, self.f[self.tet][:, None, :].expand_as(self.e), cf[self.tet][:, None, None],
                          ct[self.tet][:, None, None])
        phi = phi0
        it, settled = 0, 0
        while it < max_iters:
            ph = phi[self.others]
            fin = ph < BIG / 2
            vals = local_values(p, torch.where(fin, ph, torch.zeros_like(ph)), fin)
            new = phi.scatter_reduce(0, self.owner, vals, reduce="amin", include_self=True)
            changed = bool((new.detach() < phi.detach()).any())
            phi = new
            it += 1
            if not changed:
                settled += 1
                if settled > extra:
                    break
            else:
                settled = 0
        return phi, it


def ecg_loss(L, phi, tmpl, target):
    """Eq. (inverse_ecg): 1/(N T) sum (sum_n L_ln U(t_s - phi_n) - target)^2."""
    L = torch.tensor(np.asarray(L, np.float64))
    ts = tmpl.t0 + tmpl.dt * torch.arange(tmpl.T, dtype=torch.float64)
    xi = ts[None, :] - phi[:, None]
    U = tmpl.K0 + 0.5 * (tmpl.K1 - tmpl.K0) * (1.0 + torch.tanh(2.0 * xi / tmpl.tau))
    V = L @ U
    r = V - torch.tensor(np.asarray(target, np.float64))
    return (r * r).mean()


def gradients(mesh, fib, cf, ct, onsets, L, tmpl, target, **kw):
    """Loss and its gradients with respect to (c_f, c_t, t, x) by automatic
    differentiation through the unrolled iterations."""
    U = Unrolled(mesh, fib)
    cf_t = torch.tensor(np.asarray(cf, np.float64), requires_grad=True)
    ct_t = torch.tensor(np.asarray(ct, np.float64), requires_grad=True)
    t_t = torch.tensor(np.asarray(onsets.t, np.float64), requires_grad=True)
    if onsets.kind == 1:
        V = U.xyz[U.tets[torch.as_tensor(np.asarray(onsets.idx, np.int64))]]
        x0 = torch.einsum("kq,kqr->kr", torch.tensor(np.asarray(onsets.bary, np.float64)), V)
        x_t = x0.clone().requires_grad_(True)
    else:
        x_t = torch.zeros(len(onsets.idx), 3, dtype=torch.float64, requires_grad=True)
    phi0 = U.initial(onsets.kind, onsets.idx, t_t, x_t, cf_t, ct_t)
    phi, iters = U.solve(phi0, cf_t, ct_t, **kw)
    loss = ecg_loss(L, phi, tmpl, target)
    g = torch.autograd.grad(loss, [cf_t, ct_t, t_t, x_t], allow_unused=True)
    out = [gi.numpy() if gi is not None else np.zeros(s.shape) for gi, s in zip(g, [cf_t, ct_t, t_t, x_t])]
    return dict(loss=float(loss.detach()), phi=phi.detach().numpy(), iters=iters, d_cf=out[0], d_ct=out[1], d_t=out[2],
                d_x=out[3])
