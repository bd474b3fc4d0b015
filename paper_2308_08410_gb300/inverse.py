"""Geodesic-BP as a differentiable PyTorch operation and the Adam inverse loop.

``GeodesicEcgLoss`` wraps one forward-plus-gradient evaluation of the C ABI
(include/gbp.h): the forward pass runs the eikonal solve, the lead-field ECG
and the misfit of Eq. (inverse_ecg); the backward pass runs the frozen-graph
adjoint of Sec. II-C on the parent graph the forward solve recorded (phi is
recomputed on every call; no per-iteration solver state is stored, unlike
backpropagation through the unrolled iterations of Algorithm 2).

``InverseProblem`` holds the parameter maps (per-vertex log velocities ->
per-tet velocities, onset positions inside their tets) and runs Adam
(Sec. II-D: "gradient-based optimization utilizing ADAM").  The maps and the
optimiser are ordinary torch operations; every step of the hot path runs in
the library's kernels.
"""
from __future__ import annotations

import dataclasses
import time

import numpy as np
import torch

from . import gbp


@dataclasses.dataclass
class EvalOp:
    """Device state shared by the autograd function across calls."""
    ctx: gbp.Context
    kind: int
    on_idx: torch.Tensor
    target: torch.Tensor
    tmpl: object
    opts: object
    precision: int
    phi: torch.Tensor
    parent: torch.Tensor
    alpha: torch.Tensor
    ecg: torch.Tensor


class InverseProblem:
    """Per-vertex log-velocity fields and onset (time, position) parameters
    for a seeded problem uploaded to a context."""

    def __init__(self, ctx: gbp.Context, problem, target: np.ndarray, opts=None, precision=gbp.PREC_FP32,
                 init_log_cf=None, init_log_ct=None, init_t=None, optimise_positions=True, relocate=True):
        self.ctx = ctx
        self.p = problem
        dev = ctx.torch_device
        self.dp = gbp.setup_problem(ctx, problem)
        self.tets = torch.from_numpy(problem.mesh.tets.astype(np.int64)).to(dev)
        n_v = problem.mesh.n_v
        lcf = np.full(n_v, np.log(0.6)) if init_log_cf is None else init_log_cf
        lct = np.full(n_v, np.log(0.3)) if init_log_ct is None else init_log_ct
        t0 = problem.onsets.t if init_t is None else init_t
        self.log_cf = torch.tensor(np.asarray(lcf, np.float32), device=dev, requires_grad=True)
        self.log_ct = torch.tensor(np.asarray(lct, np.float32), device=dev, requires_grad=True)
        self.t = torch.tensor(np.asarray(t0, np.float32), device=dev, requires_grad=True)
        ons = problem.onsets
        self.kind = ons.kind
        self.optimise_positions = optimise_positions and ons.kind == gbp.ONSET_ELEMENT
        if ons.kind == gbp.ONSET_ELEMENT:
            V = problem.mesh.xyz.astype(np.float64)[problem.mesh.tets[ons.idx]]  # [K, 4, 3]
            x0 = np.einsum("kq,kqr->kr", ons.bary.astype(np.float64), V)
            M = np.concatenate([V.transpose(0, 2, 1), np.ones((ons.K, 1, 4))], axis=1)  # [K, 4, 4]
            self.Vt_inv = torch.tensor(np.linalg.inv(M), dtype=torch.float32, device=dev)
            self.x = torch.tensor(x0.astype(np.float32), device=dev, requires_grad=self.optimise_positions)
        else:
            self.Vt_inv = None
            self.x = torch.zeros(ons.K, 3, device=dev)
        self.locator = None
        if self.optimise_positions and relocate:
            from .relocate import TetLocator
            self.locator = TetLocator(problem.mesh.xyz, problem.mesh.tets)
        self.op = EvalOp(ctx=ctx, kind=ons.kind, on_idx=self.dp.on_idx,
                         target=torch.from_numpy(np.ascontiguousarray(target, np.float32)).to(dev),
                         tmpl=problem.tmpl, opts=opts if opts is not None else gbp.make_opts(),
                         precision=precision, phi=torch.empty(n_v, device=dev),
                         parent=torch.empty(n_v, dtype=torch.int32, device=dev),
                         alpha=torch.empty(n_v, 3, device=dev),
                         ecg=torch.empty(problem.L.shape[0], problem.tmpl.T, device=dev))

    def params(self):
        ps = [self.log_cf, self.log_ct, self.t]
        if self.optimise_positions:
            ps.append(self.x)
        return ps

    def tet_velocities(self):
        """Per-tet velocity = exp(mean of the four vertex log values)."""
        return VertexLogToTet.apply(self.log_cf, self.tets), VertexLogToTet.apply(self.log_ct, self.tets)

    def bary(self):
        if self.Vt_inv is None:
            return None
        xh = torch.cat([self.x.detach(), torch.ones_like(self.x[:, :1])], dim=1)
        return torch.einsum("kij,kj->ki", self.Vt_inv, xh).contiguous()

    def loss(self):
        cf, ct = self.tet_velocities()
        b = self.bary()
        return GeodesicEcgLoss.apply(cf, ct, self.t, self.x, b, self.op)

    @torch.no_grad()
    def project_positions(self, floor=1e-3):
        """Keep every onset inside the mesh: with relocation, an onset that left
        its tet moves to the tet that now contains it (relocate.py); without,
        its barycentric coordinates are clamped to >= floor in its own tet."""
        if self.Vt_inv is None:
            return
        if self.locator is not None:
            from .relocate import relocate_onsets
            relocate_onsets(self.locator, self.x, self.op.on_idx, self.Vt_inv, floor=floor)
            return
        b = self.bary().clamp_min(floor)
        b = b / b.sum(dim=1, keepdim=True)
        V = torch.from_numpy(self.p.mesh.xyz.astype(np.float32)).to(self.x.device)[self.tets[self.op.on_idx.long()]]
        self.x.copy_(torch.einsum("kq,kqr->kr", b, V))

    def run_adam(self, iters=500, lr=1e-2, log_every=0, callback=None):
        opt = torch.optim.Adam(self.params(), lr=lr)
        hist = []
        t_start = time.perf_counter()
        for it in range(iters):
            opt.zero_grad(set_to_none=True)
            loss = self.loss()
            loss.backward()
            opt.step()
            self.project_positions()
            if log_every and (it % log_every == 0 or it == iters - 1):
                hist.append((it, float(loss.item()), time.perf_counter() - t_start))
            if callback is not None:
                callback(it, loss)
        torch.cuda.synchronize()
        return hist, time.perf_counter() - t_start


class VertexLogToTet(torch.autograd.Function):
    """c_j = exp(mean of the four vertex values of log c over tet j).  The
    backward scatters g_j c_j / 4 to the tet's vertices with an atomic
    index_add (autograd's own backward of the gather sorts the indices,
    which dominates an inverse-loop step at 2M tets)."""

    @staticmethod
    def forward(fctx, logc, tets):
        c = torch.exp(logc[tets].mean(dim=1))
        fctx.save_for_backward(c, tets)
        fctx.n = logc.shape[0]
        return c

    @staticmethod
    def backward(fctx, g):
        c, tets = fctx.saved_tensors
        w = (0.25 * g * c).unsqueeze(1).expand(-1, 4).reshape(-1)
        out = torch.zeros(fctx.n, dtype=g.dtype, device=g.device)
        out.index_add_(0, tets.reshape(-1), w)
        return out, None


class GeodesicEcgLoss(torch.autograd.Function):
    """loss = 1/(N T) sum (ECG(phi(cf, ct, t, x)) - target)^2 (Eq. inverse_ecg).

    Inputs: cf, ct per tet [n_t]; t onset times [K]; x onset positions [K, 3]
    (element onsets; zeros for nodal ones), bary the barycentric coordinates
    of x in the onset tets (what the library consumes; derived from x outside
    the graph).  Forward: eikonal solve + ECG + misfit; backward: the
    frozen-graph adjoint of the parent graph recorded by this forward solve,
    which returns dL/dx directly."""

    @staticmethod
    def forward(fctx, cf, ct, t, x, bary, op):
        g = op.ctx
        g.set_velocities(cf.detach().contiguous(), ct.detach().contiguous())
        g.set_onsets(op.kind, op.on_idx, t.detach().contiguous(), bary)
        g.eikonal_solve(op.opts, phi=op.phi, parent=op.parent, alpha=op.alpha)
        ecg = g.ecg_forward(op.phi, op.tmpl, precision=op.precision, out=op.ecg)
        loss, dphi = g.ecg_loss_backward(op.phi, ecg, op.target, op.tmpl)
        fctx.op = op
        fctx.dphi = dphi
        return loss[0].clone()

    @staticmethod
    def backward(fctx, gl):
        d_cf, d_ct, d_t, d_x = fctx.op.ctx.geodesic_backward(fctx.dphi)
        return gl * d_cf, gl * d_ct, gl * d_t, gl * d_x, None, None


def run_c3(iters: int = 500, lr: float = 1e-2, n: int = 72, device: int = 0, log_every: int = 25,
           precision: int = gbp.PREC_FP32, log=print):
    """The inverse loop on the 72^3 cube (2.15M tets): Adam on the per-vertex
    log-velocity fields and the 10 onset times / positions, from the
    prior-mean start (c_f = 0.6, c_t = 0.3 mm/ms everywhere, onset times
    10 ms, onsets at the centroids of the true onset tets: relocation across
    elements is not modelled).  Target: the ground-truth ECG plus 5 % noise.
    Returns the loss history and the activation-time error against the
    ground truth before and after."""
    from . import synth as S
    p = S.make_c3(n=n)
    ctx = gbp.Context(device)
    dp = gbp.setup_problem(ctx, p)
    phi_true, _, _ = ctx.eikonal_solve()
    V = ctx.ecg_forward(phi_true, p.tmpl).cpu().numpy()
    phi_true = phi_true.clone()
    target = S.add_noise(V, p.extra["noise"], 4242)
    ons = p.onsets
    cent = np.full((ons.K, 4), 0.25, np.float32)
    p0 = S.Problem(p.name, p.mesh, p.fib, p.cf, p.ct, S.Onsets(ons.kind, ons.idx, ons.t, cent), p.L, p.tmpl,
                   p.extra)
    inv = InverseProblem(ctx, p0, target, precision=precision, init_t=np.full(ons.K, 10.0, np.float32))
    del dp

    def act_err():
        with torch.no_grad():
            cf, ct = inv.tet_velocities()
            ctx.set_velocities(cf.contiguous(), ct.contiguous())
            ctx.set_onsets(inv.kind, inv.op.on_idx, inv.t.detach().contiguous(), inv.bary())
            phi, _, _ = ctx.eikonal_solve()
            d = (phi - phi_true).double()
            return float(torch.sqrt((d * d).mean()).item()), float(d.abs().max().item())

    rmse0, max0 = act_err()
    loss0 = float(inv.loss().item())
    hist, wall = inv.run_adam(iters=iters, lr=lr, log_every=log_every,
                              callback=None)
    rmse1, max1 = act_err()
    lcf_true = torch.from_numpy(p.extra["log_cf_nodal"]).to(inv.log_cf.device)
    lct_true = torch.from_numpy(p.extra["log_ct_nodal"]).to(inv.log_ct.device)
    res = dict(workload=f"{n}^3 cube, {p.mesh.n_t} tets, {ons.K} element onsets, {p.L.shape[0]} leads, "
                        f"T={p.tmpl.T}, 5% noise",
               iters=iters, lr=lr, wall_s=wall,
               # steady state: the first iteration also loads the torch kernels
               ms_per_iter=(1e3 * (hist[-1][2] - hist[0][2]) / max(hist[-1][0] - hist[0][0], 1)
                            if len(hist) > 1 else 1e3 * wall / max(iters, 1)),
               loss0=loss0, loss_final=hist[-1][1] if hist else loss0, noise_floor=float(
                   np.mean((target - V) ** 2)),
               act_rmse_ms=(rmse0, rmse1), act_max_ms=(max0, max1),
               log_cf_mae=float((inv.log_cf.detach() - lcf_true).abs().mean().item()),
               log_ct_mae=float((inv.log_ct.detach() - lct_true).abs().mean().item()),
               log_cf_mae0=float((np.log(0.6) - lcf_true).abs().mean().item()),
               log_ct_mae0=float((np.log(0.3) - lct_true).abs().mean().item()),
               t_err_ms=(float(np.abs(10.0 - ons.t).mean()),
                         float(np.abs(inv.t.detach().cpu().numpy() - ons.t).mean())),
               history=hist)
    for it, l, tt in hist:
        log(f"iter {it:4d}  loss {l:.6g}  {tt:.2f} s")
    ctx.close()
    return res


if __name__ == "__main__":
    import argparse
    import json

    ap = argparse.ArgumentParser(description="Adam inverse loop on the 72^3 cube")
    ap.add_argument("--iters", type=int, default=500)
    ap.add_argument("--lr", type=float, default=1e-2)
    ap.add_argument("--n", type=int, default=72)
    ap.add_argument("--out", default="")
    a = ap.parse_args()
    r = run_c3(iters=a.iters, lr=a.lr, n=a.n)
    print(json.dumps({k: v for k, v in r.items() if k != "history"}))
    if a.out:
        with open(a.out, "w") as f:
            json.dump(r, f, indent=1)
