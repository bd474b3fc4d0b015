"""Geodesic-BP as a differentiable PyTorch operation and the Adam inverse loop.

``GeodesicEcgLoss`` wraps one forward-plus-gradient evaluation of the C ABI
(include/gbp.h): the forward pass runs the eikonal solve, the lead-field ECG
and the misfit of Eq. (inverse_ecg); the backward pass runs the frozen-graph
adjoint of Sec. II-C on the parent graph the forward solve recorded (phi is
recomputed on every call; no per-iteration solver state is stored, unlike
backpropagation through the unrolled iterations of Algorithm 2).

``InverseProblem`` holds the parameter maps (per-vertex log velocities ->
per-element velocities, onset positions inside their elements; tets, or
triangles for the d = 2 study of Sec. III-A) and runs Adam
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
                 init_log_cf=None, init_log_ct=None, init_t=None, optimise_positions=True, relocate=True,
                 optimise_velocities=True):
        self.ctx = ctx
        self.p = problem
        dev = ctx.torch_device
        # triangle meshes (d = 2) carry xy / tris, tet meshes xyz / tets
        self.dim = 2 if hasattr(problem.mesh, "tris") else 3
        X = problem.mesh.xy if self.dim == 2 else problem.mesh.xyz
        cells = problem.mesh.tris if self.dim == 2 else problem.mesh.tets
        self.X = np.asarray(X, np.float64)
        self.dp = gbp.setup_problem_2d(ctx, problem) if self.dim == 2 else gbp.setup_problem(ctx, problem)
        self.tets = torch.from_numpy(cells.astype(np.int64)).to(dev)
        self.optimise_velocities = optimise_velocities
        n_v = problem.mesh.n_v
        w = self.dim + 1
        lcf = np.full(n_v, np.log(0.6)) if init_log_cf is None else init_log_cf
        lct = np.full(n_v, np.log(0.3)) if init_log_ct is None else init_log_ct
        ons = problem.onsets
        t0 = ons.t if init_t is None else init_t
        self.log_cf = torch.tensor(np.asarray(lcf, np.float32), device=dev, requires_grad=optimise_velocities)
        self.log_ct = torch.tensor(np.asarray(lct, np.float32), device=dev, requires_grad=optimise_velocities)
        self.t = torch.tensor(np.asarray(t0, np.float32), device=dev, requires_grad=True)
        self.kind = ons.kind
        self.optimise_positions = optimise_positions and ons.kind == gbp.ONSET_ELEMENT
        if ons.kind == gbp.ONSET_ELEMENT:
            V = self.X[cells[ons.idx]]  # [K, d + 1, d]
            x0 = np.einsum("kq,kqr->kr", ons.bary.astype(np.float64), V)
            M = np.concatenate([V.transpose(0, 2, 1), np.ones((ons.K, 1, w))], axis=1)  # [K, d + 1, d + 1]
            self.Vt_inv = torch.tensor(np.linalg.inv(M), dtype=torch.float32, device=dev)
            self.x = torch.tensor(x0.astype(np.float32), device=dev, requires_grad=self.optimise_positions)
        else:
            self.Vt_inv = None
            self.x = torch.zeros(ons.K, self.dim, device=dev)
        self.locator = None
        if self.optimise_positions and relocate:
            from .relocate import SimplexLocator
            self.locator = SimplexLocator(self.X, cells)
        self.op = EvalOp(ctx=ctx, kind=ons.kind, on_idx=self.dp.on_idx,
                         target=torch.from_numpy(np.ascontiguousarray(target, np.float32)).to(dev),
                         tmpl=problem.tmpl, opts=opts if opts is not None else gbp.make_opts(),
                         precision=precision, phi=torch.empty(n_v, device=dev),
                         parent=torch.empty(n_v, dtype=torch.int32, device=dev),
                         alpha=torch.empty(n_v, self.dim, device=dev),
                         ecg=torch.empty(problem.L.shape[0], problem.tmpl.T, device=dev))

    def params(self):
        ps = [self.log_cf, self.log_ct, self.t] if self.optimise_velocities else [self.t]
        if self.optimise_positions:
            ps.append(self.x)
        return ps

    def tet_velocities(self):
        """Per-element velocity = exp(mean of the element's vertex log values)."""
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
        V = torch.from_numpy(self.X.astype(np.float32)).to(self.x.device)[self.tets[self.op.on_idx.long()]]
        self.x.copy_(torch.einsum("kq,kqr->kr", b, V))

    def run_adam(self, iters=500, lr=1e-2, log_every=0, callback=None, lr_sites=None):
        """Adam at lr; onset times and positions at lr_sites when given.  A
        callback(iteration, loss) that returns True ends the run after that
        iteration."""
        if lr_sites is None:
            opt = torch.optim.Adam(self.params(), lr=lr)
        else:
            site = [p for p in (self.t, self.x) if p.requires_grad]
            rest = [p for p in self.params() if all(p is not q for q in site)]
            opt = torch.optim.Adam([{"params": rest, "lr": lr}, {"params": site, "lr": lr_sites}])
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
            if callback is not None and callback(it, loss):
                if log_every and hist and hist[-1][0] != it:
                    hist.append((it, float(loss.item()), time.perf_counter() - t_start))
                break
        torch.cuda.synchronize()
        return hist, time.perf_counter() - t_start


class VertexLogToTet(torch.autograd.Function):
    """c_j = exp(mean of the w vertex values of log c over element j (w = 4
    for tets, 3 for triangles)).  The backward scatters g_j c_j / w to the
    element's vertices with an atomic index_add (autograd's own backward of
    the gather sorts the indices, which dominates an inverse-loop step at 2M
    tets)."""

    @staticmethod
    def forward(fctx, logc, tets):
        # logc [n_v] or [B, n_v] -> c [n_t] or [B, n_t]
        c = torch.exp(logc[..., tets].mean(dim=-1))
        fctx.save_for_backward(c, tets)
        fctx.shape = logc.shape
        return c

    @staticmethod
    def backward(fctx, g):
        c, tets = fctx.saved_tensors
        nw = tets.shape[1]
        w = (g * c / nw).unsqueeze(-1).expand(*c.shape, nw)
        out = torch.zeros(fctx.shape, dtype=g.dtype, device=g.device)
        out.index_add_(out.dim() - 1, tets.reshape(-1), w.reshape(*c.shape[:-1], -1))
        return out, None


class GeodesicEcgLoss(torch.autograd.Function):
    """loss = 1/(N T) sum (ECG(phi(cf, ct, t, x)) - target)^2 (Eq. inverse_ecg).

    Inputs: cf, ct per element [n_t]; t onset times [K]; x onset positions [K, d]
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
           precision: int = gbp.PREC_FP32, init: str = "surface", starts: int = 1, lr_sites: float | None = 5e-2,
           log=print):
    """The inverse loop on the 72^3 cube (2.15M tets): Adam on the per-vertex
    log-velocity fields and the 10 onset times / positions, from the
    prior-mean start (c_f = 0.6, c_t = 0.3 mm/ms everywhere, onset times
    10 ms).  init = "surface": 10 random sites on the mesh surface, which
    relocation walks through the mesh; init = "centroids": the centroids of
    the true onset tets (an informed start).  starts > 1 (surface init only)
    runs that many independent surface draws together in one batch and
    keeps the start with the lowest misfit.  lr_sites: learning rate of the
    onset times (ms) and positions (mm) (None: lr).  Target: the
    ground-truth ECG plus 5 % noise.  Returns the loss history and the
    activation-time error against the ground truth before and after."""
    from . import synth as S
    p = S.make_c3(n=n)
    ctx = gbp.Context(device)
    gbp.setup_problem(ctx, p)
    phi_true, _, _ = ctx.eikonal_solve()
    V = ctx.ecg_forward(phi_true, p.tmpl).cpu().numpy()
    phi_true = phi_true.clone()
    target = S.add_noise(V, p.extra["noise"], 4242)
    ons = p.onsets
    t10 = np.full(ons.K, 10.0, np.float32)
    if init == "surface":
        draws = [S.onsets_surface(p.mesh, ons.K, seed=777 + s_, tmin=10.0, tmax=10.0) for s_ in range(starts)]
    elif init == "centroids" and starts == 1:
        draws = [S.Onsets(ons.kind, ons.idx, t10, np.full((ons.K, 4), 0.25, np.float32))]
    else:
        raise ValueError(f"unsupported init {init!r} with {starts} starts")

    @torch.no_grad()
    def act_err(log_cf, log_ct, on_idx, t, bary):
        cells = torch.from_numpy(p.mesh.tets.astype(np.int64)).to(ctx.torch_device)
        ctx.set_velocities(VertexLogToTet.apply(log_cf, cells).contiguous(),
                           VertexLogToTet.apply(log_ct, cells).contiguous())
        ctx.set_onsets(gbp.ONSET_ELEMENT, on_idx.contiguous(), t.contiguous(), bary.contiguous())
        phi, _, _ = ctx.eikonal_solve()
        d = (phi - phi_true).double()
        return float(torch.sqrt((d * d).mean()).item()), float(d.abs().max().item())

    extra = {}
    if starts == 1:
        p0 = S.Problem(p.name, p.mesh, p.fib, p.cf, p.ct, draws[0], p.L, p.tmpl, p.extra)
        inv = InverseProblem(ctx, p0, target, precision=precision, init_t=t10)
        state = lambda: (inv.log_cf.detach(), inv.log_ct.detach(), inv.op.on_idx, inv.t.detach(),  # noqa: E731
                         inv.bary())
        rmse0, max0 = act_err(*state())
        loss0 = float(inv.loss().item())
        hist, wall = inv.run_adam(iters=iters, lr=lr, log_every=log_every, lr_sites=lr_sites)
        loss1 = hist[-1][1] if hist else loss0
        rmse1, max1 = act_err(*state())
        lcf, lct, t_fit = inv.log_cf.detach(), inv.log_ct.detach(), inv.t.detach().cpu().numpy()
    else:
        ms = MultiStartInverse(ctx, p, target, draws, precision=precision, optimise_velocities=True)
        b0 = ms.bary()
        rmse0, max0 = act_err(ms.log_cf[0].detach(), ms.log_ct[0].detach(), ms.on_idx[0], ms.t[0].detach(), b0[0])
        loss0 = float(ms.evaluate()[0].item())
        hist, wall = ms.run_adam(iters=iters, lr=lr, log_every=log_every, lr_sites=lr_sites)
        losses = ms.evaluate().detach().cpu().numpy()
        best = int(np.argmin(losses))
        loss1 = float(losses[best])
        bb = ms.bary()
        rmse1, max1 = act_err(ms.log_cf[best].detach(), ms.log_ct[best].detach(), ms.on_idx[best],
                              ms.t[best].detach(), bb[best])
        first = act_err(ms.log_cf[0].detach(), ms.log_ct[0].detach(), ms.on_idx[0], ms.t[0].detach(), bb[0])
        lcf, lct, t_fit = ms.log_cf[best].detach(), ms.log_ct[best].detach(), ms.t[best].detach().cpu().numpy()
        extra = dict(starts=starts, best_start=best, start_losses=[float(v) for v in losses],
                     start0_loss=float(losses[0]), start0_act_rmse_ms=first[0])
    lcf_true = torch.from_numpy(p.extra["log_cf_nodal"]).to(lcf.device)
    lct_true = torch.from_numpy(p.extra["log_ct_nodal"]).to(lct.device)
    res = dict(workload=f"{n}^3 cube, {p.mesh.n_t} tets, {ons.K} element onsets, {p.L.shape[0]} leads, "
                        f"T={p.tmpl.T}, 5% noise",
               init=init, iters=iters, lr=lr, lr_sites=lr_sites if lr_sites is not None else lr, wall_s=wall,
               # steady state: the first iteration also loads the torch kernels
               ms_per_iter=(1e3 * (hist[-1][2] - hist[0][2]) / max(hist[-1][0] - hist[0][0], 1)
                            if len(hist) > 1 else 1e3 * wall / max(iters, 1)),
               loss0=loss0, loss_final=loss1, noise_floor=float(np.mean((target - V) ** 2)),
               act_rmse_ms=(rmse0, rmse1), act_max_ms=(max0, max1),
               log_cf_mae=float((lcf - lcf_true).abs().mean().item()),
               log_ct_mae=float((lct - lct_true).abs().mean().item()),
               log_cf_mae0=float((np.log(0.6) - lcf_true).abs().mean().item()),
               log_ct_mae0=float((np.log(0.3) - lct_true).abs().mean().item()),
               # onset k starts in true onset k's tet only for the centroid start
               t_err_ms=((float(np.abs(10.0 - ons.t).mean()), float(np.abs(t_fit - ons.t).mean()))
                         if init == "centroids" else None),
               **extra, history=hist)
    for it, l, tt in hist:
        log(f"iter {it:4d}  loss {l:.6g}  {tt:.2f} s")
    ctx.close()
    return res


class MultiStartInverse:
    """B starts of the inverse problem run together (Sec. IV: batched
    optimisation as the way out of local minima).  Adam on every start's
    element-onset positions and times ([B, K, d], [B, K]) and, with
    optimise_velocities, its per-vertex log-velocity fields ([B, n_v], mapped
    to elements as in InverseProblem); otherwise the problem's velocities are
    kept.  Each epoch is one batched evaluation (gbp_set_onsets_batch, then
    gbp_forward_backward_batch: the FIM, parent pass and adjoint of all
    starts share their launches).  The starts stay independent: each loss
    depends on its own start only and Adam acts elementwise."""

    def __init__(self, ctx: gbp.Context, problem, target: np.ndarray, starts, opts=None, precision=gbp.PREC_FP32,
                 relocate=True, optimise_velocities=False, init_log_cf=np.log(0.6), init_log_ct=np.log(0.3)):
        self.ctx = ctx
        dev = ctx.torch_device
        self.dim = d = 2 if hasattr(problem.mesh, "tris") else 3
        X = np.asarray(problem.mesh.xy if d == 2 else problem.mesh.xyz, np.float64)
        cells = problem.mesh.tris if d == 2 else problem.mesh.tets
        (gbp.setup_problem_2d if d == 2 else gbp.setup_problem)(ctx, problem)
        self.B, self.K = B, K = len(starts), starts[0].K
        self.cf = torch.from_numpy(np.tile(problem.cf.astype(np.float32), (B, 1))).to(dev)
        self.ct = torch.from_numpy(np.tile(problem.ct.astype(np.float32), (B, 1))).to(dev)
        self.optimise_velocities = optimise_velocities
        if optimise_velocities:
            n_v = problem.mesh.n_v
            self.cells = torch.from_numpy(cells.astype(np.int64)).to(dev)
            self.log_cf = torch.full((B, n_v), float(init_log_cf), device=dev, requires_grad=True)
            self.log_ct = torch.full((B, n_v), float(init_log_ct), device=dev, requires_grad=True)
        idx = np.stack([o.idx for o in starts]).astype(np.int64)
        bary = np.stack([o.bary for o in starts]).astype(np.float64)
        V = X[cells[idx]]  # [B, K, d + 1, d]
        M = np.concatenate([V.transpose(0, 1, 3, 2), np.ones((B, K, 1, d + 1))], axis=2)
        self.Vt_inv = torch.tensor(np.linalg.inv(M), dtype=torch.float32, device=dev)
        self.on_idx = torch.from_numpy(idx.astype(np.int32)).to(dev)
        self.x = torch.tensor(np.einsum("bkq,bkqr->bkr", bary, V).astype(np.float32), device=dev,
                              requires_grad=True)
        self.t = torch.tensor(np.stack([o.t for o in starts]).astype(np.float32), device=dev, requires_grad=True)
        self.target = torch.from_numpy(np.tile(np.asarray(target, np.float32)[None], (B, 1, 1))).to(dev)
        self.tmpl = problem.tmpl
        self.opts = opts if opts is not None else gbp.make_opts()
        self.precision = precision
        self.locator = None
        if relocate:
            from .relocate import SimplexLocator
            self.locator = SimplexLocator(X, cells)
        self.out = None

    def bary(self):
        xh = torch.cat([self.x.detach(), torch.ones_like(self.x[..., :1])], dim=-1)
        return torch.einsum("bkij,bkj->bki", self.Vt_inv, xh).contiguous()

    def evaluate(self):
        """Losses [B]; the gradients land in the output dict (and, with
        optimise_velocities, in log_cf.grad / log_ct.grad)."""
        if self.optimise_velocities:
            cf = VertexLogToTet.apply(self.log_cf, self.cells)
            ct = VertexLogToTet.apply(self.log_ct, self.cells)
            self.cf, self.ct = cf.detach().contiguous(), ct.detach().contiguous()
        self.ctx.set_onsets_batch(gbp.ONSET_ELEMENT, self.on_idx, self.t.detach().contiguous(), self.bary())
        self.out = self.ctx.forward_backward_batch(self.cf, self.ct, self.target, self.tmpl, opts=self.opts,
                                                   precision=self.precision, out=self.out)
        if self.optimise_velocities:
            self.log_cf.grad = self.log_ct.grad = None
            torch.autograd.backward([cf, ct], [self.out["d_cf"], self.out["d_ct"]])
        return self.out["loss"]

    def params(self, lr, lr_sites=None):
        groups = [{"params": [self.x, self.t], "lr": lr if lr_sites is None else lr_sites}]
        if self.optimise_velocities:
            groups.append({"params": [self.log_cf, self.log_ct], "lr": lr})
        return groups

    @torch.no_grad()
    def project_positions(self, floor=1e-3):
        d = self.dim
        if self.locator is not None:
            from .relocate import relocate_onsets
            relocate_onsets(self.locator, self.x.view(-1, d), self.on_idx.view(-1),
                            self.Vt_inv.view(-1, d + 1, d + 1), floor=floor)
            return
        b = self.bary().clamp_min(floor)
        b = b / b.sum(dim=-1, keepdim=True)
        Minv = self.Vt_inv
        # x = V b with V the first d rows of M = inverse(Minv)
        self.x.copy_(torch.einsum("bkrq,bkq->bkr", torch.linalg.inv(Minv)[:, :, :d, :], b))

    def run_adam(self, iters=400, lr=0.5, log_every=0, lr_sites=None):
        opt = torch.optim.Adam(self.params(lr, lr_sites))
        hist = []
        t_start = time.perf_counter()
        for it in range(iters):
            loss = self.evaluate()
            self.x.grad = self.out["d_x"]
            self.t.grad = self.out["d_t"]
            opt.step()
            self.project_positions()
            if log_every and (it % log_every == 0 or it == iters - 1):
                hist.append((it, float(loss.min().item()), time.perf_counter() - t_start))
        torch.cuda.synchronize()
        return hist, time.perf_counter() - t_start


def run_2d(iters: int = 400, lr: float = 0.5, n_init: int = 8, starts: int = 1, device: int = 0,
           log_every: int = 20, relocate: bool = True, log=print):
    """The paper's 2-D simulation study (Sec. III-A), on synthetic geometry.
    Ground truth: 4 sites with times in [2.5, 10] ms on the 0.45 mm LV slice
    (10,440 vertices), its ECG from that mesh's lead field.  Model: the
    0.9 mm slice (2,700 vertices, 7 leads) with the true velocities, starting
    from n_init sites at 0 ms spread evenly on the mid-wall circle.  Adam on
    the sites' positions and times, 400 epochs at lr 0.5 as in the paper.
    starts > 1 runs that many starts at once (the ring turned by a fraction
    of its spacing each; start 0 is the single start) and keeps the one
    with the lowest misfit.  Reports the steady-state time per epoch, the
    misfit, and the RMSE of the activation times against the ground truth at
    the coarse vertices (which coincide with fine ones), also for the true
    sites on the coarse mesh (the floor the coarse model itself sets)."""
    import dataclasses as dc

    from . import synth as S
    ctx = gbp.Context(device)
    dev = ctx.torch_device
    fine = S.make_2d_torso(fine=True)
    gbp.setup_problem_2d(ctx, fine)
    phi_f, _, _ = ctx.eikonal_solve()
    target = ctx.ecg_forward(phi_f, fine.tmpl).cpu().numpy()
    phi_true = torch.from_numpy(phi_f.cpu().numpy().reshape(29, 360)[::2, ::2].reshape(-1)).to(dev)
    coarse = S.make_2d_torso(fine=False)
    target_d = torch.from_numpy(target).to(dev)

    def ring(offset):
        ang = offset + 2 * np.pi * np.arange(n_init) / n_init
        idx, bary = S.locate_2d(coarse.mesh, 24.5 * np.stack([np.cos(ang), np.sin(ang)], axis=1))
        return S.Onsets(S.ONSET_ELEMENT, idx.astype(np.int32), np.zeros(n_init, np.float32),
                        bary.astype(np.float32))

    cf_d = torch.from_numpy(coarse.cf).to(dev)
    ct_d = torch.from_numpy(coarse.ct).to(dev)

    @torch.no_grad()
    def evaluate_sites(idx, t, bary):
        """(misfit, activation RMSE vs truth) of one site set on the coarse mesh."""
        ctx.set_velocities(cf_d, ct_d)
        ctx.set_onsets(gbp.ONSET_ELEMENT, idx.contiguous(), t.contiguous(), bary.contiguous())
        phi, _, _ = ctx.eikonal_solve()
        V = ctx.ecg_forward(phi, coarse.tmpl)
        loss, _ = ctx.ecg_loss_backward(phi, V, target_d, coarse.tmpl)
        d = (phi - phi_true).double()
        return float(loss.item()), float(torch.sqrt((d * d).mean()).item())

    tr = coarse.onsets
    if starts == 1:
        p0 = dc.replace(coarse, onsets=ring(0.0), onset_t=np.zeros(n_init, np.float32))
        inv = InverseProblem(ctx, p0, target, optimise_velocities=False, relocate=relocate)
        loss0, rmse0 = evaluate_sites(inv.op.on_idx, inv.t.detach(), inv.bary())
        hist, wall = inv.run_adam(iters=iters, lr=lr, log_every=log_every)
        loss1, rmse1 = evaluate_sites(inv.op.on_idx, inv.t.detach(), inv.bary())
        x, t = inv.x.detach().cpu().numpy(), inv.t.detach().cpu().numpy()
        extra = {}
    else:
        ms = MultiStartInverse(ctx, coarse, target, [ring(2 * np.pi * s / (n_init * starts)) for s in range(starts)],
                               relocate=relocate)
        loss0, rmse0 = evaluate_sites(ms.on_idx[0], ms.t[0].detach(), ms.bary()[0])
        hist, wall = ms.run_adam(iters=iters, lr=lr, log_every=log_every)
        losses = ms.evaluate().cpu().numpy()
        best = int(np.argmin(losses))
        b_all = ms.bary()
        loss1, rmse1 = evaluate_sites(ms.on_idx[best], ms.t[best].detach(), b_all[best])
        first = evaluate_sites(ms.on_idx[0], ms.t[0].detach(), b_all[0])
        x, t = ms.x[best].detach().cpu().numpy(), ms.t[best].detach().cpu().numpy()
        extra = dict(starts=starts, best_start=best, start_losses=[float(v) for v in losses],
                     start0_loss=first[0], start0_act_rmse_ms=first[1])
    floor = evaluate_sites(torch.from_numpy(tr.idx).to(dev), torch.from_numpy(tr.t).to(dev),
                           torch.from_numpy(tr.bary).to(dev))
    true_pts = np.einsum("kq,kqr->kr", tr.bary.astype(np.float64),
                         coarse.mesh.xy.astype(np.float64)[coarse.mesh.tris[tr.idx]])
    res = dict(workload=f"2-D LV slice, {coarse.mesh.n_v} vertices ({coarse.mesh.n_t} triangles), "
                        f"{coarse.L.shape[0]} leads, T={coarse.tmpl.T}; truth on the {fine.mesh.n_v}-vertex slice "
                        f"with {tr.K} sites; {n_init} initial sites at 0 ms",
               iters=iters, lr=lr, wall_s=wall,
               ms_per_epoch=(1e3 * (hist[-1][2] - hist[0][2]) / max(hist[-1][0] - hist[0][0], 1)
                             if len(hist) > 1 else 1e3 * wall / max(iters, 1)),
               loss0=loss0, loss_final=loss1, act_rmse_ms=(rmse0, rmse1),
               true_sites_loss=floor[0], true_sites_act_rmse_ms=floor[1], **extra,
               sites_final=[[float(a), float(b), float(c)] for (a, b), c in zip(x, t)],
               sites_true=[[float(a), float(b), float(c)] for (a, b), c in zip(true_pts, tr.t)],
               history=hist)
    for it, l, tt in hist:
        log(f"epoch {it:4d}  loss {l:.6g}  {tt:.2f} s")
    ctx.close()
    return res


if __name__ == "__main__":
    import argparse
    import json

    ap = argparse.ArgumentParser(description="Adam inverse loops: the 72^3 cube, or the 2-D LV-slice study")
    ap.add_argument("--study", choices=["c3", "2d"], default="c3")
    ap.add_argument("--iters", type=int, default=0, help="0: 500 (c3) / 400 (2d)")
    ap.add_argument("--lr", type=float, default=0.0, help="0: 1e-2 (c3) / 0.5 (2d)")
    ap.add_argument("--n", type=int, default=72)
    ap.add_argument("--starts", type=int, default=1, help="starts run together in one batch")
    ap.add_argument("--init", choices=["surface", "centroids"], default="surface", help="c3: initial sites")
    ap.add_argument("--lr-sites", type=float, default=5e-2, help="c3: learning rate of onset times / positions")
    ap.add_argument("--out", default="")
    a = ap.parse_args()
    if a.study == "2d":
        r = run_2d(iters=a.iters or 400, lr=a.lr or 0.5, starts=a.starts)
    else:
        r = run_c3(iters=a.iters or 500, lr=a.lr or 1e-2, n=a.n, init=a.init, starts=a.starts,
                   lr_sites=a.lr_sites)
    print(json.dumps({k: v for k, v in r.items() if k != "history"}))
    if a.out:
        with open(a.out, "w") as f:
            json.dump(r, f, indent=1)
