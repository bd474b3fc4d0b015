"""Precision study of the lead-field ECG (Sec. II-D): the BF16 tensor-core
contraction with FP32 accumulation and per-lead scaling against the FP32
CUDA-core contraction on the 1M-vertex workload (100^3 cube, 12 standard
leads, T = 500 at 1 ms, phi uniform in [0, 120] ms plus smooth seeded noise):
their difference, their speed, and the difference of the misfit derivative
they lead to; then the effect of the BF16 ECG on the misfit trajectory of the
inverse problem on the biventricular mesh.  Every ECG and gradient is
computed by the library's kernels.  (Both paths' errors against the FP64
oracle on the same workload are measured by tests/test_gpu_precision.py.)
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import gbp
from . import synth as S


def _rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _time(fn, reps=20):
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def run_c4(n=100, device=0, log=print):
    mesh, L, phi, tmpl = S.make_c4(n=n)
    ctx = gbp.Context(device)
    ctx.upload_mesh(mesh.xyz, mesh.tets)
    dev = ctx.torch_device
    Ld = torch.from_numpy(np.ascontiguousarray(L, np.float32)).to(dev)
    ctx.set_leadfield(Ld)
    phid = torch.from_numpy(phi).to(dev)
    res = {"workload": f"{n}^3 cube ({mesh.n_v} vertices), {L.shape[0]} leads, T={tmpl.T}"}
    outs = {}
    for name, prec in (("fp32", gbp.PREC_FP32), ("bf16", gbp.PREC_BF16)):
        V = ctx.ecg_forward(phid, tmpl, precision=prec)
        outs[name] = V.clone()
        ms = _time(lambda: ctx.ecg_forward(phid, tmpl, precision=prec, out=V))
        res[name] = {"ms": ms, "vertex_samples_per_s": mesh.n_v * tmpl.T / (ms * 1e-3)}
    res["ecg_rel_l2_bf16_vs_fp32"] = _rel(outs["bf16"].cpu().numpy(), outs["fp32"].cpu().numpy())
    # the misfit derivative with each forward: target = FP32 ECG + 5 % noise
    target = torch.from_numpy(S.add_noise(outs["fp32"].cpu().numpy(), 0.05, 7).astype(np.float32)).to(dev)
    g = {}
    for name in ("fp32", "bf16"):
        loss, dphi = ctx.ecg_loss_backward(phid, outs[name], target, tmpl)
        g[name] = (float(loss.item()), dphi.cpu().numpy())
    res["loss"] = {"fp32": g["fp32"][0], "bf16": g["bf16"][0]}
    res["dphi_rel_l2_bf16_vs_fp32"] = _rel(g["bf16"][1], g["fp32"][1])
    ctx.close()
    log(f"ECG BF16 vs FP32 rel L2 {res['ecg_rel_l2_bf16_vs_fp32']:.3e}; "
        f"FP32 {res['fp32']['ms']:.3f} ms, BF16 {res['bf16']['ms']:.3f} ms")
    return res


def run_c2_trajectory(iters=100, lr=1e-2, device=0, log=print):
    """The inverse loop on the biventricular mesh from the prior-mean start,
    once with the FP32 ECG (iters Adam iterations) and once with the BF16 ECG
    (same target, same start) until the FP32 misfit of its iterate reaches
    the FP32 arm's final misfit, or 2 iters; returns both misfit histories and
    the time to that misfit.  A short untimed run first loads every kernel
    both arms use."""
    from .inverse import InverseProblem
    p = S.make_c2()
    ctx = gbp.Context(device)
    gbp.setup_problem(ctx, p)
    phi_true, _, _ = ctx.eikonal_solve()
    V = ctx.ecg_forward(phi_true, p.tmpl).cpu().numpy()
    target = S.add_noise(V, 0.05, 11)
    hist = {}
    goal = None  # the FP32 arm's final misfit
    for prec in (gbp.PREC_FP32, gbp.PREC_BF16):
        warm = InverseProblem(ctx, p, target, precision=prec,
                              init_log_cf=np.full(p.mesh.n_v, np.log(0.6 * 0.8)),
                              init_log_ct=np.full(p.mesh.n_v, np.log(0.3 * 0.8)),
                              init_t=(p.onsets.t + 3.0).astype(np.float32))
        warm.run_adam(iters=3, lr=lr)
    for name, prec in (("fp32", gbp.PREC_FP32), ("bf16", gbp.PREC_BF16)):
        inv = InverseProblem(ctx, p, target, precision=prec,
                             init_log_cf=np.full(p.mesh.n_v, np.log(0.6 * 0.8)),
                             init_log_ct=np.full(p.mesh.n_v, np.log(0.3 * 0.8)),
                             init_t=(p.onsets.t + 3.0).astype(np.float32))
        arrival = {}
        t_start = time.perf_counter()

        def check(it, loss, inv=inv, arrival=arrival, t_start=t_start):
            # the BF16 arm has reached the goal once the FP32 misfit of the same
            # iterate (its last forward solve) is at or below it
            if goal is None or arrival or float(loss.item()) > goal:
                return False
            op = inv.op
            e32 = ctx.ecg_forward(op.phi, op.tmpl, precision=gbp.PREC_FP32)
            l32 = float(ctx.ecg_loss_backward(op.phi, e32, op.target, op.tmpl)[0].item())
            if l32 <= goal:
                arrival.update(iteration=it, s=time.perf_counter() - t_start, bf16_misfit=float(loss.item()),
                               fp32_misfit=l32)
                return True
            return False

        if prec == gbp.PREC_BF16:
            # up to 2 iters, until the FP32 misfit of the iterate reaches the goal
            h, wall = inv.run_adam(iters=2 * iters, lr=lr, log_every=10, callback=check)
        else:
            h, wall = inv.run_adam(iters=iters, lr=lr, log_every=10)
        # the misfit of the final parameters, always with the FP32 ECG
        inv.op.precision = gbp.PREC_FP32
        final = float(inv.loss().item())
        hist[name] = {"history": h, "final_fp32_misfit": final, "wall_s": wall}
        if prec == gbp.PREC_FP32:
            goal = final
        else:
            hist[name]["reached_fp32_goal"] = arrival or None
        log(f"{name}: misfit {h[0][1]:.4g} -> {final:.4g} in {iters} iterations ({wall:.2f} s)"
            + (f"; FP32 misfit {goal:.4g} reached at {arrival}" if prec == gbp.PREC_BF16 else ""))
    ctx.close()
    return hist


if __name__ == "__main__":
    import argparse
    import json

    ap = argparse.ArgumentParser(description="BF16 vs FP32 ECG precision study")
    ap.add_argument("--n", type=int, default=100)
    ap.add_argument("--iters", type=int, default=100)
    ap.add_argument("--only", choices=["c4", "c2"], default=None, help="run one of the two studies")
    ap.add_argument("--out", default="")
    a = ap.parse_args()
    t0 = time.perf_counter()
    r = {}
    if a.only in (None, "c4"):
        r["c4"] = run_c4(a.n)
    if a.only in (None, "c2"):
        r["c2_trajectory"] = run_c2_trajectory(a.iters)
    r["wall_s"] = time.perf_counter() - t0
    s = json.dumps(r)
    print(s)
    if a.out:
        with open(a.out, "w") as f:
            f.write(s)
