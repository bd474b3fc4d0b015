#!/usr/bin/env python
"""Geodesic-BP benchmark: forward + gradient evaluations per second and
tet-updates per second on the 72^3 Kuhn cube (373,248 vertices,
2,147,466 tets), FP32 eikonal / ECG / adjoint on one GB300 per rank.

One step = a batch of B forward-plus-gradient evaluations through the C ABI
(gbp_forward_backward_batch; B = 16 starts of the inverse problem by
default, gbp_forward_backward when B = 1): per-tet metric precompute, onset
seeding, the persistent FIM eikonal solve with parent record, the parent
pass, the lead-field ECG (8 leads x 150 samples), the misfit and its
phi-derivative, and the frozen-graph adjoint to per-tet c_f, c_t, onset
times and positions.  value = evaluations / second; the same line also
reports one evaluation per step ("single").

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gbp|reference]

Under torchrun every rank runs an independent replica (the evaluation does
not shard); value = all ranks' evaluations / max-over-ranks time.
--impl reference times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRICS = {
    "c3": "Geodesic-BP fwd+grad evals/s at 2.15M tets (72^3 Kuhn cube, FP32)",
    "biv": "Geodesic-BP fwd+grad evals/s on the biventricular shell (FP32)",
}
METRIC = METRICS["c3"]
BATCH = 16                    # default problems per step (multi-start batch)
BYTES_PER_TET_UPDATE = 92.0   # algorithmic bytes per local face update
BYTES_PER_ADJ_NODE = 130.0    # algorithmic bytes per vertex of the adjoint


def workload_config(workload, n=72, h=1.0):
    if workload == "biv":
        return {
            "workload": f"c2 biventricular voxel-Kuhn shell, h={h} mm (LV wall 10 mm, RV 4 mm), rule-based "
                        "fibres -60..+60 deg, c_f/c_t 0.6/0.3 mm/ms with a 1 mm endocardial layer at 2.0 mm/ms, "
                        "5 element onsets, 12 leads from 10 torso electrodes, T=300 @ 1 ms, misfit vs noisy "
                        "target; evaluated at synth.c2_starts (tissue velocity scale exp(N(0,0.1)) per start, "
                        "5 % per-tet log noise, onset times + U(-2,2) ms)",
            "h": h,
        }
    return {
        "workload": f"Kuhn cube {n}^3 vertices (10 mm), per-node log c_f/c_t fields -> per-tet "
                    "c (exp of vertex mean), depth-rotating fibres, 10 element onsets, 8 leads "
                    "(P1 lead field, 1/r kernel, 30 mm sphere), T=150 @ 1 ms, misfit vs noisy target; "
                    "evaluated at synth.c3_starts (prior means c_f/c_t 0.6/0.3 x exp(N(0,0.1)) per start, "
                    "5 % per-vertex log noise, onset times 10 ms (+ U(-2,2) ms))",
        "n": n,
    }


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        self.file.seek(0)
        rows = [r.strip().split(",") for r in self.file.read().splitlines() if r.strip()]
        try:
            os.unlink(self.file.name)
        except OSError:
            pass
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() in ("active", "1", "yes"):
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(seconds, dist=None, device=None):
    """The job's time when every rank runs one replica: the slowest rank's
    time (all_reduce MAX; the ranks' own time on one process)."""
    if dist is None:
        return float(seconds)
    import torch
    tt = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_throughput(units_per_rank, world, seconds):
    """Whole-job throughput: world ranks each processed units_per_rank in
    `seconds`, the max-over-ranks time."""
    return world * units_per_rank / seconds


def build_inputs(workload, n=72, h=1.0, seed=0):
    from paper_2308_08410_gb300 import synth as S
    if workload == "biv":
        return S.make_c2(h=h, seed=seed)
    return S.make_c3(n=n, seed=seed)


def run_cpu_oracle_eval(p, cf, ct, ons, target):
    from oracle import oracle as O
    t0 = time.perf_counter()
    r = O.forward_backward(p.mesh, p.fib, cf, ct, ons, p.L, p.tmpl, target)
    return time.perf_counter() - t0, r


def eval_points(p, B, workload="c3"):
    """The B starts the benchmark evaluates (synth.c3_starts: the prior-mean
    velocities with a global scale per start and 5 % per-vertex log noise,
    onset times 10 ms (+ U(-2, 2) for starts 1..B-1) at the true sites;
    synth.c2_starts on the biventricular mesh).  Start 0 is the
    single-evaluation point.  Returns cf, ct [B, n_t], t [B, K] and the onsets
    of start 0."""
    from paper_2308_08410_gb300 import synth as S
    cf, ct, t = (S.c2_starts if workload == "biv" else S.c3_starts)(p, B)
    ons0 = S.Onsets(p.onsets.kind, p.onsets.idx, t[0], p.onsets.bary)
    return cf, ct, t, ons0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["gbp", "reference"], default="gbp")
    ap.add_argument("--workload", choices=["c3", "biv"], default="c3",
                    help="c3: 72^3 Kuhn cube (2.15M tets); biv: the biventricular shell (473k tets at h=1 mm)")
    ap.add_argument("--n", type=int, default=72, help="vertices per cube edge (c3)")
    ap.add_argument("--h", type=float, default=1.0, help="voxel size in mm (biv)")
    ap.add_argument("--precision", choices=["fp32", "bf16"], default="fp32")
    ap.add_argument("--local", choices=["exact", "fista"], default="exact")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--batch", type=int, default=BATCH,
                    help="problems per step (multi-start: independent parameter sets in one pass)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 0)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank == 0:
            run_reference(args, world)
        return

    import torch
    from paper_2308_08410_gb300 import gbp
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    p = build_inputs(args.workload, args.n, args.h)
    ctx = gbp.Context(local_rank)
    dp = gbp.setup_problem(ctx, p)
    dev = ctx.torch_device
    # target: the ECG of the seeded ground truth plus 5 % per-lead noise
    phi_t, _, _ = ctx.eikonal_solve()
    V_true = ctx.ecg_forward(phi_t, p.tmpl).cpu().numpy()
    from paper_2308_08410_gb300 import synth as S
    target_np = S.add_noise(V_true, 0.05, 4242)
    target = torch.from_numpy(target_np).to(dev)
    B = max(1, args.batch)
    # B starts of the inverse problem (start 0 is also the single-evaluation point)
    cfB_np, ctB_np, tB_np, ons = eval_points(p, B, args.workload)
    cf_np, ct_np = cfB_np[0], ctB_np[0]
    cf = torch.from_numpy(cf_np).to(dev)
    ct = torch.from_numpy(ct_np).to(dev)
    t_on = torch.from_numpy(ons.t).to(dev)
    opts = gbp.make_opts(local_solver=gbp.LOCAL_FISTA if args.local == "fista" else gbp.LOCAL_EXACT, n_f=32)
    prec = gbp.PREC_BF16 if args.precision == "bf16" else gbp.PREC_FP32
    out = None
    if B > 1:
        tgB_np = np.stack([target_np.astype(np.float32)] * B)
        cfB, ctB = torch.from_numpy(cfB_np).to(dev), torch.from_numpy(ctB_np).to(dev)
        tB, tgB = torch.from_numpy(tB_np).to(dev), torch.from_numpy(tgB_np).to(dev)

    def step():
        nonlocal out
        if B == 1:
            out = ctx.forward_backward(cf, ct, target, p.tmpl, t=t_on, opts=opts, precision=prec, out=out)
        else:
            out = ctx.forward_backward_batch(cfB, ctB, tgB, p.tmpl, t=tB, opts=opts, precision=prec, out=out)

    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2
    for _ in range(args.warmup):
        step()
        flush.zero_()
    torch.cuda.synchronize()
    st = ctx.stats()
    if st["status"] != 0:
        raise SystemExit(f"solve failed: {st}")

    stream = torch.cuda.current_stream(dev)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    ctx.enable_timing(True)
    ctx.reset_kernel_times()
    sampler = ClockSampler(local_rank)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    launches0 = ctx.launch_count()
    wall0 = time.perf_counter()
    for k in range(args.steps):
        evs[k][0].record(stream)
        step()
        evs[k][1].record(stream)
        flush.zero_()
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    launches = ctx.launch_count() - launches0
    clocks = sampler.stop()
    ms_steps = [a.elapsed_time(b) for a, b in evs]
    kt_ms, kt_n = ctx.kernel_times(6)
    ctx.enable_timing(False)
    st = ctx.stats()
    single = None
    if B > 1:
        # one evaluation per step (gbp_forward_backward), same timing rules
        s_out = None
        for _ in range(max(3, args.warmup)):
            s_out = ctx.forward_backward(cf, ct, target, p.tmpl, t=t_on, opts=opts, precision=prec, out=s_out)
            flush.zero_()
        s_ms = []
        for _ in range(args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s_out = ctx.forward_backward(cf, ct, target, p.tmpl, t=t_on, opts=opts, precision=prec, out=s_out)
            e1.record(stream)
            flush.zero_()
            torch.cuda.synchronize()
            s_ms.append(e0.elapsed_time(e1))
        single = {"value": world * 1e3 * len(s_ms) / sum(s_ms), "unit": "evals/s",
                  "ms_per_step": sum(s_ms) / len(s_ms), "batch": 1}
    total_s = max_over_ranks(sum(ms_steps) / 1e3, dist, dev)
    if dist is not None:
        dist.barrier()

    # e2e: the same evaluation from host buffers through the host entry points
    # (gbp_forward_backward_batch_host / gbp_forward_backward_host)
    e2e = None
    if not args.no_e2e and B > 1:
        # inputs copied from pinned host memory and outputs written back to
        # pinned host memory inside the call, every step
        hin = [torch.from_numpy(a).pin_memory().numpy() for a in (cfB_np, ctB_np, tB_np, tgB_np)]
        n_t_, K_ = cfB_np.shape[1], tB_np.shape[1]
        shapes = dict(loss=(B,), d_cf=(B, n_t_), d_ct=(B, n_t_), d_t=(B, K_), d_x=(B, K_, 3))
        hout = {k: torch.empty(v, dtype=torch.float32).pin_memory().numpy() for k, v in shapes.items()}

        def e2e_step():
            return ctx.forward_backward_batch_host(hin[0], hin[1], hin[3], p.tmpl, t=hin[2], opts=opts,
                                                   precision=prec, out=hout)

        for _ in range(max(3, args.warmup)):
            e2e_step()
        if dist is not None:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        e2e_s = max_over_ranks(time.perf_counter() - t0, dist, dev)
        e2e = {"value": job_throughput(B * args.steps, world, e2e_s), "unit": "evals/s",
               "h2d_bytes_per_step": int(sum(h.nbytes for h in hin)),
               "d2h_bytes_per_step": int(sum(h.nbytes for h in hout.values()))}
    if not args.no_e2e and B == 1:
        h_out = None
        for _ in range(max(3, args.warmup)):
            h_out = ctx.forward_backward_host(cf_np, ct_np, target_np, p.tmpl, t=ons.t, opts=opts,
                                              precision=prec, out=h_out)
        if dist is not None:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            h_out = ctx.forward_backward_host(cf_np, ct_np, target_np, p.tmpl, t=ons.t, opts=opts,
                                              precision=prec, out=h_out)
        e2e_s = max_over_ranks(time.perf_counter() - t0, dist, dev)
        n_t, K, NT = p.mesh.n_t, p.onsets.K, target_np.size
        e2e = {"value": job_throughput(args.steps, world, e2e_s), "unit": "evals/s",
               "h2d_bytes_per_step": int(4 * (2 * n_t + K + NT)),
               "d2h_bytes_per_step": int(4 * (1 + 2 * n_t + 4 * K))}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    peak, peak_kind = measured_peaks()
    steps = args.steps
    fim_ms = kt_ms[0] / max(kt_n[0], 1)
    adj_ms = kt_ms[4] / max(kt_n[4], 1)
    face_updates = st["face_updates"]
    achieved = face_updates * BYTES_PER_TET_UPDATE / (fim_ms / 1e3) / 1e9
    adj_achieved = B * p.mesh.n_v * BYTES_PER_ADJ_NODE / (adj_ms / 1e3) / 1e9
    ms_per_step = 1e3 * total_s / steps
    value = job_throughput(B * steps, world, total_s)
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        from oracle import oracle as O
        t_cpu, r = run_cpu_oracle_eval(p, cf_np, ct_np, ons, target_np)
        cpu = {"value": 1.0 / t_cpu, "unit": "evals/s", "cores": O.num_threads(), "kind": "oracle",
               "sample": "one full evaluation of the same workload (FP64 oracle: worklist Gauss-Seidel "
                         "eikonal single-threaded, ECG / misfit OpenMP, SCC adjoint serial)",
               "seconds": t_cpu, "loss_gpu": float(out["loss"].reshape(-1)[0].item()), "loss_oracle": r["loss"]}
    traffic = stored_traffic(B, args.n) if args.workload == "c3" else None
    adj_traffic = stored_traffic(B, args.n, kernel="k_adjoint") if args.workload == "c3" else None
    line = {
        "metric": METRICS[args.workload],
        "value": value,
        "unit": "evals/s",
        "n_gpus": world,
        "steps": steps,
        "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32" if args.precision == "fp32" else "f32 eikonal/adjoint, bf16 ECG",
        "data": "synthetic",
        "config": dict(workload_config(args.workload, args.n, args.h), n_v=p.mesh.n_v, n_t=p.mesh.n_t,
                       leads=int(p.L.shape[0]), T=p.tmpl.T, onsets=p.onsets.K, local_solver=args.local,
                       precision=args.precision,
                       batch=B, l2="flushed between steps (256 MB write)", parallelism="replicas"),
        "tet_updates_per_s": world * face_updates * steps / total_s,
        "fim": {"iterations": st["iterations"], "face_updates": face_updates, "candidates": st["candidates"],
                "fp64_fallbacks": st["fp64_fallbacks"], "ms": fim_ms},
        "adjoint": {"seeds": st["adj_levels"], "cycle_nodes": st["adj_cycle_nodes"],
                    "cycle_iters": st["adj_cycle_iters"], "ms": adj_ms,
                    "dataflow_ms": st["adj_dataflow_ms"], "cycle_ms": st["adj_cycle_ms"],
                    "roofline": {"bound": "hbm", "achieved": adj_achieved, "peak": peak, "unit": "GB/s",
                                 "frac": adj_achieved / peak, "traffic": adj_traffic,
                                 "traffic_over_algorithmic": (adj_traffic / (B * p.mesh.n_v * BYTES_PER_ADJ_NODE))
                                 if adj_traffic else None,
                                 "dram_frac": (adj_traffic / (adj_ms / 1e3) / 1e9 / peak) if adj_traffic else None,
                                 "achieved_basis": f"algorithmic bytes: {BYTES_PER_ADJ_NODE:g} B per vertex"}},
        "kernel_ms_per_step": {name: kt_ms[i] / steps for i, name in
                               enumerate(["fim", "parent_pass", "ecg_fwd", "ecg_bwd", "adjoint", "precompute"])},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "kernel": "k_fim",
                     "achieved_basis": f"algorithmic bytes: {BYTES_PER_TET_UPDATE:g} B per local face update "
                                       "(most gathers are served by L2)",
                     "dram_frac": (traffic / (fim_ms / 1e3) / 1e9 / peak) if traffic else None,
                     "peak_source": peak_kind},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "single": single,
        "clocks": clocks,
        "gpu_launches": int(launches),
        "wall_s": wall,
    }
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


KERNEL_SOURCES = {
    # the sources a kernel's DRAM traffic depends on (the adjoint reads the
    # record the parent pass of fim_aux.cu writes)
    "k_fim": ("fim.cu", "gbp_device.cuh"),
    "k_adjoint": ("adjoint.cu", "fim_aux.cu", "gbp_device.cuh"),
}
TRAFFIC_FILES = {"k_fim": "fim_traffic_c3_batch{batch}.txt", "k_adjoint": "adjoint_traffic_c3_batch{batch}.txt"}


_COMMENT = re.compile(r'("(?:\\.|[^"\\\n])*"|\'(?:\\.|[^\'\\\n])*\')|//[^\n]*|/\*.*?\*/', re.S)


def normalize_source(text: str) -> str:
    """C/C++/CUDA source with its comments taken out (string literals, such as
    inline PTX, kept) and every run of white space made one space."""
    return " ".join(_COMMENT.sub(lambda m: m.group(1) or "", text).split())


def kernel_hash(kernel: str = "k_fim") -> str:
    """Hash of a kernel's normalised sources (normalize_source): a stored ncu
    traffic figure applies only while it matches."""
    import hashlib
    h = hashlib.sha1()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_2308_08410_gb300", "csrc", f), encoding="utf-8") as fh:
            h.update(normalize_source(fh.read()).encode())
    return h.hexdigest()[:12]


def stored_traffic(batch, n, path=None, kernel: str = "k_fim"):
    """DRAM bytes per launch of `kernel` from the committed ncu summary for
    this workload, or None when there is none or it was taken on other kernel
    sources (its kernel_hash differs), another batch size or mesh."""
    path = path or os.path.join(ROOT, "profiles", TRAFFIC_FILES[kernel].format(batch=batch))
    try:
        with open(path) as f:
            tj = json.load(f)
    except (OSError, ValueError):
        return None
    if tj.get("kernel_hash") == kernel_hash(kernel) and tj.get("batch") == batch and tj.get("n") == n:
        return tj.get("bytes_per_launch")
    return None


def run_reference(args, world):
    """The FP64 CPU oracle, as it stands, on the host cores: each step is one
    full evaluation of the same workload (about 12 s); warm-up steps are not
    needed on the CPU and steps stop after ~150 s (the count is reported)."""
    from oracle import oracle as O
    p = build_inputs(args.workload, args.n, args.h)
    ek = O.eikonal(p.mesh, p.fib, p.cf, p.ct, p.onsets)
    from paper_2308_08410_gb300 import synth as S
    target = S.add_noise(O.ecg(p.L, ek["phi"], p.tmpl), 0.05, 4242)
    cfB, ctB, _, ons = eval_points(p, 1, args.workload)
    cf, ct = cfB[0], ctB[0]
    times = []
    t_start = time.perf_counter()
    for _ in range(max(1, args.steps)):
        dt, _ = run_cpu_oracle_eval(p, cf, ct, ons, target)
        times.append(dt)
        if time.perf_counter() - t_start > 150:
            break
    total = sum(times)
    value = len(times) / total
    line = {
        "impl": "reference",
        "metric": METRICS[args.workload],
        "value": value,
        "unit": "evals/s",
        "n_gpus": world,
        "steps": len(times),
        "warmup": 0,
        "ms_per_step": 1e3 * total / len(times),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": dict(workload_config(args.workload, args.n, args.h), n_v=p.mesh.n_v, n_t=p.mesh.n_t,
                       leads=int(p.L.shape[0]), T=p.tmpl.T, onsets=p.onsets.K, parallelism="host cores"),
        "cpu_baseline": {"value": value, "unit": "evals/s", "cores": O.num_threads(), "kind": "oracle",
                         "sample": f"{len(times)} full evaluations of the workload (steps requested "
                                   f"{args.steps}; capped near 150 s)"},
        "e2e": {"value": value, "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


if __name__ == "__main__":
    main()
