#!/usr/bin/env python3
"""Benchmark of the low-memory S_N-DG hot path on one GB300 (or N independent replicas).

A step is one pass of the whole path over the 1024 x 1024, S16 workload with 16 x 16-cell patches of
sigma_s, sigma_a ~ U[0.1, 10] (seed 1907), q = 1, eps = 1, vacuum inflow: for each scheme (standard Q1-DG,
LMDG, RLMDG) one lmdg_solve to a 1e-8 relative residual with FP32 sweeps inside FP64 iterative refinement
(FP64 Arnoldi, least squares and updates; residual sweeps in float-float, LMDG_RESID_F32X2), including the
recovery sweep that stores the angular unknowns.  The metric is transport-sweep cell-angle updates per second
over the step (every sweep the solves run); time to 1e-8 for this solver, for the same solver with FP64
residual sweeps and for the FP64 solver is reported beside it, with the final residual recomputed in FP64.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

--impl reference times the FP64 CPU oracle (test infrastructure) on a bounded sample of the same workload.
"""
import argparse
import copy
import json
import os
import tempfile
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "sweep cell·angle updates/s; GMRES time to 1e-8 resid, mixed vs FP64 (1 GB300)"
UNIT = "cell-angle updates/s"
VARIANTS = ("std", "lm", "rlm")

# FP32 operations per cell-angle update in the sweep kernel (counted from the kernel source, FMA = 2;
# reciprocals count 1): standard Q1 block solve, low-memory row-0 solve + L-row reductions, reconstructed.
FLOPS_PER_UPDATE = {"std": 90, "lm": 31, "rlm": 55}

# One ncu capture of the FP32 non-storing sweep kernels (the lean instances GMRES runs) on the 512x512 S16
# profiling case (bench.py --profile), per scheme: DRAM bytes read + written per launch (the launch shape, hence the
# partial reductions per cell, is the same at 1024x1024, so a full launch moves 4x these), issue-active % of the
# schedulers, warps active % of the maximum, and warp instructions per cell-direction update.  None until measured
# for the current kernels; must be re-measured whenever the kernel changes.
SWEEP_NCU_512 = {"std": {"dram_bytes": 68.734464e6, "issue_active_pct": 42.42, "warps_active_pct": 23.08,
                         "inst_per_update": 5.008},
                 "lm": {"dram_bytes": 36.167168e6, "issue_active_pct": 22.94, "warps_active_pct": 11.56,
                        "inst_per_update": 2.642},
                 "rlm": {"dram_bytes": 109.970176e6, "issue_active_pct": 38.22, "warps_active_pct": 22.89,
                         "inst_per_update": 5.955}}
# the pipeline of the sweep: a strip of 32 rows takes n + 31 steps and the strip above starts 32 + 8 steps later
STRIP_LAG = 40


def workload_config():
    return {"workload": "1024x1024 cells, S16 level-symmetric (144 directions), sigma_s and sigma_a piecewise "
                        "constant on 16x16-cell patches ~ U[0.1,10] (seed 1907), q=1, eps=1, vacuum inflow; "
                        "per step one mixed-precision GMRES(30) solve to 1e-8 for each of Q1-DG, LMDG, RLMDG",
            "n": 1024, "directions": 144, "eps": 1.0, "restart": 30, "tol": 1e-8,
            "l2": "flushed between steps by a 512 MB write"}


def dist_setup(ngpus):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
        return rank, ws, dist
    return 0, 1, None


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    def __init__(self, idx):
        self.idx = idx
        self.proc = None
        out = os.environ.get("LMDG_BENCH_OUT", tempfile.gettempdir())
        self.path = os.path.join(out, f"clocks_rank{idx}.csv")

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={q}", "--format=csv",
                                          "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()
            self.f.close()

    def summary(self):
        try:
            lines = [l.strip() for l in open(self.path) if l.strip() and not l.startswith("index")]
        except Exception:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["clock sampling unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in lines:
            f = [x.strip() for x in l.split(",")]
            try:
                sm.append(float(f[1].split()[0]))
                smax = float(f[2].split()[0])
            except Exception:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def aggregate(total_ms, updates, dist):
    """Whole-job figures over the ranks: the timed region is the slowest rank's, the work is every rank's
    (weak scaling: each rank runs the full workload as an independent replica; no data-path collective)."""
    if dist is None:
        return total_ms, updates
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(updates)], dtype=torch.float64, device=dev)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def host_cpu():
    """(logical cores, model string) of this host."""
    model = None
    try:
        for line in open("/proc/cpuinfo"):
            k, _, v = line.partition(":")
            if k.strip() in ("model name", "Model Name"):
                model = v.strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                k, _, v = line.partition(":")
                if k.strip() == "Model name":
                    model = v.strip()
                    break
        except Exception:
            pass
    if model is None:
        import platform
        model = platform.machine() or "unknown"
    return os.cpu_count() or 1, model


def cpu_oracle_sample(p, per_variant=16, threads=None):
    """Oracle transport sweeps (its per-direction upwind solves) on a subset of the workload's directions:
    returns (cell-angle updates/s, cores, description)."""
    import numpy as np
    from concurrent.futures import ThreadPoolExecutor
    from oracle.sweeps import SweepOracle
    so = SweepOracle(p, threads=threads)
    cores = so.threads
    rng = np.random.default_rng(0)
    X = rng.standard_normal((p.nx, 4))
    step = max(1, p.nang // per_variant)
    angles = list(range(0, p.nang, step))[:per_variant]
    jobs = []
    for l in angles:
        jobs.append(lambda l=l: so.Linv(l, so.M(l, X) + so.Q(l)))
        jobs.append(lambda l=l: so.L00inv(l, so.M0(l, X[:, 0]) + so.L01SigT(l, X[:, 1:])))
        jobs.append(lambda l=l: so.Lt00inv(l, so.M0(l, X[:, 0]) + so.L01SigT(l, X[:, 1:])))
    t = time.perf_counter()
    with ThreadPoolExecutor(cores) as ex:
        list(ex.map(lambda f: f(), jobs))
    dt = time.perf_counter() - t
    ups = len(jobs) * p.nx
    desc = (f"oracle upwind sweeps (Q1 block, L00, Ltilde00 with reconstruction) for {len(angles)} of "
            f"{p.nang} directions each on the {p.n}x{p.n} mesh, {len(jobs)} sweeps on {cores} threads")
    return ups / dt, cores, desc, dt


def run_reference(args, rank, ws):
    if rank != 0:
        return 0
    from workloads.problems import config4
    p = config4(eps=1.0)
    nproc, model = host_cpu()
    for _ in range(args.warmup):
        cpu_oracle_sample(p, per_variant=2, threads=nproc)
    vals, times = [], []
    desc = cores = None
    for _ in range(args.steps):
        v, cores, desc, dt = cpu_oracle_sample(p, per_variant=4, threads=nproc)
        vals.append(v)
        times.append(dt)
    value = len(vals) / sum(1.0 / v for v in vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc,
                             "nproc": nproc, "cpu": model},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_gpu(args, rank, ws, dist):
    import numpy as np
    import torch
    from paper_1907_01027_gb300 import Context, FP32, FP64, FP32_BF16STORE, SWEEP_FP32, SWEEP_STORE, SWEEP_SOURCE
    from paper_1907_01027_gb300 import RESID_F32X2, RESID_FP64
    from paper_1907_01027_gb300 import buildlib
    from workloads.problems import config4

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    buildlib.build()
    p = config4(eps=1.0)
    upd = p.nx * p.nang
    ctxs = {v: Context(p, v, precision=FP32, resid=RESID_F32X2, tol=1e-8, device=local) for v in VARIANTS}
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def step(stats_acc=None):
        for v in VARIANTS:
            _, _, st, rc = ctxs[v].solve(want_x=False, want_phi=True, device=True)
            if rc != 0:
                raise RuntimeError(f"{v} solve did not converge: {st}")
            if stats_acc is not None:
                stats_acc.append((v, st))

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    stats = []
    durations = []
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.fill_(float(k))
            torch.cuda.synchronize()
            e0.record()
            step(stats)
            e1.record()
            torch.cuda.synchronize()
            durations.append(e0.elapsed_time(e1))
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    total_ms = sum(durations)
    sweeps = sum(st["sweeps_fp32"] + st["sweeps_fp64"] + st["sweeps_f32x2"] for _, st in stats)
    updates = sweeps * upd
    total_ms, updates = aggregate(total_ms, updates, dist)
    value = updates / (total_ms / 1e3)
    launches = sum(st["launches"] for _, st in stats)

    # roofline of the dominant kernel (the FP32 sweep inside the solves), live from the timed region
    f32_ms = sum(st["sweep_ms_fp32"] for _, st in stats)
    f32_n = sum(st["sweeps_fp32"] for _, st in stats)
    f64_ms = sum(st["sweep_ms_fp64"] for _, st in stats)
    f64_n = sum(st["sweeps_fp64"] for _, st in stats)
    f2_ms = sum(st["sweep_ms_f32x2"] for _, st in stats)
    f2_n = sum(st["sweeps_f32x2"] for _, st in stats)
    flops = sum(FLOPS_PER_UPDATE[v] * st["sweeps_fp32"] * upd for v, st in stats)
    fp32_peak = 152 * 128 * 2 * 2.07e9 / 1e12
    achieved = flops / (f32_ms / 1e3) / 1e12 if f32_ms > 0 else None
    scale = (p.n / 512) ** 2
    measured = all(SWEEP_NCU_512[v]["dram_bytes"] is not None for v in VARIANTS)
    traffic = (sum(SWEEP_NCU_512[v]["dram_bytes"] * scale * st["sweeps_fp32"] for v, st in stats) / max(1, f32_n)
               if measured else None)
    # the binding resource of the non-storing sweeps: instruction issue along the wavefront.  Critical path: the
    # dependent steps of the last strip, (n + 31) + STRIP_LAG (strips - 1); its time per step from the launch time
    strips = (p.n + 31) // 32
    cp_steps = (p.n + 31) + STRIP_LAG * (strips - 1)
    issue = {"critical_path_steps": cp_steps,
             "ns_per_step": (f32_ms / max(1, f32_n)) * 1e6 / cp_steps if f32_n else None,
             "issue_active_pct": {v: SWEEP_NCU_512[v]["issue_active_pct"] for v in VARIANTS},
             "warps_active_pct": {v: SWEEP_NCU_512[v]["warps_active_pct"] for v in VARIANTS},
             "warp_inst_per_update": {v: SWEEP_NCU_512[v]["inst_per_update"] for v in VARIANTS},
             "source": "issue and warp figures from one ncu capture of the 512x512 profiling case (bench.py "
                       "--profile), the kernels' launch shape being the same at 1024x1024"}
    roofline = {"bound": "alu", "kernel": "sweep_kernel<float> (all three schemes, non-storing)",
                "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": (achieved / fp32_peak) if achieved else None, "traffic": traffic,
                "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of the 512x512 profiling "
                                  "case, per scheme, scaled by the cell count and averaged over the timed "
                                  "launches",
                "peak_source": "FP32 CUDA-core peak from unit counts and clock: 152 SMs x 128 lanes x 2 x 2.07 GHz",
                "avg_launch_ms": f32_ms / max(1, f32_n), "launches": f32_n, "binding": issue,
                "flops_per_update": FLOPS_PER_UPDATE,
                "f32x2_sweep_avg_ms": f2_ms / max(1, f2_n), "f32x2_sweeps": f2_n,
                "fp64_sweep_avg_ms": f64_ms / max(1, f64_n) if f64_n else None, "fp64_sweeps": f64_n}
    clocks = clk.summary()

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None,
           "dtype": "f32 sweeps, f32x2 (float-float) residual sweeps, f64 refinement", "data": "synthetic",
           "config": workload_config(), "roofline": roofline, "clocks": clocks, "gpu_launches": launches}

    # time to 1e-8: mixed (from the timed region) vs FP64 (one solve each, after it)
    ttr = {}
    phis = {}
    for v in VARIANTS:
        mixed = [st for vv, st in stats if vv == v]
        ttr[v] = {"mixed_ms": sum(s["time_ms"] for s in mixed) / len(mixed),
                  "mixed_iters": mixed[-1]["iters"], "mixed_refinements": mixed[-1]["refinements"],
                  "mixed_sweeps_fp32": mixed[-1]["sweeps_fp32"], "mixed_sweeps_f32x2": mixed[-1]["sweeps_f32x2"],
                  "mixed_resid": mixed[-1]["resid"] / mixed[-1]["resid0"]}
        # the same solve's final residual recomputed with FP64 sweeps: ||K x - b'|| / ||b'||
        xs, phis[v], _, _ = ctxs[v].solve(want_x=True, want_phi=True, device=True)
        ttr[v]["mixed_kappa_est"] = mixed[-1]["kappa_est"]
        r = ctxs[v].sweep(xs, flags=SWEEP_SOURCE)
        b = ctxs[v].sweep(torch.zeros_like(xs), flags=SWEEP_SOURCE)
        ttr[v]["mixed_resid_fp64_check"] = float(torch.linalg.norm(r) / torch.linalg.norm(b))
        # the mixed solver with FP64 residual sweeps
        ctx = Context(p, v, precision=FP32, resid=RESID_FP64, tol=1e-8, device=local)
        ctx.solve(want_x=False, want_phi=True, device=True)
        torch.cuda.synchronize()
        e0.record()
        _, _, st, rc = ctx.solve(want_x=False, want_phi=True, device=True)
        e1.record()
        torch.cuda.synchronize()
        ttr[v].update({"mixed_fp64resid_ms": e0.elapsed_time(e1), "mixed_fp64resid_status": rc,
                       "mixed_fp64resid_sweeps_fp64": st["sweeps_fp64"],
                       "fp64_residual_sweep_avg_ms": st["sweep_ms_fp64"] / max(1, st["sweeps_fp64"]),
                       "f32x2_residual_sweep_avg_ms": mixed[-1]["sweep_ms_f32x2"] /
                       max(1, mixed[-1]["sweeps_f32x2"])})
        ctx.close()
    if not args.skip_fp64:
        for v in VARIANTS:
            ctx = Context(p, v, precision=FP64, tol=1e-8, device=local)
            torch.cuda.synchronize()
            e0.record()
            _, phi64, st, rc = ctx.solve(want_x=False, want_phi=True, device=True)
            e1.record()
            torch.cuda.synchronize()
            # error of the mixed solution against the FP64 one, and the bound the solves' kappa_est states: two
            # solutions with relative residuals below tol differ by at most about 2 kappa tol in the unknowns GMRES
            # sees, u = M^-1 x (M the right preconditioner: the identity for Q1-DG, so there the bound is on phi;
            # the Jacobi scaling of the slope block for LMDG and RLMDG, whose phi differences it does not bound)
            kap = max(st["kappa_est"], ttr[v]["mixed_kappa_est"])
            ttr[v].update({"fp64_ms": e0.elapsed_time(e1), "fp64_iters": st["iters"], "fp64_status": rc,
                           "fp64_sweep_avg_ms": st["sweep_ms_fp64"] / max(1, st["sweeps_fp64"]),
                           "fp64_kappa_est": st["kappa_est"],
                           "mixed_vs_fp64_phi_rel": float(torch.linalg.norm(phis[v] - phi64) /
                                                          torch.linalg.norm(phi64)),
                           "bound_2_kappa_tol_preconditioned_unknowns": 2 * kap * 1e-8})
            ctx.close()
    out["gmres_time_to_1e-8"] = ttr

    # storing sweeps (recovery): HBM roofline of the FP32 sweeps that write the angular unknowns -- Q1-DG psi
    # (16 B per update), LMDG psi0 in FP32 (4 B) and in bfloat16 (2 B)
    hbm = peaks().get("hbm_gbs")
    x = torch.randn(p.nx, 4, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    e2 = torch.cuda.Event(enable_timing=True)
    e3 = torch.cuda.Event(enable_timing=True)

    def storing(c, psi_bytes, kernel):
        for _ in range(3):
            c.sweep(x, y, flags=SWEEP_FP32 | SWEEP_STORE | SWEEP_SOURCE)
        torch.cuda.synchronize()
        reps = 5
        e0.record()
        for _ in range(reps):
            flush.fill_(1.0)
            c.sweep(x, y, flags=SWEEP_FP32 | SWEEP_STORE | SWEEP_SOURCE)
        e1.record()
        torch.cuda.synchronize()
        e2.record()
        for _ in range(reps):
            flush.fill_(1.0)
        e3.record()
        torch.cuda.synchronize()
        ms = (e0.elapsed_time(e1) - e2.elapsed_time(e3)) / reps
        nbytes = upd * psi_bytes + p.nx * (32 + 4 * 3 + 16) + p.nx * 32
        ach = nbytes / (ms / 1e3) / 1e9
        return {"bound": "hbm", "kernel": kernel, "achieved": ach, "peak": hbm, "unit": "GB/s",
                "frac": ach / hbm if hbm else None, "ms": ms, "algorithmic_bytes": nbytes,
                "psi_bytes_per_update": psi_bytes, "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"}

    bf = Context(p, "lm", precision=FP32_BF16STORE, device=local)
    out["roofline_storing_sweep"] = storing(ctxs["std"], 16, "sweep_kernel<float, Q1-DG, store> + epilogue")
    out["roofline_storing_sweeps"] = {
        "std_fp32": out["roofline_storing_sweep"],
        "lm_fp32": storing(ctxs["lm"], 4, "sweep_kernel<float, LMDG, store psi0 fp32> + epilogue"),
        "lm_bf16": storing(bf, 2, "sweep_kernel<float, LMDG, store psi0 bf16> + epilogue")}
    bf.close()

    # diffusive regime: the same workload at eps = 1e-3, GMRES right-preconditioned by the vertex diffusion
    # correction (precond = 2), time to 1e-8 with FP32 sweeps and FP64 residual sweeps against the FP64 solver
    if not args.skip_diffusive:
        out["gmres_time_to_1e-8_eps1e-3"] = diffusive_times(args, local)
    if not args.skip_configs:
        out["other_configs"] = other_configs(local)

    # end to end through the public API with host buffers: setup from host arrays, solve, phi back to host; the
    # host arrays (the problem's cross sections, source and quadrature, and phi) live in pinned memory
    def pinned(a):
        t = torch.empty(np.shape(a), dtype=torch.float64, pin_memory=True).numpy()
        t[...] = a
        return t
    ph = copy.copy(p)
    for f in ("ox", "oy", "w", "sigma_s", "sigma_a", "q"):
        setattr(ph, f, pinned(getattr(p, f)))
    phi_h = {v: pinned(np.zeros((p.nx, 4))) for v in VARIANTS}
    e2e_ms, e2e_upd = 0.0, 0
    part_ms = {"setup": 0.0, "solve": 0.0, "destroy": 0.0}
    h2d = d2h = 0
    for k in range(max(1, args.steps)):
        for v in VARIANTS:
            t0 = time.perf_counter()
            ctx = Context(ph, v, precision=FP32, resid=RESID_F32X2, tol=1e-8, device=local)
            t1 = time.perf_counter()
            _, phi, st, rc = ctx.solve(want_x=False, want_phi=True, device=False, phi_out=phi_h[v])
            t2 = time.perf_counter()
            ctx.close()
            torch.cuda.synchronize()
            t3 = time.perf_counter()
            e2e_ms += 1e3 * (t3 - t0)
            part_ms["setup"] += 1e3 * (t1 - t0)
            part_ms["solve"] += 1e3 * (t2 - t1)
            part_ms["destroy"] += 1e3 * (t3 - t2)
            e2e_upd += (st["sweeps_fp32"] + st["sweeps_fp64"] + st["sweeps_f32x2"]) * upd
            if k == 0:
                h2d += 8 * (3 * p.nang + 2 * p.nx + 4 * p.nx)
                d2h += phi.nbytes
    out["e2e"] = {"value": e2e_upd / (e2e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                  "d2h_bytes_per_step": d2h,
                  "what": "lmdg_setup from pinned host arrays + lmdg_solve (LMDG_HOST_PTRS, phi to a pinned host "
                          "array) + destroy, three schemes per step",
                  "ms_per_step": {k: t / max(1, args.steps) for k, t in part_ms.items()}}

    if rank == 0 and ws == 1 and not args.skip_cpu:
        nproc, model = host_cpu()
        v, cores, desc, dt = cpu_oracle_sample(p, per_variant=16, threads=nproc)
        v1, _, desc1, dt1 = cpu_oracle_sample(p, per_variant=2, threads=1)
        out["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc,
                               "seconds": dt, "nproc": nproc, "cpu": model,
                               "one_thread": {"value": v1, "sample": desc1, "seconds": dt1}}
    if rank == 0:
        print(json.dumps(out), flush=True)
    for c in ctxs.values():
        c.close()
    return 0


# iteration caps of the eps = 1e-3 solves (GMRES iterations, all refinement steps)
DIFFUSIVE_MAX_ITERS = {"std": 2000, "lm": 3000, "rlm": 1500}
# lmdg_options.precond of the eps = 1e-3 solves: 2 (vertex correction) or 3 (with the cell-block step); measured at
# 1024^2 S16 mixed: Q1-DG 68 / 72 iterations, LMDG 227 / 210, RLMDG 1350 / 1200
DIFFUSIVE_PRECOND = {"std": 2, "lm": 3, "rlm": 3}


def diffusive_times(args, local):
    """Time to 1e-8 at eps = 1e-3 on the 1024^2 S16 patch medium (sigma_t h from 0.1 to 10): per scheme the mixed
    solver (FP32 sweeps, FP64 residual sweeps, FP64 refinement) and the FP64 solver, both with the vertex diffusion
    correction (DIFFUSIVE_PRECOND: with the cell-block step for LMDG and RLMDG, which takes fewer iterations there,
    without it for Q1-DG, which takes more), one timed solve each after the context's workspace is allocated."""
    import numpy as np
    import torch
    from paper_1907_01027_gb300 import Context, FP32, FP64, RESID_FP64
    from workloads.problems import config4
    p = config4(eps=1e-3)
    res = {}
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for v in VARIANTS:
        res[v] = {}
        for mode, kw in (("mixed", dict(precision=FP32, resid=RESID_FP64)), ("fp64", dict(precision=FP64))):
            if args.skip_fp64 and mode == "fp64":
                continue
            ctx = Context(p, v, precond=DIFFUSIVE_PRECOND[v], tol=1e-8, max_iters=DIFFUSIVE_MAX_ITERS[v],
                          device=local, **kw)
            ctx.precond_apply(np.zeros((p.nx, 4)))          # allocates the Krylov workspace outside the timing
            torch.cuda.synchronize()
            e0.record()
            _, _, st, rc = ctx.solve(want_x=False, want_phi=True, device=True)
            e1.record()
            torch.cuda.synchronize()
            res[v][mode] = {"ms": e0.elapsed_time(e1), "status": rc, "precond": DIFFUSIVE_PRECOND[v],
                            "iters": st["iters"],
                            "refinements": st["refinements"], "resid": st["resid"] / st["resid0"],
                            "sweeps_fp32": st["sweeps_fp32"], "sweeps_fp64": st["sweeps_fp64"],
                            "sweep_ms_fp32": st["sweep_ms_fp32"], "sweep_ms_fp64": st["sweep_ms_fp64"]}
            ctx.close()
    res["note"] = ("status 0: converged to 1e-8; -5: iteration cap reached (resid is then the relative residual "
                   "reached)")
    return res


def other_configs(local):
    """The workload configurations besides the benchmark's own, timed on the GPU (one solve each after a warm-up
    solve in the same context; CUDA events): the 32^2 S4 FP64 case to 1e-10 (GMRES; source iteration is not
    built), the 256^2 S8 diffusion-limit sweep (Q1-DG against LMDG, FP64, to 1e-8; the vertex correction with the
    cell-block step for eps < 1), the 512^2 S12 block medium (RLMDG, FP64 and mixed to 1e-8) and the adjoint
    workload (256^2 S8 bumps: Q1-DG and LMDG gradients, FP64 and mixed)."""
    import numpy as np
    import torch
    from paper_1907_01027_gb300 import Context, FP32, FP64, RESID_F32X2
    from workloads.problems import config1, config2, config3, config5
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    def timed_solve(p, variant, **kw):
        ctx = Context(p, variant, device=local, **kw)
        ctx.solve(want_x=False, want_phi=True, device=True)
        torch.cuda.synchronize()
        e0.record()
        _, _, st, rc = ctx.solve(want_x=False, want_phi=True, device=True)
        e1.record()
        torch.cuda.synchronize()
        ctx.close()
        return {"ms": e0.elapsed_time(e1), "status": rc, "iters": st["iters"], "resid": st["resid"] / st["resid0"],
                "updates_per_s": (st["sweeps_fp64"] + st["sweeps_fp32"] + st["sweeps_f32x2"]) * p.nx * p.nang /
                (e0.elapsed_time(e1) / 1e3)}

    out = {}
    p1 = config1()
    out["32x32_S4_fp64_to_1e-10"] = {v: timed_solve(p1, v, precision=FP64, tol=1e-10) for v in VARIANTS}
    out["256x256_S8_fp64_to_1e-8"] = {}
    for eps in (1.0, 1e-2, 1e-4):
        p2 = config2(eps=eps)
        kw = dict(precision=FP64, tol=1e-8, max_iters=3000)
        if eps < 1:
            kw["precond"] = 3
        out["256x256_S8_fp64_to_1e-8"][f"eps={eps:g}"] = {v: timed_solve(p2, v, **kw) for v in ("std", "lm")}
    p3 = config3()
    out["512x512_S12_blocks_rlm_to_1e-8"] = {
        "fp64": timed_solve(p3, "rlm", precision=FP64, tol=1e-8, max_iters=5000),
        "mixed": timed_solve(p3, "rlm", precision=FP32, resid=RESID_F32X2, tol=1e-8, max_iters=5000)}
    p5 = config5()
    g = np.ascontiguousarray(p5.info["detector"])
    adj = {}
    for v in ("std", "lm"):
        for mode, kw in (("fp64", dict(precision=FP64)), ("mixed", dict(precision=FP32))):
            ctx = Context(p5, v, tol=1e-10, device=local, **kw)
            ctx.adjoint(g)
            t = time.perf_counter()
            J, _, _, _, st = ctx.adjoint(g)
            adj[f"{v}_{mode}"] = {"ms": 1e3 * (time.perf_counter() - t), "J": J, "iters": st["iters"]}
            ctx.close()
    out["256x256_S8_adjoint_gradients"] = adj
    return out


def run_profile(args):
    """Small case for ncu: 512x512 cells, S16, the bench media; per pass the three FP32 non-storing sweeps (as
    inside GMRES: Q1-DG, LMDG, RLMDG), an FP32 Q1-DG storing sweep (psi 604 MB, larger than L2), the three
    FP64 source sweeps (the refinement residual of LMDG_RESID_FP64) and the three float-float source sweeps (that
    of LMDG_RESID_F32X2); two rounds (sweep kernels 1-10 untimed, 11-20 for the capture)."""
    import torch
    from paper_1907_01027_gb300 import Context, FP32, SWEEP_FP32, SWEEP_STORE, SWEEP_SOURCE, SWEEP_F32X2
    from workloads.problems import config4
    torch.cuda.set_device(0)
    p = config4(eps=1.0, n=512)
    ctx = {v: Context(p, v, precision=FP32) for v in ("std", "lm", "rlm")}
    x = torch.randn(p.nx, 4, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    for _ in range(2):
        for v in ("std", "lm", "rlm"):
            ctx[v].sweep(x, y, flags=SWEEP_FP32)
        ctx["std"].sweep(x, y, flags=SWEEP_FP32 | SWEEP_STORE | SWEEP_SOURCE)
        for v in ("std", "lm", "rlm"):
            ctx[v].sweep(x, y, flags=SWEEP_SOURCE)
        for v in ("std", "lm", "rlm"):
            ctx[v].sweep(x, y, flags=SWEEP_SOURCE | SWEEP_F32X2)
        torch.cuda.synchronize()
    for c in ctx.values():
        c.close()
    print("profile case done", flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300")
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-diffusive", action="store_true", help="leave out the eps = 1e-3 solves")
    ap.add_argument("--skip-configs", action="store_true", help="leave out the other workload configurations")
    ap.add_argument("--profile", action="store_true", help="small fixed case for ncu captures")
    args = ap.parse_args()
    if args.profile:
        return run_profile(args)
    if args.warmup < 3:
        args.warmup = 3
    rank, ws, dist = dist_setup(args.gpus)
    try:
        if args.impl == "reference":
            return run_reference(args, rank, ws)
        return run_gpu(args, rank, ws, dist)
    finally:
        if dist:
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
