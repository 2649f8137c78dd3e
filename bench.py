#!/usr/bin/env python
"""Time-to-solution benchmark of the GB300 sweeping preconditioner.

Workload: the 100^3 converging-lens problem, c(x) = 1 - 0.4 exp(-32 |x - 0.5|^2), omega for 10
points per minimum wavelength, PML of 8 points on all faces, 4-plane panels padded with 8 PML
planes, nested-dissection leaf 64, one Gaussian shot (sigma = 2h) at (0.5, 0.5, 0.1), GMRES(20) to
a relative residual of 1e-5, complex128 on the GPU.  One step = the whole hot path on one problem:
setup (factor every panel) + GMRES solve to 1e-5 (all preconditioner applications and matvecs).

One JSON line is printed by rank 0.  Before the timed region the library's sweep autotuner picks
the sweep schedule once per precision (`--no-tune` keeps the defaults).  The line also carries
the complex64 path on the same workload (`mixed`; `--no-mixed` skips it) and the CPU oracle's
extrapolated time (`cpu_baseline`; `--no-cpu-baseline` skips it).  `--workload batch16` prints the
same kind of line for 16 independent problems of uneven size in one batched handle instead.
`--impl reference` times the complex128 CPU oracle on a bounded sample of the default workload
(see `reference_main`).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GMRES solve time & iters to 1e-5; front TFLOP/s; sweep GB/s; mixed vs FP64"
UNIT = "solves/s"          # problems taken from c(x) and f to a solution at 1e-5 (setup + GMRES) per second
WORKLOAD = "lens100"
FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12   # SMs x FP64 flop/clk/SM (2 FMA) x max SM clock


GRID_N = 100


def workload():
    from paper_1204_0111_gb300 import workloads as wl
    return wl.cube_lens(GRID_N)


def config_dict(w, nrhs, extra=None):
    d = {"workload": f"{WORKLOAD}: {w.n}^3 converging lens, gamma {w.gamma}, panels of {w.panel_depth} + pad {w.pad}, "
                     f"leaf {w.leaf}, {nrhs} shot, GMRES({w.k}) to {w.tol:g}",
         "n": w.n, "N": w.N, "omega": w.omega, "pml_gamma": w.gamma, "panel_depth": w.panel_depth, "pad": w.pad,
         "leaf": w.leaf, "nrhs": nrhs, "gmres_k": w.k, "tol": w.tol,
         "l2": "inputs larger than L2 (factors of ~15 GB stream per apply)"}
    if extra:
        d.update(extra)
    return d


# ---------------------------------------------------------------------------------------------
# CPU oracle sample (run in a spawned process so that BLAS threading and CUDA state stay clean)
# ---------------------------------------------------------------------------------------------
def _oracle_sample(args):
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    os.environ["OMP_NUM_THREADS"] = "1"
    sys.path.insert(0, ROOT)
    import numpy as np

    from oracle import discretize as dz
    from oracle import multifrontal as mf
    from oracle import panels as pn
    from oracle import symbolic as sy
    w = workload()
    p = dz.Helmholtz(w.c, w.h, w.omega, w.gamma, w.pml_C, w.alpha)
    plan = pn.panel_plan(p.nz, p.gamma, w.panel_depth)
    z0, z1 = plan[1]
    t0 = time.perf_counter()
    ap = pn.aux_problem(p, z0, z1, w.pad)
    sym = sy.nested_dissection(ap.nx, ap.ny, ap.depth, w.leaf)
    fr = mf.factor(ap.H, sym)
    t1 = time.perf_counter()
    v = np.zeros(ap.H.shape[0], dtype=np.complex128)
    v[ap.lead * p.nx * p.ny:] = w.rhs()[0][z0 * p.nx * p.ny:z1 * p.nx * p.ny]
    mf.solve(fr, sym, v)
    t2 = time.perf_counter()
    A = dz.operator_A(p)
    x = w.rhs()[0]
    t3 = time.perf_counter()
    A @ x
    t4 = time.perf_counter()
    return {"t_factor": t1 - t0, "t_T": t2 - t1, "t_matvec": t4 - t3, "m": len(plan)}


def oracle_estimate(iters, k=20):
    """Seconds per solve of the oracle, extrapolated from a one-panel sample: m panel factorisations,
    iters x (2m - 1) panel solves plus iters + restarts true-residual matvecs; Arnoldi (k^2 N) is
    counted from the measured matvec rate as 8 vector passes per matvec-equivalent."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Pool(1) as pool:
        s = pool.apply(_oracle_sample, ((),))
    m = s["m"]
    t_setup = m * s["t_factor"]
    t_apply = (2 * m - 1) * s["t_T"]
    t_mv = s["t_matvec"]
    restarts = max(1, math.ceil(iters / k))
    t_solve = iters * (t_apply + t_mv) + restarts * t_mv + iters * (iters + 1) / 2 / 4 * t_mv
    total = t_setup + t_solve
    sample = (f"one {w_desc()} panel factorisation ({s['t_factor']:.2f} s) + one panel solve ({s['t_T']:.3f} s) + "
              f"one sparse matvec ({s['t_matvec']:.4f} s), single thread, extrapolated to m={m} panels, "
              f"{iters} GMRES iterations")
    return total, sample, s


def w_desc():
    return f"{GRID_N}x{GRID_N}x12"


def cpu_cores():
    return os.cpu_count() or 1


# ---------------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_uuid=None):
        self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if device_uuid:
            cmd += ["-i", device_uuid]
        try:
            self.p = subprocess.Popen(cmd, stdout=self.tmp, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is not None:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
        self.tmp.flush()
        self.tmp.seek(0)
        rows = [r.strip().split(",") for r in self.tmp.read().splitlines() if r.strip()]
        os.unlink(self.tmp.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def traffic_from_profiles(kernel):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        kv = dict(t.split("=", 1) for t in line.split() if "=" in t)
        if kv.get("kernel") != kernel or kv.get("workload") != WORKLOAD:
            continue
        src = os.path.join(ROOT, "paper_1204_0111_gb300", "csrc", kv.get("source", ""))
        if not os.path.exists(src):
            return None
        if hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] != kv.get("sha", ""):
            return None
        return float(kv["bytes_per_launch"])
    return None


SETUP_KERNELS = ("k_assemble", "k_diag_ldlt", "k_panel_right", "k_panel_left", "k_gemm", "k_copy_linv", "k_tc_gemm",
                 "k_tc_pack", "k_scale_zd")
SWEEP_KERNELS = ("k_sweep", "k_solve_fwd", "k_solve_bwd")


def max_over_ranks(x, device=None):
    """The largest value of a per-rank float over all ranks (the slowest rank's time); the value
    itself when no process group is running."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, units_per_rank, seconds_max):
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return world * units_per_rank / seconds_max


def _agg(stat_list):
    agg = {}
    for st in stat_list:
        for k, v in st.items():
            g = agg.setdefault(k, {"launches": 0, "total_ms": 0.0, "flops": 0.0, "bytes": 0.0})
            for f in g:
                g[f] += v[f]
    return agg


def kernel_table(stats):
    return {k: {"launches": v["launches"], "ms_per_step": v["total_ms"],
                "tflops": v["flops"] / max(v["total_ms"], 1e-9) / 1e9,
                "gbs": v["bytes"] / max(v["total_ms"], 1e-9) / 1e6} for k, v in sorted(stats.items())}


def summarize(stats_timed, stats_full, infos, factor_bytes, steps):
    """Roofline of the dominant kernel and the per-kernel detail from psp_stats records.

    stats_timed: one record per timed step (setup kernels timed with CUDA events);
    stats_full: one step with every launch timed (kernel-time shares)."""
    agg = _agg(stats_timed)
    host = {k[5:]: v["total_ms"] / steps for k, v in agg.items() if k.startswith("host:")}
    agg = {k: v for k, v in agg.items() if not k.startswith("host:")}
    full = {k: v for k, v in stats_full.items() if not k.startswith("host:")}
    launches = int(sum(v["launches"] for v in agg.values()))
    tot_all = sum(v["total_ms"] for v in full.values()) or 1.0
    top_name = max(full.items(), key=lambda kv: kv[1]["total_ms"])[0]
    if agg.get(top_name, {}).get("total_ms", 0) > 0:
        tk, tv = top_name, agg[top_name]
    else:
        tk, tv = max(agg.items(), key=lambda kv: kv[1]["total_ms"])
    achieved = tv["flops"] / max(tv["total_ms"] * 1e-3, 1e-12) / 1e12
    roofline = {"kernel": tk, "bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic_from_profiles(tk),
                "peak_source": "FP64 CUDA-core peak derived: 152 SMs x 4 flop/clk x 2.07 GHz (complex128 path)",
                "kernel_share": full.get(tk, {"total_ms": 0.0})["total_ms"] / tot_all,
                "timing": "achieved from CUDA events around every launch of this kernel inside the timed region; "
                          "share from one fully instrumented step after it"}
    setup_ms = sum(v["total_ms"] for k, v in agg.items() if k in SETUP_KERNELS) / steps
    setup_flops = sum(v["flops"] for k, v in agg.items() if k in SETUP_KERNELS)
    sweep = [v for k, v in full.items() if k in SWEEP_KERNELS]
    sweep_ms = sum(v["total_ms"] for v in sweep)
    sweep_bytes = sum(v["bytes"] for v in sweep)
    applies = max(infos[-1]["applies"], 1)
    detail = {
        "gmres_iters": infos[-1]["iterations"],
        "relres": max(i["relres_max"] for i in infos),
        "setup_kernel_ms": setup_ms,
        "solve_wall_ms": statistics.mean(i["solve_ms"] for i in infos),
        "apply_ms": sweep_ms / applies,
        "front_tflops": setup_flops / max(setup_ms * steps * 1e-3, 1e-12) / 1e12,
        "sweep_gbs": sweep_bytes / max(sweep_ms * 1e-3, 1e-12) / 1e9,
        "factor_bytes": factor_bytes,
        "host_setup_ms": host,
        "kernels": kernel_table(full),
    }
    return roofline, detail, launches


# ---------------------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------------------
def gpu_main(a):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1204_0111_gb300 import psp

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    w = workload()
    nrhs = 1
    c_dev = torch.from_numpy(w.c).to(dev)
    f_host = w.rhs()
    f_dev = torch.from_numpy(f_host).to(dev)
    u_dev = torch.zeros_like(f_dev)
    stream = torch.cuda.current_stream(dev)

    sched = {}

    def step(precision="c128", stats=0):
        P = psp.SweepingPreconditioner(c_dev, w.h, w.omega, w.gamma, w.panel_depth, pad=w.pad, leaf=w.leaf,
                                       pml_C=w.pml_C, alpha=w.alpha, precision=precision, collect_stats=stats,
                                       **sched.get(precision, {}))
        info = P.solve(f_dev, u_dev, tol=w.tol, k=w.k, maxit=400)
        st = P.stats() if stats else None
        fb = P.info()["factor_bytes"]
        P.close()
        return info, st, fb

    def barrier():
        if world > 1:
            dist.barrier()

    # sweep schedule from the library's autotuner, once per precision, before any timed work
    tuning = {}
    for prec in () if a.no_tune else ("c128",) + (() if a.no_mixed else ("c64",)):
        P = psp.SweepingPreconditioner(c_dev, w.h, w.omega, w.gamma, w.panel_depth, pad=w.pad, leaf=w.leaf,
                                       pml_C=w.pml_C, alpha=w.alpha, precision=prec)
        t = P.tune_sweep(nrhs=nrhs, reps=3)
        P.close()
        tuning[prec] = t
        sched[prec] = {"sweep_level_tasks": t["sweep_level_tasks"], "sweep_ctas_per_sm": t["sweep_ctas_per_sm"],
                       "sweep_rhs_group": t["sweep_rhs_group"]}
    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        uuid = None
    clocks = ClockSampler(uuid)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    infos, stats_all = [], []
    fbytes = 0
    for _ in range(a.steps):
        info, st, fbytes = step(stats=2)      # CUDA events around the setup kernels only
        infos.append(info)
        stats_all.append(st)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    ms_max = max_over_ranks(ms, dev)
    value = job_rate(world, a.steps, ms_max / 1e3)

    _, full_st, _ = step(stats=1)       # one extra step, every launch timed, after the timed region
    roofline, detail, launches = summarize(stats_all, full_st, infos, fbytes, a.steps)

    # end to end through the public API with pinned host buffers (copies inside the timed region)
    c_pin = torch.from_numpy(w.c).pin_memory()
    f_pin = torch.from_numpy(f_host).pin_memory()
    u_pin = torch.zeros_like(f_pin).pin_memory()
    e2e_steps = max(1, min(a.steps, 2))
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        P = psp.SweepingPreconditioner(c_pin, w.h, w.omega, w.gamma, w.panel_depth, pad=w.pad, leaf=w.leaf,
                                       pml_C=w.pml_C, alpha=w.alpha, **sched.get("c128", {}))
        P.solve(f_pin, u_pin, tol=w.tol, k=w.k, maxit=400)
        P.close()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    e2e = {"value": job_rate(world, e2e_steps, max_over_ranks(t1 - t0, dev)), "unit": UNIT,
           "h2d_bytes_per_step": int(c_pin.numel() * 8 + f_pin.numel() * 16),
           "d2h_bytes_per_step": int(u_pin.numel() * 16)}

    # mixed precision (complex64 fronts and sweeps, complex128 GMRES) on the same workload
    mixed = None
    if not a.no_mixed:
        step("c64")
        torch.cuda.synchronize()
        m0 = torch.cuda.Event(enable_timing=True)
        m1 = torch.cuda.Event(enable_timing=True)
        msteps = max(1, min(a.steps, 3))
        m0.record(stream)
        minfo = None
        mstats = []
        for _ in range(msteps):
            minfo, mst, _ = step("c64", stats=2)
            mstats.append(mst)
        m1.record(stream)
        torch.cuda.synchronize()
        mms = m0.elapsed_time(m1) / msteps
        _, mfull, _ = step("c64", stats=1)      # instrumented step, outside the timed region
        mhost = {k[5:]: v["total_ms"] for k, v in mfull.items() if k.startswith("host:")}
        mfull = {k: v for k, v in mfull.items() if not k.startswith("host:")}
        magg = _agg(mstats)
        # apply error of the complex64 preconditioner against the complex128 one
        P128 = psp.SweepingPreconditioner(c_dev, w.h, w.omega, w.gamma, w.panel_depth, pad=w.pad, leaf=w.leaf)
        P64 = psp.SweepingPreconditioner(c_dev, w.h, w.omega, w.gamma, w.panel_depth, pad=w.pad, leaf=w.leaf,
                                         precision="c64")
        g = torch.Generator(device="cpu").manual_seed(0)
        r = torch.complex(torch.randn(w.N, generator=g, dtype=torch.float64),
                          torch.randn(w.N, generator=g, dtype=torch.float64)).reshape(1, -1).to(dev)
        o128 = torch.empty_like(r)
        o64 = torch.empty_like(r)
        P128.apply(r, o128)
        P64.apply(r, o64)
        torch.cuda.synchronize()
        err = float(torch.linalg.norm(o64 - o128) / torch.linalg.norm(o128))
        P128.close()
        P64.close()
        mixed = {"value": 1e3 / mms, "unit": UNIT, "ms_per_step": mms, "gmres_iters": minfo["iterations"],
                 "relres": minfo["relres_max"], "apply_rel_err_vs_c128": err,
                 "speedup_vs_c128": (ms_max / a.steps) / mms, "dtype": "c64 fronts/sweeps, f64 GMRES",
                 "setup_kernel_ms": sum(v["total_ms"] for k, v in magg.items() if not k.startswith("host:")) / msteps,
                 "host_setup_ms": mhost,
                 "kernels": kernel_table(mfull)}

    if rank == 0:
        cpu = None
        if not a.no_cpu_baseline:
            t_cpu, sample, _ = oracle_estimate(detail["gmres_iters"], w.k)
            cpu = {"value": 1.0 / t_cpu, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                   "seconds_per_solve": t_cpu}
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": ms_max / a.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": config_dict(w, nrhs, {"parallelism": f"replicas x{world}" if world > 1 else "single GPU"}),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches // a.steps,
                "clocks": clk, "detail": dict(detail, sweep_tuning=tuning), "mixed": mixed}
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------------------------
# batching workload: 16 independent problems of uneven size in one handle (not the default line)
# ---------------------------------------------------------------------------------------------
BATCH_UNIT = "batch solves/s"   # all 16 problems x 8 shots from c(x) and f to 1e-5 (setup + GMRES) per second


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        return json.load(open(path)), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def roofline_generic(name, v, share, timing):
    """Roofline line for one kernel of the complex64 path from its psp_stats record."""
    pk, src = _peaks()
    ms = max(v["total_ms"], 1e-9)
    if name == "k_tc_gemm":
        peak = pk["bf16_tflops"] * 1.1 / 2.25     # TF32 dense = bf16 x the nominal 1.1 / 2.25 ratio
        ach = v["flops"] / ms / 1e9
        return {"kernel": name, "bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "traffic": None, "kernel_share": share, "timing": timing,
                "peak_source": f"TF32 dense from the {src} bf16 peak x 1.1/2.25; achieved counts useful complex "
                               "flops (8 per complex MAC), the split-TF32 3M scheme executes 18 per 8"}
    if name in ("k_sweep", "k_assemble", "k_tc_pack", "k_matvec", "k_multiaxpy"):
        peak = pk["hbm_gbs"]
        ach = v["bytes"] / ms / 1e6
        return {"kernel": name, "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                "frac": ach / peak, "traffic": None, "kernel_share": share, "timing": timing,
                "peak_source": f"{src} HBM copy bandwidth"}
    peak = 152 * 128 * 2 * 2.07e9 / 1e12          # FP32 lanes x FMA x max SM clock
    ach = v["flops"] / ms / 1e9
    return {"kernel": name, "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
            "traffic": None, "kernel_share": share, "timing": timing,
            "peak_source": "FP32 CUDA-core peak derived: 152 SMs x 128 lanes x 2 flop x 2.07 GHz"}


def batch_main(a):
    import numpy as np
    import torch

    from paper_1204_0111_gb300 import psp
    from paper_1204_0111_gb300 import workloads as wl

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    ws = [wl.cube_smooth(k) for k in range(16)]
    nrhs = 8
    prs = [dict(c=torch.from_numpy(w.c).to(dev), h=w.h, omega=w.omega, gamma=w.gamma, panel_depth=w.panel_depth)
           for w in ws]
    f_host = np.concatenate([w.rhs().reshape(-1) for w in ws])
    f_dev = torch.from_numpy(f_host).to(dev)
    u_dev = torch.zeros_like(f_dev)
    stream = torch.cuda.current_stream(dev)

    pml_C = ws[0].pml_C        # one PML amplitude for the whole batch (the same for every problem)
    B = psp.SweepingPreconditionerBatch(prs, precision="c64", pml_C=pml_C)
    tuning = B.tune_sweep(nrhs=nrhs, reps=2)     # the library's autotuner, before any timed work
    B.close()
    sched = {"sweep_level_tasks": tuning["sweep_level_tasks"], "sweep_ctas_per_sm": tuning["sweep_ctas_per_sm"],
             "sweep_rhs_group": tuning["sweep_rhs_group"], "pml_C": pml_C}

    def step(stats=0, problems=prs, f=f_dev, u=u_dev):
        B = psp.SweepingPreconditionerBatch(problems, precision="c64", collect_stats=stats, **sched)
        info = B.solve(f, u, tol=1e-5, k=20, maxit=400)
        st = B.stats() if stats else None
        fb = B.info()["factor_bytes"]
        B.close()
        return info, st, fb

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    infos, stats_all = [], []
    fbytes = 0
    for _ in range(a.steps):
        info, st, fbytes = step(stats=2)
        infos.append(info)
        stats_all.append(st)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    _, full_st, _ = step(stats=1)
    agg = {k: v for k, v in _agg(stats_all).items() if not k.startswith("host:")}
    full = {k: v for k, v in full_st.items() if not k.startswith("host:")}
    tot = sum(v["total_ms"] for v in full.values()) or 1.0
    top = max(full.items(), key=lambda kv: kv[1]["total_ms"])[0]
    if agg.get(top, {}).get("total_ms", 0) > 0:
        roof = roofline_generic(top, agg[top], full[top]["total_ms"] / tot,
                                "CUDA events around every launch of this kernel inside the timed region")
    else:
        roof = roofline_generic(top, full[top], full[top]["total_ms"] / tot,
                                "CUDA events around every launch in one instrumented step after the timed region")
    # end to end with pinned host buffers
    c_pin = [torch.from_numpy(w.c).pin_memory() for w in ws]
    f_pin = torch.from_numpy(f_host).pin_memory()
    u_pin = torch.zeros_like(f_pin).pin_memory()
    prs_h = [dict(p, c=cp) for p, cp in zip(prs, c_pin)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    step(problems=prs_h, f=f_pin, u=u_pin)
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    sizes = [w.n for w in ws]
    line = {"metric": METRIC, "value": a.steps / (ms / 1e3), "unit": BATCH_UNIT, "n_gpus": 1, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": ms / a.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c64 fronts/sweeps, f64 GMRES", "data": "synthetic",
            "config": {"workload": "batch16: 16 independent problems n = 40 + 8 (k mod 11), smooth random velocity "
                                   "c = 2 + 0.5 tanh(g), gamma 8, PML amplitude 10 (4 relative to c < 2.5), panels of "
                                   "4 + pad 8, leaf 64, 8 shots each below the top PML, GMRES(20) to 1e-05, complex64 "
                                   "fronts",
                       "sizes": sizes, "nrhs_per_problem": nrhs, "points": int(sum(w.N for w in ws)),
                       "l2": "inputs larger than L2", "parallelism": "single GPU, one batched handle"},
            "roofline": roof, "cpu_baseline": None,
            "e2e": {"value": 1.0 / t_e2e, "unit": BATCH_UNIT, "h2d_bytes_per_step": int(sum(c.numel() * 8 for c in c_pin)
                                                                                    + f_pin.numel() * 16),
                    "d2h_bytes_per_step": int(u_pin.numel() * 16)},
            "gpu_launches": int(sum(v["launches"] for v in agg.values()) // a.steps), "clocks": clk,
            "detail": {"gmres_iters": infos[-1]["iterations"], "relres": max(i["relres_max"] for i in infos),
                       "applies": infos[-1]["applies"], "factor_bytes": fbytes, "sweep_tuning": tuning,
                       "host_setup_ms": {k[5:]: v["total_ms"] for k, v in full_st.items() if k.startswith("host:")},
                       "kernels": kernel_table(full)}}
    print(json.dumps(line))


# ---------------------------------------------------------------------------------------------
# reference arm: the complex128 CPU oracle, as it stands, on a bounded sample per step
# ---------------------------------------------------------------------------------------------
def reference_main(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    iters = a.ref_iters
    total_s, sample, s = None, None, None
    for _ in range(a.warmup if a.warmup < 1 else 1):
        oracle_estimate(iters)
    times = []
    for _ in range(a.steps):
        t0 = time.perf_counter()
        total_s, sample, s = oracle_estimate(iters)
        times.append(time.perf_counter() - t0)
    w = workload()
    value = 1.0 / total_s
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": 1e3 * total_s, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": config_dict(w, 1, {"parallelism": "CPU oracle, single thread"}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample + f" (GMRES iteration count {iters} from the GPU path)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "sample_wall_s": statistics.mean(times)}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="skip the sweep autotuner (library defaults); keeps the "
                    "first timed step the first launches of the run, for launch-list captures")
    ap.add_argument("--ref-iters", type=int, default=18, help="GMRES iterations assumed by the reference arm")
    ap.add_argument("--n", type=int, default=100, help="grid points per axis (100 = the benchmark workload; "
                    "smaller sizes are for profiling captures)")
    ap.add_argument("--workload", choices=["lens", "batch16"], default="lens",
                    help="lens: the converging-lens problem of --n (default); batch16: 16 independent problems "
                         "in one batched handle, complex64")
    a = ap.parse_args()
    global GRID_N, WORKLOAD
    GRID_N = a.n
    WORKLOAD = f"lens{a.n}"
    if a.warmup < 3 and a.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if a.impl == "reference":
        reference_main(a)
    elif a.workload == "batch16":
        batch_main(a)
    else:
        gpu_main(a)


if __name__ == "__main__":
    main()
