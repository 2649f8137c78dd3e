#!/usr/bin/env python
"""Time-to-solution benchmark of the GB300 sweeping preconditioner.

Workload: the 100^3 converging-lens problem, c(x) = 1 - 0.4 exp(-32 |x - 0.5|^2), omega for 10
points per minimum wavelength, PML of 8 points on all faces, 4-plane panels padded with 8 PML
planes, nested-dissection leaf 64, one Gaussian shot (sigma = 2h) at (0.5, 0.5, 0.1), GMRES(20) to
a relative residual of 1e-5, complex128 on the GPU.  One step = the whole hot path on one problem:
setup (factor every panel) + GMRES solve to 1e-5 (all preconditioner applications and matvecs).

One JSON line is printed by rank 0.  Before the timed region the library's sweep autotuner picks
the sweep schedule once per precision (`--no-tune` keeps the defaults).  Besides the contract's keys
the line carries:
  mixed        the complex64 path (complex64 fronts and sweeps, complex128 GMRES) on the same workload;
  rooflines    achieved fraction of the measured peak for each kernel family the metric names
               (complex128 GEMM and sweep, complex64 sweep, complex64 front phase on the tensor pipe);
  peaks        the FP64 / FP32 CUDA-core peaks measured here (cuBLAS DGEMM / SGEMM through torch);
  salt256      the largest single-GPU workload: 256^3 salt body, 32 shots, GMRES(30), complex64;
  layered200   the 200^3 layered and faulted model, GMRES(20), complex64;
  batch16      16 independent problems of uneven size in one batched handle, 8 shots each, complex64;
  cpu_baseline the CPU oracle on all host cores, a bounded sample extrapolated to one solve.
`--no-mixed`, `--no-extra` (skip salt256 / layered200 / batch16) and `--no-cpu-baseline` skip parts.
`--workload batch16` prints a full line for the batch instead; `--workload gamma` prints the waveguide
model's GMRES iterations against PML thickness (§3).  `--impl reference` times the
complex128 CPU oracle on a bounded sample of the default workload per step (see reference_main).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import platform
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
# FP64 CUDA-core peak from unit counts: 152 SMs x 2 DFMA per SM clock x 2 flop x 2.07 GHz
FP64_DERIVED_TFLOPS = 152 * 4 * 2.07e9 / 1e12
FP32_DERIVED_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # FP32 lanes x FMA x max SM clock
TF32_PER_BF16 = 1.1 / 2.25                            # nominal dense TF32 / bf16 tensor rates
TC_EXECUTED_PER_USEFUL = 18.0 / 8.0                   # 3M x (hi.hi + hi.lo + lo.hi) TF32 products per complex MAC
GEMM_3M_EXECUTED_PER_USEFUL = 6.0 / 8.0               # CUDA-core complex GEMM: 3 real FMAs per complex MAC (8 flops)

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
# CPU oracle sample: one panel factorisation per host core, concurrently, plus one panel solve and
# one sparse matvec; run in spawned processes (single-threaded BLAS each) so that no worker is
# forked from a process that holds a CUDA context
# ---------------------------------------------------------------------------------------------
def _oracle_worker(job):
    panel, timed_solve, n = job
    global GRID_N
    GRID_N = n
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
    z0, z1 = plan[panel]
    t0 = time.perf_counter()
    ap = pn.aux_problem(p, z0, z1, w.pad)
    sym = sy.nested_dissection(ap.nx, ap.ny, ap.depth, w.leaf)
    fr = mf.factor(ap.H, sym)
    t1 = time.perf_counter()
    out = {"t_factor": t1 - t0, "panel": panel}
    if timed_solve:
        v = np.zeros(ap.H.shape[0], dtype=np.complex128)
        v[ap.lead * p.nx * p.ny:] = w.rhs()[0][z0 * p.nx * p.ny:z1 * p.nx * p.ny]
        mf.solve(fr, sym, v)
        t2 = time.perf_counter()
        A = dz.operator_A(p)
        x = w.rhs()[0]
        t3 = time.perf_counter()
        A @ x
        t4 = time.perf_counter()
        out.update(t_T=t2 - t1, t_matvec=t4 - t3)
    return out


def cpu_cores():
    return os.cpu_count() or 1


def cpu_model():
    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
        for line in r.stdout.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.processor() or platform.machine()


class OracleSampler:
    """A pool of one spawned single-threaded process per host core; each sample factors one interior
    panel per core at the same time (the panel factorisations are independent, Alg. 1.4) and times
    one panel solve and one sparse matvec."""

    def __init__(self, cores=None):
        import multiprocessing as mp
        from oracle import panels as pn
        self.cores = cores or cpu_cores()
        w = workload()
        self.m = len(pn.panel_plan(w.n, w.gamma, w.panel_depth))
        self.k = w.k
        self.pool = mp.get_context("spawn").Pool(self.cores)
        self.pool.map(_noop, range(self.cores))   # start the workers before timing

    def sample(self):
        jobs = [(1 + i % (self.m - 1), i == 0, GRID_N) for i in range(self.cores)]
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_worker, jobs, chunksize=1)
        wall = time.perf_counter() - t0
        solve = next(r for r in res if "t_T" in r)
        return {"t_batch": max(r["t_factor"] for r in res), "t_T": solve["t_T"], "t_matvec": solve["t_matvec"],
                "wall": wall}

    def close(self):
        self.pool.close()
        self.pool.join()


def _noop(_):
    return 0


def oracle_extrapolate(s, m, cores, iters, k):
    """Seconds per solve of the oracle from one sample: ceil(m / cores) rounds of concurrent panel
    factorisations, then GMRES with iters x (2m - 1) sequential panel solves (Alg. 1.5 is a chain),
    iters + restarts true-residual / Krylov matvecs, and Gram-Schmidt counted as iters (iters + 1) / 2
    vector passes at a quarter of a matvec each."""
    t_setup = math.ceil(m / cores) * s["t_batch"]
    t_apply = (2 * m - 1) * s["t_T"]
    restarts = max(1, math.ceil(iters / k))
    t_solve = iters * (t_apply + s["t_matvec"]) + restarts * s["t_matvec"] + iters * (iters + 1) / 2 / 4 * s["t_matvec"]
    formula = (f"ceil(m/cores) x t_batch + iters x ((2m - 1) t_T + t_mv) + restarts x t_mv + "
               f"iters (iters + 1) / 8 x t_mv with m = {m}, cores = {cores}, iters = {iters}, restarts = {restarts}")
    return t_setup + t_solve, formula


def oracle_baseline(iters, k=20, sampler=None):
    own = sampler is None
    sampler = sampler or OracleSampler()
    try:
        s = sampler.sample()
    finally:
        if own:
            sampler.close()
    total, formula = oracle_extrapolate(s, sampler.m, sampler.cores, iters, k)
    sample = (f"{sampler.cores} concurrent {GRID_N}x{GRID_N}x12 panel factorisations ({s['t_batch']:.2f} s, one per "
              f"core) + one panel solve ({s['t_T']:.3f} s) + one sparse matvec ({s['t_matvec']:.4f} s), "
              f"single-threaded BLAS per process")
    return {"value": 1.0 / total, "unit": UNIT, "cores": sampler.cores, "kind": "oracle", "sample": sample,
            "cpu_model": cpu_model(), "nproc": cpu_cores(), "seconds_per_solve": total, "extrapolated": True,
            "formula": formula, "sample_wall_s": s["wall"],
            "iterations": iters, "iterations_source": "the GPU complex128 path's GMRES count on this workload "
            "(the oracle's own count equals the GPU path's within +-1 on every parity case of the tests)"}


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


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        return json.load(open(path)), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def measure_alu_peaks(dev):
    """FP64 and FP32 CUDA-core peaks measured here: best of five cuBLAS DGEMM / SGEMM (TF32 off) calls
    through torch.  A DGEMM rate above the unit-count figure would mean an emulated FP64 GEMM; the
    derived figure is used then."""
    import torch
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    out = {}
    try:
        for name, dt, n, derived in (("fp64", torch.float64, 4096, FP64_DERIVED_TFLOPS),
                                     ("fp32", torch.float32, 8192, FP32_DERIVED_TFLOPS)):
            g = torch.Generator(device=dev).manual_seed(1)
            a = torch.randn(n, n, dtype=dt, device=dev, generator=g)
            b = torch.randn(n, n, dtype=dt, device=dev, generator=g)
            for _ in range(2):
                torch.matmul(a, b)
            best = float("inf")
            for _ in range(5):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b)
                e1.record()
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1))
            meas = 2.0 * n ** 3 / (best * 1e-3) / 1e12
            if meas > 1.05 * derived:
                out[f"{name}_tflops"] = derived
                out[f"{name}_source"] = (f"derived from unit counts ({derived:.3f}); cuBLAS {n}^3 measured "
                                         f"{meas:.3f}, above it, so treated as emulated")
            else:
                out[f"{name}_tflops"] = meas
                out[f"{name}_source"] = f"measured: best of 5 cuBLAS {name.upper()} GEMMs {n}^3 (derived {derived:.3f})"
            del a, b
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    torch.cuda.empty_cache()
    return out


def _agg(stat_list):
    agg = {}
    for st in stat_list:
        for k, v in st.items():
            g = agg.setdefault(k, {"launches": 0, "total_ms": 0.0, "flops": 0.0, "bytes": 0.0, "extra_flops": 0.0})
            for f in g:
                g[f] += v.get(f, 0.0)
    return agg


def kernel_table(stats):
    return {k: {"launches": v["launches"], "ms_per_step": v["total_ms"],
                "tflops": v["flops"] / max(v["total_ms"], 1e-9) / 1e9,
                "si_tflops": v.get("extra_flops", 0.0) / max(v["total_ms"], 1e-9) / 1e9,
                "gbs": v["bytes"] / max(v["total_ms"], 1e-9) / 1e6} for k, v in sorted(stats.items())}


def summarize(stats_timed, stats_full, infos, factor_bytes, steps, fp64_peak=FP64_DERIVED_TFLOPS,
              fp64_source="derived from unit counts"):
    """Roofline of the dominant kernel and the per-kernel detail from psp_stats records.

    stats_timed: one record per timed step (setup kernels timed with CUDA events);
    stats_full: one step with every launch timed (kernel-time shares).  Achieved flops count the
    plain multifrontal work (LDL^T, F_BL L^{-T}, Schur update); the selective-inversion flops the
    kernel also executes are reported beside it."""
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
    sec = max(tv["total_ms"] * 1e-3, 1e-12)
    achieved = tv["flops"] / sec / 1e12
    # the complex products are 3M (3 real FMAs = 6 executed flops per 8 counted), so in counted complex
    # flops the FP64 pipe's ceiling is its peak x 8/6
    peak = fp64_peak / GEMM_3M_EXECUTED_PER_USEFUL
    executed = (tv["flops"] + tv.get("extra_flops", 0.0)) * GEMM_3M_EXECUTED_PER_USEFUL / sec / 1e12
    roofline = {"kernel": tk, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic_from_profiles(tk),
                "achieved_incl_si": (tv["flops"] + tv.get("extra_flops", 0.0)) / sec / 1e12,
                "fp64_executed": executed, "fp64_pipe_frac": executed / fp64_peak,
                "peak_source": f"FP64 CUDA-core peak ({fp64_source}) x 8/6: the 3M complex products execute 6 real "
                               "flops per 8 counted, so 8/6 of the FP64 rate is the ceiling in counted flops; "
                               "fp64_pipe_frac = executed FP64 flops (algorithmic + selective inversion) over the "
                               "FP64 peak",
                "kernel_share": full.get(tk, {"total_ms": 0.0})["total_ms"] / tot_all,
                "work": "algorithmic flops of the plain multifrontal factorisation (8 per complex MAC); "
                        "achieved_incl_si adds the selective-inversion flops the kernel also executes",
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


def roofline_generic(name, v, share, timing, alu_peaks=None):
    """Roofline line for one kernel from its psp_stats record."""
    pk, src = _peaks()
    alu_peaks = alu_peaks or {}
    ms = max(v["total_ms"], 1e-9)
    if name == "k_tc_gemm":
        peak = pk["bf16_tflops"] * TF32_PER_BF16
        ach = v["flops"] / ms / 1e9
        useful_all = v["flops"] + v.get("extra_flops", 0.0)
        return {"kernel": name, "bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "traffic": None, "kernel_share": share, "timing": timing,
                "achieved_incl_si": useful_all / ms / 1e9,
                "executed": useful_all * TC_EXECUTED_PER_USEFUL / ms / 1e9,
                "executed_frac": useful_all * TC_EXECUTED_PER_USEFUL / ms / 1e9 / peak,
                "peak_source": f"TF32 dense from the {src} bf16 peak x 1.1/2.25 (of {src}); achieved counts the "
                               "algorithmic complex flops (8 per complex MAC), executed the split-TF32 3M products "
                               "(18 real TF32 flops per useful complex MAC)"}
    if name in ("k_sweep", "k_assemble", "k_tc_pack", "k_matvec", "k_multiaxpy", "k_solve_fwd", "k_solve_bwd"):
        peak = pk["hbm_gbs"]
        ach = v["bytes"] / ms / 1e6
        return {"kernel": name, "bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                "frac": ach / peak, "traffic": None, "kernel_share": share, "timing": timing,
                "peak_source": f"{src} HBM copy bandwidth (of {src})"}
    peak = alu_peaks.get("fp32_tflops", FP32_DERIVED_TFLOPS)
    ach = v["flops"] / ms / 1e9
    return {"kernel": name, "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
            "traffic": None, "kernel_share": share, "timing": timing,
            "peak_source": alu_peaks.get("fp32_source", "FP32 CUDA-core peak derived: 152 SMs x 128 lanes x 2 flop x "
                                                        "2.07 GHz")}


def rooflines(full128, full64, alu):
    """Achieved fraction of the measured peak for each kernel family the metric names, from one
    instrumented step of each path (every launch timed with CUDA events on the launch stream)."""
    pk, src = _peaks()
    out = []
    fp64 = alu.get("fp64_tflops", FP64_DERIVED_TFLOPS)
    if full128:
        tot = sum(v["total_ms"] for k, v in full128.items() if not k.startswith("host:")) or 1.0
        g = full128.get("k_gemm")
        if g and g["total_ms"] > 0:
            sec = g["total_ms"] * 1e-3
            pk3 = fp64 / GEMM_3M_EXECUTED_PER_USEFUL
            exe = (g["flops"] + g["extra_flops"]) * GEMM_3M_EXECUTED_PER_USEFUL / sec / 1e12
            out.append({"path": "c128", "kernel": "k_gemm", "bound": "alu", "unit": "TFLOP/s",
                        "achieved": g["flops"] / sec / 1e12, "peak": pk3, "frac": g["flops"] / sec / 1e12 / pk3,
                        "achieved_incl_si": (g["flops"] + g["extra_flops"]) / sec / 1e12,
                        "fp64_executed": exe, "fp64_pipe_frac": exe / fp64, "kernel_share": g["total_ms"] / tot,
                        "peak_source": "FP64 peak x 8/6 (3M products): " + alu.get("fp64_source", "derived")})
        s = full128.get("k_sweep")
        if s and s["total_ms"] > 0:
            sec = s["total_ms"] * 1e-3
            out.append({"path": "c128", "kernel": "k_sweep", "bound": "alu", "unit": "TFLOP/s",
                        "achieved": s["flops"] / sec / 1e12, "peak": fp64, "frac": s["flops"] / sec / 1e12 / fp64,
                        "hbm_gbs": s["bytes"] / sec / 1e9, "hbm_frac": s["bytes"] / sec / 1e9 / pk["hbm_gbs"],
                        "kernel_share": s["total_ms"] / tot, "peak_source": alu.get("fp64_source", "derived"),
                        "note": "8 FP64 flops per complex128 factor entry per right-hand side: FP64-bound"})
    if full64:
        f64 = {k: v for k, v in full64.items() if not k.startswith("host:")}
        tot = sum(v["total_ms"] for v in f64.values()) or 1.0
        s = f64.get("k_sweep")
        if s and s["total_ms"] > 0:
            r = roofline_generic("k_sweep", s, s["total_ms"] / tot, "instrumented step", alu)
            r["path"] = "c64"
            out.append(r)
        setup = [v for k, v in f64.items() if k in SETUP_KERNELS]
        sms = sum(v["total_ms"] for v in setup)
        if sms > 0:
            tf32 = pk["bf16_tflops"] * TF32_PER_BF16
            useful = sum(v["flops"] for v in setup)
            si = sum(v.get("extra_flops", 0.0) for v in setup)
            tc = f64.get("k_tc_gemm", {"flops": 0.0, "extra_flops": 0.0})
            exe = (tc["flops"] + tc.get("extra_flops", 0.0)) * TC_EXECUTED_PER_USEFUL
            out.append({"path": "c64", "kernel": "front phase (all setup kernels)", "bound": "tensor",
                        "unit": "TFLOP/s", "achieved": useful / (sms * 1e-3) / 1e12, "peak": tf32,
                        "frac": useful / (sms * 1e-3) / 1e12 / tf32,
                        "achieved_incl_si": (useful + si) / (sms * 1e-3) / 1e12,
                        "tensor_executed": exe / (sms * 1e-3) / 1e12, "setup_kernel_ms": sms,
                        "kernel_share": sms / tot,
                        "peak_source": f"TF32 dense = {src} bf16 x 1.1/2.25 (of {src})"})
        t = f64.get("k_tc_gemm")
        if t and t["total_ms"] > 0:
            r = roofline_generic("k_tc_gemm", t, t["total_ms"] / tot, "instrumented step", alu)
            r["path"] = "c64"
            out.append(r)
    return out


# ---------------------------------------------------------------------------------------------
# the other configurations, one object each (a single timed step after the kernels are warm)
# ---------------------------------------------------------------------------------------------
def extra_workload(name, w, precision, dev, sched=None, maxit=400, desc="", tune_nrhs=0):
    import torch

    from paper_1204_0111_gb300 import psp
    stream = torch.cuda.current_stream(dev)
    c_dev = torch.from_numpy(w.c).to(dev)
    tuning = None
    if tune_nrhs > 0:
        # the sweep autotuner on a handle of its own, before the timed step, for the right-hand sides one
        # GMRES run carries
        P = psp.SweepingPreconditioner(c_dev, w.h, w.omega, w.gamma, w.panel_depth, pad=w.pad, leaf=w.leaf,
                                       pml_C=w.pml_C, alpha=w.alpha, precision=precision, **(sched or {}))
        tuning = P.tune_sweep(nrhs=tune_nrhs, reps=1)
        P.close()
        torch.cuda.empty_cache()
        sched = dict(sched or {}, sweep_level_tasks=tuning["sweep_level_tasks"],
                     sweep_ctas_per_sm=tuning["sweep_ctas_per_sm"], sweep_rhs_group=tuning["sweep_rhs_group"],
                     sweep_min_rows=tuning["sweep_min_rows"], sweep_max_rows=tuning["sweep_max_rows"],
                     sweep_claim_ahead=tuning["sweep_claim_ahead"])
    f = w.rhs()
    f_dev = torch.from_numpy(f).to(dev)
    u_dev = torch.zeros_like(f_dev)
    torch.cuda.synchronize()
    clocks = ClockSampler()
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e0.record(stream)
    t0 = time.perf_counter()
    P = psp.SweepingPreconditioner(c_dev, w.h, w.omega, w.gamma, w.panel_depth, pad=w.pad, leaf=w.leaf,
                                   pml_C=w.pml_C, alpha=w.alpha, precision=precision, collect_stats=1,
                                   **(sched or {}))
    e1.record(stream)
    info = P.solve(f_dev, u_dev, tol=w.tol, k=w.k, maxit=maxit)
    e2.record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    clk = clocks.stop()
    st = P.stats()
    pinfo = P.info()
    P.close()
    del c_dev, f_dev, u_dev
    torch.cuda.empty_cache()
    full = {k: v for k, v in st.items() if not k.startswith("host:")}
    tot = sum(v["total_ms"] for v in full.values()) or 1.0
    top = max(full.items(), key=lambda kv: kv[1]["total_ms"])[0]
    roof = roofline_generic(top, full[top], full[top]["total_ms"] / tot,
                            "CUDA events around every launch of this kernel in the timed step")
    sw = full.get("k_sweep", {"total_ms": 0.0, "bytes": 0.0})
    ms = e0.elapsed_time(e2)
    return {"workload": desc or w.name, "n": w.n, "N": w.N, "nrhs": int(f.shape[0]), "gmres_k": w.k, "tol": w.tol,
            "precision": precision, "steps": 1, "warmup": 0,
            "warmup_note": "the library's kernels were warmed by the lens steps in the same process",
            "ms_per_step": ms, "value": 1e3 / ms, "unit": "solves/s (all right-hand sides)", "wall_s": wall,
            "setup_ms": e0.elapsed_time(e1), "solve_ms": e1.elapsed_time(e2), "gmres_iters": info["iterations"],
            "relres_max": info["relres_max"], "converged": info["converged"], "gmres_groups": info["groups"],
            "applies": info["applies"], "panels": pinfo["panels"], "fronts": pinfo["fronts"],
            "factor_bytes": pinfo["factor_bytes"],
            "apply_ms": sw["total_ms"] / max(info["applies"], 1),
            "sweep_gbs": sw["bytes"] / max(sw["total_ms"] * 1e-3, 1e-12) / 1e9,
            "roofline": roof, "clocks": clk, "kernels": kernel_table(full), "sweep_tuning": tuning,
            "host_setup_ms": {k[5:]: v["total_ms"] for k, v in st.items() if k.startswith("host:")}}


# ---------------------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------------------
def gpu_main(a):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1204_0111_gb300 import psp
    from paper_1204_0111_gb300 import workloads as wl

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

    main_prec = a.precision

    def step(precision=None, stats=0):
        precision = precision or main_prec
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

    alu = {} if a.no_peaks else measure_alu_peaks(dev)
    # the library's autotuners, once per precision, before any timed work: the factor form and tensor-core
    # threshold for the expected number of applications (psp_tune_setup), then the sweep schedule
    tuning, setup_tuning = {}, {}
    for prec in () if a.no_tune else (main_prec,) + (() if a.no_mixed or main_prec == "c64" else ("c64",)):
        P = psp.SweepingPreconditioner(c_dev, w.h, w.omega, w.gamma, w.panel_depth, pad=w.pad, leaf=w.leaf,
                                       pml_C=w.pml_C, alpha=w.alpha, precision=prec)
        ts = P.tune_setup(nrhs=nrhs, expected_applies=a.expected_applies) if a.si == "auto" else \
            {"selective_inversion": a.si, "tc_min_dim": 0, "tuned": False}
        t = P.tune_sweep(nrhs=nrhs, reps=3)
        P.close()
        tuning[prec] = t
        setup_tuning[prec] = ts
        sched[prec] = {"sweep_level_tasks": t["sweep_level_tasks"], "sweep_ctas_per_sm": t["sweep_ctas_per_sm"],
                       "sweep_rhs_group": t["sweep_rhs_group"], "sweep_min_rows": t["sweep_min_rows"],
                       "sweep_max_rows": t["sweep_max_rows"], "sweep_claim_ahead": t["sweep_claim_ahead"],
                       "selective_inversion": ts["selective_inversion"],
                       "tc_min_dim": ts["tc_min_dim"] if prec == "c64" else 0}
    if a.no_tune and a.si != "auto":
        for prec in ("c128", "c64"):
            sched.setdefault(prec, {})["selective_inversion"] = a.si
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
    roofline, detail, launches = summarize(stats_all, full_st, infos, fbytes, a.steps,
                                           alu.get("fp64_tflops", FP64_DERIVED_TFLOPS), alu.get("fp64_source", ""))

    # end to end through the public API with pinned host buffers (copies inside the timed region)
    c_pin = torch.from_numpy(w.c).pin_memory()
    f_pin = torch.from_numpy(f_host).pin_memory()
    u_pin = torch.zeros_like(f_pin).pin_memory()
    e2e_steps = 0 if a.no_e2e else max(1, min(a.steps, 5))
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        P = psp.SweepingPreconditioner(c_pin, w.h, w.omega, w.gamma, w.panel_depth, pad=w.pad, leaf=w.leaf,
                                       pml_C=w.pml_C, alpha=w.alpha, precision=main_prec,
                                       **sched.get(main_prec, {}))
        P.solve(f_pin, u_pin, tol=w.tol, k=w.k, maxit=400)
        P.close()
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    e2e = None if a.no_e2e else {
        "value": job_rate(world, e2e_steps, max_over_ranks(t1 - t0, dev)), "unit": UNIT, "steps": e2e_steps,
        "h2d_bytes_per_step": int(c_pin.numel() * 8 + f_pin.numel() * 16), "d2h_bytes_per_step": int(u_pin.numel() * 16)}

    # mixed precision (complex64 fronts and sweeps, complex128 GMRES) on the same workload
    mixed, mfull = None, None
    if not a.no_mixed and main_prec == "c128":
        step("c64")
        torch.cuda.synchronize()
        m0 = torch.cuda.Event(enable_timing=True)
        m1 = torch.cuda.Event(enable_timing=True)
        msteps = max(1, min(a.steps, 5))
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
        mkern = {k: v for k, v in mfull.items() if not k.startswith("host:")}
        magg = _agg(mstats)
        # apply error of the complex64 preconditioner against the complex128 one
        P128 = psp.SweepingPreconditioner(c_dev, w.h, w.omega, w.gamma, w.panel_depth, pad=w.pad, leaf=w.leaf,
                                          pml_C=w.pml_C, alpha=w.alpha)
        P64 = psp.SweepingPreconditioner(c_dev, w.h, w.omega, w.gamma, w.panel_depth, pad=w.pad, leaf=w.leaf,
                                         pml_C=w.pml_C, alpha=w.alpha, precision="c64")
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
        del o128, o64, r
        mixed = {"value": 1e3 / mms, "unit": UNIT, "ms_per_step": mms, "steps": msteps,
                 "gmres_iters": minfo["iterations"], "relres": minfo["relres_max"], "apply_rel_err_vs_c128": err,
                 "speedup_vs_c128": (ms_max / a.steps) / mms, "dtype": "c64 fronts/sweeps, f64 GMRES",
                 "setup_kernel_ms": sum(v["total_ms"] for k, v in magg.items() if not k.startswith("host:")) / msteps,
                 "apply_ms": mkern.get("k_sweep", {"total_ms": 0.0})["total_ms"] / max(minfo["applies"], 1),
                 "host_setup_ms": mhost, "kernels": kernel_table(mkern)}
    roofs = rooflines({k: v for k, v in full_st.items() if not k.startswith("host:")}, mfull, alu)

    # setup and application of each factor form (selective inversion, §2.2 and Table 2's trade)
    si_forms = {}
    if not a.no_mixed and main_prec == "c128":
        for prec in ("c128", "c64"):
            for form in ("extended", "paper", "none"):
                kw = {k: v for k, v in sched.get(prec, {}).items() if k != "selective_inversion"}
                P = psp.SweepingPreconditioner(c_dev, w.h, w.omega, w.gamma, w.panel_depth, pad=w.pad, leaf=w.leaf,
                                               pml_C=w.pml_C, alpha=w.alpha, precision=prec, collect_stats=1,
                                               selective_inversion=form, **kw)
                uu = torch.empty_like(f_dev)
                P.apply(f_dev, uu)
                P.stats(reset=True)
                for _ in range(3):
                    P.apply(f_dev, uu)
                st = {k: v for k, v in P.stats().items() if not k.startswith("host:")}
                fb = P.info()["factor_bytes"]
                P.close()
                P = psp.SweepingPreconditioner(c_dev, w.h, w.omega, w.gamma, w.panel_depth, pad=w.pad, leaf=w.leaf,
                                               pml_C=w.pml_C, alpha=w.alpha, precision=prec, collect_stats=2,
                                               selective_inversion=form, **kw)
                su = {k: v for k, v in P.stats().items() if k in SETUP_KERNELS}
                P.close()
                sw = st.get("k_sweep", {"total_ms": 0.0})
                si_forms[f"{prec}/{form}"] = {
                    "setup_kernel_ms": sum(v["total_ms"] for v in su.values()),
                    "setup_algorithmic_tflop": sum(v["flops"] for v in su.values()) / 1e12,
                    "setup_si_tflop": sum(v["extra_flops"] for v in su.values()) / 1e12,
                    "apply_ms": sw["total_ms"] / 3, "factor_bytes": fb}

    # the other configurations (rank 0 of a single-GPU run only)
    extras = {}
    if not a.no_extra and world == 1:
        torch.cuda.empty_cache()
        ws = wl.cube_salt(256)
        extras["salt256"] = extra_workload(
            "salt256", ws, "c64", dev, maxit=400, tune_nrhs=8,
            desc=f"salt256: 256^3 salt body in a 1.5-4.5 depth gradient, 8 points per wavelength, gamma 12, panels "
                 f"of 8 + pad 8, leaf 64, PML amplitude 4 relative to c_max, 32 shots on an 8 x 4 grid below the "
                 f"top PML, GMRES(30) to 1e-05, complex64 fronts and sweeps, complex128 GMRES")
        wly = wl.cube_layered(200)
        extras["layered200"] = extra_workload(
            "layered200", wly, "c64", dev, maxit=600, tune_nrhs=1,
            desc="layered200: 200^3, 12 dipping layers c ~ U(1.5, 6) and 2 planar faults (seed 3), 10 points per "
                 "wavelength at c_min, gamma 10, panels of 4 + pad 10, PML amplitude 4 relative to c_max, one shot "
                 "at (0.5, 0.5, 0.1), GMRES(20) to 1e-05, complex64 fronts and sweeps, complex128 GMRES")
        extras["batch16"] = batch_object(dev, steps=1, warmup=1)

    if rank == 0:
        cpu = None
        if not a.no_cpu_baseline:
            cpu = oracle_baseline(detail["gmres_iters"], w.k)
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
                "warmup": a.warmup, "ms_per_step": ms_max / a.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64" if main_prec == "c128" else "c64 fronts/sweeps, f64 GMRES",
                "data": "synthetic",
                "config": config_dict(w, nrhs, {"parallelism": f"replicas x{world}" if world > 1 else "single GPU"}),
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches // a.steps,
                "clocks": clk, "peaks": alu, "rooflines": roofs,
                "detail": dict(detail, sweep_tuning=tuning, setup_tuning=setup_tuning, chosen=sched),
                "si_forms": si_forms,
                "mixed": mixed}
        line.update(extras)
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------------------------
# batching workload: 16 independent problems of uneven size in one handle
# ---------------------------------------------------------------------------------------------
BATCH_UNIT = "batch solves/s"   # all 16 problems x 8 shots from c(x) and f to 1e-5 (setup + GMRES) per second


def batch_object(dev, steps, warmup, with_e2e=False):
    import numpy as np
    import torch

    from paper_1204_0111_gb300 import psp
    from paper_1204_0111_gb300 import workloads as wl

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
             "sweep_rhs_group": tuning["sweep_rhs_group"], "sweep_max_rows": tuning["sweep_max_rows"],
             "sweep_claim_ahead": tuning["sweep_claim_ahead"], "pml_C": pml_C}

    def step(stats=0, problems=prs, f=f_dev, u=u_dev):
        B = psp.SweepingPreconditionerBatch(problems, precision="c64", collect_stats=stats, **sched)
        info = B.solve(f, u, tol=1e-5, k=20, maxit=400)
        st = B.stats() if stats else None
        fb = B.info()["factor_bytes"]
        B.close()
        return info, st, fb

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    infos, stats_all = [], []
    fbytes = 0
    for _ in range(steps):
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
    out = {"workload": "batch16: 16 independent problems n = 40 + 8 (k mod 11), smooth random velocity "
                       "c = 2 + 0.5 tanh(g), gamma 8, PML amplitude 10 (4 relative to c < 2.5), panels of "
                       "4 + pad 8, leaf 64, 8 shots each below the top PML, GMRES(20) to 1e-05, complex64 fronts",
           "sizes": [w.n for w in ws], "nrhs_per_problem": nrhs, "points": int(sum(w.N for w in ws)),
           "value": steps / (ms / 1e3), "unit": BATCH_UNIT, "steps": steps, "warmup": warmup,
           "ms_per_step": ms / steps, "roofline": roof, "clocks": clk,
           "gpu_launches": int(sum(v["launches"] for v in agg.values()) // steps),
           "gmres_iters": infos[-1]["iterations"], "relres": max(i["relres_max"] for i in infos),
           "applies": infos[-1]["applies"], "factor_bytes": fbytes, "sweep_tuning": tuning,
           "host_setup_ms": {k[5:]: v["total_ms"] for k, v in full_st.items() if k.startswith("host:")},
           "kernels": kernel_table(full)}
    if with_e2e:
        c_pin = [torch.from_numpy(w.c).pin_memory() for w in ws]
        f_pin = torch.from_numpy(f_host).pin_memory()
        u_pin = torch.zeros_like(f_pin).pin_memory()
        prs_h = [dict(p, c=cp) for p, cp in zip(prs, c_pin)]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step(problems=prs_h, f=f_pin, u=u_pin)
        torch.cuda.synchronize()
        t_e2e = time.perf_counter() - t0
        out["e2e"] = {"value": 1.0 / t_e2e, "unit": BATCH_UNIT,
                      "h2d_bytes_per_step": int(sum(c.numel() * 8 for c in c_pin) + f_pin.numel() * 16),
                      "d2h_bytes_per_step": int(u_pin.numel() * 16)}
    return out


def salt_main(a):
    """The salt workload of --n as one line (a profiling aid; the default line carries salt256).  With
    --apply-only: setup, then --steps timed applications to --apply-nrhs shots (after --warmup
    untimed ones and, unless --no-tune, the sweep autotuner), no GMRES."""
    import torch

    from paper_1204_0111_gb300 import psp
    from paper_1204_0111_gb300 import workloads as wl
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    w = wl.cube_salt(a.n)
    if not a.apply_only:
        for _ in range(a.warmup):
            extra_workload("salt", w, "c64", dev)
        o = extra_workload("salt", w, "c64", dev, desc=f"salt{a.n}")
        print(json.dumps(o))
        return
    c_dev = torch.from_numpy(w.c).to(dev)
    P = psp.SweepingPreconditioner(c_dev, w.h, w.omega, w.gamma, w.panel_depth, pad=w.pad, leaf=w.leaf,
                                   pml_C=w.pml_C, alpha=w.alpha, precision="c64", collect_stats=1)
    tuning = None if a.no_tune else P.tune_sweep(nrhs=a.apply_nrhs, reps=1)
    f = torch.from_numpy(w.rhs()[:a.apply_nrhs].copy()).to(dev)
    u = torch.empty_like(f)
    for _ in range(a.warmup):
        P.apply(f, u)
    P.stats(reset=True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(a.steps):
        P.apply(f, u)
    e1.record()
    torch.cuda.synchronize()
    st = P.stats()
    sw = st["k_sweep"]
    print(json.dumps({"workload": f"salt{a.n} apply, {a.apply_nrhs} shots, complex64", "steps": a.steps,
                      "apply_ms": e0.elapsed_time(e1) / a.steps, "sweep_ms": sw["total_ms"] / a.steps,
                      "sweep_gbs": sw["bytes"] / max(sw["total_ms"] * 1e-3, 1e-12) / 1e9,
                      "factor_bytes": P.info()["factor_bytes"], "sweep_tuning": tuning}))
    P.close()


def gamma_main(a):
    """PML thickness (§3): the waveguide model with the paper's settings (4-plane panels, damping 7,
    PML amplitude 2 relative to its fastest speed, its four forcing functions, 10 points per
    wavelength), GMRES(20) to 1e-5 on all four, for gamma = 5, 6, 8, 10 PML points at --n and at
    twice --n (twice the frequency at the same resolution per wavelength).  The paper reports 52
    iterations with 5 points at 500^3 and 27 with 6, and that half the frequency needs the 27 with 5
    points.  One JSON object; complex64 fronts and sweeps, complex128 GMRES."""
    import torch

    from paper_1204_0111_gb300 import psp
    from paper_1204_0111_gb300 import workloads as wl
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    rows = []
    for n in (a.n, 2 * a.n):
        for gamma in (5, 6, 8, 10):
            w = wl.cube_paper("waveguide", n, gamma=gamma)
            c_dev = torch.from_numpy(w.c).to(dev)
            f = torch.from_numpy(w.forcing).to(dev)
            u = torch.zeros_like(f)
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record()
            P = psp.SweepingPreconditioner(c_dev, w.h, w.omega, w.gamma, w.panel_depth, pad=w.pad, leaf=w.leaf,
                                           pml_C=w.pml_C, alpha=w.alpha, precision="c64")
            e1.record()
            info = P.solve(f, u, tol=1e-5, k=20, maxit=400)
            e2.record()
            torch.cuda.synchronize()
            rows.append({"n": n, "gamma": gamma, "iterations": info["iterations"], "converged": info["converged"],
                         "relres_max": info["relres_max"], "setup_ms": e0.elapsed_time(e1),
                         "solve_ms": e1.elapsed_time(e2), "panels": P.info()["panels"]})
            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
            P.close()
            del c_dev, f, u
            torch.cuda.empty_cache()
    print(json.dumps({"workload": "waveguide (paper §3), PML thickness sweep", "precision": "c64 fronts, c128 GMRES",
                      "rhs": "the paper's four forcing functions", "gmres_k": 20, "tol": 1e-5, "rows": rows}))


def batch_main(a):
    import torch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    o = batch_object(dev, a.steps, a.warmup, with_e2e=True)
    line = {"metric": METRIC, "value": o["value"], "unit": BATCH_UNIT, "n_gpus": 1, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": o["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c64 fronts/sweeps, f64 GMRES", "data": "synthetic",
            "config": {"workload": o["workload"], "sizes": o["sizes"], "nrhs_per_problem": o["nrhs_per_problem"],
                       "points": o["points"], "l2": "inputs larger than L2",
                       "parallelism": "single GPU, one batched handle"},
            "roofline": o["roofline"], "cpu_baseline": None, "e2e": o["e2e"], "gpu_launches": o["gpu_launches"],
            "clocks": o["clocks"],
            "detail": {k: o[k] for k in ("gmres_iters", "relres", "applies", "factor_bytes", "sweep_tuning",
                                         "host_setup_ms", "kernels")}}
    print(json.dumps(line))


# ---------------------------------------------------------------------------------------------
# reference arm: the complex128 CPU oracle, as it stands, on a bounded sample per step
# ---------------------------------------------------------------------------------------------
def reference_main(a):
    """Each step is one bounded sample of the oracle on the default workload: one panel factorisation
    per host core at the same time, one panel solve and one sparse matvec.  `ms_per_step` is that
    sample's measured wall time; `value` is the solves/s the samples extrapolate to (formula in
    `extrapolated`).  The GMRES iteration count is taken from the GPU path (--ref-iters)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    iters = a.ref_iters
    sampler = OracleSampler()
    try:
        for _ in range(min(a.warmup, 1)):
            sampler.sample()
        times, samples = [], []
        for _ in range(a.steps):
            t0 = time.perf_counter()
            samples.append(sampler.sample())
            times.append(time.perf_counter() - t0)
    finally:
        sampler.close()
    med = {k: statistics.median(s[k] for s in samples) for k in ("t_batch", "t_T", "t_matvec", "wall")}
    total, formula = oracle_extrapolate(med, sampler.m, sampler.cores, iters, sampler.k)
    w = workload()
    value = 1.0 / total
    sample = (f"{sampler.cores} concurrent {GRID_N}x{GRID_N}x12 panel factorisations (median {med['t_batch']:.2f} s) "
              f"+ one panel solve ({med['t_T']:.3f} s) + one sparse matvec ({med['t_matvec']:.4f} s) per step")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": 1e3 * statistics.mean(times), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": config_dict(w, 1, {"parallelism": f"CPU oracle, {sampler.cores} processes x 1 thread"}),
            "extrapolated": {"seconds_per_solve": total, "formula": formula, "iterations": iters,
                             "iterations_source": "the GPU complex128 path's count on this workload (--ref-iters); "
                                                  "the oracle's own count equals it within +-1 on the parity cases"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": sampler.cores, "kind": "oracle", "sample": sample,
                             "cpu_model": cpu_model(), "nproc": cpu_cores()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "step_note": "a step is one bounded sample (ms_per_step is its measured wall time); value is the "
                         "extrapolated whole-solve rate"}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-mixed", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="skip the salt256, layered200 and batch16 objects")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling captures)")
    ap.add_argument("--no-peaks", action="store_true", help="skip the FP64/FP32 GEMM peak measurement (profiling "
                    "captures; the derived peaks are used)")
    ap.add_argument("--apply-only", action="store_true", help="--workload salt: time applications only")
    ap.add_argument("--apply-nrhs", type=int, default=8, help="--workload salt --apply-only: shots per application")
    ap.add_argument("--si", choices=["auto", "extended", "paper", "none"], default="auto",
                    help="factor form (selective inversion) of the timed path: auto = psp_tune_setup's choice")
    ap.add_argument("--precision", choices=["c128", "c64"], default="c128",
                    help="precision of the timed lens path (c128 = the benchmark; c64 for profiling captures)")
    ap.add_argument("--no-tune", action="store_true", help="skip the sweep autotuner (library defaults); keeps the "
                    "first timed step the first launches of the run, for launch-list captures")
    ap.add_argument("--ref-iters", type=int, default=18, help="GMRES iterations assumed by the reference arm")
    ap.add_argument("--expected-applies", type=int, default=18, help="applications per solve the setup autotuner "
                    "weighs the setup against (lens100: 18 GMRES iterations, one application each)")
    ap.add_argument("--n", type=int, default=100, help="grid points per axis (100 = the benchmark workload; "
                    "smaller sizes are for profiling captures)")
    ap.add_argument("--workload", choices=["lens", "batch16", "salt", "gamma"], default="lens",
                    help="lens: the converging-lens problem of --n (default); batch16: 16 independent problems "
                         "in one batched handle, complex64; salt: the salt-body workload of --n alone (32 shots, "
                         "GMRES(30), complex64), for profiling captures; gamma: the waveguide model's iterations "
                         "against PML thickness at --n and 2 --n")
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
    elif a.workload == "salt":
        salt_main(a)
    elif a.workload == "gamma":
        gamma_main(a)
    else:
        gpu_main(a)


if __name__ == "__main__":
    main()
