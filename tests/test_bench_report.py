"""bench.py's report building (no GPU): roofline, kernel shares and detail from psp_stats records."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def rec(launches, ms, flops, bytes_, extra=0.0):
    return {"launches": launches, "total_ms": ms, "flops": flops, "bytes": bytes_, "extra_flops": extra}


def test_summarize_picks_dominant_kernel_and_computes_rates(bench):
    timed = [{"k_gemm": rec(100, 1000.0, 1e12, 1e9), "k_assemble": rec(10, 50.0, 1e9, 5e10),
              "k_sweep": rec(19, 0.0, 5e11, 3e11), "host:plan_tasks": rec(0, 70.0, 0, 0)}] * 2
    full = {"k_gemm": rec(100, 1000.0, 1e12, 1e9), "k_assemble": rec(10, 50.0, 1e9, 5e10),
            "k_sweep": rec(19, 400.0, 5e11, 3e11), "host:plan_tasks": rec(0, 70.0, 0, 0)}
    infos = [{"iterations": 18, "relres_max": 6e-6, "solve_ms": 900.0, "applies": 19}] * 2
    roof, detail, launches = bench.summarize(timed, full, infos, 16e9, 2)
    assert roof["kernel"] == "k_gemm"
    assert roof["achieved"] == pytest.approx(1.0)              # 2e12 flop / 2 s
    # 3M complex products: the ceiling in counted flops is the FP64 peak x 8/6
    assert roof["frac"] == pytest.approx(1.0 / (bench.FP64_DERIVED_TFLOPS * 8 / 6))
    assert roof["kernel_share"] == pytest.approx(1000.0 / 1450.0)
    assert launches == 2 * 129
    assert detail["apply_ms"] == pytest.approx(400.0 / 19)
    assert detail["sweep_gbs"] == pytest.approx(3e11 / 0.4 / 1e9)
    assert detail["host_setup_ms"] == {"plan_tasks": 70.0}
    assert "host:plan_tasks" not in detail["kernels"]
    assert detail["setup_kernel_ms"] == pytest.approx(1050.0)


def test_summarize_falls_back_when_dominant_kernel_untimed(bench):
    timed = [{"k_gemm": rec(100, 10.0, 1e10, 0), "k_sweep": rec(19, 0.0, 5e11, 3e11)}]
    full = {"k_gemm": rec(100, 10.0, 1e10, 0), "k_sweep": rec(19, 400.0, 5e11, 3e11)}
    infos = [{"iterations": 18, "relres_max": 6e-6, "solve_ms": 900.0, "applies": 19}]
    roof, _, _ = bench.summarize(timed, full, infos, 1, 1)
    assert roof["kernel"] == "k_gemm" and roof["kernel_share"] == pytest.approx(10 / 410)


def test_gpu_main_uses_only_defined_names(bench):
    import dis
    code = bench.gpu_main.__code__
    names = {ins.argval for ins in dis.get_instructions(code) if ins.opname in ("LOAD_GLOBAL",)}
    for n in names:
        assert hasattr(bench, n) or n in dir(__builtins__) or n in __builtins__, n


def test_roofline_generic_bounds_and_rates(bench):
    # the sweep against HBM: algorithmic bytes over event time
    r = bench.roofline_generic("k_sweep", rec(27, 1000.0, 1e12, 5e11), 0.9, "t")
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert abs(r["achieved"] - 500.0) < 1e-9 and abs(r["frac"] - 500.0 / r["peak"]) < 1e-12
    # the tensor-core GEMM against the TF32 peak derived from the bf16 one
    t = bench.roofline_generic("k_tc_gemm", rec(16, 100.0, 1e13, 1e10), 0.1, "t")
    assert t["bound"] == "tensor" and abs(t["achieved"] - 100.0) < 1e-9
    pk, _ = bench._peaks()
    assert abs(t["peak"] - pk["bf16_tflops"] * 1.1 / 2.25) < 1e-9
    # a CUDA-core kernel against the FP32 ALU peak
    g = bench.roofline_generic("k_gemm", rec(10, 10.0, 1e11, 1e9), 0.05, "t")
    assert g["bound"] == "alu" and abs(g["peak"] - 152 * 128 * 2 * 2.07e9 / 1e12) < 1e-9


def test_job_rate_counts_every_rank(bench):
    assert bench.job_rate(4, 5, 2.0) == 10.0


def test_summarize_counts_algorithmic_flops_and_reports_si_beside(bench):
    timed = [{"k_gemm": rec(10, 1000.0, 1e12, 0, extra=2.5e11)}]
    full = {"k_gemm": rec(10, 1000.0, 1e12, 0, extra=2.5e11)}
    infos = [{"iterations": 3, "relres_max": 1e-6, "solve_ms": 1.0, "applies": 4}]
    roof, _, _ = bench.summarize(timed, full, infos, 1, 1, fp64_peak=1.25, fp64_source="x")
    assert roof["achieved"] == pytest.approx(1.0) and roof["frac"] == pytest.approx(0.8 * 6 / 8)
    assert roof["achieved_incl_si"] == pytest.approx(1.25)
    assert roof["fp64_executed"] == pytest.approx(1.25 * 6 / 8) and roof["fp64_pipe_frac"] == pytest.approx(0.75)


def test_rooflines_cover_the_metric_families(bench):
    full128 = {"k_gemm": rec(10, 2000.0, 2e12, 1e9, extra=5e11), "k_sweep": rec(19, 1000.0, 4e11, 3e11)}
    full64 = {"k_gemm": rec(10, 60.0, 5e11, 1e9), "k_tc_gemm": rec(16, 30.0, 2.5e12, 1e10, extra=5e11),
              "k_assemble": rec(12, 40.0, 1e9, 4e10), "k_sweep": rec(19, 300.0, 5e11, 5e11)}
    alu = {"fp64_tflops": 1.2, "fp64_source": "m", "fp32_tflops": 70.0, "fp32_source": "m"}
    out = {(r["path"], r["kernel"]): r for r in bench.rooflines(full128, full64, alu)}
    g = out[("c128", "k_gemm")]
    assert g["achieved"] == pytest.approx(1.0) and g["frac"] == pytest.approx(1.0 / (1.2 * 8 / 6))
    assert g["fp64_pipe_frac"] == pytest.approx(1.25 * 0.75 / 1.2)
    assert g["achieved_incl_si"] == pytest.approx(1.25)
    s64 = out[("c64", "k_sweep")]
    assert s64["bound"] == "hbm" and s64["achieved"] == pytest.approx(5e11 / 0.3 / 1e9)
    fp = out[("c64", "front phase (all setup kernels)")]
    assert fp["bound"] == "tensor" and fp["setup_kernel_ms"] == pytest.approx(130.0)
    assert fp["achieved"] == pytest.approx((5e11 + 2.5e12 + 1e9) / 0.13 / 1e12)
    assert fp["tensor_executed"] == pytest.approx(3e12 * 18 / 8 / 0.13 / 1e12)
    tc = out[("c64", "k_tc_gemm")]
    assert tc["executed"] == pytest.approx(3e12 * 18 / 8 / 0.03 / 1e12)


def test_oracle_extrapolation_formula(bench):
    s = {"t_batch": 10.0, "t_T": 0.2, "t_matvec": 0.01}
    total, formula = bench.oracle_extrapolate(s, m=23, cores=16, iters=18, k=20)
    expect = 2 * 10.0 + 18 * (45 * 0.2 + 0.01) + 1 * 0.01 + 18 * 19 / 8 * 0.01
    assert total == pytest.approx(expect) and "cores = 16" in formula
