"""bench.py's roofline bookkeeping (host logic, no GPU): which peak each kernel
category is measured against, and the DRAM-traffic ratios taken from ncu."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_fp64_gram_schmidt_is_measured_against_the_fp64_pipe():
    B = _bench()
    # one multi-dot launch of 120 FP64 vectors of 655,360 entries in 174 us (1 FMA per 8 bytes)
    m, n, t_ms = 120, 655360, 0.174
    prof = {"multidot": (t_ms, 1, 8.0 * (m + 1) * n, 2.0 * m * n)}
    r = B.roofline(prof, "multidot", "fp64", "burgers_nx128_n1024")
    assert r["bound"] == "alu" and r["peak"] == B.FP64_TFLOPS_MEASURED
    assert abs(r["achieved"] - 2.0 * m * n / (t_ms / 1e3) / 1e12) < 1e-3
    # the ncu capture of this kernel on this workload: DRAM bytes = algorithmic bytes
    assert r["traffic"] == round(8.0 * (m + 1) * n)


def test_pair_gram_schmidt_is_measured_against_hbm():
    B = _bench()
    m, n, t_ms = 120, 655360, 0.111
    prof = {"pair_dot": (t_ms, 1, 8.0 * (m + 1) * n, 2.0 * m * n),
            "pair_axpy": (t_ms, 1, 8.0 * (m + 2) * n, 2.0 * m * n)}
    hbm, _ = B.measured_peaks()
    for cat in ("pair_dot", "pair_axpy"):
        r = B.roofline(prof, cat, "fp64", "burgers_nx128_n1024")
        assert r["bound"] == "hbm" and r["peak"] == hbm and r["unit"] == "GB/s"
        assert abs(r["frac"] - prof[cat][2] / (t_ms / 1e3) / 1e9 / hbm) < 1e-3
    assert B.roofline(prof, "pair_dot", "fp64", "burgers_nx128_n1024")["traffic"] is not None


def test_fp32_modes_measure_the_vcycle_against_fp32_and_krylov_against_fp64():
    B = _bench()
    prof = {"block_solve": (1.0, 10, 1e9, 5e12), "multidot": (1.0, 10, 1e9, 5e12)}
    assert B.roofline(prof, "block_solve", "fp32")["peak"] == B.FP32_TFLOPS_MEASURED
    assert B.roofline(prof, "multidot", "fp32")["peak"] == B.FP64_TFLOPS_MEASURED
    assert B.roofline({}, "multidot", "fp64")["bound"] is None
