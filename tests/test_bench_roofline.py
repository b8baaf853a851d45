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
    assert r["bound"] == "alu" and r["peak"] == B.PEAKS["fp64_tflops"]
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
    assert B.roofline(prof, "block_solve", "fp32")["peak"] == B.PEAKS["fp32_tflops"]
    assert B.roofline(prof, "multidot", "fp32")["peak"] == B.PEAKS["fp64_tflops"]
    assert B.roofline({}, "multidot", "fp64")["bound"] is None


def test_probe_rate_replaces_the_nominal_peak():
    B = _bench()
    prof = {"multidot": (0.174, 1, 8.0 * 121 * 655360, 2.0 * 120 * 655360)}
    B.PEAKS.update(fp64_tflops=1.2, source="measured in this run")
    r = B.roofline(prof, "multidot", "fp64")
    assert r["peak"] == 1.2 and "measured in this run" in r["peak_source"]


def test_extrapolation_sums_restart_cycles():
    B = _bench()
    # t_j = 2 + 0.5 j exactly: a solve of 7 iterations at restart 4 visits j = 0,1,2,3,0,1,2
    times = [2.0 + 0.5 * j for j in range(6)]
    secs, a, b = B.extrapolate_solve(times, 7, 4)
    assert abs(a - 2.0) < 1e-12 and abs(b - 0.5) < 1e-12
    assert abs(secs - sum(2.0 + 0.5 * j for j in (0, 1, 2, 3, 0, 1, 2))) < 1e-9


def test_error_vs_oracle_reads_the_stored_samples():
    import numpy as np
    B = _bench()
    g = B.golden_direct("vdp_n256")
    assert g is not None and g["relres"] < 1e-11
    torch = __import__("pytest").importorskip("torch")
    x = np.zeros(g["length"])
    for rec in g["types"].values():
        x[np.asarray(rec["indices"])] = rec["values"]
    e = B.error_vs_oracle(torch.tensor(x), "vdp_n256")
    assert e["max_type_rel_err"] == 0.0
    assert e["samples"] == sum(len(r["indices"]) for r in g["types"].values()) == 4 * 512 + 256
    x[g["types"]["mu"]["indices"][3]] += 1e-6 * g["types"]["mu"]["max_abs"]
    e = B.error_vs_oracle(torch.tensor(x), "vdp_n256")
    assert abs(e["per_type"]["mu"] - 1e-6) < 1e-9 and e["per_type"]["u"] == 0.0


def test_oracle_sample_runs_in_a_thread_sized_interpreter():
    """The CPU-baseline legs time the oracle in a fresh interpreter whose BLAS pools are sized by the
    environment (1 thread and every core); a short sample of van der Pol nt = 256 completes iterations."""
    for threads in (1, 2):
        times = _bench().oracle_sample_threads("vdp_n256", 1.0, 1.0, 400, "inject", threads)
        assert len(times) >= 5 and all(t > 0 for t in times)
