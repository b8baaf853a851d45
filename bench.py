#!/usr/bin/env python
"""Benchmark: augmented-system solves per second to a 1e-8 relative residual.

One step = one fgmres_solve from x0 = 0 on one right-hand side: flexible GMRES
preconditioned by the time-multigrid V-cycle (block-Jacobi smoothing,
residual/restriction, prolongation, coarse GMRES with SGS), every kernel of the
path running in libpintmg on one GB300.  Default workload: viscous Burgers
control, P1 elements on nx = 128 interior nodes, nt = 1024 steps, nu = 0.01,
3-level V-cycle with 4/4 block-Jacobi sweeps, FP64, synthetic seeded inputs.

Prints one JSON line (rank 0).  Under torchrun every rank solves its own
system (different seed) with no collective on the data path: weak scaling.
--impl reference times the CPU oracle (FP64, scipy) on a bounded sample of
the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2405_04808_gb300 import replicas as RP  # noqa: E402
from paper_2405_04808_gb300 import workloads as W  # noqa: E402

METRIC = "augmented solves/s to 1e-8 rel. residual: plain FP64 MG vs mixed/learned/batched"
UNIT = "solves/s"
RTOL = 1e-8
L2_FLUSH_BYTES = 512 << 20   # > 129 MB L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="burgers_nx128_n1024", choices=sorted(W.WORKLOADS))
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "fp32s", "bf16"],
                    help="fp32: V-cycle in FP32; fp32s: smoother and transfers in FP32, coarse solve in FP64; "
                         "bf16: the FP32 V-cycle with the smoothing levels' bands stored in BF16")
    ap.add_argument("--restart", type=int, default=None,
                    help="FGMRES restart length (default: the workload's, from a sweep of solve times)")
    ap.add_argument("--krylov-basis", default="fp64", choices=["fp64", "pair", "pair_dcgs2"],
                    help="FGMRES basis storage: FP64 (the plain method, default) or FP32 pairs with compensated "
                         "dot products (an option: ~48-bit basis)")
    ap.add_argument("--omega", type=float, default=1.0,
                    help="block-Jacobi relaxation weight; 1 is the paper's sweep (Eq. jacobi-aj)")
    ap.add_argument("--restrict", default="inject", choices=["inject", "transpose"],
                    help="residual restriction of the V-cycle: the variable formulas of Sec. 5.3.1 (inject, the "
                         "paper as written) or the transpose of the interpolation")
    ap.add_argument("--maxit", type=int, default=2000)
    ap.add_argument("--no-c3", action="store_true", help="skip the Burgers nx=512, nt=8192 block")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true", help="skip the mixed-precision / relaxed-sweep variants")
    ap.add_argument("--host-loops", action="store_true",
                    help="time host-driven Krylov loops instead of one CUDA graph per solve")
    ap.add_argument("--allow-partial", action="store_true",
                    help="accept solves stopped by --maxit (bounded profiler captures only)")
    ap.add_argument("--cpu-sample-seconds", type=float, default=20.0)
    ap.add_argument("--learned-pairs", type=int, default=2000,
                    help="training pairs for the learned coarse correction variant (0 skips it)")
    ap.add_argument("--learned-epochs", type=int, default=4)
    ap.add_argument("--no-batch", action="store_true", help="skip the batched and learned variants")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the library's default SGS chain and dot blocking instead of mg_autotune's")
    # internal: time an oracle sample in this (fresh) interpreter and print the per-iteration times
    ap.add_argument("--oracle-sample", default=None, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.restart is None:
        args.restart = W.WORKLOADS[args.workload].get("restart", 400)
    return args


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        if self.path and os.path.exists(self.path):
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, val in zip(names, parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(nm)
            os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return d.get("hbm_gbs", 6777.0), "measured"
    return 6800.0, "fallback"


# Arithmetic peaks for the ALU-bound kernels.  The FP64 (and FP32) rates are
# measured in this process by the library's FMA-rate probe (probe_fp_rates);
# until then the nominal GB300 FP64 rate (1.25 TFLOP/s, 152 SMs at 2.07 GHz)
# and a nominal FP32 rate (152 SMs x 128 FMA/clk x 2 flop x 2.07 GHz) stand in.
PEAKS = {"fp64_tflops": 1.25, "fp32_tflops": 80.5, "source": "nominal (probe not run)"}


def probe_fp_rates(P, torch, dev, stream):
    """FP64 and FP32 FMA rates of this GPU: mg_probe_fma timed with CUDA events on
    the launching stream (one warm-up launch, best of three), clocks sampled
    during the timed launches.  Updates PEAKS and returns the record."""
    blocks = 8 * torch.cuda.get_device_properties(dev).multi_processor_count
    out = {"blocks": blocks, "threads": P.PROBE_THREADS, "chains_per_thread": P.PROBE_CHAINS}
    with ClockSampler(torch.cuda.current_device()) as clk:
        for label, prec, dtype, iters in (("fp64", P.MG_PRECISION_FP64, torch.float64, 20000),
                                          ("fp32", P.MG_PRECISION_FP32, torch.float32, 400000)):
            sink = torch.empty(blocks * P.PROBE_THREADS, dtype=dtype, device=dev)
            P.mg_probe_fma(prec, blocks, iters, sink.data_ptr(), stream)
            best = None
            for _ in range(3):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                flops = P.mg_probe_fma(prec, blocks, iters, sink.data_ptr(), stream)
                e1.record()
                torch.cuda.synchronize(dev)
                ms = e0.elapsed_time(e1)
                best = ms if best is None else min(best, ms)
            out[f"{label}_tflops"] = round(flops / (best / 1e3) / 1e12, 4)
            out[f"{label}_ms"] = round(best, 3)
            del sink
    out["clocks"] = clk.summary()
    PEAKS.update(fp64_tflops=out["fp64_tflops"], fp32_tflops=out["fp32_tflops"],
                 source="measured in this run by mg_probe_fma (independent FMA chains, CUDA events)")
    return out


# DRAM traffic / algorithmic bytes of a dominant kernel from an ncu capture of
# the same workload (dram__bytes_read.sum + dram__bytes_write.sum per launch);
# valid while the kernel is unchanged since that capture
TRAFFIC_RATIO = {
    ("burgers_nx128_n1024", "multidot", "fp64"): (1.00, "profiles/multidot_burgers_nx128_n1024.md"),
    ("burgers_nx128_n1024", "pair_dot", "fp64"): (1.00, "profiles/multidot_pair_tma_burgers_nx128_n1024.md"),
    ("burgers_nx128_n1024", "block_solve", "fp64"): (1.10, "profiles/block_solve_tri2_burgers_nx128_n1024.md"),
}


def roofline(prof, dominant, precision, workload=None):
    """Roofline object of the dominant kernel category from the library's
    event timings and its algorithmic byte / flop models (per launch).

    FP64 kernels are judged against the larger of their HBM time and their
    FP64-FMA time (PEAKS), FP32 kernels likewise with the FP32 rate; the
    pair-basis Gram-Schmidt kernels (pair_dot, pair_axpy) stream FP32 pairs
    and are judged against HBM only."""
    hbm, peak_kind = measured_peaks()
    ms, n, nbytes, nflops = prof.get(dominant, (0.0, 0, 0.0, 0.0))
    if not n or ms <= 0:
        return {"bound": None, "kernel": dominant, "note": "no timed launches"}
    t = ms / 1e3
    bw = nbytes / t / 1e9
    fl = nflops / t / 1e12
    # the Krylov kernels are FP64 in every mode; the V-cycle's follow the precision mode
    # (the coarse SGS stays FP64 in fp32s)
    pair = dominant in ("pair_dot", "pair_axpy")
    fp64_kernel = not pair and (precision == "fp64" or dominant in ("multidot", "axpy_scale", "arnoldi_scalar", "apply")
                                or (precision == "fp32s" and dominant == "sgs_chain"))
    alu_peak = PEAKS["fp64_tflops"] if fp64_kernel else PEAKS["fp32_tflops"]
    t_hbm = nbytes / (hbm * 1e9)
    t_alu = 0.0 if pair else nflops / (alu_peak * 1e12)
    common = {"kernel": dominant, "launches": n, "avg_launch_us": round(ms * 1e3 / n, 3),
              "bytes_per_launch": round(nbytes / n), "flops_per_launch": round(nflops / n),
              "traffic": None}
    ratio = TRAFFIC_RATIO.get((workload, dominant, precision))
    if ratio:
        common["traffic"] = round(ratio[0] * nbytes / n)
        common["traffic_source"] = f"{ratio[1]}: ncu DRAM bytes = {ratio[0]} x algorithmic bytes"
    if t_alu > t_hbm:
        return {"bound": "alu", "achieved": round(fl, 4), "peak": alu_peak, "unit": "TFLOP/s",
                "frac": round(fl / alu_peak, 4), "achieved_gbs": round(bw, 1), "hbm_peak_gbs": hbm,
                "peak_source": f"{'FP64' if fp64_kernel else 'FP32'} FMA rate, {PEAKS['source']}", **common}
    return {"bound": "hbm", "achieved": round(bw, 1), "peak": hbm, "unit": "GB/s", "frac": round(bw / hbm, 4),
            "achieved_tflops": round(fl, 4), "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)", **common}


#: the reading of the cycle that reproduces Tables 3-4's logarithmic iteration growth:
#: residual restricted by the transpose of the interpolation, weighted sweeps
PAPER_BEHAVIOUR = {"omega": 2.0 / 3.0, "restrict": "transpose", "restart": 60}


def golden_direct(workload):
    path = os.path.join(ROOT, "tests", "golden", "direct_samples.json")
    if not os.path.exists(path):
        return None
    return json.load(open(path)).get(workload)


def error_vs_oracle(x, workload):
    """Largest sampled entry error of each variable type against the oracle's direct
    solution (tests/golden/direct_samples.json, SuperLU), relative to that type's
    largest magnitude; None when no samples are stored for the workload."""
    g = golden_direct(workload)
    if g is None or g["length"] != x.numel():
        return None
    xc = x.detach().cpu().numpy()
    per = {}
    for t, rec in g["types"].items():
        idx = np.asarray(rec["indices"])
        per[t] = float(np.max(np.abs(xc[idx] - np.asarray(rec["values"]))) / rec["max_abs"])
    return {"max_type_rel_err": max(per.values()), "per_type": {k: float(f"{v:.3e}") for k, v in per.items()},
            "samples": sum(len(r["indices"]) for r in g["types"].values()),
            "source": "tests/golden/direct_samples.json (oracle direct solve, oracle/direct_samples.py)"}


def measure(P, torch, prob, wl, args, precision, omega, steps, warmup, dev, stream, world, want_e2e, levels=None,
            basis=None, restrict="inject", restart=None, workload=None):
    """Per-kernel shares and the roofline from one event-bracketed, host-driven
    solve (kernels inside a captured graph cannot be bracketed); then warm-up,
    `steps` timed solves and the end-to-end solves in the timed mode
    (default: one CUDA graph per solve with device-side loops)."""
    prec = {"fp64": P.MG_PRECISION_FP64, "fp32": P.MG_PRECISION_FP32, "fp32s": P.MG_PRECISION_FP32_SMOOTH,
            "bf16": P.MG_PRECISION_BF16_BANDS}[precision]
    lv = levels or wl["levels"]
    restart = restart or args.restart
    workload = workload or args.workload
    b = torch.tensor(prob.b, device=dev)
    x = torch.empty_like(b)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    tuned = {}

    def setup(device_loops):
        h = P.mg_setup(prob, levels=lv, nu_pre=wl["nu_pre"], nu_post=wl["nu_post"], precision=prec,
                       omega=omega, device_loops=device_loops, krylov_basis=basis or args.krylov_basis,
                       restrict=restrict, stream=stream)
        if not args.no_autotune:
            # the library's autotuner: SGS chain evaluation and dot-product blocking for this
            # shape, timed once per process (outside the timed region) and cached
            try:
                chain, vb = P.mg_autotune(h, stream)
            except Exception:
                P.mg_destroy(h)
                raise
            tuned.update(chain=chain, dot_vb=vb,
                         block_warps=[P.mg_block_mapping(h, l) for l in range(lv - 1)])
        return h

    def solve(h, bp, xp):
        code, info = P.fgmres_solve(h, bp, xp, RTOL, args.maxit, restart, stream)
        if code != P.MG_OK and not (args.allow_partial and code == P.MG_NOT_CONVERGED):
            raise RuntimeError(f"fgmres_solve: {P.mg_status_string(code)} (iters {info.iters}, "
                               f"relres {info.relres:.2e}, true {info.true_relres:.2e})")
        return info

    # 1. profiled, host-driven solve: shares of every kernel category, the dominant one's roofline
    hp = setup(False)
    try:
        solve(hp, b.data_ptr(), x.data_ptr())
        P.mg_profile_enable(hp, P.PROFILE_ALL)
        flush.zero_()
        solve(hp, b.data_ptr(), x.data_ptr())
        shares = P.mg_profile_read(hp)
        P.mg_profile_enable(hp, 0)
    finally:
        P.mg_destroy(hp)
    dominant = max(shares, key=lambda k: shares[k][0])
    # 2. timed solves
    t0 = time.perf_counter()
    h = setup(not args.host_loops)
    torch.cuda.synchronize(dev)
    setup_ms = (time.perf_counter() - t0) * 1e3
    try:
        for _ in range(warmup):
            flush.zero_()
            solve(h, b.data_ptr(), x.data_ptr())
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        launches0 = P.mg_launch_count(h)
        infos = []
        with ClockSampler(torch.cuda.current_device()) as clk:
            for i in range(steps):
                flush.zero_()
                ev[i][0].record()
                infos.append(solve(h, b.data_ptr(), x.data_ptr()))
                ev[i][1].record()
            torch.cuda.synchronize(dev)
        launches = P.mg_launch_count(h) - launches0
        gl = P.mg_graph_launches(h)
        graph_launches = (None if gl[0] != P.MG_OK else
                          {"fixed": gl[1], "per_fgmres_iteration": gl[2], "per_coarse_iteration": gl[3]})
        if world > 1:
            torch.distributed.barrier()
        local_ms = sum(a.elapsed_time(bb) for a, bb in ev)
        value = RP.job_throughput(local_ms / 1e3, steps, world, device=dev)
        total_ms = 1e3 * world * steps / value   # the slowest rank's time
        out = {"value": value, "ms_per_step": total_ms / steps, "x": x.clone(),
               "iters": [i.iters for i in infos], "true_relres": max(i.true_relres for i in infos),
               "coarse_iters_per_vcycle": sum(i.coarse_iters for i in infos) / max(1, sum(i.vcycles for i in infos)),
               "setup_ms": setup_ms, "launches": launches, "graph_launches": graph_launches,
               "shares": shares, "dominant": dominant,
               "roofline": roofline(shares, dominant, precision, workload if levels is None else None),
               "category_rooflines": {k: roofline(shares, k, precision, workload if levels is None else None)
                                      for k in shares if shares[k][1] and shares[k][2] > 0},
               "error_vs_oracle": error_vs_oracle(x, workload),
               "autotune": dict(tuned) or None,
               "clocks": clk.summary()}
        if want_e2e:
            # end to end through the public API with pinned host buffers
            bh = torch.tensor(prob.b).pin_memory()
            xh = torch.empty_like(bh).pin_memory()
            solve(h, bh.data_ptr(), xh.data_ptr())   # capture for the staging buffers (not timed)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            for _ in range(steps):
                solve(h, bh.data_ptr(), xh.data_ptr())
            e2e_value = RP.job_throughput(time.perf_counter() - t0, steps, world, device=dev)
            out["e2e"] = {"value": round(e2e_value, 4), "unit": UNIT,
                          "h2d_bytes_per_step": 8 * prob.size, "d2h_bytes_per_step": 8 * prob.size}
        return out
    finally:
        P.mg_destroy(h)


def measure_batch(P, torch, args, dev, stream, omega, restrict, restart):
    """The batched workload (64 uneven systems: van der Pol nt 512-16384,
    Burgers nx 64-256 x nt 512-4096, 4 levels each): one graph launch for all
    systems (FP64, and with the FP32 V-cycle) against one plain FP64 solve at a
    time.  The cycle of the paper-behaviour reading (residual restricted by the
    transpose of the interpolation, weighted sweeps): with the literal cycle the
    larger members do not converge within the iteration cap."""
    import os
    systems = W.batch_uneven(workers=max(1, min(16, os.cpu_count() or 1)))
    res = {"systems": len(systems), "unknowns": int(sum(p.size for p, _ in systems)), "omega": omega,
           "restrict": restrict, "restart": restart,
           "workload": "64 uneven systems: vdP nt 512-16384, Burgers nx 64-256 x nt 512-4096"}
    for label, prec, reps in (("sequential_fp64", P.MG_PRECISION_FP64, 1), ("batched_fp64", P.MG_PRECISION_FP64, 2),
                              ("batched_fp32_vcycle", P.MG_PRECISION_FP32, 2)):
        hs, bs, xs = [], [], []
        try:
            for prob, opts in systems:
                hs.append(P.mg_setup(prob, omega=omega, precision=prec, restrict=restrict, stream=stream, **opts))
                bs.append(torch.tensor(prob.b, device=dev))
                xs.append(torch.empty_like(bs[-1]))
            tuned = None
            if label.startswith("batched"):
                # the autotuner picks each shape's chain evaluation and dot blocking (cached per shape)
                t0 = time.perf_counter()
                picks = [P.mg_autotune(h, stream) for h in hs]
                tuned = {"ms": round((time.perf_counter() - t0) * 1e3, 1),
                         "chains": {c: sum(1 for p_ in picks if p_[0] == c) for c in P.SGS_CHAINS},
                         "dot_vb": {str(v): sum(1 for p_ in picks if p_[1] == v) for v in (4, 8, 16)}}

            def run_once():
                if label.startswith("sequential"):
                    iters = []
                    for h, b, x in zip(hs, bs, xs):
                        code, info = P.fgmres_solve(h, b.data_ptr(), x.data_ptr(), RTOL, args.maxit, restart, stream)
                        if code != P.MG_OK:
                            raise RuntimeError("batch member did not converge")
                        iters.append(info.iters)
                    return iters
                code, infos = P.fgmres_solve_batched(hs, [b.data_ptr() for b in bs], [x.data_ptr() for x in xs],
                                                     RTOL, args.maxit, restart, stream)
                if code != P.MG_OK:
                    raise RuntimeError(f"batched solve: {P.mg_status_string(code)}")
                return [i.iters for i in infos]

            run_once()
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                iters = run_once()
            e1.record()
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1) / reps
            res[label] = {"solves_per_s": round(len(systems) / (ms / 1e3), 3), "ms_per_batch": round(ms, 3),
                          "iters_min_max": [min(iters), max(iters)]}
            if tuned:
                res[label]["autotune"] = tuned
        finally:
            for h in hs:
                P.mg_destroy(h)
            del bs, xs
            torch.cuda.empty_cache()
    return res


def measure_paper_behaviour(P, torch, prob, wl, args, dev, stream, world, variant_entry):
    """The headline workload under the reading that reproduces Tables 3-4's
    iteration growth (residual restricted by the transpose of the
    interpolation, weighted sweeps omega = 2/3, restart 60): the same metric
    end to end and on the device, its kernel shares and roofline, and its
    precision / basis variants."""
    pb = PAPER_BEHAVIOUR
    m = measure(P, torch, prob, wl, args, "fp64", pb["omega"], args.steps, args.warmup, dev, stream, world, True,
                restrict=pb["restrict"], restart=pb["restart"])
    out = {"reading": "residual restricted by the transpose of the interpolation (R = P^T), block-Jacobi sweeps "
                      "weighted by omega = 2/3; Sec. 5.3.1 as written injects, Eq. (jacobi-aj) is undamped",
           "value": round(m["value"], 4), "unit": UNIT, "ms_per_step": round(m["ms_per_step"], 3),
           "fgmres_iters": m["iters"], "true_relres": m["true_relres"], "error_vs_oracle": m["error_vs_oracle"],
           "oracle_iters": oracle_iterations(args.workload, pb["omega"], pb["restart"], pb["restrict"]),
           "coarse_iters_per_vcycle": round(m["coarse_iters_per_vcycle"], 3), "setup_ms": round(m["setup_ms"], 2),
           "e2e": m["e2e"], "gpu_launches": m["launches"], "graph_launches": m["graph_launches"],
           "roofline": m["roofline"],
           "category_rooflines": {k: {"bound": v["bound"], "frac": v.get("frac"), "achieved": v.get("achieved"),
                                      "unit": v.get("unit"), "avg_launch_us": v.get("avg_launch_us")}
                                  for k, v in m["category_rooflines"].items()},
           "kernel_shares": {k: {"ms": round(v[0], 3), "launches": v[1]} for k, v in m["shares"].items() if v[1]},
           "clocks": m["clocks"], "omega": pb["omega"], "restrict": pb["restrict"], "restart": pb["restart"],
           "variants": {}}
    for name, prec, kb in (("fp32_vcycle", "fp32", None), ("fp32_smoother_fp64_coarse", "fp32s", None),
                           ("bf16_bands_fp32_vcycle", "bf16", None), ("pair_krylov_basis", "fp64", "pair"),
                           ("pair_dcgs2_krylov_basis", "fp64", "pair_dcgs2")):
        v = measure(P, torch, prob, wl, args, prec, pb["omega"], max(1, min(args.steps, 3)), 1, dev, stream, world,
                    False, basis=kb, restrict=pb["restrict"], restart=pb["restart"])
        out["variants"][name] = variant_entry(v, prec, pb["omega"], None, kb, pb["restrict"], pb["restart"])
    return out


C3_WORKLOAD = "burgers_nx512_n8192"


def measure_c3(P, torch, args, dev, stream, world):
    """Burgers nx = 512, nt = 8192 (21 M unknowns, 168 MB per FP64 vector, four
    levels, 4/4 sweeps), the mixed-precision configuration: the paper-behaviour
    reading in FP64, with the FP32 V-cycle, with FP32 smoothing and an FP64
    coarse solve, and with the FP32 V-cycle reading BF16 bands; each solve's
    iterations at 1e-8 and its FP64 true residual
    (the library's operator; the oracle's assembled operator checks the same
    residual in tests/test_gpu_fullsize.py)."""
    wl = W.WORKLOADS[C3_WORKLOAD]
    prob = wl["make"]()
    pb = PAPER_BEHAVIOUR
    res = {"workload": C3_WORKLOAD, "n": prob.n, "p": prob.p, "unknowns": prob.size, "levels": wl["levels"],
           "omega": pb["omega"], "restrict": pb["restrict"], "restart": pb["restart"]}
    ref_x = None
    for name, prec in (("fp64", "fp64"), ("fp32_vcycle", "fp32"), ("fp32_smoother_fp64_coarse", "fp32s"),
                       ("bf16_bands_fp32_vcycle", "bf16")):
        v = measure(P, torch, prob, wl, args, prec, pb["omega"], max(1, min(args.steps, 3)), 1, dev, stream, world,
                    False, restrict=pb["restrict"], restart=pb["restart"], workload=C3_WORKLOAD)
        entry = {"value": round(v["value"], 4), "unit": UNIT, "ms_per_step": round(v["ms_per_step"], 3),
                 "fgmres_iters": v["iters"][0], "true_relres": v["true_relres"],
                 "coarse_iters_per_vcycle": round(v["coarse_iters_per_vcycle"], 3), "setup_ms": round(v["setup_ms"], 1),
                 "dominant_kernel": v["dominant"], "roofline": v["roofline"],
                 "category_rooflines": {k: {"bound": c["bound"], "frac": c.get("frac"), "achieved": c.get("achieved"),
                                            "unit": c.get("unit")} for k, c in v["category_rooflines"].items()},
                 "kernel_shares": {k: {"ms": round(c[0], 3), "launches": c[1]} for k, c in v["shares"].items() if c[1]},
                 "clocks": v["clocks"]}
        if ref_x is None:
            ref_x = v["x"]
        else:
            entry["solution_rel_diff_vs_fp64"] = float(torch.linalg.vector_norm(v["x"] - ref_x) /
                                                       torch.linalg.vector_norm(ref_x))
        res[name] = entry
        del v
        torch.cuda.empty_cache()
    return res


def oracle_full_solve(prob, wl, reading):
    """One complete oracle solve (FGMRES to 1e-8 from x0 = 0, SuperLU
    factorisations included) on the host cores, once with the BLAS thread pool
    limited to one thread and once unrestricted."""
    from oracle import augmented as O
    try:
        from threadpoolctl import threadpool_limits
    except ImportError:   # not installed on every host
        threadpool_limits = None
    out = {"kind": "oracle", "reading": f"omega {reading['omega']:.4g}, restrict {reading['restrict']}, "
                                        f"restart {reading['restart']}"}
    for label, limit in (("threads_1", 1), ("threads_all", None)):
        if limit is not None and threadpool_limits is None:
            continue
        ctx = threadpool_limits(limits=limit) if (limit is not None) else _Null()
        with ctx:
            t0 = time.perf_counter()
            hier = O.Hierarchy(prob, O.MGOptions(levels=wl["levels"], nu_pre=wl["nu_pre"], nu_post=wl["nu_post"],
                                                 omega=reading["omega"], restrict=reading["restrict"]))
            x, res, tr = hier.solve(prob.b, rtol=RTOL, maxit=2000, restart=reading["restart"])
            secs = time.perf_counter() - t0
        out[label] = {"seconds": round(secs, 2), "solves_per_s": round(1.0 / secs, 5), "iters": res.iters,
                      "true_relres": tr, "cores": 1 if limit == 1 else os.cpu_count()}
    return out


class _Null:
    def __enter__(self):
        return self

    def __exit__(self, *exc):
        return False


LEARNED_WORKLOAD = "burgers_nx256_n4096"


def measure_learned(P, torch, args, dev, stream, omega, restrict, restart):
    """The learned coarse correction on its own workload (Burgers nx=256,
    nt=4096): collect the plain method's coarse pairs from seeded runs
    (host-driven solves with recording), train the network with the library's
    kernels, then time graph-mode solves of a held-out system with and
    without it.  The cycle of the paper-behaviour reading (residual restricted
    by the transpose of the interpolation, weighted sweeps): the literal cycle
    does not reach 1e-8 within 3000 iterations here."""
    from paper_2405_04808_gb300 import learned as LN
    wl = W.WORKLOADS[LEARNED_WORKLOAD]
    settings = dict(levels=wl["levels"], nu_pre=wl["nu_pre"], nu_post=wl["nu_post"], omega=omega, restrict=restrict)
    res = {"workload": LEARNED_WORKLOAD, "restart": restart, "omega": omega, "restrict": restrict,
           "levels": wl["levels"], "admit": 0.5,
           "inference": "bf16 on the tensor cores (tcgen05.mma kind::f16, M=128 positions, accumulators in TMEM), fp32 accumulation"}
    t0 = time.perf_counter()
    import os
    per = 20  # a solve to 1e-12 records one pair per FGMRES iteration (about 25 here)
    nprob = (args.learned_pairs + per - 1) // per
    train_probs = W.make_many(LEARNED_WORKLOAD, [wl["seed"] + 1 + k for k in range(nprob)],
                              workers=max(1, min(16, os.cpu_count() or 1)))
    R, Y = LN.collect_pairs(train_probs, settings, args.learned_pairs, rtol=1e-12, restart=restart,
                            per_problem=per)
    torch.cuda.synchronize(dev)
    res["pairs"] = int(R.shape[0])
    res["collect_s"] = round(time.perf_counter() - t0, 2)
    _, _, T, X = R.shape
    # two networks from the same initial parameters and pairs: the mean squared error against the
    # coarse solutions, and the residual metric of the first training system's coarse operator (the
    # quantity the admission test measures)
    nets = {}
    hm = P.mg_setup(train_probs[0], stream=stream, **settings)
    try:
        fl = 3 * 2.0 * T * X * 21 * (5 * 32 + 32 * 32 + 32 * 32 + 32 * 5) * R.shape[0] * args.learned_epochs
        res["coarse_shape"] = [5, T, X]
        res["epochs"] = args.learned_epochs
        for name, metric in (("mse", None), ("metric", hm)):
            # the metric-trained network starts from a zero output layer (proposal 0, residual r)
            nets[name] = LN.new_net(wl["seed"], zero_output=metric is not None)
            t0 = time.perf_counter()
            losses = LN.train(nets[name], R, Y, epochs=args.learned_epochs, batch=8, lr=1e-3, seed=1, metric=metric)
            torch.cuda.synchronize(dev)
            train_s = time.perf_counter() - t0
            res[f"train_{name}"] = {"loss": "mean((net(r) - y)^2)" if metric is None else
                                    "mean((A_c (net(r) - y))^2), A_c the coarse operator of training system 0",
                                    "train_s": round(train_s, 2), "epoch_loss": [round(float(l), 5) for l in losses],
                                    "train_tflops_conv": round(fl / train_s / 1e12, 2)}
    finally:
        P.mg_destroy(hm)
    try:
        del R, Y
        prob = wl["make"]()
        b = torch.tensor(prob.b, device=dev)
        x = torch.empty_like(b)
        for name, nt in (("plain", None), ("learned_mse", nets["mse"]), ("learned", nets["metric"])):
            # kernel shares (net inference included) from one profiled host-driven solve
            hp = P.mg_setup(prob, device_loops=False, stream=stream, **settings)
            try:
                if nt:
                    P.mg_attach_coarse_net(hp, nt, admit=0.5, bf16=True)
                P.fgmres_solve(hp, b.data_ptr(), x.data_ptr(), RTOL, args.maxit, restart, stream)
                P.mg_profile_enable(hp, P.PROFILE_ALL)
                P.fgmres_solve(hp, b.data_ptr(), x.data_ptr(), RTOL, args.maxit, restart, stream)
                shares = P.mg_profile_read(hp)
                P.mg_profile_enable(hp, 0)
            finally:
                P.mg_destroy(hp)
            h = P.mg_setup(prob, stream=stream, **settings)
            try:
                if nt:
                    P.mg_attach_coarse_net(h, nt, admit=0.5, bf16=True)
                code, info = P.fgmres_solve(h, b.data_ptr(), x.data_ptr(), RTOL, args.maxit, restart, stream)
                if code != P.MG_OK and nt is None:
                    raise RuntimeError(f"learned variant {name}: {P.mg_status_string(code)}")
                torch.cuda.synchronize(dev)
                reps = max(1, min(args.steps, 3))
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(reps):
                    code, info = P.fgmres_solve(h, b.data_ptr(), x.data_ptr(), RTOL, args.maxit, restart,
                                                stream)
                e1.record()
                torch.cuda.synchronize(dev)
                ms = e0.elapsed_time(e1) / reps
            finally:
                P.mg_destroy(h)
            # a network's admitted proposals can stall FGMRES: then the solve rate is that of unconverged solves
            entry = {"status": P.mg_status_string(code), "converged": code == P.MG_OK,
                     "solves_per_s": round(1e3 / ms, 4) if code == P.MG_OK else 0.0, "ms_per_solve": round(ms, 2),
                     "fgmres_iters": info.iters,
                     "true_relres": info.true_relres, "coarse_gmres_iters": info.coarse_iters,
                     "coarse_solves_by_network": info.coarse_learned, "vcycles": info.vcycles,
                     "kernel_shares": {k: round(v[0], 3) for k, v in shares.items() if v[1]}}
            if "net_coarse" in shares and shares["net_coarse"][1]:
                ms_net, n_net, _, fl_net = shares["net_coarse"]
                total = sum(v[0] for v in shares.values())
                entry.update(net_share=round(ms_net / total, 4), net_tflops=round(fl_net / ms_net / 1e9, 2))
            res[name] = entry
        res["speedup_learned_vs_plain"] = round(res["learned"]["solves_per_s"] / res["plain"]["solves_per_s"], 4)
        res["speedup_learned_mse_vs_plain"] = round(res["learned_mse"]["solves_per_s"] /
                                                    res["plain"]["solves_per_s"], 4)
    finally:
        for nt in nets.values():
            P.mg_net_destroy(nt)
    return res


def run_native(args):
    import torch

    from paper_2405_04808_gb300 import pintmg as P

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev).cuda_stream
    wl = W.WORKLOADS[args.workload]
    prob = wl["make"](seed=RP.rank_seed(wl["seed"], rank))
    fp_probe = probe_fp_rates(P, torch, dev, stream)
    main = measure(P, torch, prob, wl, args, args.precision, args.omega, args.steps, args.warmup, dev, stream,
                   world, True, restrict=args.restrict)

    def variant_entry(v, prec, om, lv, kb, restrict, restart):
        # the variant's solution against the headline solve's (both to a 1e-8 relative residual)
        xdiff = float(torch.linalg.vector_norm(v["x"] - main["x"]) / torch.linalg.vector_norm(main["x"]))
        return {"value": round(v["value"], 4), "unit": UNIT, "ms_per_step": round(v["ms_per_step"], 3),
                "fgmres_iters": v["iters"][0], "true_relres": v["true_relres"],
                "error_vs_oracle": v["error_vs_oracle"], "solution_rel_diff_vs_main": xdiff,
                "precision": prec, "omega": om, "restrict": restrict, "restart": restart,
                "levels": lv or wl["levels"], "krylov_basis": kb or args.krylov_basis,
                "coarse_iters_per_vcycle": round(v["coarse_iters_per_vcycle"], 3),
                "setup_ms": round(v["setup_ms"], 1),
                "dominant_kernel": v["dominant"], "roofline_frac": v["roofline"].get("frac")}

    variants = {}
    paper = None
    if not args.no_variants:
        # (name, precision, omega, levels, basis): the other Krylov basis, the mixed-precision
        # V-cycle, and the paper's serial baseline of Sec. 6.3 (SGS-GMRES, no multigrid), whose
        # block Gauss-Seidel chains run here as a parallel scan in time
        other = "fp64" if args.krylov_basis == "pair" else "pair"
        for name, prec, om, lv, kb in ((f"{other}_krylov_basis", args.precision, args.omega, None, other),
                                       ("pair_dcgs2_krylov_basis", args.precision, args.omega, None, "pair_dcgs2"),
                                       ("fp32_vcycle", "fp32", args.omega, None, None),
                                       ("fp32_smoother_fp64_coarse", "fp32s", args.omega, None, None),
                                       ("sgs_gmres_no_multigrid", "fp64", 1.0, 1, None)):
            if prec == args.precision and om == args.omega and lv is None and kb is None:
                continue
            v = measure(P, torch, prob, wl, args, prec, om, max(1, min(args.steps, 3)), 1, dev, stream, world, False,
                        levels=lv, basis=kb, restrict=args.restrict)
            variants[name] = variant_entry(v, prec, om, lv, kb, args.restrict, args.restart)
        paper = measure_paper_behaviour(P, torch, prob, wl, args, dev, stream, world, variant_entry)
    c3 = None if (args.no_variants or args.no_c3) else measure_c3(P, torch, args, dev, stream, world)
    batch = None if (args.no_variants or args.no_batch) else measure_batch(P, torch, args, dev, stream,
                                                                           omega=PAPER_BEHAVIOUR["omega"],
                                                                           restrict=PAPER_BEHAVIOUR["restrict"],
                                                                           restart=PAPER_BEHAVIOUR["restart"])
    learned = (None if (args.no_variants or args.no_batch or args.learned_pairs <= 0)
               else measure_learned(P, torch, args, dev, stream, **PAPER_BEHAVIOUR))
    out = {
        "metric": METRIC, "value": round(main["value"], 4), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(main["ms_per_step"], 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64",
        "data": "synthetic (seeded iterate and N(0,1) right-hand side)",
        "config": {"workload": args.workload, "n": prob.n, "p": prob.p, "q": prob.q,
                   "levels": wl["levels"], "nu_pre": wl["nu_pre"], "nu_post": wl["nu_post"],
                   "unknowns": prob.size, "rtol": RTOL, "restart": args.restart, "precision": args.precision,
                   "krylov_basis": ("FP64 entries rounded to ~48 bits as FP32 pairs; compensated (Dot2) dot products "
                                    "and axpys against them, FP64 reductions" if args.krylov_basis == "pair"
                                    else "FP64"),
                   "omega": args.omega, "restrict": args.restrict,
                   "l2": "flushed (512 MB write) before every timed step",
                   "solve": "host-driven loops" if args.host_loops else
                            "one CUDA graph per solve (FGMRES and coarse GMRES loops as conditional nodes)",
                   "roofline_source": "event-bracketed kernels of one host-driven solve of the same system",
                   "parallelism": f"replicas{world}"},
        "fgmres_iters": main["iters"], "true_relres": main["true_relres"],
        "error_vs_oracle": main["error_vs_oracle"],
        "coarse_iters_per_vcycle": round(main["coarse_iters_per_vcycle"], 3),
        "setup_ms": round(main["setup_ms"], 2),
        "e2e": main["e2e"],
        "gpu_launches": main["launches"],
        "graph_launches": main["graph_launches"],
        "autotune": main["autotune"],
        "roofline": main["roofline"],
        "category_rooflines": {k: {"bound": v["bound"], "frac": v.get("frac"), "achieved": v.get("achieved"),
                                   "unit": v.get("unit"), "avg_launch_us": v.get("avg_launch_us")}
                               for k, v in main["category_rooflines"].items()},
        "kernel_shares": {k: {"ms": round(v[0], 3), "launches": v[1]} for k, v in main["shares"].items() if v[1]},
        "variants": variants,
        "paper_behaviour": paper,
        "c3": c3,
        "fp_rate_probe": fp_probe,
        "batched": batch,
        "learned_coarse": learned,
        "clocks": main["clocks"],
    }
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(prob, wl, args, main["iters"])
        if paper is not None:
            paper["cpu_full_solve"] = oracle_full_solve(prob, wl, PAPER_BEHAVIOUR)
    if world > 1:
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


def oracle_iterations(workload, omega, restart, restrict="inject"):
    """The oracle's own FGMRES iteration count for a full solve of this
    workload (tests/golden/oracle_iterations.json, written by
    oracle/measure_iterations.py), or None."""
    rec = oracle_record(workload, omega, restart, restrict)
    return rec["iters"] if rec else None


def oracle_record(workload, omega, restart, restrict="inject"):
    path = os.path.join(ROOT, "tests", "golden", "oracle_iterations.json")
    if not os.path.exists(path):
        return None
    key = f"{workload}/omega={float(omega)}/restart={restart}"
    if restrict == "transpose":
        key += "/restrict=transpose"
    rec = json.load(open(path)).get(key)
    if rec and rec.get("restart") == restart and rec.get("rtol") == RTOL:
        return rec
    return None


def oracle_sample(prob, wl, omega, seconds, restart, restrict="inject", limit=True):
    """Time the oracle as it stands: its FGMRES on this system for about
    `seconds` (setup, i.e. the sparse LU factorisations, excluded), with the
    BLAS thread pool limited to one thread where threadpoolctl is available
    (limit=False: as the environment sized it).  Returns the duration of every
    completed FGMRES iteration (V-cycle, operator product and the modified
    Gram-Schmidt of that iteration), in seconds."""
    from oracle import augmented as O
    ctx = _Null()
    if limit:
        try:
            from threadpoolctl import threadpool_limits
            ctx = threadpool_limits(limits=1)
        except ImportError:
            pass
    with ctx:
        hier = O.Hierarchy(prob, O.MGOptions(levels=wl["levels"], nu_pre=wl["nu_pre"], nu_post=wl["nu_post"],
                                             omega=omega, restrict=restrict))
        lev = hier.fine
        bt = lev.to_time_major(prob.b)
        hier.vcycle(0, bt)  # builds the factorisations
        stamps = []

        class Stop(Exception):
            pass

        def prec(v):
            stamps.append(time.perf_counter())   # start of an iteration
            if stamps[-1] - stamps[0] > seconds:
                raise Stop()
            return hier.vcycle(0, v)

        try:
            O.fgmres(lambda v: lev.At @ v, prec, bt, rtol=RTOL, maxit=100000, restart=restart)
        except Stop:
            pass
    return [b - a for a, b in zip(stamps, stamps[1:])]


BLAS_THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS",
                    "VECLIB_MAXIMUM_THREADS", "NUMEXPR_NUM_THREADS")


def oracle_sample_threads(workload, omega, seconds, restart, restrict, threads):
    """oracle_sample in a fresh interpreter whose BLAS thread pools are sized to
    `threads` through the environment before numpy loads (the one portable
    way to size them without threadpoolctl).  The child runs this file with
    --oracle-sample and imports no torch.  Returns the per-iteration times."""
    spec = json.dumps({"workload": workload, "omega": omega, "seconds": seconds, "restart": restart,
                       "restrict": restrict})
    env = dict(os.environ)
    for var in BLAS_THREAD_VARS:
        env[var] = str(threads)
    res = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample", spec], env=env,
                         capture_output=True, text=True, timeout=30 * seconds + 300, check=True)
    return json.loads(res.stdout.strip().splitlines()[-1])["times"]


def oracle_sample_main(spec):
    d = json.loads(spec)
    wl = W.WORKLOADS[d["workload"]]
    times = oracle_sample(wl["make"](), wl, d["omega"], d["seconds"], d["restart"], d["restrict"], limit=False)
    print(json.dumps({"times": times}), flush=True)


def extrapolate_solve(times, iters, restart):
    """Seconds of a full solve of `iters` FGMRES iterations at this restart from
    sampled per-iteration durations: t_j = a + b j in the basis index j (the
    V-cycle and operator product are constant, the Gram-Schmidt sweep grows
    with j), fitted by least squares over the sampled iterations and summed
    over the solve's restart cycles."""
    j = np.arange(len(times), dtype=np.float64)
    if len(times) >= 3:
        b, a = np.polyfit(j, np.asarray(times), 1)
        b = max(b, 0.0)
        a = float(np.mean(times) - b * np.mean(j))
    else:
        a, b = float(np.mean(times)), 0.0
    idx = np.arange(iters) % restart
    return float(np.sum(a + b * idx)), a, b


def cpu_baseline(prob, wl, args, gpu_iters):
    """The oracle as it stands on the host cores, twice: BLAS pools of one
    thread and of every core (SuperLU and scipy's sparse products are
    single-threaded either way; only the dense BLAS calls can use more).  The
    faster leg is the value, its thread count the cores."""
    rec = oracle_record(args.workload, args.omega, args.restart, args.restrict)
    n_it = rec["iters"] if rec else int(round(statistics.mean(gpu_iters)))
    src = "the oracle's own full-solve count" if rec else "the GPU solve's count"
    nproc = os.cpu_count() or 1
    legs = {}
    for threads in sorted({1, nproc}):
        times = oracle_sample_threads(args.workload, args.omega, args.cpu_sample_seconds, args.restart,
                                      args.restrict, threads)
        secs, a, b = extrapolate_solve(times, n_it, args.restart)
        legs[threads] = {"value": round(1.0 / secs, 6), "threads": threads, "sampled_iterations": len(times),
                         "fit_ms": [round(a * 1e3, 2), round(b * 1e3, 4)]}
    best = max(legs.values(), key=lambda v: v["value"])
    a_ms, b_ms = best["fit_ms"]
    out = {"value": best["value"], "unit": UNIT, "cores": best["threads"], "kind": "oracle", "extrapolated": True,
           "sampled_iterations": best["sampled_iterations"],
           "legs": {f"{t}_threads": v for t, v in legs.items()},
           "sample": f"{best['sampled_iterations']} timed oracle FGMRES iterations of this solve ({best['threads']} "
                     f"BLAS threads, the faster of 1 and {nproc}; SuperLU factorisations excluded), fitted as "
                     f"{a_ms:.0f} ms + {b_ms:.2f} ms per basis vector and summed over {n_it} iterations at restart "
                     f"{args.restart} ({src}); scipy/SuperLU on the host cores of the GPU box"}
    if rec and rec.get("seconds"):
        out["recorded_full_solve_s"] = rec["seconds"]
        out["recorded_full_solve_note"] = ("one complete oracle solve, timed when oracle/measure_iterations.py "
                                           "recorded the count (build host, not the GPU box)")
    return out


def run_reference(args):
    """--impl reference: the CPU oracle as it stands.  A full solve of the
    literal cycle takes minutes, so each step times a bounded sample of the
    solve's iterations and the line reports the extrapolated full-solve rate
    (marked "extrapolated")."""
    rank, world, local = dist_env()
    if rank != 0:
        return
    per_step = max(5.0, min(30.0, 150.0 / max(1, args.steps + args.warmup)))
    rec = oracle_record(args.workload, args.omega, args.restart, args.restrict)
    n_it = rec["iters"] if rec else None
    nproc = os.cpu_count() or 1
    solve_s, sampled, wall = [], 0, time.perf_counter()
    for k in range(args.warmup + args.steps):
        times = oracle_sample_threads(args.workload, args.omega, per_step, args.restart, args.restrict, nproc)
        if k >= args.warmup and n_it:
            solve_s.append(extrapolate_solve(times, n_it, args.restart)[0])
            sampled += len(times)
    wall = time.perf_counter() - wall
    secs = statistics.mean(solve_s) if solve_s else None
    value = round(1.0 / secs, 6) if secs else None
    line = {"metric": METRIC, "impl": "reference", "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(secs * 1e3, 1) if secs else None,
            "extrapolated": True, "sampled_iterations": sampled, "sample_seconds_per_step": per_step,
            "wall_s": round(wall, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded iterate and N(0,1) right-hand side)",
            "config": {"workload": args.workload, "restart": args.restart, "omega": args.omega,
                       "restrict": args.restrict, "rtol": RTOL},
            "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": nproc, "extrapolated": True,
                             "sample": f"per step about {per_step:.0f} s of timed oracle FGMRES iterations ({nproc} "
                                       f"BLAS threads; SuperLU and the sparse products use one), fitted in the basis "
                                       f"index and summed over the oracle's {n_it} "
                                       f"iterations per full solve at restart {args.restart}; ms_per_step is that "
                                       f"extrapolated full solve, not the sample"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    if rec and rec.get("seconds"):
        line["recorded_full_solve_s"] = rec["seconds"]
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.oracle_sample:
        oracle_sample_main(args.oracle_sample)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
