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
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32", "fp32s"],
                    help="fp32: V-cycle in FP32; fp32s: smoother and transfers in FP32, coarse solve in FP64")
    ap.add_argument("--restart", type=int, default=None,
                    help="FGMRES restart length (default: the workload's, from a sweep of solve times)")
    ap.add_argument("--krylov-basis", default="fp64", choices=["fp64", "pair"],
                    help="FGMRES basis storage: FP64 (the plain method, default) or FP32 pairs with compensated "
                         "dot products (an option: ~48-bit basis)")
    ap.add_argument("--omega", type=float, default=1.0,
                    help="block-Jacobi relaxation weight; 1 is the paper's sweep (Eq. jacobi-aj)")
    ap.add_argument("--maxit", type=int, default=2000)
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


# FP64 peak of this GB300 for the ALU-bound kernels: 152 SMs x 4 sub-partitions
# x 0.5 FP64 FMA/clk x 2 flop x 2.07 GHz = 1.259 TFLOP/s nominal; a
# throughput probe (independent FMA chains, 4+ warps per SM) measured
# 1.196 TFLOP/s, which is the peak used here.
FP64_TFLOPS_MEASURED = 1.196
FP32_TFLOPS_MEASURED = 74.2


# DRAM traffic / algorithmic bytes of a dominant kernel from an ncu capture of
# the same workload (dram__bytes_read.sum + dram__bytes_write.sum per launch);
# valid while the kernel is unchanged since that capture
TRAFFIC_RATIO = {
    ("burgers_nx128_n1024", "multidot", "fp64"): (1.00, "profiles/multidot_burgers_nx128_n1024.md"),
    ("burgers_nx128_n1024", "pair_dot", "fp64"): (1.00, "profiles/multidot_pair_tma_burgers_nx128_n1024.md"),
    ("burgers_nx128_n1024", "block_solve", "fp64"): (1.21, "profiles/block_solve_tri2_burgers_nx128_n1024.md"),
}


def roofline(prof, dominant, precision, workload=None):
    """Roofline object of the dominant kernel category from the library's
    event timings and its algorithmic byte / flop models (per launch)."""
    hbm, peak_kind = measured_peaks()
    ms, n, nbytes, nflops = prof.get(dominant, (0.0, 0, 0.0, 0.0))
    if not n or ms <= 0:
        return {"bound": None, "kernel": dominant, "note": "no timed launches"}
    t = ms / 1e3
    bw = nbytes / t / 1e9
    fl = nflops / t / 1e12
    # the Krylov kernels are FP64 in every mode; the V-cycle's follow the precision mode
    # (the coarse SGS stays FP64 in fp32s)
    # the pair-basis Gram-Schmidt kernels (pair_dot, pair_axpy) run in FP32 arithmetic, ~6 FP32
    # operations per FP64-equivalent flop counted in their models
    pair = dominant in ("pair_dot", "pair_axpy")
    fp64_kernel = not pair and (precision == "fp64" or dominant in ("multidot", "axpy_scale", "arnoldi_scalar", "apply")
                                or (precision == "fp32s" and dominant == "sgs_chain"))
    alu_peak = FP64_TFLOPS_MEASURED if fp64_kernel else FP32_TFLOPS_MEASURED / (6.0 if pair else 1.0)
    t_hbm = nbytes / (hbm * 1e9)
    t_alu = nflops / (alu_peak * 1e12)
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
                "peak_source": "measured FP64 FMA probe (1.196 of 1.259 nominal TFLOP/s)" if fp64_kernel
                else ("measured FP32 FMA probe / 6 FP32 operations per counted flop" if pair
                      else "measured FP32 FMA probe"), **common}
    return {"bound": "hbm", "achieved": round(bw, 1), "peak": hbm, "unit": "GB/s", "frac": round(bw / hbm, 4),
            "achieved_tflops": round(fl, 4), "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)", **common}


def measure(P, torch, prob, wl, args, precision, omega, steps, warmup, dev, stream, world, want_e2e, levels=None,
            basis=None):
    """Per-kernel shares and the roofline from one event-bracketed, host-driven
    solve (kernels inside a captured graph cannot be bracketed); then warm-up,
    `steps` timed solves and the end-to-end solves in the timed mode
    (default: one CUDA graph per solve with device-side loops)."""
    prec = {"fp64": P.MG_PRECISION_FP64, "fp32": P.MG_PRECISION_FP32, "fp32s": P.MG_PRECISION_FP32_SMOOTH}[precision]
    lv = levels or wl["levels"]
    b = torch.tensor(prob.b, device=dev)
    x = torch.empty_like(b)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    tuned = {}

    def setup(device_loops):
        h = P.mg_setup(prob, levels=lv, nu_pre=wl["nu_pre"], nu_post=wl["nu_post"], precision=prec,
                       omega=omega, device_loops=device_loops, krylov_basis=basis or args.krylov_basis,
                       stream=stream)
        if not args.no_autotune:
            # the library's autotuner: SGS chain evaluation and dot-product blocking for this
            # shape, timed once per process (outside the timed region) and cached
            try:
                chain, vb = P.mg_autotune(h, stream)
            except Exception:
                P.mg_destroy(h)
                raise
            tuned.update(chain=chain, dot_vb=vb)
        return h

    def solve(h, bp, xp):
        code, info = P.fgmres_solve(h, bp, xp, RTOL, args.maxit, args.restart, stream)
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
        if world > 1:
            torch.distributed.barrier()
        local_ms = sum(a.elapsed_time(bb) for a, bb in ev)
        value = RP.job_throughput(local_ms / 1e3, steps, world, device=dev)
        total_ms = 1e3 * world * steps / value   # the slowest rank's time
        out = {"value": value, "ms_per_step": total_ms / steps, "x": x.clone(),
               "iters": [i.iters for i in infos], "true_relres": max(i.true_relres for i in infos),
               "coarse_iters_per_vcycle": sum(i.coarse_iters for i in infos) / max(1, sum(i.vcycles for i in infos)),
               "setup_ms": setup_ms, "launches": launches, "shares": shares, "dominant": dominant,
               "roofline": roofline(shares, dominant, precision, args.workload if levels is None else None),
               "category_rooflines": {k: roofline(shares, k, precision, args.workload if levels is None else None)
                                      for k in shares if shares[k][1] and shares[k][2] > 0},
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


def measure_batch(P, torch, args, dev, stream, omega=0.7, restart=100):
    """The batched workload (64 uneven systems: van der Pol nt 512-16384,
    Burgers nx 64-256 x nt 512-4096, 4 levels each): one graph launch for all
    systems (FP64, and with the FP32 V-cycle) against one plain FP64 solve at a
    time.  Relaxed sweeps (omega = 0.7, an option outside the paper): with the
    literal sweeps the larger members do not converge within the iteration cap."""
    import os
    systems = W.batch_uneven(workers=max(1, min(16, os.cpu_count() or 1)))
    res = {"systems": len(systems), "unknowns": int(sum(p.size for p, _ in systems)), "omega": omega,
           "restart": restart, "workload": "64 uneven systems: vdP nt 512-16384, Burgers nx 64-256 x nt 512-4096"}
    for label, prec, reps in (("sequential_fp64", P.MG_PRECISION_FP64, 1), ("batched_fp64", P.MG_PRECISION_FP64, 2),
                              ("batched_fp32_vcycle", P.MG_PRECISION_FP32, 2)):
        hs, bs, xs = [], [], []
        try:
            for prob, opts in systems:
                hs.append(P.mg_setup(prob, omega=omega, precision=prec, stream=stream, **opts))
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


LEARNED_WORKLOAD = "burgers_nx256_n4096"


def measure_learned(P, torch, args, dev, stream, omega=0.7):
    """The learned coarse correction on its own workload (Burgers nx=256,
    nt=4096): collect the plain method's coarse pairs from seeded runs
    (host-driven solves with recording), train the network with the library's
    kernels, then time graph-mode solves of a held-out system with and
    without it.  Relaxed sweeps (omega = 0.7, an option outside the paper):
    the literal sweeps do not reach 1e-8 within 3000 iterations here."""
    from paper_2405_04808_gb300 import learned as LN
    wl = W.WORKLOADS[LEARNED_WORKLOAD]
    settings = dict(levels=wl["levels"], nu_pre=wl["nu_pre"], nu_post=wl["nu_post"], omega=omega)
    restart = wl.get("restart", 400)
    res = {"workload": LEARNED_WORKLOAD, "restart": restart, "omega": omega, "levels": wl["levels"], "admit": 0.5,
           "inference": "bf16 on the tensor cores (mma.sync m16n8k16), fp32 accumulation"}
    t0 = time.perf_counter()
    import os
    per = 90  # a solve records one pair per FGMRES iteration (95 here)
    nprob = (args.learned_pairs + per - 1) // per
    train_probs = W.make_many(LEARNED_WORKLOAD, [wl["seed"] + 1 + k for k in range(nprob)],
                              workers=max(1, min(16, os.cpu_count() or 1)))
    R, Y = LN.collect_pairs(train_probs, settings, args.learned_pairs, restart=restart, per_problem=per)
    torch.cuda.synchronize(dev)
    res["pairs"] = int(R.shape[0])
    res["collect_s"] = round(time.perf_counter() - t0, 2)
    _, _, T, X = R.shape
    net = LN.new_net(wl["seed"])
    try:
        t0 = time.perf_counter()
        losses = LN.train(net, R, Y, epochs=args.learned_epochs, batch=8, lr=1e-3, seed=1)
        torch.cuda.synchronize(dev)
        train_s = time.perf_counter() - t0
        # forward + backward ~ 3x the forward's 2 * T * X * 21 * sum(C_in * C_out) flops per sample
        fl = 3 * 2.0 * T * X * 21 * (5 * 32 + 32 * 32 + 32 * 32 + 32 * 5) * R.shape[0] * args.learned_epochs
        res.update(epochs=args.learned_epochs, train_s=round(train_s, 2),
                   train_loss_normalised=[round(float(l), 4) for l in losses],
                   train_tflops=round(fl / train_s / 1e12, 2), coarse_shape=[5, T, X])
        del R, Y
        prob = wl["make"]()
        b = torch.tensor(prob.b, device=dev)
        x = torch.empty_like(b)
        for name, nt in (("plain", None), ("learned", net)):
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
                if code != P.MG_OK:
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
            entry = {"solves_per_s": round(1e3 / ms, 4), "ms_per_solve": round(ms, 2), "fgmres_iters": info.iters,
                     "true_relres": info.true_relres, "coarse_gmres_iters": info.coarse_iters,
                     "coarse_solves_by_network": info.coarse_learned}
            if "net_coarse" in shares and shares["net_coarse"][1]:
                ms_net, n_net, _, fl_net = shares["net_coarse"]
                total = sum(v[0] for v in shares.values())
                entry.update(net_share=round(ms_net / total, 4), net_tflops=round(fl_net / ms_net / 1e9, 2))
            res[name] = entry
        res["speedup_learned_vs_plain"] = round(res["learned"]["solves_per_s"] / res["plain"]["solves_per_s"], 4)
    finally:
        P.mg_net_destroy(net)
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
    main = measure(P, torch, prob, wl, args, args.precision, args.omega, args.steps, args.warmup, dev, stream,
                   world, True)
    variants = {}
    if not args.no_variants:
        # (name, precision, omega, levels): the mixed-precision V-cycle, relaxed sweeps (an option
        # outside the paper), and the paper's serial baseline of Sec. 6.3 (SGS-GMRES, no multigrid),
        # whose block Gauss-Seidel chains run here as a parallel scan in time
        other = "fp64" if args.krylov_basis == "pair" else "pair"
        for name, prec, om, lv, kb in ((f"{other}_krylov_basis", args.precision, args.omega, None, other),
                                       ("fp32_vcycle", "fp32", args.omega, None, None),
                                       ("fp32_smoother_fp64_coarse", "fp32s", args.omega, None, None),
                                       ("omega0.7_fp64", "fp64", 0.7, None, None),
                                       ("omega0.7_fp32_vcycle", "fp32", 0.7, None, None),
                                       ("omega0.7_fp32_smoother_fp64_coarse", "fp32s", 0.7, None, None),
                                       ("sgs_gmres_no_multigrid", "fp64", 1.0, 1, None)):
            if prec == args.precision and om == args.omega and lv is None and kb is None:
                continue
            v = measure(P, torch, prob, wl, args, prec, om, max(1, min(args.steps, 3)), 1, dev, stream, world, False,
                        levels=lv, basis=kb)
            # the variant's solution against the headline solve's (both to a 1e-8 relative residual)
            xdiff = float(torch.linalg.vector_norm(v["x"] - main["x"]) / torch.linalg.vector_norm(main["x"]))
            variants[name] = {"value": round(v["value"], 4), "unit": UNIT, "ms_per_step": round(v["ms_per_step"], 3),
                              "fgmres_iters": v["iters"][0], "true_relres": v["true_relres"],
                              "solution_rel_diff_vs_main": xdiff,
                              "precision": prec, "omega": om, "levels": lv or wl["levels"],
                              "krylov_basis": kb or args.krylov_basis,
                              "coarse_iters_per_vcycle": round(v["coarse_iters_per_vcycle"], 3),
                              "setup_ms": round(v["setup_ms"], 1),
                              "dominant_kernel": v["dominant"], "roofline_frac": v["roofline"].get("frac")}
    batch = None if (args.no_variants or args.no_batch) else measure_batch(P, torch, args, dev, stream)
    learned = (None if (args.no_variants or args.no_batch or args.learned_pairs <= 0)
               else measure_learned(P, torch, args, dev, stream))
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
                   "omega": args.omega, "l2": "flushed (512 MB write) before every timed step",
                   "solve": "host-driven loops" if args.host_loops else
                            "one CUDA graph per solve (FGMRES and coarse GMRES loops as conditional nodes)",
                   "roofline_source": "event-bracketed kernels of one host-driven solve of the same system",
                   "parallelism": f"replicas{world}"},
        "fgmres_iters": main["iters"], "true_relres": main["true_relres"],
        "coarse_iters_per_vcycle": round(main["coarse_iters_per_vcycle"], 3),
        "setup_ms": round(main["setup_ms"], 2),
        "e2e": main["e2e"],
        "gpu_launches": main["launches"],
        "autotune": main["autotune"],
        "roofline": main["roofline"],
        "category_rooflines": {k: {"bound": v["bound"], "frac": v.get("frac"), "achieved": v.get("achieved"),
                                   "unit": v.get("unit"), "avg_launch_us": v.get("avg_launch_us")}
                               for k, v in main["category_rooflines"].items()},
        "kernel_shares": {k: {"ms": round(v[0], 3), "launches": v[1]} for k, v in main["shares"].items() if v[1]},
        "variants": variants,
        "batched": batch,
        "learned_coarse": learned,
        "clocks": main["clocks"],
    }
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(prob, wl, args, main["iters"])
    if world > 1:
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


def oracle_iterations(workload, omega, restart):
    """The oracle's own FGMRES iteration count for a full solve of this
    workload (tests/golden/oracle_iterations.json, written by
    oracle/measure_iterations.py), or None."""
    path = os.path.join(ROOT, "tests", "golden", "oracle_iterations.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path)).get(f"{workload}/omega={float(omega)}/restart={restart}")
    if rec and rec.get("restart") == restart and rec.get("rtol") == RTOL:
        return rec["iters"]
    return None


def oracle_sample(prob, wl, omega, seconds):
    """Time the oracle as it stands: its FGMRES on this system for about
    `seconds` (setup, i.e. the sparse LU factorisations, excluded).  Returns
    (seconds per FGMRES iteration, iterations run)."""
    from oracle import augmented as O
    hier = O.Hierarchy(prob, O.MGOptions(levels=wl["levels"], nu_pre=wl["nu_pre"], nu_post=wl["nu_post"],
                                         omega=omega))
    lev = hier.fine
    bt = lev.to_time_major(prob.b)
    hier.vcycle(0, bt)  # builds the factorisations
    count = [0]
    t0 = time.perf_counter()

    class Stop(Exception):
        pass

    def prec(v):
        count[0] += 1
        return hier.vcycle(0, v)

    def apply_A(v):
        if time.perf_counter() - t0 > seconds:
            raise Stop()
        return lev.At @ v

    try:
        O.fgmres(apply_A, prec, bt, rtol=RTOL, maxit=100000, restart=400)
    except Stop:
        pass
    el = time.perf_counter() - t0
    return el / max(1, count[0]), count[0]


def cpu_baseline(prob, wl, args, gpu_iters):
    per_iter, k = oracle_sample(prob, wl, args.omega, args.cpu_sample_seconds)
    n_or = oracle_iterations(args.workload, args.omega, args.restart)
    n_it = n_or if n_or is not None else statistics.mean(gpu_iters)
    src = "the oracle's own full-solve count" if n_or is not None else "the GPU solve's count"
    return {"value": round(1.0 / (per_iter * n_it), 6), "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{k} oracle FGMRES iterations ({per_iter * 1e3:.0f} ms each, first iterations of the "
                      f"solve, SuperLU factorisations excluded) scaled by {n_it:.0f} iterations per solve "
                      f"({src}); scipy/SuperLU, host cores of the GPU box"}


def run_reference(args):
    """--impl reference: the CPU oracle as it stands, a bounded sample per step."""
    rank, world, local = dist_env()
    if rank != 0:
        return
    wl = W.WORKLOADS[args.workload]
    prob = wl["make"]()
    per_step = max(5.0, min(30.0, 150.0 / max(1, args.steps + args.warmup)))
    times = []
    for k in range(args.warmup + args.steps):
        per_iter, cnt = oracle_sample(prob, wl, args.omega, per_step)
        if k >= args.warmup:
            times.append(per_iter)
    per_iter = statistics.mean(times)
    n_or = oracle_iterations(args.workload, args.omega, args.restart)
    value = None if n_or is None else round(1.0 / (per_iter * n_or), 6)
    line = {"metric": METRIC, "impl": "reference", "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(per_iter * (n_or or 0) * 1e3, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded iterate and N(0,1) right-hand side)",
            "config": {"workload": args.workload, "restart": args.restart, "omega": args.omega, "rtol": RTOL},
            "cpu_baseline": {"value": value, "unit": UNIT, "kind": "oracle", "cores": os.cpu_count(),
                             "sample": f"per step about {per_step:.0f} s of oracle FGMRES iterations "
                                       f"({per_iter * 1e3:.0f} ms each) scaled by the oracle's {n_or} "
                                       f"iterations per full solve"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
