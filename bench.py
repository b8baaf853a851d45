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
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--restart", type=int, default=200)
    ap.add_argument("--maxit", type=int, default=2000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--allow-partial", action="store_true",
                    help="accept solves stopped by --maxit (bounded profiler captures only)")
    ap.add_argument("--cpu-sample-seconds", type=float, default=20.0)
    return ap.parse_args()


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


# FP64 FMA rate of this GB300 (measured: 1.196 TFLOP/s = 0.598 T FMA/s with
# every SM sub-partition busy); the ALU peak for the FP64 kernels.
FP64_TFLOPS_MEASURED = 1.196


def algorithmic_cost(category: str, wl: dict, prob, precision: str):
    """Algorithmic bytes and FP64 flops of ONE launch of a kernel category at the fine level.

    block_solve (one block-Jacobi sweep, tridiagonal): per time block it reads
    the right-hand side (4p+q), the two coupling vectors (2p), the N, V, Z bands
    (9p) and the LDL^T factor (3p), and writes the block (4p+q); flops: 3
    tridiagonal products (18p), the pentadiagonal solve (2 x 4p + p) and three
    transposed products (18p) = 45p per block.
    """
    p, q, n = prob.p, prob.q, prob.n
    wsz = 8 if precision == "fp64" else 4
    if category == "block_solve":
        bytes_per_block = wsz * ((4 * p + q) * 2 + 2 * p + 9 * p + 3 * p)
        flops_per_block = 45 * p
        return bytes_per_block * (n + 1), flops_per_block * (n + 1)
    return None, None


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
    prob = wl["make"](seed=2000 + 17 * rank) if rank else wl["make"]()
    precision = P.MG_PRECISION_FP64 if args.precision == "fp64" else P.MG_PRECISION_FP32
    t0 = time.perf_counter()
    h = P.mg_setup(prob, levels=wl["levels"], nu_pre=wl["nu_pre"], nu_post=wl["nu_post"], precision=precision,
                   stream=stream)
    torch.cuda.synchronize(dev)
    setup_ms = (time.perf_counter() - t0) * 1e3
    n = prob.size
    b = torch.tensor(prob.b, device=dev)
    x = torch.empty_like(b)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def solve():
        code, info = P.fgmres_solve(h, b.data_ptr(), x.data_ptr(), RTOL, args.maxit, args.restart, stream)
        if code != P.MG_OK and not (args.allow_partial and code == P.MG_NOT_CONVERGED):
            raise RuntimeError(f"fgmres_solve: {P.mg_status_string(code)} (iters {info.iters}, "
                               f"relres {info.relres:.2e}, true {info.true_relres:.2e})")
        return info

    for _ in range(args.warmup):
        flush.zero_()
        solve()
    # one fully profiled solve: per-category kernel time shares
    P.mg_profile_enable(h, P.PROFILE_ALL)
    flush.zero_()
    solve()
    shares = P.mg_profile_read(h)
    P.mg_profile_enable(h, 0)
    dominant = max(shares, key=lambda k: shares[k][0])

    # timed region: device-resident inputs, L2 flushed before every step,
    # the dominant kernel category bracketed by CUDA events on the library's stream
    P.mg_profile_enable(h, 1 << P.PROFILE_CATEGORIES.index(dominant))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    launches0 = P.mg_launch_count(h)
    infos = []
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record()
            infos.append(solve())
            ev[i][1].record()
        torch.cuda.synchronize(dev)
    launches = P.mg_launch_count(h) - launches0
    prof = P.mg_profile_read(h)
    P.mg_profile_enable(h, 0)
    if world > 1:
        torch.distributed.barrier()
    step_ms = [a.elapsed_time(bb) for a, bb in ev]
    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    value = world * args.steps / (total_ms / 1e3)

    # end to end through the public API with pinned host buffers
    bh = torch.tensor(prob.b).pin_memory()
    xh = torch.empty_like(bh).pin_memory()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        code, info = P.fgmres_solve(h, bh.data_ptr(), xh.data_ptr(), RTOL, args.maxit, args.restart, stream)
        if code != P.MG_OK and not (args.allow_partial and code == P.MG_NOT_CONVERGED):
            raise RuntimeError("e2e solve failed")
    e2e_s = time.perf_counter() - t0
    e2e_value = world * args.steps / e2e_s
    if world > 1:
        t = torch.tensor([e2e_s], device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        e2e_value = world * args.steps / float(t.item())

    # roofline of the dominant kernel
    hbm, peak_kind = measured_peaks()
    cat_ms, cat_n = prof.get(dominant, (0.0, 0))
    roof = None
    if cat_n:
        per_launch_s = cat_ms / cat_n / 1e3
        bytes_l, flops_l = algorithmic_cost(dominant, wl, prob, args.precision)
        if bytes_l is not None:
            bw = bytes_l / per_launch_s / 1e9
            fl = flops_l / per_launch_s / 1e12
            # FP64 arithmetic on this part is slower than its HBM: report the binding roof
            t_hbm = bytes_l / (hbm * 1e9)
            t_alu = flops_l / (FP64_TFLOPS_MEASURED * 1e12) if args.precision == "fp64" else 0.0
            if t_alu > t_hbm:
                roof = {"bound": "alu", "achieved": round(fl, 4), "peak": FP64_TFLOPS_MEASURED,
                        "unit": "TFLOP/s", "frac": round(fl / FP64_TFLOPS_MEASURED, 4), "traffic": None,
                        "kernel": dominant, "alu_peak_source": "measured FP64 FMA probe",
                        "achieved_gbs": round(bw, 1), "hbm_peak_gbs": hbm}
            else:
                roof = {"bound": "hbm", "achieved": round(bw, 1), "peak": hbm, "unit": "GB/s",
                        "frac": round(bw / hbm, 4), "traffic": None, "kernel": dominant,
                        "peak_source": peak_kind}
        else:
            roof = {"bound": None, "kernel": dominant, "note": "no algorithmic model for this category"}
        roof["avg_launch_us"] = round(per_launch_s * 1e6, 3)
        roof["launches_in_timed_region"] = cat_n

    iters = [i.iters for i in infos]
    out = {
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(total_ms / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32+f64",
        "data": "synthetic (seeded iterate and N(0,1) right-hand side)",
        "config": {"workload": args.workload, "n": prob.n, "p": prob.p, "q": prob.q,
                   "levels": wl["levels"], "nu_pre": wl["nu_pre"], "nu_post": wl["nu_post"],
                   "unknowns": n, "rtol": RTOL, "restart": args.restart, "precision": args.precision,
                   "l2": "flushed (512 MB write) before every timed step", "parallelism": f"replicas{world}"},
        "fgmres_iters": iters, "true_relres": max(i.true_relres for i in infos),
        "coarse_iters_per_vcycle": round(sum(i.coarse_iters for i in infos) / max(1, sum(i.vcycles for i in infos)), 3),
        "setup_ms": round(setup_ms, 2),
        "e2e": {"value": round(e2e_value, 4), "unit": UNIT, "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * n},
        "gpu_launches": launches,
        "roofline": roof,
        "kernel_shares": {k: {"ms": round(v[0], 3), "launches": v[1]} for k, v in shares.items() if v[1]},
        "clocks": clk.summary(),
    }
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(prob, wl, iters, args.cpu_sample_seconds)
    P.mg_destroy(h)
    if world > 1:
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


def cpu_baseline(prob, wl, gpu_iters, seconds):
    """The oracle as it stands, on a bounded sample: FGMRES iterations of the
    same system until `seconds` elapse; solves/s = 1 / (time per iteration x the
    GPU solve's iteration count).  Oracle setup (sparse LU) is excluded, like
    the GPU's mg_setup."""
    from oracle import augmented as O
    hier = O.Hierarchy(prob, O.MGOptions(levels=wl["levels"], nu_pre=wl["nu_pre"], nu_post=wl["nu_post"]))
    lev = hier.fine
    bt = lev.to_time_major(prob.b)
    # warm the factorisations once (setup), then time iterations
    hier.vcycle(0, bt)
    count = [0]
    t0 = time.perf_counter()

    def prec(v):
        count[0] += 1
        return hier.vcycle(0, v)

    class Stop(Exception):
        pass

    def apply_A(v):
        if time.perf_counter() - t0 > seconds:
            raise Stop()
        return lev.At @ v

    try:
        O.fgmres(apply_A, prec, bt, rtol=RTOL, maxit=100000, restart=200)
    except Stop:
        pass
    el = time.perf_counter() - t0
    per_iter = el / max(1, count[0])
    iters = statistics.mean(gpu_iters)
    return {"value": round(1.0 / (per_iter * iters), 6), "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{count[0]} oracle FGMRES iterations in {el:.1f} s on this system; "
                      f"scaled by the GPU solve's {iters:.1f} iterations per solve"}


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    wl = W.WORKLOADS[args.workload]
    prob = wl["make"]()
    from oracle import augmented as O
    hier = O.Hierarchy(prob, O.MGOptions(levels=wl["levels"], nu_pre=wl["nu_pre"], nu_post=wl["nu_post"]))
    hier.vcycle(0, hier.fine.to_time_major(prob.b))
    # a step: a bounded sample of the solve (the oracle's FGMRES for a fixed
    # number of iterations), scaled to solves/s by the iteration count the
    # oracle needs for a full solve at this size (measured once below on the
    # same sample budget)
    per_step = max(1.0, 60.0 / max(1, args.steps + args.warmup))
    lev = hier.fine
    bt = lev.to_time_major(prob.b)
    times, its = [], []
    for k in range(args.warmup + args.steps):
        cnt = [0]
        t0 = time.perf_counter()

        def prec(v):
            cnt[0] += 1
            return hier.vcycle(0, v)

        class Stop(Exception):
            pass

        def apply_A(v):
            if time.perf_counter() - t0 > per_step:
                raise Stop()
            return lev.At @ v

        try:
            O.fgmres(apply_A, prec, bt, rtol=RTOL, maxit=100000, restart=200)
        except Stop:
            pass
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
            its.append(cnt[0])
    per_iter = sum(times) / max(1, sum(its))
    est_iters = float(os.environ.get("PINTMG_REF_ITERS", "0")) or None
    value = None if est_iters is None else 1.0 / (per_iter * est_iters)
    line = {"metric": METRIC, "impl": "reference", "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * sum(times) / len(times), 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": args.workload},
            "oracle_ms_per_fgmres_iteration": round(per_iter * 1e3, 2),
            "cpu_baseline": {"value": value, "kind": "oracle", "cores": os.cpu_count(),
                             "sample": f"{sum(its)} oracle FGMRES iterations over {len(times)} steps"},
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
