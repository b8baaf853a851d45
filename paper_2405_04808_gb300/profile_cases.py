"""Small, self-contained GPU cases for kernel profiling (ncu): the learned
coarse correction's kernels at the Burgers nx=256, nt=4096 coarse shape
(5 x 512 x 256 per sample), and a fixed-length FGMRES cycle whose basis
outgrows L2 (Burgers nx=128, nt=256: 163,840 entries per vector, 121 basis
vectors = 159 MB) for the Gram-Schmidt kernels.

    python -m paper_2405_04808_gb300.profile_cases conv_fwd_bf16
    python -m paper_2405_04808_gb300.profile_cases conv_fwd_fp32
    python -m paper_2405_04808_gb300.profile_cases train_step
    python -m paper_2405_04808_gb300.profile_cases fgmres_cycle [--basis pair|fp64]
    python -m paper_2405_04808_gb300.profile_cases vcycle [--restrict transpose|inject]
    python -m paper_2405_04808_gb300.profile_cases vcycle_p512 [--restrict transpose|inject]
    python -m paper_2405_04808_gb300.profile_cases sharded_fgmres [--reps N]

sharded_fgmres: the FGMRES around the time-sharded V-cycle (timeshard.py) on
one GPU with 1, 2 and 4 ranks held in one process (their kernels run one after
another), against fgmres_solve on the same handle: steps, wall time per solve
and the solutions' difference (Burgers nx=128, nt=1024, the paper-behaviour
cycle, restart 60, rtol 1e-8).

vcycle: V-cycles of the benchmark system (Burgers nx=128, nt=1024, 3 levels,
4/4 sweeps; weighted sweeps omega = 2/3 with the transposed restriction by
default), one mg_vcycle per repetition, host-driven, so every kernel of the
cycle launches on its own.  vcycle_p512: the same with the large blocks of
the nx = 512 system (Burgers nx=512, nt=2048, nu = 0.005: p = 512).

Each case runs a warm-up and then `--reps` launches of the kernels it names,
and exits non-zero on any library error.

    python -m paper_2405_04808_gb300.profile_cases summarize LAUNCHES.csv

condenses an ncu launch list (``--metrics gpu__time_duration.sum --csv``) to
launches, total time and share per kernel name; an optional third argument is a
regular expression of kernel names to leave out (e.g. the set-up kernels).
"""
from __future__ import annotations

import argparse
import sys

import numpy as np


def summarize(path: str, exclude: str = "") -> str:
    """Markdown table of an ncu CSV launch list: launches, total ms and share per kernel
    (kernels whose name matches the regular expression `exclude` left out)."""
    import csv
    import io
    import re
    rows = []
    with open(path, newline="") as f:
        text = f.read()
    start = text.find('"ID"')
    for r in csv.DictReader(io.StringIO(text[start:])):
        if r.get("Metric Name") == "gpu__time_duration.sum":
            v = float(r["Metric Value"].replace(",", ""))
            unit = r.get("Metric Unit", "")
            scale = {"nsecond": 1e-6, "usecond": 1e-3, "msecond": 1.0, "second": 1e3}.get(unit, 1e-6)
            name = r["Kernel Name"]
            name = name.split("(")[0].replace("void ", "") if "(" in name else name
            if exclude and re.search(exclude, name):
                continue
            rows.append((name, v * scale))
    tot = {}
    for name, ms in rows:
        n, t = tot.get(name, (0, 0.0))
        tot[name] = (n + 1, t + ms)
    total = sum(t for _, t in tot.values()) or 1.0
    out = [f"{len(rows)} launches, {total:.1f} ms in all", "", "| kernel | launches | total ms | share |",
           "|---|---|---|---|"]
    for name, (n, t) in sorted(tot.items(), key=lambda kv: -kv[1][1]):
        out.append(f"| {name} | {n} | {t:.3f} | {100 * t / total:.1f} % |")
    return "\n".join(out)


def main(argv=None):
    argv = sys.argv[1:] if argv is None else argv
    if argv and argv[0] == "summarize":
        print(summarize(argv[1], argv[2] if len(argv) > 2 else ""))
        return 0
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["conv_fwd_bf16", "conv_fwd_fp32", "train_step", "fgmres_cycle", "vcycle",
                                     "vcycle_p512", "sharded_fgmres"])
    ap.add_argument("--restrict", default="transpose", choices=["transpose", "inject"])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--basis", default="pair", choices=["pair", "fp64"])
    args = ap.parse_args(argv)
    import torch

    from . import pintmg as P
    from . import workloads as W
    if args.case in ("vcycle", "vcycle_p512"):
        # vcycle_p512: the C3 discretisation (nx = 512, nu = 0.005) at nt = 2048 (42 MB per vector)
        prob = (W.burgers(nx=128, n=1024, nu=0.01, seed=2000) if args.case == "vcycle" else
                W.burgers(nx=512, n=2048, nu=0.005, seed=3000))
        omega = 2.0 / 3.0 if args.restrict == "transpose" else 1.0
        h = P.mg_setup(prob, levels=3, nu_pre=4, nu_post=4, omega=omega, restrict=args.restrict,
                       device_loops=False)
        try:
            r = torch.tensor(prob.b, dtype=torch.float64, device="cuda")
            y = torch.empty_like(r)
            for _ in range(1 + args.reps):
                code = P.mg_vcycle(h, r.data_ptr(), y.data_ptr())
                if code != P.MG_OK:
                    raise P.PintmgError(code, "mg_vcycle")
            torch.cuda.synchronize()
            print(f"vcycle ({args.restrict}): {1 + args.reps} cycles, |y| = {float(torch.linalg.norm(y)):.6e}")
        finally:
            P.mg_destroy(h)
        return 0
    if args.case == "sharded_fgmres":
        import time

        from . import timeshard as TS
        prob = W.burgers(nx=128, n=1024, nu=0.01, seed=2200)
        levels, rtol, restart = 3, 1e-8, 60
        h = P.mg_setup(prob, levels=levels, nu_pre=4, nu_post=4, omega=2.0 / 3.0, restrict="transpose")
        try:
            b = torch.tensor(prob.b, dtype=torch.float64, device="cuda")
            ref = torch.zeros_like(b)

            def timed(fn):
                fn()  # warm-up
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                for _ in range(args.reps):
                    out = fn()
                torch.cuda.synchronize()
                return out, (time.perf_counter() - t0) / args.reps

            def solve_ref():
                code, info = P.fgmres_solve(h, b.data_ptr(), ref.data_ptr(), rtol, 2000, restart)
                if code != P.MG_OK:
                    raise P.PintmgError(code, "fgmres_solve")
                return info.iters
            iters, sec = timed(solve_ref)
            print(f"fgmres_solve: {iters} steps, {sec * 1e3:.2f} ms per solve")
            layouts = [TS.Layout(P.mg_level_info(h, lv)[0], prob.p, prob.q) for lv in range(levels)]
            for world in (1, 2, 4):
                part = TS.Partition(prob.n, levels, world)
                ranks = list(range(world))
                cyc = TS.ShardedVCycle(part, layouts, [TS.LibraryEngine(P, h) for _ in ranks], ranks,
                                       TS.LocalExchange(world), 4, 4,
                                       lambda k: torch.zeros(k, dtype=torch.float64, device="cuda"))
                solver = TS.ShardedFGMRES(cyc, restart)
                res, sec = timed(lambda: solver.solve([b.clone() for _ in ranks], rtol, 2000))
                x = torch.full_like(b, float("nan"))
                for r in ranks:
                    j0, j1 = part.blocks(r, 0)
                    for j in range(j0, j1):
                        for sl in layouts[0].block(j):
                            x[sl] = res.x[r][sl]
                diff = float(torch.linalg.norm(x - ref) / torch.linalg.norm(ref))
                print(f"sharded, {world} rank(s) in one process: {res.iters} steps, {sec * 1e3:.2f} ms per solve, "
                      f"|x - x_ref| / |x_ref| = {diff:.2e}")
        finally:
            P.mg_destroy(h)
        return 0
    if args.case == "fgmres_cycle":
        # 120 FGMRES iterations without restart (tolerance out of reach): the
        # basis grows to 121 vectors; host-driven loops launch each kernel alone
        prob = W.burgers(nx=128, n=256, seed=2100)
        h = P.mg_setup(prob, levels=3, nu_pre=4, nu_post=4, device_loops=False, krylov_basis=args.basis)
        try:
            b = torch.tensor(prob.b, dtype=torch.float64, device="cuda")
            x = torch.empty_like(b)
            code, info = P.fgmres_solve(h, b.data_ptr(), x.data_ptr(), 1e-300, 120, 120)
            torch.cuda.synchronize()
            if code not in (P.MG_OK, P.MG_NOT_CONVERGED):
                raise P.PintmgError(code, "fgmres_solve")
            print(f"fgmres_cycle ({args.basis}): {info.iters} iterations, relres {info.relres:.2e}")
        finally:
            P.mg_destroy(h)
        return 0
    T, X = 512, 256
    net = P.mg_net_create(W.net_init_params(1).astype(np.float32))
    try:
        g = torch.Generator(device="cuda").manual_seed(0)
        if args.case.startswith("conv_fwd"):
            x = torch.randn((1, 5, T, X), device="cuda", generator=g)
            y = torch.empty_like(x)
            bf16 = args.case.endswith("bf16")
            for _ in range(1 + args.reps):
                P.mg_net_forward(net, x.data_ptr(), 1, T, X, y.data_ptr(), bf16=bf16)
        else:
            B = args.batch
            x = torch.randn((B, 5, T, X), device="cuda", generator=g)
            t = torch.randn_like(x)
            for _ in range(1 + args.reps):
                P.mg_net_loss_grad(net, x.data_ptr(), t.data_ptr(), B, T, X)
                P.mg_net_adam_step(net, 1e-3)
        torch.cuda.synchronize()
    finally:
        P.mg_net_destroy(net)
    return 0


if __name__ == "__main__":
    sys.exit(main())
