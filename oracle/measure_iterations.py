"""Run the oracle's own FGMRES to convergence on the benchmark workloads and
record its iteration counts (tests/golden/oracle_iterations.json).

Calls only oracle/ and the input generator.  Slow (the Burgers nx=128 solve
takes about 15 minutes on 8 CPU cores); the CPU-reference arm of bench.py
scales its bounded per-iteration timing by these counts.  Keys:
"<workload>/omega=<omega>/restart=<restart>", at each workload's restart,
for the cycle as written (injection of the residual); the cycle with the
residual restricted by the transpose of the interpolation and weighted sweeps
(omega = 2/3, restart 60) adds "/restrict=transpose".
"""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import augmented as O  # noqa: E402
from paper_2405_04808_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(ROOT, "tests", "golden", "oracle_iterations.json")


#: the weighted sweep that goes with restriction by the transpose of the interpolation
OMEGA_TRANSPOSE = 2.0 / 3.0
RESTART_TRANSPOSE = 60


def key(name, omega, restart, restrict="inject"):
    k = f"{name}/omega={float(omega)}/restart={restart}"
    return k + "/restrict=transpose" if restrict == "transpose" else k


def measure(name, rtol=1e-8, restart=None, maxit=2000, omega=1.0, restrict="inject"):
    wl = W.WORKLOADS[name]
    restart = restart or wl.get("restart", 400)
    prob = wl["make"]()
    h = O.Hierarchy(prob, O.MGOptions(levels=wl["levels"], nu_pre=wl["nu_pre"], nu_post=wl["nu_post"], omega=omega,
                                      restrict=restrict))
    t0 = time.time()
    x, res, true_rel = h.solve(prob.b, rtol=rtol, maxit=maxit, restart=restart)
    return {"workload": name, "rtol": rtol, "restart": restart, "maxit": maxit, "omega": omega,
            "restrict": restrict, "iters": res.iters, "relres": res.relres, "true_relres": true_rel,
            "seconds": round(time.time() - t0, 1)}


if __name__ == "__main__":
    args = sys.argv[1:]
    only_transpose = "--transpose-only" in args
    names = [a for a in args if not a.startswith("--")] or ["vdp_n256", "burgers_nx128_n1024"]
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    runs = [] if only_transpose else [dict(omega=1.0), dict(omega=0.7)]
    runs.append(dict(omega=OMEGA_TRANSPOSE, restrict="transpose", restart=RESTART_TRANSPOSE))
    for nm in names:
        for kw in runs:
            rec = measure(nm, **kw)
            k = key(nm, rec["omega"], rec["restart"], rec["restrict"])
            data[k] = rec
            print(k, data[k], flush=True)
            with open(OUT, "w") as fh:
                json.dump(data, fh, indent=1, sort_keys=True)
