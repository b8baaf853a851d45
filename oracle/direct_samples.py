"""Sampled entries of the oracle's direct solution of the benchmark workloads
(tests/golden/direct_samples.json), for comparing a GPU solve with the exact
answer x* = A^-1 b of the lifted system (Sec. 5.1, Eq. augsys-aj).

Calls only oracle/ and the input generator.  The direct solve is SuperLU on
the assembled type-major matrix (``augmented.direct_solve``, about 10 s for
the Burgers nx=128, nt=1024 system).  For every variable type (u, v, z,
lambda, mu) it stores the largest magnitude of that type and 512 entries at
evenly spaced positions of the type's block, with their indices in the full
type-major vector; values are written with Python's round-trip float repr.
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import augmented as O  # noqa: E402
from paper_2405_04808_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(ROOT, "tests", "golden", "direct_samples.json")
PER_TYPE = 512


def samples(name):
    wl = W.WORKLOADS[name]
    prob = wl["make"]()
    t0 = time.time()
    x = O.direct_solve(prob)
    secs = time.time() - t0
    off = O.type_major_offsets(prob.n, prob.p, prob.q)
    types = {}
    for t, label in zip("uvzlm", ("u", "v", "z", "lambda", "mu")):
        width = prob.q if t == "z" else prob.p
        start, length = off[t], prob.n * width
        idx = np.unique(np.linspace(0, length - 1, PER_TYPE).round().astype(np.int64)) + start
        types[label] = {"max_abs": float(np.max(np.abs(x[start:start + length]))),
                        "indices": [int(i) for i in idx], "values": [float(x[i]) for i in idx]}
    residual = float(np.linalg.norm(prob.b - O.Level(O.raw_from_problem(prob)).A @ x) / np.linalg.norm(prob.b))
    return {"workload": name, "n": prob.n, "p": prob.p, "q": prob.q, "length": prob.size,
            "norm": float(np.linalg.norm(x)), "relres": residual, "seconds": round(secs, 1), "types": types}


if __name__ == "__main__":
    names = sys.argv[1:] or ["vdp_n256", "burgers_nx128_n1024"]
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for nm in names:
        data[nm] = samples(nm)
        print(nm, data[nm]["relres"], data[nm]["seconds"], flush=True)
        with open(OUT, "w") as fh:
            json.dump(data, fh, indent=0, sort_keys=True)
