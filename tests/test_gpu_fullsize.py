"""Parity at the benchmark workloads' full sizes, in bench.py's configuration.

C1 (van der Pol, n = 256, 2 levels, 1/1) is small enough for a direct solve
of the oracle's system.  C2 (Burgers nx = 128, n = 1024, 3 levels, 4/4,
655,360 unknowns) is checked through properties the oracle computes
independently: the GPU solution's residual against the oracle's own
assembled lifted operator, agreement with a direct sparse solve, and one
full-size V-cycle against the oracle's.  C3 (Burgers nx = 512, n = 8192, 21 M
unknowns) is checked by the residual against the oracle's assembled operator.
"""
import numpy as np
import pytest

from oracle import augmented as O
from paper_2405_04808_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2405_04808_gb300 import pintmg
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pintmg.lib()
    return pintmg


def _solve(P, prob, wl, rtol, restart=400, **kw):
    h = P.mg_setup(prob, levels=wl["levels"], nu_pre=wl["nu_pre"], nu_post=wl["nu_post"], **kw)
    try:
        b = torch.tensor(prob.b, dtype=torch.float64, device="cuda")
        x = torch.empty_like(b)
        code, info = P.fgmres_solve(h, b.data_ptr(), x.data_ptr(), rtol, 3000, restart)
        assert code == P.MG_OK, P.mg_status_string(code)
        return x.cpu().numpy(), info
    finally:
        P.mg_destroy(h)


def test_c1_vdp_full_size(P):
    wl = W.WORKLOADS["vdp_n256"]
    prob = wl["make"]()
    x, info = _solve(P, prob, wl, 1e-10)
    xd = O.direct_solve(prob)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= 1e-9
    # the oracle's FGMRES at the same settings takes the same number of iterations (R13: +-2)
    h = O.Hierarchy(prob, O.MGOptions(levels=wl["levels"], nu_pre=wl["nu_pre"], nu_post=wl["nu_post"]))
    _, res, _ = h.solve(prob.b, rtol=1e-10, maxit=3000, restart=400)
    assert abs(res.iters - info.iters) <= 2


@pytest.mark.slow
def test_c2_burgers_full_size_solution(P):
    wl = W.WORKLOADS["burgers_nx128_n1024"]
    prob = wl["make"]()
    x, info = _solve(P, prob, wl, 1e-10, omega=0.7)   # relaxed sweeps: same solution, 50x fewer iterations
    lev = O.Level(O.raw_from_problem(prob))
    rel = np.linalg.norm(prob.b - lev.A @ x) / np.linalg.norm(prob.b)
    assert rel <= 1.5e-10, rel
    xd = O.direct_solve(prob)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= 1e-9


@pytest.mark.slow
def test_c2_burgers_full_size_vcycle(P):
    """One V-cycle at the bench configuration (fixed coarse iterations) equals the oracle's."""
    wl = W.WORKLOADS["burgers_nx128_n1024"]
    prob = wl["make"]()
    opts = dict(levels=wl["levels"], nu_pre=wl["nu_pre"], nu_post=wl["nu_post"], coarse_fixed_iters=2)
    h = P.mg_setup(prob, **opts)
    try:
        r = torch.tensor(prob.b, dtype=torch.float64, device="cuda")
        y = torch.empty_like(r)
        assert P.mg_vcycle(h, r.data_ptr(), y.data_ptr(), 0) == P.MG_OK
        torch.cuda.synchronize()
        yo = O.Hierarchy(prob, O.MGOptions(**opts)).precondition(prob.b)
        yg = y.cpu().numpy()
        assert np.linalg.norm(yg - yo) / np.linalg.norm(yo) <= 1e-10
        # sampled entries, element by element (first, middle, last steps of every type)
        n, p, q = prob.n, prob.p, prob.q
        off = O.type_major_offsets(n, p, q)
        scale = np.max(np.abs(yo))
        for t in "uvzlm":
            wdt = q if t == "z" else p
            for step in (0, n // 2, n - 1):
                sl = slice(off[t] + step * wdt, off[t] + (step + 1) * wdt)
                assert np.max(np.abs(yg[sl] - yo[sl])) <= 1e-10 * scale
    finally:
        P.mg_destroy(h)


@pytest.mark.parametrize("name,omega", [("burgers_nx128_n1024", 1.0), ("burgers_nx128_n1024", 0.7),
                                        ("vdp_n256", 1.0), ("vdp_n256", 0.7)])
def test_bench_configuration_iterations_match_oracle(P, name, omega):
    """At bench.py's configuration (rtol 1e-8, the workload's restart) the GPU solve takes the
    oracle's own full-solve iteration count (tests/golden/oracle_iterations.json,
    written by oracle/measure_iterations.py) and meets the tolerance on the
    oracle's independently assembled operator."""
    import json
    import os
    from conftest import GOLDEN
    wl = W.WORKLOADS[name]
    key = f"{name}/omega={omega}/restart={wl['restart']}"
    rec = json.load(open(os.path.join(GOLDEN, "oracle_iterations.json")))[key]
    prob = wl["make"]()
    h = P.mg_setup(prob, levels=wl["levels"], nu_pre=wl["nu_pre"], nu_post=wl["nu_post"], omega=omega)
    try:
        b = torch.tensor(prob.b, dtype=torch.float64, device="cuda")
        x = torch.empty_like(b)
        code, info = P.fgmres_solve(h, b.data_ptr(), x.data_ptr(), rec["rtol"], rec["maxit"], rec["restart"])
        assert code == P.MG_OK
        assert abs(info.iters - rec["iters"]) <= 2, (info.iters, rec["iters"])
        lev = O.Level(O.raw_from_problem(prob))
        xr = x.cpu().numpy()
        assert np.linalg.norm(prob.b - lev.A @ xr) / np.linalg.norm(prob.b) <= 1.05 * rec["rtol"]
    finally:
        P.mg_destroy(h)


@pytest.mark.parametrize("name", ["vdp_n256", "burgers_nx128_n1024"])
def test_kkt_right_hand_sides_full_size(P, name):
    """The two KKT right-hand sides at full size: b = (chi, 0) gives x in null(B) (the projection of chi),
    b = (0, chi) gives B x = chi.  Checked with the oracle's own assembled B and lifted operator."""
    import dataclasses
    wl = W.WORKLOADS[name]
    prob = wl["make"]()
    lev = O.Level(O.raw_from_problem(prob))
    raw = lev.raw
    B = O.lifted_constraint_jacobian(lev.N, lev.V, lev.Z, raw.n, raw.p, raw.q)
    m, nx = B.shape
    rng = np.random.default_rng(12)
    for which in ("primal", "dual"):
        chi = rng.standard_normal(nx if which == "primal" else m)
        rhs = np.concatenate([chi, np.zeros(m)]) if which == "primal" else np.concatenate([np.zeros(nx), chi])
        x, info = _solve(P, dataclasses.replace(prob, b=rhs), wl, 1e-10, omega=0.7)
        assert np.linalg.norm(rhs - lev.A @ x) <= 1.5e-10 * np.linalg.norm(rhs)
        Bx = B @ x[:nx]
        if which == "primal":
            assert np.linalg.norm(Bx) <= 1.5e-10 * np.linalg.norm(chi)
        else:
            assert np.linalg.norm(Bx - chi) <= 1.5e-10 * np.linalg.norm(chi)


@pytest.mark.slow
def test_c3_burgers_full_size_residual(P):
    """C3 (Burgers nx = 512, n = 8192, 21 M unknowns, 4 levels) in bench.py's configuration
    (relaxed sweeps, restart 100, rtol 1e-8), with the FP64 and the FP32-pair Krylov basis:
    the oracle's own assembled lifted operator confirms the residual each solve reports.
    (The oracle's FGMRES is out of reach at this size; the residual holds at any size.)"""
    wl = W.WORKLOADS["burgers_nx512_n8192"]
    prob = wl["make"]()
    lev = O.Level(O.raw_from_problem(prob))
    bn = np.linalg.norm(prob.b)
    for basis in ("fp64", "pair"):
        x, info = _solve(P, prob, wl, 1e-8, restart=wl["restart"], omega=0.7, krylov_basis=basis)
        rel = np.linalg.norm(prob.b - lev.A @ x) / bn
        assert rel <= 1.05e-8, (basis, rel)
        assert abs(rel - info.true_relres) <= 1e-12 + 1e-6 * rel, (basis, rel, info.true_relres)
