"""All block-Jacobi sweeps of a smoothing level in one cooperative launch
(k_sweeps_tri2, an option: PINTMG_PERSIST=1) against one launch per sweep
(k_block_solve_tri2, the default): the same arithmetic in the same order, so
bitwise-equal V-cycles and solves; and the bounded wait of that kernel, made
to run out without a GPU fault."""
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


CASES = [
    # (problem, options)
    (lambda: W.burgers(nx=128, n=64, seed=301), dict(levels=3, nu_pre=4, nu_post=4, omega=2.0 / 3.0,
                                                     restrict="transpose")),   # p = 128: compile-time chunks
    (lambda: W.burgers(nx=40, n=32, seed=302), dict(levels=2, nu_pre=2, nu_post=3)),         # ragged chunks
    (lambda: W.burgers(nx=7, n=16, seed=303, theta=0.5), dict(levels=2, nu_pre=1, nu_post=2, omega=0.7)),
    (lambda: W.burgers(nx=64, n=32, seed=304), dict(levels=3, nu_pre=3, nu_post=1, precision=1)),  # FP32 cycle
    (lambda: W.burgers(nx=128, n=8, seed=305), dict(levels=2, nu_pre=4, nu_post=4)),          # 9 blocks
]


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _run(P, prob, opts, monkeypatch, persist):
    monkeypatch.setenv("PINTMG_PERSIST", "1" if persist else "0")
    h = P.mg_setup(prob, **opts)
    monkeypatch.delenv("PINTMG_PERSIST")
    try:
        b = _dev(prob.b)
        y = torch.empty_like(b)
        n0 = P.mg_launch_count(h)
        assert P.mg_vcycle(h, b.data_ptr(), y.data_ptr(), 0) == P.MG_OK
        launches = P.mg_launch_count(h) - n0
        x = torch.empty_like(b)
        code, info = P.fgmres_solve(h, b.data_ptr(), x.data_ptr(), 1e-10, 2000, 300)
        torch.cuda.synchronize()
        assert code == P.MG_OK, P.mg_status_string(code)
        return y.cpu().numpy(), x.cpu().numpy(), info.iters, launches
    finally:
        P.mg_destroy(h)


@pytest.mark.parametrize("case", range(len(CASES)))
def test_persistent_sweeps_equal_separate_launches(P, monkeypatch, case):
    make, opts = CASES[case]
    prob = make()
    y1, x1, it1, l1 = _run(P, prob, opts, monkeypatch, True)
    y0, x0, it0, l0 = _run(P, prob, opts, monkeypatch, False)
    assert np.array_equal(y1, y0)
    assert it1 == it0 and np.array_equal(x1, x0)
    # the fused path was taken where it applies (p <= 128 and 16-byte coefficient rows:
    # p even in FP64, a multiple of 4 in FP32): one launch per smoothing instead of one per sweep
    fp32 = opts.get("precision", 0) == 1
    eligible = prob.p <= 128 and prob.p % (4 if fp32 else 2) == 0
    sweeps = (opts["nu_pre"] + opts["nu_post"]) * (opts["levels"] - 1)
    fused = sum(1 for k in ("nu_pre", "nu_post") if opts[k] > 0) * (opts["levels"] - 1)
    assert l0 - l1 == (sweeps - fused if eligible else 0), (l0, l1)
    # and the solve is the direct solution
    xd = O.direct_solve(prob)
    assert np.linalg.norm(x1 - xd) <= 1e-9 * np.linalg.norm(xd)


@pytest.mark.parametrize("loops", [True, False])
def test_persistent_sweep_wait_runs_out_without_a_fault(P, monkeypatch, loops):
    """Failure detection without a GPU fault: with the test hook set, block 0
    never publishes its coupling, so block 1's wait for it runs out (2 s); the
    kernel records it and finishes without further waits, and the solve (and a
    single V-cycle) report MG_ERR_TIMEOUT.  The context stays usable: a new
    handle afterwards solves to the direct solution."""
    import time
    prob = W.burgers(nx=40, n=32, seed=306)
    opts = dict(levels=2, nu_pre=2, nu_post=2, device_loops=loops)
    monkeypatch.setenv("PINTMG_TEST_SWEEP_STALL", "1")
    monkeypatch.setenv("PINTMG_PERSIST", "1")
    h = P.mg_setup(prob, **opts)
    monkeypatch.delenv("PINTMG_TEST_SWEEP_STALL")
    try:
        b = _dev(prob.b)
        x = torch.empty_like(b)
        t0 = time.time()
        code, info = P.fgmres_solve(h, b.data_ptr(), x.data_ptr(), 1e-10, 6, 6)
        assert code == P.MG_ERR_TIMEOUT, P.mg_status_string(code)
        y = torch.empty_like(b)
        assert P.mg_vcycle(h, b.data_ptr(), y.data_ptr(), 0) == P.MG_ERR_TIMEOUT
        assert time.time() - t0 < 60.0
    finally:
        P.mg_destroy(h)
    h = P.mg_setup(prob, **opts)
    monkeypatch.delenv("PINTMG_PERSIST")
    try:
        b = _dev(prob.b)
        x = torch.empty_like(b)
        code, info = P.fgmres_solve(h, b.data_ptr(), x.data_ptr(), 1e-10, 2000, 300)
        assert code == P.MG_OK
        xd = O.direct_solve(prob)
        assert np.linalg.norm(x.cpu().numpy() - xd) <= 1e-9 * np.linalg.norm(xd)
    finally:
        P.mg_destroy(h)
