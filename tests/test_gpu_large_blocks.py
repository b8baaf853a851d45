"""Tridiagonal blocks larger than one warp's registers hold (p = 512): the
block solve in three launches (right-hand sides, pentadiagonal solves,
outputs) against the one-warp kernel it replaces, which forms every entry by
the same operations: bitwise-equal V-cycles for both couplings of V and Z,
relaxed and undamped sweeps, FP64, FP32 and BF16 bands; and a solve against
the oracle's direct solution."""
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


def _vcycle(P, prob, split, monkeypatch, **opts):
    monkeypatch.setenv("PINTMG_SPLIT_BS", "1" if split else "0")
    h = P.mg_setup(prob, **opts)
    monkeypatch.delenv("PINTMG_SPLIT_BS")
    try:
        r = torch.tensor(np.random.default_rng(5).standard_normal(prob.size), dtype=torch.float64, device="cuda")
        y = torch.empty_like(r)
        assert P.mg_vcycle(h, r.data_ptr(), y.data_ptr()) == P.MG_OK
        torch.cuda.synchronize()
        return y.cpu().numpy()
    finally:
        P.mg_destroy(h)


@pytest.mark.parametrize("theta", [1.0, 0.5])            # V = kappa Z (one product) and the general path
@pytest.mark.parametrize("precision", ["fp64", "fp32", "bf16"])
@pytest.mark.parametrize("omega,restrict", [(1.0, "inject"), (2.0 / 3.0, "transpose")])
def test_split_block_solve_is_bitwise_the_one_warp_solve(P, monkeypatch, theta, precision, omega, restrict):
    prob = W.burgers(nx=512, n=16, seed=31, theta=theta)
    prec = {"fp64": P.MG_PRECISION_FP64, "fp32": P.MG_PRECISION_FP32, "bf16": P.MG_PRECISION_BF16_BANDS}[precision]
    opts = dict(levels=3, nu_pre=2, nu_post=2, omega=omega, restrict=restrict, precision=prec)
    a = _vcycle(P, prob, True, monkeypatch, **opts)
    b = _vcycle(P, prob, False, monkeypatch, **opts)
    assert np.isfinite(a).all() and np.linalg.norm(a) > 0
    assert np.array_equal(a, b)


def test_split_block_solve_reaches_the_direct_solution(P):
    prob = W.burgers(nx=512, n=32, seed=32)
    h = P.mg_setup(prob, levels=3, nu_pre=2, nu_post=2, omega=2.0 / 3.0, restrict="transpose")
    try:
        b = torch.tensor(prob.b, dtype=torch.float64, device="cuda")
        x = torch.zeros_like(b)
        st, info = P.fgmres_solve(h, b.data_ptr(), x.data_ptr(), 1e-11, maxit=300, restart=60)
        assert st == P.MG_OK
    finally:
        P.mg_destroy(h)
    ref = O.direct_solve(prob)
    xs = x.cpu().numpy()
    assert np.linalg.norm(xs - ref) <= 1e-9 * np.linalg.norm(ref)


@pytest.mark.parametrize("loops", [True, False])
def test_split_kernels_give_the_same_solve(P, monkeypatch, loops):
    """FGMRES with restarts (operator products with the basis copy, restart residuals, sweeps, transfers) on
    p = 512 blocks: the per-entry kernels and the one-warp kernels give the same bits."""
    prob = W.burgers(nx=512, n=32, seed=33)
    out = []
    for split in ("1", "0"):
        monkeypatch.setenv("PINTMG_SPLIT_BS", split)
        h = P.mg_setup(prob, levels=3, nu_pre=2, nu_post=2, omega=2.0 / 3.0, restrict="transpose",
                       device_loops=loops)
        monkeypatch.delenv("PINTMG_SPLIT_BS")
        try:
            b = torch.tensor(prob.b, dtype=torch.float64, device="cuda")
            x = torch.zeros_like(b)
            st, info = P.fgmres_solve(h, b.data_ptr(), x.data_ptr(), 1e-10, maxit=300, restart=4)
            assert st == P.MG_OK
            out.append((x.cpu().numpy(), info.iters, info.true_relres))
        finally:
            P.mg_destroy(h)
    assert out[0][1] == out[1][1] and out[0][2] == out[1][2] and np.array_equal(out[0][0], out[1][0])
