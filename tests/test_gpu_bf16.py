"""BF16 storage of the N, V, Z~ bands (MG_PRECISION_BF16_BANDS): the V-cycle
in FP32 with BF16 bands on every smoothing level, against the oracle's cycle
on the same BF16-rounded bands (FP64 arithmetic), and FGMRES (FP64, exact
operator) reaching the direct solution of the unrounded system."""
import numpy as np
import pytest

from oracle import augmented as O
from paper_2405_04808_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SOLVE_RTOL = 1e-9


@pytest.fixture(scope="module")
def P():
    from paper_2405_04808_gb300 import pintmg
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pintmg.lib()
    return pintmg


CASES = [
    (lambda: W.burgers(nx=40, n=32, seed=501), dict(levels=2, nu_pre=2, nu_post=2)),
    (lambda: W.burgers(nx=128, n=64, seed=502), dict(levels=3, nu_pre=4, nu_post=4, omega=2.0 / 3.0,
                                                     restrict="transpose")),
    (lambda: W.burgers(nx=130, n=16, seed=503), dict(levels=2, nu_pre=1, nu_post=2)),   # unstaged kernels
    (lambda: W.burgers(nx=24, n=32, seed=504, theta=0.5), dict(levels=3, nu_pre=2, nu_post=1)),  # V != kappa Z
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_bf16_band_vcycle_matches_oracle_on_rounded_bands(P, case):
    make, opts = CASES[case]
    prob = make()
    opts = dict(opts, coarse_fixed_iters=2)
    h = P.mg_setup(prob, precision=P.MG_PRECISION_BF16_BANDS, **opts)
    try:
        r = torch.tensor(prob.b, dtype=torch.float64, device="cuda")
        y = torch.empty_like(r)
        assert P.mg_vcycle(h, r.data_ptr(), y.data_ptr(), 0) == P.MG_OK
        torch.cuda.synchronize()
        yg = y.cpu().numpy()
    finally:
        P.mg_destroy(h)
    yb = O.Hierarchy(prob, O.MGOptions(bands="bf16", **opts)).precondition(prob.b)
    y64 = O.Hierarchy(prob, O.MGOptions(**opts)).precondition(prob.b)
    err_b = np.linalg.norm(yg - yb) / np.linalg.norm(yb)
    err_64 = np.linalg.norm(yg - y64) / np.linalg.norm(y64)
    # FP32 arithmetic on the same rounded bands; the rounding itself moves the cycle much further
    assert err_b <= 1e-3, err_b
    assert err_b <= 0.2 * err_64, (err_b, err_64)


@pytest.mark.parametrize("case", range(len(CASES)))
def test_bf16_band_preconditioned_fgmres_reaches_fp64_solution(P, case):
    make, opts = CASES[case]
    prob = make()
    h = P.mg_setup(prob, precision=P.MG_PRECISION_BF16_BANDS, **opts)
    try:
        b = torch.tensor(prob.b, dtype=torch.float64, device="cuda")
        x = torch.empty_like(b)
        code, info = P.fgmres_solve(h, b.data_ptr(), x.data_ptr(), 1e-10, 3000, 300)
        assert code == P.MG_OK, P.mg_status_string(code)
        assert info.true_relres <= 2e-10
    finally:
        P.mg_destroy(h)
    xd = O.direct_solve(prob)
    assert np.linalg.norm(x.cpu().numpy() - xd) <= SOLVE_RTOL * np.linalg.norm(xd)


def test_bf16_bands_need_the_tridiagonal_layout(P):
    with pytest.raises(P.PintmgError) as e:
        P.mg_setup(W.vdp(n=16, seed=505), levels=2, precision=P.MG_PRECISION_BF16_BANDS)
    assert e.value.code == P.MG_ERR_UNSUPPORTED
