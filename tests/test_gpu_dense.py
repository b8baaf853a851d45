"""Dense local blocks beyond 4 x 4 (a warp per time block, p, q <= 32): the
V-cycle against the oracle, FGMRES against the direct solve, the same system
in the dense and the tridiagonal layouts, and the size limit."""
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
    (lambda: W.coupled(p=12, q=6, n=32, seed=801), dict(levels=3, nu_pre=2, nu_post=2)),
    (lambda: W.coupled(p=5, q=1, n=48, seed=802), dict(levels=2, nu_pre=1, nu_post=1, omega=2.0 / 3.0,
                                                       restrict="transpose")),
    (lambda: W.coupled(p=32, q=32, n=16, seed=803), dict(levels=2, nu_pre=3, nu_post=2)),   # the largest block
    (lambda: W.coupled(p=32, q=3, n=32, seed=804), dict(levels=3, nu_pre=2, nu_post=1, end_rule=1)),
    (lambda: W.dense_copy(W.burgers(nx=20, n=32, seed=805)), dict(levels=2, nu_pre=2, nu_post=2)),
]


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("case", range(len(CASES)))
def test_dense_warp_vcycle_matches_oracle(P, case):
    make, opts = CASES[case]
    prob = make()
    opts = dict(opts, coarse_fixed_iters=3)
    h = P.mg_setup(prob, **opts)
    try:
        rd = _dev(prob.b)
        yd = torch.empty_like(rd)
        assert P.mg_vcycle(h, rd.data_ptr(), yd.data_ptr(), 0) == P.MG_OK
        torch.cuda.synchronize()
        yo = O.Hierarchy(prob, O.MGOptions(**opts)).precondition(prob.b)
        err = np.linalg.norm(yd.cpu().numpy() - yo) / np.linalg.norm(yo)
        assert err <= 1e-10, err
    finally:
        P.mg_destroy(h)


@pytest.mark.parametrize("case", range(len(CASES)))
def test_dense_warp_fgmres_matches_direct_solve(P, case):
    make, opts = CASES[case]
    prob = make()
    for loops in (True, False):
        h = P.mg_setup(prob, device_loops=loops, **opts)
        try:
            b = _dev(prob.b)
            x = torch.empty_like(b)
            code, info = P.fgmres_solve(h, b.data_ptr(), x.data_ptr(), 1e-10, 2000, 500)
            assert code == P.MG_OK, P.mg_status_string(code)
            xd = O.direct_solve(prob)
            assert np.linalg.norm(x.cpu().numpy() - xd) <= 1e-9 * np.linalg.norm(xd)
        finally:
            P.mg_destroy(h)


def test_dense_and_tridiagonal_layouts_agree(P):
    """The same Burgers system stored tridiagonal (warp-scan LDL^T) and dense (warp Cholesky)."""
    prob = W.burgers(nx=24, n=64, seed=806)
    outs = []
    for pr in (prob, W.dense_copy(prob)):
        h = P.mg_setup(pr, levels=3, nu_pre=2, nu_post=2, coarse_fixed_iters=3)
        try:
            rd = _dev(pr.b)
            yd = torch.empty_like(rd)
            assert P.mg_vcycle(h, rd.data_ptr(), yd.data_ptr(), 0) == P.MG_OK
            torch.cuda.synchronize()
            outs.append(yd.cpu().numpy())
        finally:
            P.mg_destroy(h)
    assert np.linalg.norm(outs[0] - outs[1]) <= 1e-10 * np.linalg.norm(outs[0])


def test_dense_blocks_beyond_32_are_unsupported(P):
    with pytest.raises(P.PintmgError) as e:
        P.mg_setup(W.coupled(p=33, q=2, n=8, seed=807), levels=2)
    assert e.value.code == P.MG_ERR_UNSUPPORTED
