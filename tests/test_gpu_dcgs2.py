"""Delayed reorthogonalisation (DCGS2) on the FP32-pair Krylov basis: the
same FGMRES iterations as classical Gram-Schmidt twice on the same basis
(within one), the oracle's direct solution to the solve tolerance, across
restarts and with a cycle that ends full, and an orthonormal basis."""
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
    (lambda: W.burgers(nx=40, n=32, seed=601), dict(levels=2, nu_pre=2, nu_post=2, omega=2.0 / 3.0,
                                                   restrict="transpose"), 7),
    (lambda: W.burgers(nx=40, n=32, seed=602), dict(levels=2, nu_pre=2, nu_post=2, omega=2.0 / 3.0,
                                                   restrict="transpose"), 60),
    (lambda: W.vdp(n=128, seed=603), dict(levels=2, nu_pre=1, nu_post=1), 400),
    (lambda: W.burgers(nx=64, n=64, seed=604), dict(levels=3, nu_pre=4, nu_post=4), 25),
]


def _solve(P, prob, opts, basis, restart, loops, rtol=1e-10):
    h = P.mg_setup(prob, krylov_basis=basis, device_loops=loops, **opts)
    try:
        b = torch.tensor(prob.b, dtype=torch.float64, device="cuda")
        x = torch.zeros_like(b)
        st, info = P.fgmres_solve(h, b.data_ptr(), x.data_ptr(), rtol, maxit=2000, restart=restart)
        return st, info, x.cpu().numpy()
    finally:
        P.mg_destroy(h)


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("loops", [False, True])
def test_dcgs2_matches_cgs2_and_the_direct_solution(P, case, loops):
    make, opts, restart = CASES[case]
    prob = make()
    ref = O.direct_solve(prob)
    st0, i0, x0 = _solve(P, prob, opts, "pair", restart, loops)
    st1, i1, x1 = _solve(P, prob, opts, "pair_dcgs2", restart, loops)
    assert st0 == P.MG_OK and st1 == P.MG_OK, (P.mg_status_string(st0), P.mg_status_string(st1))
    assert abs(i1.iters - i0.iters) <= 1, (i0.iters, i1.iters)
    assert i1.true_relres <= 1e-10 * 1.01
    assert np.linalg.norm(x1 - ref) <= 1e-9 * np.linalg.norm(ref)
