"""The autotuner: its choices keep the results (bitwise for the dot-product
blocking, to the solve tolerance for the chain evaluation), and a second
handle of the same shape takes the cached choice."""
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


@pytest.mark.parametrize("make,settings", [
    (lambda: W.burgers(nx=64, n=64, seed=71), dict(levels=3, nu_pre=2, nu_post=2)),
    (lambda: W.vdp(n=128, seed=72), dict(levels=2, nu_pre=1, nu_post=1)),
    (lambda: W.burgers(nx=48, n=32, seed=73), dict(levels=2, nu_pre=1, nu_post=1, precision=1)),
])
def test_autotuned_solve_keeps_the_solution(P, make, settings):
    prob = make()
    ref = O.direct_solve(prob)
    b = torch.tensor(prob.b, dtype=torch.float64, device="cuda")
    xs, choices, maps = [], [], []
    for tune in (False, True, True):
        h = P.mg_setup(prob, **settings)
        try:
            if tune:
                choices.append(P.mg_autotune(h))
            maps.append([P.mg_block_mapping(h, l) for l in range(settings["levels"])])
            x = torch.zeros_like(b)
            st, info = P.fgmres_solve(h, b.data_ptr(), x.data_ptr(), 1e-10, maxit=1500, restart=200)
            assert st == P.MG_OK
            xs.append(x.cpu().numpy())
        finally:
            P.mg_destroy(h)
    assert choices[0] == choices[1]                      # the second handle takes the cached choice
    chain, vb = choices[0]
    assert chain in P.SGS_CHAINS and vb in (4, 8, 16)
    for x in xs:
        assert np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref)
    assert np.array_equal(xs[1], xs[2]) and maps[1] == maps[2]
    assert all(m in (1, 2) for mm in maps for m in mm)
    if chain == "scan" and maps[0] == maps[1]:           # default chain and block mapping: only the blocking
        assert np.array_equal(xs[0], xs[1])
