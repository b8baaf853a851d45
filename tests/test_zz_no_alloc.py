"""The residual check that allocates nothing agrees with fgmres_solve's own
true residual, call after call (its scratch is a shared static device array)."""
import numpy as np
import pytest

from paper_2405_04808_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# both sides run the same FP64 kernels in the same reduction order; allow
# rounding-level differences only
RTOL = 1e-12


@pytest.fixture(scope="module")
def P():
    from paper_2405_04808_gb300 import pintmg
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pintmg.lib()
    return pintmg


@pytest.mark.parametrize("make", [lambda: W.burgers(nx=40, n=32, seed=151), lambda: W.vdp(n=64, seed=152)],
                         ids=["burgers", "vdp"])
def test_noalloc_residual_matches_solver(P, make):
    prob = make()
    h = P.mg_setup(prob, levels=2, nu_pre=2, nu_post=2)
    try:
        b = torch.tensor(prob.b, dtype=torch.float64, device="cuda")
        x = torch.empty_like(b)
        code, info = P.fgmres_solve(h, b.data_ptr(), x.data_ptr(), 1e-9, 2000, 400)
        assert code == P.MG_OK
        out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
        for _ in range(2):  # two calls in a row reuse the same static scratch
            out.fill_(-1.0)
            assert P.mg_true_residual_noalloc(h, b.data_ptr(), x.data_ptr(), out.data_ptr(), 0) == P.MG_OK
            torch.cuda.synchronize()
            rel = float(out[1])
            assert abs(rel - info.true_relres) <= RTOL * max(info.true_relres, 1e-300)
            assert abs(float(out[0]) - rel * float(torch.linalg.norm(b))) <= 1e-12 * float(out[0]) + 1e-300
        # against the oracle's assembled lifted operator (Fig. 4): ||b - A x|| / ||b|| in FP64 on the host
        from oracle import augmented as O
        A = O.Level(O.raw_from_problem(prob)).A
        xh = x.cpu().numpy()
        want = float(np.linalg.norm(prob.b - A @ xh) / np.linalg.norm(prob.b))
        # (a residual near 1e-9 carries cancellation error of order eps * ||A|| ||x|| / ||b|| from either side)
        assert abs(float(out[1]) - want) <= 1e-4 * want + 1e-14, (float(out[1]), want)
        # a different x gives its own residual (nothing stale from the previous call)
        xz = torch.zeros_like(b)
        assert P.mg_true_residual_noalloc(h, b.data_ptr(), xz.data_ptr(), out.data_ptr(), 0) == P.MG_OK
        torch.cuda.synchronize()
        assert abs(float(out[1]) - 1.0) <= 1e-14
    finally:
        P.mg_destroy(h)


def test_noalloc_rejects_vectors_beyond_its_scratch(P):
    prob = W.burgers(nx=16, n=16384, seed=153)   # n (4p+q) = 1,310,720 > 2^20
    h = P.mg_setup(prob, levels=2)
    try:
        n = prob.size
        b = torch.zeros(n, dtype=torch.float64, device="cuda")
        out = torch.zeros(2, dtype=torch.float64, device="cuda")
        code = P.mg_true_residual_noalloc(h, b.data_ptr(), b.data_ptr(), out.data_ptr(), 0)
        assert code == P.MG_ERR_ARG
        assert "exceeds" in P.mg_last_cuda_error()
    finally:
        P.mg_destroy(h)
