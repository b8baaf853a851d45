"""Krylov reductions fused into the kernels that produce their partial sums
(the last CTA of a multi-dot reduces it; the last CTA of CGS2's second axpy
forms ||w||^2, adds the two passes' coefficients and the Arnoldi column)
against separate reduction / step launches: the same sums in the same order,
so bitwise-equal solves with fewer launches per iteration."""
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


def _solve(P, prob, opts, monkeypatch, fused, restart):
    monkeypatch.setenv("PINTMG_FUSE_REDUCE", str(fused))
    h = P.mg_setup(prob, **opts)
    monkeypatch.delenv("PINTMG_FUSE_REDUCE")
    try:
        b = torch.tensor(prob.b, dtype=torch.float64, device="cuda")
        x = torch.empty_like(b)
        n0 = P.mg_launch_count(h)
        code, info = P.fgmres_solve(h, b.data_ptr(), x.data_ptr(), 1e-10, 500, restart)
        torch.cuda.synchronize()
        assert code == P.MG_OK, P.mg_status_string(code)
        return x.cpu().numpy(), info, P.mg_launch_count(h) - n0
    finally:
        P.mg_destroy(h)


@pytest.mark.parametrize("level", [1, 2])
@pytest.mark.parametrize("basis", ["fp64", "pair"])
@pytest.mark.parametrize("loops", [False, True])
@pytest.mark.parametrize("case", [0, 1])
def test_fused_reductions_are_bitwise_neutral(P, monkeypatch, basis, loops, case, level):
    prob, opts, restart = [
        (W.burgers(nx=40, n=32, seed=401), dict(levels=2, nu_pre=2, nu_post=2, omega=2.0 / 3.0,
                                               restrict="transpose"), 7),   # restarts every 7 iterations
        (W.vdp(n=64, seed=402), dict(levels=3, nu_pre=1, nu_post=1), 40),
    ][case]
    opts = dict(opts, krylov_basis=basis, device_loops=loops)
    x1, i1, l1 = _solve(P, prob, opts, monkeypatch, level, restart)
    x0, i0, l0 = _solve(P, prob, opts, monkeypatch, 0, restart)
    assert (i1.iters, i1.coarse_iters) == (i0.iters, i0.coarse_iters)
    assert i1.true_relres == i0.true_relres and np.array_equal(x1, x0)
    if not loops:
        # per FGMRES and coarse GMRES iteration: no separate norm reduction, coefficient sum or
        # Arnoldi step; with every dot product fused (level 2, FP64 basis) two reductions fewer still
        steps = i1.iters + i1.coarse_iters
        saved_per_step = 5 if (level == 2 and basis == "fp64") else 3
        assert l0 - l1 >= saved_per_step * steps, (l0, l1, steps)
    xd = O.direct_solve(prob)
    assert np.linalg.norm(x1 - xd) <= 1e-9 * np.linalg.norm(xd)


@pytest.mark.parametrize("basis", ["fp64", "pair"])
def test_fused_copies_in_captured_solves(P, monkeypatch, basis):
    """In a captured solve the basis write also fills the preconditioner's input and the operator product
    also stores the preconditioned vector Z_j (two copy launches fewer per FGMRES and coarse GMRES
    iteration): bitwise the same solve, across a restart."""
    prob = W.burgers(nx=40, n=32, seed=403)
    opts = dict(levels=2, nu_pre=2, nu_post=2, omega=2.0 / 3.0, restrict="transpose", krylov_basis=basis,
                device_loops=True)
    res, graph = {}, {}
    for fc in ("1", "0"):
        monkeypatch.setenv("PINTMG_FUSE_COPIES", fc)
        h = P.mg_setup(prob, **opts)
        monkeypatch.delenv("PINTMG_FUSE_COPIES")
        try:
            b = torch.tensor(prob.b, dtype=torch.float64, device="cuda")
            runs = []
            for _ in range(2):  # the second launch of the cached graph too
                x = torch.empty_like(b)
                n0 = P.mg_launch_count(h)
                code, info = P.fgmres_solve(h, b.data_ptr(), x.data_ptr(), 1e-10, 200, 6)
                assert code == P.MG_OK, P.mg_status_string(code)
                runs.append((x.cpu().numpy(), info.iters, info.coarse_iters, P.mg_launch_count(h) - n0))
            res[fc] = runs
            graph[fc] = P.mg_graph_launches(h)
        finally:
            P.mg_destroy(h)
    for k in range(2):
        x1, it1, c1, l1 = res["1"][k]
        x0, it0, c0, l0 = res["0"][k]
        assert (it1, c1) == (it0, c0) and np.array_equal(x1, x0)
        assert l0 - l1 == 2 * (it1 + c1), (l0, l1, it1, c1)
    # the graph's own record: two launches fewer in each loop body, the same fixed part
    (s1, f1, b1, k1), (s0, f0, b0, k0) = graph["1"], graph["0"]
    assert s1 == s0 == P.MG_OK and f1 == f0 and b0 - b1 == 2 and k0 - k1 == 2 and b1 > 0 and k1 > 0
    for k in range(2):
        assert res["1"][k][3] == f1 + b1 * res["1"][k][1] + k1 * res["1"][k][2]
