"""The V-cycle sharded by time (paper_2405_04808_gb300.timeshard) on the GPU
through the library's time-range entry points, with two and three ranks held
in one process (their kernels run one after another; no kernel waits on
another): the same cycle as mg_vcycle on the whole system."""
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
    # (problem, options, world, bitwise): the transposed restriction uses the cycle's own kernels
    (lambda: W.burgers(nx=128, n=64, seed=701), dict(levels=3, nu_pre=4, nu_post=4, omega=2.0 / 3.0,
                                                     restrict="transpose"), 2, True),
    (lambda: W.burgers(nx=40, n=96, seed=702), dict(levels=3, nu_pre=2, nu_post=1, restrict="transpose",
                                                    end_rule=1), 3, True),
    (lambda: W.vdp(n=64, seed=703), dict(levels=2, nu_pre=1, nu_post=2, restrict="transpose"), 2, True),
    # injection: the cycle fuses residual and restriction, the range path does not (equal to rounding)
    (lambda: W.burgers(nx=40, n=32, seed=704), dict(levels=2, nu_pre=2, nu_post=2), 2, False),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_sharded_vcycle_matches_mg_vcycle(P, case):
    from paper_2405_04808_gb300 import timeshard as TS
    make, opts, world, bitwise = CASES[case]
    prob = make()
    h = P.mg_setup(prob, coarse_fixed_iters=3, **opts)
    try:
        b = torch.tensor(prob.b, dtype=torch.float64, device="cuda")
        ref = torch.empty_like(b)
        assert P.mg_vcycle(h, b.data_ptr(), ref.data_ptr(), 0) == P.MG_OK
        levels = opts["levels"]
        layouts = [TS.Layout(P.mg_level_info(h, lv)[0], prob.p, prob.q) for lv in range(levels)]
        part = TS.Partition(prob.n, levels, world)
        ranks = list(range(world))
        engines = [TS.LibraryEngine(P, h) for _ in ranks]
        cyc = TS.ShardedVCycle(part, layouts, engines, ranks, TS.LocalExchange(world), opts["nu_pre"],
                               opts["nu_post"], lambda k: torch.zeros(k, dtype=torch.float64, device="cuda"))
        y = cyc.vcycle(0, [b.clone() for _ in ranks])
        torch.cuda.synchronize()
        got = torch.full_like(b, float("nan"))
        for r in ranks:
            j0, j1 = part.blocks(r, 0)
            for j in range(j0, j1):
                for sl in layouts[0].block(j):
                    got[sl] = y[r][sl]
        g, want = got.cpu().numpy(), ref.cpu().numpy()
        assert not np.isnan(g).any()
        if bitwise:
            assert np.array_equal(g, want)
        else:
            assert np.linalg.norm(g - want) <= 1e-12 * np.linalg.norm(want)
    finally:
        P.mg_destroy(h)


def test_range_entry_points_reject_bad_ranges(P):
    prob = W.burgers(nx=16, n=16, seed=705)
    h = P.mg_setup(prob, levels=2)
    try:
        v = torch.zeros(prob.size, dtype=torch.float64, device="cuda")
        with pytest.raises(P.PintmgError):
            P.mg_range_sweep(h, 0, 4, 4, v.data_ptr(), 0, v.data_ptr() + 8)     # empty range
        with pytest.raises(P.PintmgError):
            P.mg_range_sweep(h, 1, 0, 4, v.data_ptr(), 0, v.data_ptr() + 8)     # the coarsest level
        with pytest.raises(P.PintmgError):
            P.mg_range_restrict(h, 0, 3, 9, v.data_ptr(), v.data_ptr())          # odd start
        with pytest.raises(P.PintmgError):
            P.mg_range_residual(h, 0, 0, 18, v.data_ptr(), v.data_ptr(), v.data_ptr())  # past n + 1
    finally:
        P.mg_destroy(h)


def _owned_index(layout, j0, j1):
    return np.concatenate([np.arange(sl.start, sl.stop) for j in range(j0, j1) for sl in layout.block(j)])


@pytest.mark.parametrize("j0,j1", [(0, 5), (5, 17), (16, 17), (0, 17), (7, 8)])
def test_range_krylov_entry_points(P, j0, j1):
    """mg_range_dots / mg_range_axpy / mg_range_scale against numpy on the
    entries of blocks [j0, j1); the other entries are left as they were."""
    from paper_2405_04808_gb300 import timeshard as TS
    prob = W.burgers(nx=24, n=16, seed=706)
    h = P.mg_setup(prob, levels=2)
    try:
        n, length = P.mg_level_info(h, 0)
        lay = TS.Layout(n, prob.p, prob.q)
        idx = _owned_index(lay, j0, j1)
        rng = np.random.default_rng(707)
        k = 11
        Vh = rng.standard_normal((k, length + 3))          # stride > length
        wh, ch = rng.standard_normal(length), rng.standard_normal(k)
        V = torch.tensor(Vh, device="cuda")
        w = torch.tensor(wh, device="cuda")
        c = torch.tensor(ch, device="cuda")
        out = torch.full((k,), np.nan, dtype=torch.float64, device="cuda")
        P.mg_range_dots(h, 0, j0, j1, V.data_ptr(), V.stride(0), k, w.data_ptr(), out.data_ptr())
        want = Vh[:, idx] @ wh[idx]
        assert np.allclose(out.cpu().numpy(), want, rtol=1e-12, atol=1e-12 * np.abs(Vh[:, idx]).sum())
        P.mg_range_axpy(h, 0, j0, j1, V.data_ptr(), V.stride(0), k, c.data_ptr(), -1.0, w.data_ptr())
        got = w.cpu().numpy()
        ref = wh.copy()
        ref[idx] -= ch @ Vh[:, idx]
        assert np.allclose(got, ref, rtol=0, atol=1e-12 * (1 + np.abs(Vh).max() * np.abs(ch).sum()))
        rest = np.setdiff1d(np.arange(length), idx)
        assert np.array_equal(got[rest], wh[rest])
        a = torch.tensor([0.375], dtype=torch.float64, device="cuda")
        y = torch.zeros(length, dtype=torch.float64, device="cuda")
        P.mg_range_scale(h, 0, j0, j1, w.data_ptr(), a.data_ptr(), y.data_ptr())
        yh = y.cpu().numpy()
        assert np.array_equal(yh[idx], 0.375 * got[idx]) and not yh[rest].any()
        for bad in (0, 513):
            with pytest.raises(P.PintmgError):
                P.mg_range_dots(h, 0, j0, j1, V.data_ptr(), V.stride(0), bad, w.data_ptr(), out.data_ptr())
        with pytest.raises(P.PintmgError):
            P.mg_range_axpy(h, 0, j0, j1, V.data_ptr(), length - 1, k, c.data_ptr(), 1.0, w.data_ptr())
        with pytest.raises(P.PintmgError):
            P.mg_range_residual(h, 0, j0, j1, w.data_ptr(), 0, w.data_ptr())      # r aliases y
    finally:
        P.mg_destroy(h)


def test_range_residual_without_b_is_the_operator_product(P):
    from paper_2405_04808_gb300 import timeshard as TS
    prob = W.burgers(nx=24, n=16, seed=708)
    h = P.mg_setup(prob, levels=2)
    try:
        n, length = P.mg_level_info(h, 0)
        lay = TS.Layout(n, prob.p, prob.q)
        y = torch.tensor(np.random.default_rng(709).standard_normal(length), device="cuda")
        zero = torch.zeros_like(y)
        neg, ay = torch.empty_like(y), torch.empty_like(y)
        P.mg_range_residual(h, 0, 3, 11, y.data_ptr(), zero.data_ptr(), neg.data_ptr())
        P.mg_range_residual(h, 0, 3, 11, y.data_ptr(), 0, ay.data_ptr())
        idx = _owned_index(lay, 3, 11)
        assert np.array_equal(ay.cpu().numpy()[idx], -neg.cpu().numpy()[idx])
    finally:
        P.mg_destroy(h)


FGMRES_CASES = [
    # (problem, options, world, restart)
    (lambda: W.burgers(nx=64, n=64, seed=710), dict(levels=3, nu_pre=2, nu_post=2, omega=2.0 / 3.0,
                                                    restrict="transpose"), 2, 40),
    (lambda: W.burgers(nx=40, n=96, seed=711), dict(levels=3, nu_pre=2, nu_post=1, restrict="transpose",
                                                    end_rule=1, omega=2.0 / 3.0), 3, 8),
]


@pytest.mark.parametrize("case", range(len(FGMRES_CASES)))
def test_sharded_fgmres_matches_fgmres_solve(P, case):
    """FGMRES around the sharded cycle, ranks held in one process, all vector
    work through the range entry points: the step count of fgmres_solve and
    its solution to the tolerance; one rank and several take the same steps."""
    from paper_2405_04808_gb300 import timeshard as TS
    make, opts, world, restart = FGMRES_CASES[case]
    prob = make()
    rtol = 1e-10
    h = P.mg_setup(prob, coarse_fixed_iters=3, **opts)
    try:
        b = torch.tensor(prob.b, dtype=torch.float64, device="cuda")
        ref = torch.zeros_like(b)
        st, info = P.fgmres_solve(h, b.data_ptr(), ref.data_ptr(), rtol, maxit=400, restart=restart)
        assert st == P.MG_OK
        levels = opts["levels"]
        layouts = [TS.Layout(P.mg_level_info(h, lv)[0], prob.p, prob.q) for lv in range(levels)]
        sols = []
        for wd in (world, 1):
            part = TS.Partition(prob.n, levels, wd)
            ranks = list(range(wd))
            engines = [TS.LibraryEngine(P, h) for _ in ranks]
            cyc = TS.ShardedVCycle(part, layouts, engines, ranks, TS.LocalExchange(wd), opts["nu_pre"],
                                   opts["nu_post"], lambda k: torch.zeros(k, dtype=torch.float64, device="cuda"))
            res = TS.ShardedFGMRES(cyc, restart).solve([b.clone() for _ in ranks], rtol, 400)
            torch.cuda.synchronize()
            x = np.full(prob.size, np.nan)
            for r in ranks:
                idx = _owned_index(layouts[0], *part.blocks(r, 0))
                x[idx] = res.x[r].cpu().numpy()[idx]
            assert not np.isnan(x).any()
            sols.append((res.iters, x))
        want = ref.cpu().numpy()
        exact = O.direct_solve(prob)
        for iters, x in sols:
            assert abs(iters - info.iters) <= 1
            assert np.linalg.norm(x - exact) <= 1e-7 * np.linalg.norm(exact)
            assert np.linalg.norm(x - want) <= 1e-7 * np.linalg.norm(want)
        assert sols[0][0] == sols[1][0]
        assert np.linalg.norm(sols[0][1] - sols[1][1]) <= 1e-10 * np.linalg.norm(sols[1][1])
    finally:
        P.mg_destroy(h)
