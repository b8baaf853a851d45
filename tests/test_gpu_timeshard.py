"""The V-cycle sharded by time (paper_2405_04808_gb300.timeshard) on the GPU
through the library's time-range entry points, with two and three ranks held
in one process (their kernels run one after another; no kernel waits on
another): the same cycle as mg_vcycle on the whole system."""
import numpy as np
import pytest

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
