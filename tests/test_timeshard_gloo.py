"""The V-cycle sharded by time across two gloo processes (CPU), each rank
running its blocks with the oracle and exchanging the range-end couplings,
residual blocks and coarse corrections by torch.distributed: the same bits as
the unsharded cycle.  Also the partition's invariants, the same cycle with
all ranks in one process, and FGMRES around the sharded cycle (the dot
products summed over the processes): the oracle's FGMRES iterations and
solution."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")

CASES = {
    # (problem, options, world)
    "burgers_transpose": (dict(kind="burgers", nx=12, n=32, seed=601),
                          dict(levels=3, nu_pre=2, nu_post=2, omega=2.0 / 3.0, restrict="transpose"), 2),
    "vdp_inject": (dict(kind="vdp", n=64, seed=602), dict(levels=3, nu_pre=1, nu_post=2, end_rule=1), 2),
    "burgers_four_ranks": (dict(kind="burgers", nx=8, n=64, seed=603),
                           dict(levels=2, nu_pre=3, nu_post=1, restrict="transpose"), 4),
}


def _problem(spec):
    from paper_2405_04808_gb300 import workloads as W
    spec = dict(spec)
    kind = spec.pop("kind")
    return W.burgers(**spec) if kind == "burgers" else W.vdp(**spec)


def _cycle(prob, opts, world, ranks, exchange):
    from oracle import augmented as O
    from paper_2405_04808_gb300 import timeshard as TS
    from shard_oracle_engine import OracleEngine
    hier = O.Hierarchy(prob, O.MGOptions(coarse_fixed_iters=3, **opts))
    part = TS.Partition(prob.n, opts["levels"], world)
    layouts = [TS.Layout(lev.n, lev.p, lev.q) for lev in hier.levels]
    engines = [OracleEngine(hier, layouts, part, r) for r in ranks]
    cyc = TS.ShardedVCycle(part, layouts, engines, ranks, exchange, opts["nu_pre"], opts["nu_post"],
                           lambda k: torch.zeros(k, dtype=torch.float64))
    b = [torch.from_numpy(prob.b.copy()) for _ in ranks]
    y = cyc.vcycle(0, b)
    return hier, part, layouts, y


def _reference(prob, opts):
    from oracle import augmented as O
    return O.Hierarchy(prob, O.MGOptions(coarse_fixed_iters=3, **opts)).precondition(prob.b)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, name, out):
    import torch.distributed as dist

    from paper_2405_04808_gb300 import timeshard as TS
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        spec, opts, _ = CASES[name]
        prob = _problem(spec)
        _, part, layouts, y = _cycle(prob, opts, world, [rank], TS.DistExchange(dist, rank, world))
        j0, j1 = part.blocks(rank, 0)
        mine = {}
        for j in range(j0, j1):
            for sl in layouts[0].block(j):
                mine[(sl.start, sl.stop)] = y[0][sl].numpy().copy()
        out[rank] = mine
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("name", sorted(CASES))
def test_sharded_vcycle_over_gloo_ranks_equals_one_process(name):
    import torch.multiprocessing as mp
    spec, opts, world = CASES[name]
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, name, out), nprocs=world, join=True)
    prob = _problem(spec)
    ref = _reference(prob, opts)
    y = np.full(prob.size, np.nan)
    for r in range(world):
        for (a, b), vals in out[r].items():
            y[a:b] = vals
    assert not np.isnan(y).any()          # the ranks' blocks cover the vector
    assert np.array_equal(y, ref)         # bitwise the unsharded cycle


FGMRES_CASES = {
    # (problem, options, world, rtol, restart)
    "burgers_two_ranks": (dict(kind="burgers", nx=12, n=32, seed=611),
                          dict(levels=3, nu_pre=2, nu_post=2, omega=2.0 / 3.0, restrict="transpose"), 2, 1e-10, 40),
    "vdp_four_ranks_restarted": (dict(kind="vdp", n=64, seed=612),
                                 dict(levels=2, nu_pre=2, nu_post=2, omega=2.0 / 3.0, restrict="transpose"), 4, 1e-9,
                                 6),
}


def _fgmres(prob, opts, world, ranks, exchange, rtol, restart, maxit=200):
    from paper_2405_04808_gb300 import timeshard as TS
    hier, part, layouts, _ = _cycle(prob, dict(opts, nu_pre=0, nu_post=0), world, ranks, exchange)
    from shard_oracle_engine import OracleEngine
    engines = [OracleEngine(hier, layouts, part, r) for r in ranks]
    cyc = TS.ShardedVCycle(part, layouts, engines, ranks, exchange, opts["nu_pre"], opts["nu_post"],
                           lambda k: torch.zeros(k, dtype=torch.float64))
    solver = TS.ShardedFGMRES(cyc, restart)
    res = solver.solve([torch.from_numpy(prob.b.copy()) for _ in ranks], rtol, maxit)
    return part, layouts, res


def _assemble(prob, part, layouts, xs_by_rank):
    x = np.full(prob.size, np.nan)
    for r, xr in xs_by_rank.items():
        j0, j1 = part.blocks(r, 0)
        for j in range(j0, j1):
            for sl in layouts[0].block(j):
                x[sl] = xr[sl]
    return x


def _fgmres_worker(rank, world, port, name, out):
    import torch.distributed as dist

    from paper_2405_04808_gb300 import timeshard as TS
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        spec, opts, _, rtol, restart = FGMRES_CASES[name]
        _, _, res = _fgmres(_problem(spec), opts, world, [rank], TS.DistExchange(dist, rank, world), rtol, restart)
        out[rank] = (res.x[0].numpy().copy(), res.iters, res.history)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("name", sorted(FGMRES_CASES))
def test_sharded_fgmres_over_gloo_ranks(name):
    """The processes take the same steps (the summed dot products are the same
    on every one), the same number as the oracle's FGMRES with the unsharded
    cycle, and the solution meets the tolerance against the direct solve."""
    import torch.multiprocessing as mp

    from oracle import augmented as O
    spec, opts, world, rtol, restart = FGMRES_CASES[name]
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_fgmres_worker, args=(world, port, name, out), nprocs=world, join=True)
    prob = _problem(spec)
    iters = {out[r][1] for r in range(world)}
    assert len(iters) == 1 and all(out[r][2] == out[0][2] for r in range(world))   # identical decisions
    from paper_2405_04808_gb300 import timeshard as TS
    part = TS.Partition(prob.n, opts["levels"], world)
    hier = O.Hierarchy(prob, O.MGOptions(coarse_fixed_iters=3, **opts))
    layouts = [TS.Layout(lev.n, lev.p, lev.q) for lev in hier.levels]
    x = _assemble(prob, part, layouts, {r: out[r][0] for r in range(world)})
    assert not np.isnan(x).any()
    _, ref, _ = hier.solve(prob.b, rtol=rtol, maxit=200, restart=restart)
    assert ref.iters < 200 and abs(out[0][1] - ref.iters) <= 1   # CGS2 here, modified Gram-Schmidt there
    exact = O.direct_solve(prob)
    assert np.linalg.norm(prob_residual(prob, x)) <= 10 * rtol * np.linalg.norm(prob.b)
    assert np.linalg.norm(x - exact) <= 1e-6 * np.linalg.norm(exact)


def prob_residual(prob, x):
    from oracle import augmented as O
    return prob.b - O.Level(O.raw_from_problem(prob)).A @ x


@pytest.mark.parametrize("name", sorted(FGMRES_CASES))
def test_sharded_fgmres_in_one_process_matches_one_rank(name):
    """All ranks in one process against the same solver on one rank: the same
    step count and the solution to rounding (only the order of the sums of
    the dot products differs)."""
    from paper_2405_04808_gb300 import timeshard as TS
    spec, opts, world, rtol, restart = FGMRES_CASES[name]
    prob = _problem(spec)
    part, layouts, res = _fgmres(prob, opts, world, list(range(world)), TS.LocalExchange(world), rtol, restart)
    p1, l1, res1 = _fgmres(prob, opts, 1, [0], TS.LocalExchange(1), rtol, restart)
    x = _assemble(prob, part, layouts, {r: res.x[r].numpy() for r in range(world)})
    x1 = _assemble(prob, p1, l1, {0: res1.x[0].numpy()})
    assert res.iters == res1.iters
    assert np.linalg.norm(x - x1) <= 1e-10 * np.linalg.norm(x1)


def test_sharded_fgmres_sums_twice_per_step():
    """One sum for |b|, one per restart cycle for beta, two per Arnoldi step
    (the second Gram-Schmidt pass carries the norm)."""
    from paper_2405_04808_gb300 import timeshard as TS

    class Counting(TS.LocalExchange):
        calls = 0

        def allreduce(self, vals):
            Counting.calls += 1
            super().allreduce(vals)

    spec, opts, world, rtol, restart = FGMRES_CASES["vdp_four_ranks_restarted"]
    _, _, res = _fgmres(_problem(spec), opts, world, list(range(world)), Counting(world), rtol, restart)
    cycles = -(-res.iters // restart)
    assert res.iters > restart and Counting.calls == 1 + cycles + 2 * res.iters


def test_sharded_fgmres_stops_at_maxit_and_restarts_every_step():
    """maxit reached before the tolerance: the step count is maxit and the
    estimate above rtol; restart = 1 (a restart every step): the same steps as
    one rank and an estimate that falls."""
    from paper_2405_04808_gb300 import timeshard as TS
    spec, opts, world, rtol, _ = FGMRES_CASES["vdp_four_ranks_restarted"]
    prob = _problem(spec)
    _, _, res = _fgmres(prob, opts, world, list(range(world)), TS.LocalExchange(world), rtol, 6, maxit=5)
    assert res.iters == 5 and res.est > rtol and len(res.history) == 5
    _, _, r4 = _fgmres(prob, opts, world, list(range(world)), TS.LocalExchange(world), rtol, 1, maxit=12)
    _, _, r1 = _fgmres(prob, opts, 1, [0], TS.LocalExchange(1), rtol, 1, maxit=12)
    assert r4.iters == r1.iters == 12
    assert np.allclose(r4.history, r1.history, rtol=1e-8, atol=0)
    assert r4.history[-1] < r4.history[0]


def test_sharded_fgmres_zero_rhs_and_restart_bounds():
    from paper_2405_04808_gb300 import timeshard as TS
    prob = _problem(dict(kind="vdp", n=16, seed=613))
    prob.b[:] = 0.0
    _, _, res = _fgmres(prob, dict(levels=2, nu_pre=1, nu_post=1), 2, [0, 1], TS.LocalExchange(2), 1e-8, 5)
    assert res.iters == 0 and all(float(v.abs().max()) == 0.0 for v in res.x)
    with pytest.raises(ValueError):
        TS.ShardedFGMRES(None, 512)


@pytest.mark.parametrize("name", sorted(CASES))
def test_sharded_vcycle_in_one_process_equals_unsharded(name):
    from paper_2405_04808_gb300 import timeshard as TS
    spec, opts, world = CASES[name]
    prob = _problem(spec)
    _, part, layouts, y = _cycle(prob, opts, world, list(range(world)), TS.LocalExchange(world))
    got = np.full(prob.size, np.nan)
    for r in range(world):
        j0, j1 = part.blocks(r, 0)
        for j in range(j0, j1):
            for sl in layouts[0].block(j):
                got[sl] = y[r][sl].numpy()
    assert np.array_equal(got, _reference(prob, opts))


def test_partition_ranges():
    from paper_2405_04808_gb300 import timeshard as TS
    for n, levels, world in [(32, 3, 2), (64, 2, 4), (1024, 3, 8), (48, 4, 3)]:
        part = TS.Partition(n, levels, world)
        for lv in range(levels):
            nl = n >> lv
            ranges = [part.blocks(r, lv) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == nl + 1
            assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))   # contiguous, disjoint
            assert all(j1 > j0 for j0, j1 in ranges)
            if lv < levels - 1:
                assert all(j0 % 2 == 0 for j0, _ in ranges)                 # even boundaries to restrict from
    with pytest.raises(ValueError):
        TS.Partition(30, 3, 2)          # n not divisible by 4
    with pytest.raises(ValueError):
        TS.Partition(16, 3, 5)          # more ranks than units of 4 steps


def test_layout_blocks_cover_the_vector_once():
    from paper_2405_04808_gb300 import timeshard as TS
    lay = TS.Layout(6, 3, 2)
    seen = np.zeros(lay.length, dtype=int)
    for j in range(lay.n + 1):
        for sl in lay.block(j):
            seen[sl] += 1
    assert (seen == 1).all()


def test_merged_slices_cover_the_same_entries():
    from paper_2405_04808_gb300 import timeshard as TS
    lay = TS.Layout(16, 3, 2)
    for j0, j1 in [(0, 5), (4, 9), (12, 17), (16, 17), (0, 17)]:
        sl = sum((lay.block(j) for j in range(j0, j1)), [])
        m = TS.merged(sl)
        a, b = np.zeros(lay.length, int), np.zeros(lay.length, int)
        for x in sl:
            a[x] += 1
        for x in m:
            b[x] += 1
        assert (a == b).all() and len(m) <= 5                # one run per type at most
        assert all(x.stop < y.start for x, y in zip(m, m[1:]))
