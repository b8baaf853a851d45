"""The V-cycle sharded by time across two gloo processes (CPU), each rank
running its blocks with the oracle and exchanging the range-end couplings,
residual blocks and coarse corrections by torch.distributed: the same bits as
the unsharded cycle.  Also the partition's invariants and the same cycle with
all ranks in one process."""
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
