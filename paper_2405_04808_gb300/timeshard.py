"""The V-cycle sharded across processes by time (one GPU per process).

Each process owns a contiguous range of time blocks on every level of the
hierarchy and runs the cycle's steps on its range with the library's
time-range entry points (``mg_range_sweep``, ``mg_range_residual``,
``mg_range_restrict``, ``mg_range_prolong``); only the couplings at the range
ends cross processes.  Time block j of a level holds u_j, z_j, lambda_j and
v_{j-1}, mu_{j-1} (the blocks of Fig. 5).  Per level and cycle:

* before every sweep after the first and before the residual: u_{j1-1} goes to
  the right neighbour, mu_{j0-1} to the left one (2p values per boundary);
* after the residual: the last two blocks of each range's residual go to the
  right neighbour (the restriction of Sec. 5.3.1 reads fine steps 2K-1..2K+1);
* after the coarser level's correction: the first coarse block of each range
  goes to the left neighbour (linear interpolation reads coarse step K+1);
* the coarsest level is gathered to every process and solved there (GMRES
  with SGS is serial in time, Sec. 5.3.4), each process keeping the whole
  coarse correction.

Range boundaries are multiples of 2^(levels-1) fine blocks, so every level's
boundaries are even.  Every exchanged entry is the value a single process would
have read, and every block is computed by the same kernel as in the unsharded
cycle, so the sharded cycle gives the same bits.

``ShardedFGMRES`` is the outer solver of Sec. 6 around that cycle: FGMRES
whose vectors are sharded the same way.  Each Arnoldi step exchanges the
couplings of z_j before the operator product and sums partial dot products
over the processes twice (the two classical Gram-Schmidt passes, the second
with the norm); the small Hessenberg least-squares problem is replicated on every
process, which all hold the same summed values and so take the same decisions.

Two exchangers: ``DistExchange`` moves the boundary slices between processes
with torch.distributed point-to-point operations (NCCL between GPUs, gloo on
CPU); ``LocalExchange`` holds all ranks in one process and copies between them
(the ranks' kernels still run one after another, none waits on another).  An
engine runs one rank's steps: ``LibraryEngine`` calls the library; any object
with the same methods can stand in.
"""
from __future__ import annotations

import dataclasses


class Partition:
    """Fine time blocks 0..n split into `world` contiguous ranges whose interior
    boundaries are multiples of 2^(levels - 1); level l's ranges are the fine
    ones shifted right by l (the last range always ends at n_l + 1)."""

    def __init__(self, n: int, levels: int, world: int):
        unit = 1 << (levels - 1)
        if n % unit:
            raise ValueError("n must be divisible by 2^(levels - 1)")
        units = n // unit
        if world < 1 or world > units:
            raise ValueError(f"cannot split {units} units of {unit} steps over {world} ranks")
        self.n, self.levels, self.world = n, levels, world
        self.cuts = [(r * units // world) * unit for r in range(world)] + [n + 1]

    def blocks(self, rank: int, level: int):
        """(j0, j1): the blocks [j0, j1) of level `level` owned by `rank`."""
        j0 = self.cuts[rank] >> level
        j1 = (self.cuts[rank + 1] >> level) if rank + 1 < self.world else (self.n >> level) + 1
        return j0, j1


def merged(slices):
    """the same entries as a list of slices, adjacent ones joined (in order of start)"""
    out = []
    for sl in sorted(slices, key=lambda t: t.start):
        if out and out[-1].stop == sl.start:
            out[-1] = slice(out[-1].start, sl.stop)
        else:
            out.append(sl)
    return out


@dataclasses.dataclass
class Layout:
    """Offsets of one level's type-major vector (u, v, z, lambda, mu)."""
    n: int
    p: int
    q: int

    def step(self, kind: str, t: int):
        """slice of the entries of type `kind` at step t"""
        n, p, q = self.n, self.p, self.q
        start = {"u": t * p, "v": n * p + t * p, "z": 2 * n * p + t * q, "l": 2 * n * p + n * q + t * p,
                 "m": 3 * n * p + n * q + t * p}[kind]
        return slice(start, start + (q if kind == "z" else p))

    def block(self, j: int):
        """slices of time block j's entries"""
        out = []
        if j < self.n:
            out += [self.step(k, j) for k in ("u", "z", "l")]
        if j >= 1:
            out += [self.step(k, j - 1) for k in ("v", "m")]
        return out

    @property
    def length(self):
        return self.n * (4 * self.p + self.q)


class LibraryEngine:
    """One rank's cycle steps through the library's time-range entry points on
    full level-length torch vectors on the handle's GPU."""

    def __init__(self, P, h, stream=0):
        self.P, self.h, self.stream = P, h, stream

    def sweep(self, level, j0, j1, r, yold, y):
        self.P.mg_range_sweep(self.h, level, j0, j1, r.data_ptr(), yold.data_ptr() if yold is not None else 0,
                              y.data_ptr(), self.stream)

    def residual(self, level, j0, j1, y, b, r):
        self.P.mg_range_residual(self.h, level, j0, j1, y.data_ptr(), b.data_ptr(), r.data_ptr(), self.stream)

    def restrict(self, level, j0, j1, r, rc):
        self.P.mg_range_restrict(self.h, level, j0, j1, r.data_ptr(), rc.data_ptr(), self.stream)

    def prolong(self, level, j0, j1, ec, y):
        self.P.mg_range_prolong(self.h, level, j0, j1, ec.data_ptr(), y.data_ptr(), self.stream)

    def coarse_solve(self, rc, yc):
        self.P.mg_coarse_solve(self.h, rc.data_ptr(), yc.data_ptr(), self.stream)

    # -- the Krylov vector work on the rank's entries (level 0 of FGMRES) ------------
    def apply(self, level, j0, j1, y, out):
        """out = A~ y on the rows of blocks [j0, j1)"""
        self.P.mg_range_residual(self.h, level, j0, j1, y.data_ptr(), 0, out.data_ptr(), self.stream)

    def dots(self, level, j0, j1, V, k, w):
        """the rank's shares V_i . w, i < k (V: rows of a 2-D tensor), as a device tensor"""
        import torch
        out = torch.empty(k, dtype=torch.float64, device=w.device)
        self.P.mg_range_dots(self.h, level, j0, j1, V.data_ptr(), V.stride(0), k, w.data_ptr(), out.data_ptr(),
                             self.stream)
        return out

    def axpy(self, level, j0, j1, V, k, c, sign, w):
        """w += sign sum_i c[i] V_i on the rank's entries (c: k host values)"""
        import torch
        cd = torch.tensor(c[:k], dtype=torch.float64, device=w.device)
        self.P.mg_range_axpy(self.h, level, j0, j1, V.data_ptr(), V.stride(0), k, cd.data_ptr(), sign, w.data_ptr(),
                             self.stream)

    def scale(self, level, j0, j1, x, a, y):
        """y = a x on the rank's entries (a: a host value)"""
        import torch
        ad = torch.tensor([a], dtype=torch.float64, device=x.device)
        self.P.mg_range_scale(self.h, level, j0, j1, x.data_ptr(), ad.data_ptr(), y.data_ptr(), self.stream)


class LocalExchange:
    """All ranks in one process: boundary slices are copied between their vectors."""

    def __init__(self, world):
        self.world = world

    def swap(self, vecs, sends, recvs=None):
        """sends: per source rank a list of (destination rank, slices); the
        destination's entries at those slices take the source's values (the
        receive list, which a process-per-rank exchange needs, is implied)."""
        for src, items in enumerate(sends):
            for dst, sls in items:
                for sl in sls:
                    vecs[dst][sl] = vecs[src][sl]

    def allreduce(self, vals):
        """every held rank's values become the sum over the ranks (in rank order)"""
        total = vals[0].clone()
        for v in vals[1:]:
            total += v
        for v in vals:
            v.copy_(total)

    def gather(self, vecs, owned):
        """every rank's vector gets every rank's owned slices"""
        for src in range(self.world):
            for dst in range(self.world):
                if dst != src:
                    for sl in owned[src]:
                        vecs[dst][sl] = vecs[src][sl]


class DistExchange:
    """One rank per process: boundary slices move by torch.distributed
    point-to-point operations (sends and receives posted together)."""

    def __init__(self, dist, rank, world):
        self.dist, self.rank, self.world = dist, rank, world

    def swap(self, vecs, sends, recvs):
        """sends: this rank's (destination, slices) list; recvs: its (source,
        slices) list; the received values land at those slices."""
        import torch
        (vec,) = vecs
        ops, landing = [], []
        for dst, sls in sends[0]:
            ops.append(self.dist.P2POp(self.dist.isend, torch.cat([vec[sl] for sl in sls]).contiguous(), dst))
        for src, sls in recvs:
            buf = torch.empty(sum(sl.stop - sl.start for sl in sls), dtype=vec.dtype, device=vec.device)
            ops.append(self.dist.P2POp(self.dist.irecv, buf, src))
            landing.append((buf, sls))
        if ops:
            for req in self.dist.batch_isend_irecv(ops):
                req.wait()
        for buf, sls in landing:
            off = 0
            for sl in sls:
                k = sl.stop - sl.start
                vec[sl] = buf[off:off + k]
                off += k

    def allreduce(self, vals):
        """the values become the sum over the processes (the same on every one)"""
        self.dist.all_reduce(vals[0])

    def gather(self, vecs, owned):
        import torch
        (vec,) = vecs
        sizes = [sum(sl.stop - sl.start for sl in owned[r]) for r in range(self.world)]
        top = max(sizes)
        mine = torch.zeros(top, dtype=vec.dtype, device=vec.device)   # equal sizes for every backend
        mine[:sizes[self.rank]] = torch.cat([vec[sl] for sl in owned[self.rank]])
        bufs = [torch.empty(top, dtype=vec.dtype, device=vec.device) for _ in sizes]
        self.dist.all_gather(bufs, mine)
        for r in range(self.world):
            if r != self.rank:
                off = 0
                for sl in owned[r]:
                    k = sl.stop - sl.start
                    vec[sl] = bufs[r][off:off + k]
                    off += k


class ShardedVCycle:
    """The V-cycle of Alg. 1 (generalised to `levels` levels) over a time
    partition.  ranks: the ranks this process holds (all of them with a
    LocalExchange, its own one with a DistExchange); engines: one per held rank.
    The cycle's smoothing counts are nu_pre / nu_post (the handle's)."""

    def __init__(self, part: Partition, layouts, engines, ranks, exchange, nu_pre, nu_post, zeros):
        self.part, self.layouts, self.engines, self.ranks = part, layouts, engines, list(ranks)
        self.ex, self.nu_pre, self.nu_post, self.zeros = exchange, nu_pre, nu_post, zeros

    # -- who sends what -------------------------------------------------------------
    def _coupling_sends(self, level, held):
        """u_{j1-1} to the right neighbour, mu_{j0-1} to the left one"""
        lay = self.layouts[level]
        out = []
        for r in held:
            j0, j1 = self.part.blocks(r, level)
            items = []
            if r + 1 < self.part.world and j1 - 1 < lay.n:
                items.append((r + 1, [lay.step("u", j1 - 1)]))
            if r > 0 and j0 >= 1:
                items.append((r - 1, [lay.step("m", j0 - 1)]))
            out.append(items)
        return out

    def _coupling_recvs(self, level, r):
        lay = self.layouts[level]
        j0, j1 = self.part.blocks(r, level)
        items = []
        if r > 0:
            items.append((r - 1, [lay.step("u", j0 - 1)]))
        if r + 1 < self.part.world:
            items.append((r + 1, [lay.step("m", j1 - 1)]))
        return items

    def _residual_sends(self, level, held):
        """the last two blocks of each range to the right neighbour"""
        lay = self.layouts[level]
        out = []
        for r in held:
            j0, j1 = self.part.blocks(r, level)
            items = []
            if r + 1 < self.part.world:
                items.append((r + 1, merged(lay.block(j1 - 2) + lay.block(j1 - 1))))
            out.append(items)
        return out

    def _residual_recvs(self, level, r):
        lay = self.layouts[level]
        j0, _ = self.part.blocks(r, level)
        return [(r - 1, merged(lay.block(j0 - 2) + lay.block(j0 - 1)))] if r > 0 else []

    def _coarse_sends(self, level, held):
        """the first block of each coarse range to the left neighbour"""
        lay = self.layouts[level]
        out = []
        for r in held:
            j0, _ = self.part.blocks(r, level)
            out.append([(r - 1, lay.block(j0))] if r > 0 else [])
        return out

    def _coarse_recvs(self, level, r):
        lay = self.layouts[level]
        _, j1 = self.part.blocks(r, level)
        return [(r + 1, lay.block(j1))] if r + 1 < self.part.world else []

    def _exchange(self, vecs, sends, recvs_of):
        self.ex.swap(vecs, sends, recvs_of(self.ranks[0]) if len(self.ranks) == 1 else None)

    # -- the cycle ------------------------------------------------------------------
    def vcycle(self, level, b):
        """b: per held rank the level's right-hand side (valid on its blocks);
        returns per held rank the cycle's output (valid on its blocks)."""
        last = self.part.levels - 1
        lay = self.layouts[level]
        if level == last:
            owned = [merged(sum((lay.block(j) for j in range(*self.part.blocks(r, level))), []))
                     for r in range(self.part.world)]
            self.ex.gather(b, owned)
            y = [self.zeros(lay.length) for _ in self.ranks]
            for k, e in enumerate(self.engines):
                e.coarse_solve(b[k], y[k])
            return y
        rng = [self.part.blocks(r, level) for r in self.ranks]
        y = [self.zeros(lay.length) for _ in self.ranks]
        t = [self.zeros(lay.length) for _ in self.ranks]
        couple = (self._coupling_sends(level, self.ranks), lambda r: self._coupling_recvs(level, r))
        for k in range(self.nu_pre):
            if k:
                self._exchange(y, *couple)
            for i, e in enumerate(self.engines):
                e.sweep(level, *rng[i], b[i], y[i] if k else None, t[i])
            y, t = t, y
        self._exchange(y, *couple)
        res = t
        for i, e in enumerate(self.engines):
            e.residual(level, *rng[i], y[i], b[i], res[i])
        self._exchange(res, self._residual_sends(level, self.ranks), lambda r: self._residual_recvs(level, r))
        clay = self.layouts[level + 1]
        bc = [self.zeros(clay.length) for _ in self.ranks]
        for i, e in enumerate(self.engines):
            e.restrict(level, *rng[i], res[i], bc[i])
        ec = self.vcycle(level + 1, bc)
        if level + 1 < last:
            self._exchange(ec, self._coarse_sends(level + 1, self.ranks), lambda r: self._coarse_recvs(level + 1, r))
        for i, e in enumerate(self.engines):
            e.prolong(level, *rng[i], ec[i], y[i])
        t = [self.zeros(lay.length) for _ in self.ranks]
        for k in range(self.nu_post):
            self._exchange(y, *couple)
            for i, e in enumerate(self.engines):
                e.sweep(level, *rng[i], b[i], y[i], t[i])
            y, t = t, y
        return y


@dataclasses.dataclass
class ShardedResult:
    x: list          # per held rank the solution (valid on its level-0 blocks)
    iters: int
    est: float       # |g_{k+1}| / ||b||, the last residual estimate
    history: list


class ShardedFGMRES:
    """Restarted flexible GMRES (x0 = 0) preconditioned by a ShardedVCycle, on
    vectors sharded like the cycle's level 0 (Sec. 6's outer solver).

    Per Arnoldi step j: z_j = M(v_j) by the sharded cycle; its couplings
    u_{j1-1} / mu_{j0-1} cross the range ends; w = A~ z_j on the rank's rows;
    classical Gram-Schmidt twice (h = V^T w summed over the processes, w -= V h,
    twice), two sums over the processes per step: the second also carries
    |w|^2 before its update, and |w - V h2|^2 = |w|^2 - |h2|^2 for orthonormal
    V (a third sum takes the norm itself when that drops below half of |w|^2);
    the Hessenberg column by Givens rotations, replicated; v_{j+1} = w / h_{j+1,j}.  Stops when the estimate
    |g_{j+1}| <= rtol ||b||, at a breakdown (h_{j+1,j} = 0) or after maxit
    steps; restarts every `restart` steps from the true residual.  The
    engines' apply / dots / axpy / scale run the vector work; the exchange's
    allreduce sums the partial dot products."""

    def __init__(self, cycle: ShardedVCycle, restart: int):
        if restart < 1 or restart > 511:
            raise ValueError("restart must be in [1, 511]")
        self.cyc, self.m = cycle, restart

    def _sum(self, shares):
        """shares: per held rank a tensor of partial sums; their sum on the host"""
        self.cyc.ex.allreduce(shares)
        return shares[0].cpu().numpy().astype(float)

    def _couple(self, vecs):
        cyc = self.cyc
        cyc._exchange(vecs, cyc._coupling_sends(0, cyc.ranks), lambda r: cyc._coupling_recvs(0, r))

    def solve(self, b, rtol: float, maxit: int) -> ShardedResult:
        import math

        import numpy as np
        cyc = self.cyc
        E, lay = cyc.engines, cyc.layouts[0]
        rng = [cyc.part.blocks(r, 0) for r in cyc.ranks]
        held = range(len(cyc.ranks))
        zeros = cyc.zeros
        x = [zeros(lay.length) for _ in held]
        bnorm = math.sqrt(self._sum([E[i].dots(0, *rng[i], b[i].view(1, -1), 1, b[i]) for i in held])[0])
        if bnorm == 0.0:
            return ShardedResult(x, 0, 0.0, [])
        m = self.m
        V = [zeros((m + 1) * lay.length).view(m + 1, lay.length) for _ in held]
        Z = [zeros(m * lay.length).view(m, lay.length) for _ in held]
        total, est, history, start = 0, 1.0, [], True
        while total < maxit:
            if start:  # x0 = 0: the residual is b
                for i in held:
                    V[i][0].copy_(b[i])
            else:
                self._couple(x)
                for i in held:
                    E[i].residual(0, *rng[i], x[i], b[i], V[i][0])
            start = False
            beta = math.sqrt(self._sum([E[i].dots(0, *rng[i], V[i][0:1], 1, V[i][0]) for i in held])[0])
            if beta == 0.0:
                est = 0.0
                break
            for i in held:
                E[i].scale(0, *rng[i], V[i][0], 1.0 / beta, V[i][0])
            mm = min(m, maxit - total)
            H = np.zeros((mm + 1, mm))
            cs, sn, g = np.zeros(mm), np.zeros(mm), np.zeros(mm + 1)
            g[0] = beta
            k, done = 0, False
            for j in range(mm):
                z = cyc.vcycle(0, [V[i][j] for i in held])
                for i in held:
                    Z[i][j].copy_(z[i])
                zj = [Z[i][j] for i in held]
                self._couple(zj)
                w = [V[i][j + 1] for i in held]
                for i in held:
                    E[i].apply(0, *rng[i], zj[i], w[i])
                # classical Gram-Schmidt twice; the second sum also carries |w|^2 (w is row j + 1 of V)
                h = self._sum([E[i].dots(0, *rng[i], V[i], j + 1, w[i]) for i in held])
                for i in held:
                    E[i].axpy(0, *rng[i], V[i], j + 1, h, -1.0, w[i])
                d = self._sum([E[i].dots(0, *rng[i], V[i], j + 2, w[i]) for i in held])
                h2, w2 = d[:j + 1], d[j + 1]
                for i in held:
                    E[i].axpy(0, *rng[i], V[i], j + 1, h2, -1.0, w[i])
                h = h + h2
                hn2 = w2 - float(h2 @ h2)  # |w - V h2|^2 with V orthonormal
                if not hn2 > 0.5 * w2:  # the second pass removed much of w: take the norm itself
                    hn2 = self._sum([E[i].dots(0, *rng[i], V[i][j + 1:j + 2], 1, w[i]) for i in held])[0]
                hn = math.sqrt(max(hn2, 0.0))
                H[:j + 1, j], H[j + 1, j] = h, hn
                for t in range(j):  # earlier rotations
                    a, c = H[t, j], H[t + 1, j]
                    H[t, j], H[t + 1, j] = cs[t] * a + sn[t] * c, -sn[t] * a + cs[t] * c
                a, c = H[j, j], H[j + 1, j]
                d = math.hypot(a, c)
                cs[j], sn[j] = (1.0, 0.0) if d == 0.0 else (a / d, c / d)
                H[j, j], H[j + 1, j] = cs[j] * a + sn[j] * c, 0.0
                g[j + 1], g[j] = -sn[j] * g[j], cs[j] * g[j]
                k, total = j + 1, total + 1
                est = abs(g[j + 1]) / bnorm
                history.append(est)
                if hn != 0.0:
                    for i in held:
                        E[i].scale(0, *rng[i], w[i], 1.0 / hn, w[i])
                if hn == 0.0 or est <= rtol:
                    done = True
                    break
            y = np.zeros(k)
            for t in range(k - 1, -1, -1):
                y[t] = (g[t] - H[t, t + 1:k] @ y[t + 1:k]) / H[t, t]
            for i in held:
                E[i].axpy(0, *rng[i], Z[i], k, y, 1.0, x[i])
            if done or total >= maxit:
                break
        return ShardedResult(x, total, est, history)
