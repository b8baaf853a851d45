"""An engine for paper_2405_04808_gb300.timeshard that runs one rank's cycle
steps with the CPU oracle (test infrastructure): each step is the oracle's
whole-level operation (block-Jacobi sweep, residual, sparse restriction or
interpolation) on the rank's full-length vectors, of which only the rank's
blocks are kept.  The oracle's operations couple neighbouring blocks only, so
the entries a rank keeps depend on its blocks and the exchanged boundary
values alone.  The Krylov vector work of the sharded FGMRES (operator
product, dot products, updates) runs on the rank's entries with numpy."""
import numpy as np
import torch

from oracle import augmented as O


class OracleEngine:
    def __init__(self, hier: O.Hierarchy, layouts, part, rank):
        self.hier, self.layouts, self.part, self.rank = hier, layouts, part, rank

    def _keep(self, level, j0, j1, src_type_major, dst):
        lay = self.layouts[level]
        for j in range(j0, j1):
            for sl in lay.block(j):
                dst[sl] = torch.from_numpy(src_type_major[sl])

    def _tm(self, level, x):
        return self.hier.levels[level].to_time_major(x.numpy())

    def _ty(self, level, y):
        return self.hier.levels[level].to_type_major(y)

    def sweep(self, level, j0, j1, r, yold, y):
        lev = self.hier.levels[level]
        y0 = np.zeros(lev.size) if yold is None else self._tm(level, yold)
        ynew = O.jacobi_sweep(lev, self._tm(level, r), y0, self.hier.opts.omega)
        self._keep(level, j0, j1, self._ty(level, ynew), y)

    def residual(self, level, j0, j1, y, b, r):
        lev = self.hier.levels[level]
        res = self._tm(level, b) - lev.At @ self._tm(level, y)
        self._keep(level, j0, j1, self._ty(level, res), r)

    def restrict(self, level, j0, j1, r, rc):
        rcoarse = self.hier.R[level] @ self._tm(level, r)
        self._keep(level + 1, j0 // 2, (j1 + 1) // 2, self._ty(level + 1, rcoarse), rc)

    def prolong(self, level, j0, j1, ec, y):
        ynew = self._tm(level, y) + self.hier.P[level] @ self._tm(level + 1, ec)
        self._keep(level, j0, j1, self._ty(level, ynew), y)

    def coarse_solve(self, rc, yc):
        last = len(self.hier.levels) - 1
        yc[:] = torch.from_numpy(self._ty(last, self.hier.coarse_solve(last, self._tm(last, rc))))

    # -- the sharded FGMRES's vector work on the rank's entries --------------------
    def _owned(self, level, j0, j1):
        lay = self.layouts[level]
        return np.concatenate([np.arange(sl.start, sl.stop) for j in range(j0, j1) for sl in lay.block(j)])

    def apply(self, level, j0, j1, y, out):
        lev = self.hier.levels[level]
        self._keep(level, j0, j1, self._ty(level, lev.At @ self._tm(level, y)), out)

    def dots(self, level, j0, j1, V, k, w):
        idx = self._owned(level, j0, j1)
        return torch.from_numpy(V[:k].numpy()[:, idx] @ w.numpy()[idx])

    def axpy(self, level, j0, j1, V, k, c, sign, w):
        idx = self._owned(level, j0, j1)
        wn = w.numpy()
        wn[idx] += sign * (np.asarray(c[:k]) @ V[:k].numpy()[:, idx])

    def scale(self, level, j0, j1, x, a, y):
        idx = self._owned(level, j0, j1)
        y.numpy()[idx] = a * x.numpy()[idx]
