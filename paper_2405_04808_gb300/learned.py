"""Learned coarse-grid correction: data collection and training driver.

Orchestration only: the plain method's coarse solves are recorded by the
library (mg_record_coarse) during host-driven FGMRES solves, and the network
is trained by the library's own forward, backward and Adam kernels
(mg_net_train).  PyTorch provides the device buffers.
"""
from __future__ import annotations

import numpy as np

from . import pintmg as P
from . import workloads as W


def collect_pairs(problems, settings: dict, max_pairs: int, rtol: float = 1e-8, maxit: int = 2000,
                  restart: int = 400, per_problem: int | None = None):
    """Record (r / rms(r), y / rms(r)) coarse pairs (rms(r) = ||r|| / sqrt(len r)) of the plain method (GMRES + SGS
    coarse solves inside FGMRES) from a list of problems with the same coarse
    shape.  Returns device tensors R, Y of shape (count, 5, T, X) (FP32)."""
    import torch
    R = Y = None
    count = 0
    shape = None
    for prob in problems:
        if count >= max_pairs:
            break
        h = P.mg_setup(prob, device_loops=False, **settings)
        try:
            T, X = P.mg_coarse_shape(h)
            if shape is None:
                shape = (T, X)
                R = torch.empty((max_pairs, 5, T, X), dtype=torch.float32, device="cuda")
                Y = torch.empty_like(R)
            elif shape != (T, X):
                raise ValueError("problems differ in coarse shape")
            want = max_pairs - count if per_problem is None else min(per_problem, max_pairs - count)
            P.mg_record_coarse(h, R[count].data_ptr(), Y[count].data_ptr(), want)
            b = torch.tensor(prob.b, dtype=torch.float64, device="cuda")
            x = torch.zeros_like(b)
            P.fgmres_solve(h, b.data_ptr(), x.data_ptr(), rtol, maxit=maxit, restart=restart)
            torch.cuda.synchronize()
            count += P.mg_recorded_pairs(h)
        finally:
            P.mg_destroy(h)
    return R[:count], Y[:count]


def train(net, R, Y, epochs: int, batch: int = 16, lr: float = 1e-3, seed: int = 0, normalize: bool = True,
          metric=None):
    """Minibatch Adam on (R, Y) with the library's kernels (per-channel
    normalised by default); returns per-epoch losses.  metric: a handle whose
    coarse operator A_c defines the residual-metric loss mean((A_c (net(r) -
    y))^2) (mg_net_set_metric); None: the mean squared error."""
    count, _, T, X = R.shape
    P.mg_net_set_metric(net, metric)
    try:
        return P.mg_net_train(net, R.data_ptr(), Y.data_ptr(), count, T, X, batch, epochs, lr, seed, normalize)
    finally:
        P.mg_net_set_metric(net, None)


def new_net(seed: int, zero_output: bool = False):
    """A network with the seeded initial parameters (workloads.net_init_params)."""
    return P.mg_net_create(W.net_init_params(seed, zero_output).astype(np.float32))
