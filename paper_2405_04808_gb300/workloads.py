"""Seeded synthetic workloads: the raw inputs of an augmented-system solve.

This module is the only code shared by the CUDA path and the CPU oracle.  It
holds no arithmetic of the solver itself (no scaling, no lifting, no
multigrid): it draws a problem instance and evaluates the model ODE's
right-hand side f and its Jacobians at a seeded iterate.  Everything it returns
is in physical (unscaled) coordinates; the solver side forms the scaled blocks
of Sec. 4.1 from it.

Two model problems, shaped like the paper's Sec. 6 workloads:

* van der Pol control (Sec. 6.1): p = 2 states, q = 1 control entering the
  second equation, mu = 1, theta = 0.5, M = I, u(0) = (1, 1) absorbed by the
  shift u <- u + chi of the footnote to Sec. 1.
* viscous Burgers control (Sec. 6.2) with P1 finite elements on nx interior
  nodes of [0, 1] (homogeneous Dirichlet ends), M = (h/6) tridiag(1, 4, 1),
  stiffness K = (1/h) tridiag(-1, 2, -1), a Galerkin convective term C(u) and
  distributed control entering as M z; theta = 1 (backward Euler).

The "SQP iterate" at which the Jacobians are taken is the paper's setting
with unavailable data replaced by seeded draws: a control z_k ~ N(0, s^2) per
step (and per node), the state from the theta-method forward solve (Eq. 8,
Newton per step) and the virtual states equal to the states (v = u, which the
forward solve satisfies).  The right-hand side b ~ N(0, 1) fills all
n (4p + q) entries of the lifted system.

Random numbers: splitmix64 used as a counter-based generator,
``out_i = mix64(key + (i + 1) * 0x9E3779B97F4A7C15)`` with Vigna's mix64
finaliser, ``key = mix64(seed * 65536 + stream)``; uniforms are the top 53
bits; normals come from Box-Muller on consecutive pairs.  Streams: 1 control,
2 right-hand side, 3 Burgers mode numbers, 4 Burgers mode amplitudes, 5 the
coarse-correction network's initial weights.

Matrix formats (the C-ABI's): a "dense" problem stores every p x p or p x q
block row-major; a "tridiag" problem (q == p) stores every p x p tridiagonal
matrix as three length-p rows: band[0][i] = A[i, i-1] (band[0][0] = 0),
band[1][i] = A[i, i], band[2][i] = A[i, i+1] (band[2][p-1] = 0).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

STREAM_CONTROL = 1
STREAM_RHS = 2
STREAM_MODES = 3
STREAM_AMPL = 4
STREAM_NET_INIT = 5
STREAM_COUPLING = 6


def _mix64(z):
    with np.errstate(over="ignore"):
        z = np.asarray(z, dtype=np.uint64)
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def random_u64(seed: int, stream: int, count: int) -> np.ndarray:
    """``count`` splitmix64 outputs of (seed, stream), counter-based."""
    key = _mix64(np.uint64((int(seed) * 65536 + int(stream)) % (1 << 64)))
    with np.errstate(over="ignore"):
        ctr = np.arange(1, count + 1, dtype=np.uint64)
        return _mix64(key + ctr * _GOLDEN)


def uniform(seed: int, stream: int, count: int) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits."""
    return (random_u64(seed, stream, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, stream: int, count: int) -> np.ndarray:
    """Standard normals by Box-Muller on consecutive uniform pairs."""
    m = (count + 1) // 2
    u = uniform(seed, stream, 2 * m)
    r = np.sqrt(-2.0 * np.log1p(-u[0::2]))
    ang = 2.0 * math.pi * u[1::2]
    out = np.empty(2 * m)
    out[0::2] = r * np.cos(ang)
    out[1::2] = r * np.sin(ang)
    return out[:count]


# --------------------------------------------------------------------------
# banded helpers (format conversion only)

def band_to_dense(band: np.ndarray) -> np.ndarray:
    """(3, p) tridiagonal band -> dense (p, p)."""
    p = band.shape[-1]
    a = np.diag(band[1])
    if p > 1:
        a += np.diag(band[0][1:], -1) + np.diag(band[2][:-1], 1)
    return a


def _band_matvec(band: np.ndarray, x: np.ndarray) -> np.ndarray:
    y = band[1] * x
    y[1:] += band[0][1:] * x[:-1]
    y[:-1] += band[2][:-1] * x[1:]
    return y


def _solve_tridiag(band: np.ndarray, r: np.ndarray) -> np.ndarray:
    """Banded LU (LAPACK gbsv via scipy) for the forward solve's Newton steps."""
    from scipy.linalg import solve_banded
    ab = np.zeros((3, band.shape[1]))
    ab[0, 1:] = band[2][:-1]
    ab[1, :] = band[1]
    ab[2, :-1] = band[0][1:]
    return solve_banded((1, 1), ab, r)


# --------------------------------------------------------------------------
# model problems

@dataclasses.dataclass
class VanDerPol:
    """van der Pol control on [0, T] mapped to [0, 1] (Sec. 6.1).

    u1' = T (u2 + [z1]),  u2' = T (mu (1 - u1^2) u2 - u1 + z_last);
    q = 1 puts the single control in the second equation, q = 2 puts one
    control in each (the paper's form).
    """
    mu: float = 1.0
    u_init: tuple = (1.0, 1.0)
    q: int = 1
    T: float = 1.0
    p: int = 2
    kind: str = "dense"

    def f(self, u, z):
        z1 = z[0] if self.q == 2 else 0.0
        return self.T * np.array([u[1] + z1, self.mu * (1.0 - u[0] ** 2) * u[1] - u[0] + z[-1]])

    def dfdu(self, u, z):
        return self.T * np.array([[0.0, 1.0],
                                  [-2.0 * self.mu * u[0] * u[1] - 1.0, self.mu * (1.0 - u[0] ** 2)]])

    def dfdz(self, u, z):
        if self.q == 2:
            return self.T * np.eye(2)
        return self.T * np.array([[0.0], [1.0]])

    def mass(self):
        return np.eye(2)


@dataclasses.dataclass
class BurgersFE:
    """M u' = -nu K u - C(u) + M z with P1 elements on nx interior nodes (Sec. 6.2)."""
    nx: int
    nu: float
    kind: str = "tridiag"

    @property
    def p(self):
        return self.nx

    @property
    def q(self):
        return self.nx

    @property
    def h(self):
        return 1.0 / (self.nx + 1)

    def mass(self):
        h = self.h
        band = np.zeros((3, self.nx))
        band[0][1:] = h / 6.0
        band[1][:] = 4.0 * h / 6.0
        band[2][:-1] = h / 6.0
        return band

    def stiffness(self):
        h = self.h
        band = np.zeros((3, self.nx))
        band[0][1:] = -1.0 / h
        band[1][:] = 2.0 / h
        band[2][:-1] = -1.0 / h
        return band

    @staticmethod
    def _padded(u):
        return np.concatenate(([0.0], u, [0.0]))

    def convection(self, u):
        """C_i(u) = (u_{i+1}^2 + u_i u_{i+1} - u_{i-1} u_i - u_{i-1}^2) / 6, u_0 = u_{nx+1} = 0."""
        w = self._padded(u)
        um, uc, up = w[:-2], w[1:-1], w[2:]
        return (up * up + uc * up - um * uc - um * um) / 6.0

    def f(self, u, z):
        return (-self.nu * _band_matvec(self.stiffness(), u) - self.convection(u)
                + _band_matvec(self.mass(), z))

    def dfdu(self, u, z):
        w = self._padded(u)
        um, uc, up = w[:-2], w[1:-1], w[2:]
        dc = np.zeros((3, self.nx))
        dc[0] = (-2.0 * um - uc) / 6.0
        dc[1] = (up - um) / 6.0
        dc[2] = (uc + 2.0 * up) / 6.0
        dc[0][0] = 0.0
        dc[2][-1] = 0.0
        return -self.nu * self.stiffness() - dc

    def dfdz(self, u, z):
        return self.mass()

    def initial_state(self, seed):
        """Sum of four sine modes, wavenumbers U{1..8}, amplitudes U(-1, 1), max |u0| <= 1."""
        km = 1 + np.floor(8.0 * uniform(seed, STREAM_MODES, 4)).astype(int)
        am = 2.0 * uniform(seed, STREAM_AMPL, 4) - 1.0
        x = self.h * np.arange(1, self.nx + 1)
        u0 = np.zeros(self.nx)
        for k, a in zip(km, am):
            u0 += a * np.sin(math.pi * k * x)
        peak = np.max(np.abs(u0))
        if peak > 1.0:
            u0 /= peak
        return u0


@dataclasses.dataclass
class CoupledCubic:
    """A dense test model (no counterpart in the paper's Sec. 6; it exercises the
    dense block layout): u' = A u - 0.1 u^3 + B z with seeded A = -I + G / (2 sqrt p),
    B = H / sqrt q (G, H standard normal, stream 6), M = I; d_u f = A - 0.3 diag(u^2)
    is dense and d_z f = B is constant, so the control is separable."""
    p: int
    q: int
    seed: int
    kind: str = "dense"

    def __post_init__(self):
        g = normal(self.seed, STREAM_COUPLING, self.p * self.p + self.p * self.q)
        self.A = -np.eye(self.p) + g[:self.p * self.p].reshape(self.p, self.p) / (2.0 * math.sqrt(self.p))
        self.B = g[self.p * self.p:].reshape(self.p, self.q) / math.sqrt(self.q)

    def f(self, u, z):
        return self.A @ u - 0.1 * u ** 3 + self.B @ z

    def dfdu(self, u, z):
        return self.A - 0.3 * np.diag(u ** 2)

    def dfdz(self, u, z):
        return self.B.copy()

    def mass(self):
        return np.eye(self.p)

    def initial_state(self, seed):
        return normal(seed, STREAM_MODES, self.p)


# --------------------------------------------------------------------------
# problem instance

@dataclasses.dataclass
class Problem:
    """Raw inputs of one augmented system, in the C-ABI's formats.

    Index convention (0-based step t = k - 1 of the paper's k = 1..n):
      Ju_cur[t]  = d_u f(u_{t+1}, z_{t+1})   (physical point)
      Ju_prev[t] = d_u f(v_t, z_{t+1})       (v_0 = the initial state)
      Jz_cur[t], Jz_prev[t] likewise for d_z f; when ``jz_const`` the two
      arrays hold one matrix (leading dimension 1) used at every step.
    """
    kind: str
    n: int
    p: int
    q: int
    theta: float
    gamma: float
    M: np.ndarray
    Ju_cur: np.ndarray
    Ju_prev: np.ndarray
    Jz_cur: np.ndarray
    Jz_prev: np.ndarray
    jz_const: bool
    b: np.ndarray                 # type-major right-hand side, length n (4p + q)
    model: object = None
    u_phys: np.ndarray = None     # (n + 1, p) states u_0..u_n, physical
    z_phys: np.ndarray = None     # (n, q) controls z_1..z_n

    @property
    def dt(self):
        return 1.0 / self.n

    @property
    def size(self):
        return self.n * (4 * self.p + self.q)


def _forward_solve(model, u0, z, n, theta, tol=1e-14, maxit=30):
    """theta-method time stepping (Eq. 8) with Newton per step: the seeded iterate."""
    dt = 1.0 / n
    us = [np.array(u0, dtype=np.float64)]
    dense = model.kind == "dense"
    Mm = model.mass()
    for k in range(n):
        up = us[-1]
        zk = z[k]
        fp = model.f(up, zk)
        Mup = Mm @ up if dense else _band_matvec(Mm, up)
        u = up.copy()
        for _ in range(maxit):
            Mu = Mm @ u if dense else _band_matvec(Mm, u)
            res = Mu - Mup - dt * (theta * model.f(u, zk) + (1.0 - theta) * fp)
            J = model.dfdu(u, zk)
            if dense:
                step = np.linalg.solve(Mm - theta * dt * J, -res)
            else:
                step = _solve_tridiag(Mm - theta * dt * J, -res)
            u = u + step
            if np.max(np.abs(step)) <= tol * (1.0 + np.max(np.abs(u))):
                break
        us.append(u)
    return np.array(us)


def make_problem(model, n: int, theta: float, gamma: float, seed: int,
                 z_sigma: float, u_init=None) -> Problem:
    """Draw the iterate and the right-hand side and evaluate the raw Jacobians."""
    p, q = model.p, model.q
    z = z_sigma * normal(seed, STREAM_CONTROL, n * q).reshape(n, q)
    if u_init is None:
        u_init = model.initial_state(seed) if hasattr(model, "initial_state") else np.zeros(p)
    us = _forward_solve(model, u_init, z, n, theta)
    vs = us  # the iterate satisfies v = u
    Ju_cur = np.array([model.dfdu(us[t + 1], z[t]) for t in range(n)])
    Ju_prev = np.array([model.dfdu(vs[t], z[t]) for t in range(n)])
    if isinstance(model, BurgersFE):
        Jz_cur = model.dfdz(None, None)[None]
        Jz_prev = Jz_cur.copy()
        jz_const = True
    else:
        Jz_cur = np.array([model.dfdz(us[t + 1], z[t]) for t in range(n)])
        Jz_prev = np.array([model.dfdz(vs[t], z[t]) for t in range(n)])
        jz_const = False
    b = normal(seed, STREAM_RHS, n * (4 * p + q))
    return Problem(kind=model.kind, n=n, p=p, q=q, theta=theta, gamma=gamma,
                   M=model.mass(), Ju_cur=Ju_cur, Ju_prev=Ju_prev,
                   Jz_cur=Jz_cur, Jz_prev=Jz_prev, jz_const=jz_const, b=b,
                   model=model, u_phys=us, z_phys=z)


# --------------------------------------------------------------------------
# the named workloads

def vdp(n: int = 256, seed: int = 1000, gamma: float = 100.0, mu: float = 1.0) -> Problem:
    """van der Pol control, p = 2, q = 1, theta = 0.5, z ~ N(0, 0.1^2) on [0, 1]."""
    m = VanDerPol(mu=mu)
    return make_problem(m, n=n, theta=0.5, gamma=gamma, seed=seed, z_sigma=0.1,
                        u_init=np.array(m.u_init))


def vdp_paper(n: int = 64, seed: int = 1, gamma: float = 100.0) -> Problem:
    """The paper's van der Pol setting of Sec. 6.1 (mu = 0.1, T = 8, q = 2,
    u(0) = (1, 1), theta = 0.5) at a first-iterate-like point: z = 0 and the
    state from the forward solve."""
    m = VanDerPol(mu=0.1, q=2, T=8.0)
    return make_problem(m, n=n, theta=0.5, gamma=gamma, seed=seed, z_sigma=0.0,
                        u_init=np.array(m.u_init))


def coupled(p: int = 12, q: int = 6, n: int = 64, seed: int = 7000, gamma: float = 100.0) -> Problem:
    """The dense test model CoupledCubic, theta = 0.5, z ~ N(0, 0.1^2) per step and control."""
    return make_problem(CoupledCubic(p=p, q=q, seed=seed), n=n, theta=0.5, gamma=gamma, seed=seed, z_sigma=0.1)


def dense_copy(prob: Problem) -> Problem:
    """The same problem with every block stored dense (a tridiagonal problem in the dense layout)."""
    if prob.kind == "dense":
        return prob
    dense = lambda arr: np.array([band_to_dense(a) for a in arr])
    return dataclasses.replace(prob, kind="dense", M=band_to_dense(prob.M), Ju_cur=dense(prob.Ju_cur),
                               Ju_prev=dense(prob.Ju_prev), Jz_cur=dense(prob.Jz_cur), Jz_prev=dense(prob.Jz_prev))


def burgers(nx: int = 128, n: int = 1024, nu: float = 0.01, seed: int = 2000,
            gamma: float = 100.0, theta: float = 1.0) -> Problem:
    """Viscous Burgers control with P1 elements, z ~ N(0, 0.05^2) per node and step."""
    return make_problem(BurgersFE(nx=nx, nu=nu), n=n, theta=theta, gamma=gamma,
                        seed=seed, z_sigma=0.05)


#: the solver settings that go with each named workload (levels, smoothing,
#: FGMRES restart length; the restart lengths of the first two come from a
#: sweep of the solve time: at restart 250 Burgers nx=128 takes 487 iterations,
#: unrestarted 446 but with longer orthogonalisations; van der Pol converges
#: unrestarted in 382)
WORKLOADS = {
    "vdp_n256": dict(make=lambda seed=1000: vdp(n=256, seed=seed), seed=1000, levels=2, nu_pre=1, nu_post=1,
                     restart=400),
    "burgers_nx128_n1024": dict(make=lambda seed=2000: burgers(nx=128, n=1024, nu=0.01, seed=seed), seed=2000,
                                levels=3, nu_pre=4, nu_post=4, restart=250),
    "burgers_nx128_n8192": dict(make=lambda seed=2500: burgers(nx=128, n=8192, nu=0.01, seed=seed), seed=2500,
                                levels=3, nu_pre=4, nu_post=4, restart=250),
    "burgers_nx512_n8192": dict(make=lambda seed=3000: burgers(nx=512, n=8192, nu=0.005, seed=seed), seed=3000,
                                levels=4, nu_pre=4, nu_post=4, restart=100),
    # the learned coarse correction's workload: training pairs come from seeded
    # runs (seeds 5001, 5002, ...), the timed solve uses seed 5000
    "burgers_nx256_n4096": dict(make=lambda seed=5000: burgers(nx=256, n=4096, nu=0.01, seed=seed), seed=5000,
                                levels=4, nu_pre=4, nu_post=4, restart=400),
}


def batch_mix(seed: int = 4000, count: int = 32):
    """Uneven systems for batched solves: van der Pol with nt 256 / 512 and
    Burgers with nx 32 / 64 and nt 256 / 512, distinct seeded iterates; each
    with its own solver settings (3 levels; 1/1 sweeps for van der Pol, 4/4
    for Burgers).  Returns [(Problem, settings)]."""
    out = []
    for k in range(count):
        sd = seed + k
        if k % 2 == 0:
            nt = 256 if (k // 2) % 2 == 0 else 512
            out.append((vdp(n=nt, seed=sd), dict(levels=3, nu_pre=1, nu_post=1)))
        else:
            nx = 32 if (k // 2) % 2 == 0 else 64
            nt = 256 if (k // 4) % 2 == 0 else 512
            out.append((burgers(nx=nx, n=nt, seed=sd), dict(levels=3, nu_pre=4, nu_post=4)))
    return out


def _batch_member(k: int, seed: int):
    vdp_nt = (512, 1024, 2048, 4096, 8192, 16384)
    bg = [(nx, nt) for nt in (512, 1024, 2048, 4096) for nx in (64, 128, 256)]
    sd = seed + k
    if k % 2 == 0:
        return vdp(n=vdp_nt[(k // 2) % len(vdp_nt)], seed=sd), dict(levels=4, nu_pre=1, nu_post=1)
    nx, nt = bg[(k // 2) % len(bg)]
    return burgers(nx=nx, n=nt, seed=sd), dict(levels=4, nu_pre=4, nu_post=4)


def _make_named(name: str, seed: int):
    return WORKLOADS[name]["make"](seed=seed)


def make_many(name: str, seeds, workers: int = 1):
    """The named workload at several seeds (a spawned process pool when workers > 1)."""
    seeds = list(seeds)
    if workers <= 1:
        return [_make_named(name, sd) for sd in seeds]
    import concurrent.futures as cf
    import multiprocessing as mp
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_make_named, [name] * len(seeds), seeds))


def batch_uneven(seed: int = 6000, count: int = 64, workers: int = 1):
    """The batched workload: `count` systems at distinct seeded iterates, half
    van der Pol with nt cycling through 512 ... 16384, half Burgers with
    (nx, nt) cycling through {64, 128, 256} x {512, 1024, 2048, 4096}; every
    system with 4 levels (1/1 sweeps for van der Pol, 4/4 for Burgers).
    workers > 1 builds the members in a spawned process pool (the forward
    solves are per-step Python loops).  Returns [(Problem, settings)]."""
    if workers <= 1:
        return [_batch_member(k, seed) for k in range(count)]
    import concurrent.futures as cf
    import multiprocessing as mp
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        return list(ex.map(_batch_member, range(count), [seed] * count))


# --------------------------------------------------------------------------
# the learned coarse correction's network: initial parameters

NET_CHANNELS = (5, 32, 32, 32, 5)
NET_KT, NET_KX = 3, 7


def net_init_params(seed: int, zero_output: bool = False) -> np.ndarray:
    """Initial parameters of the coarse-correction network, flat in the C-ABI's
    layout (per layer: weights [out][in][time tap][space tap], then biases):
    weights uniform in +-sqrt(6 / fan_in) (He et al. 2015), biases zero.
    zero_output: the last layer's weights zero too, so the untrained network
    proposes e = 0 (residual r; used with the residual-metric loss, where a
    random output's error is amplified by the coarse operator)."""
    sizes = [(co * ci * NET_KT * NET_KX, co, ci * NET_KT * NET_KX)
             for ci, co in zip(NET_CHANNELS[:-1], NET_CHANNELS[1:])]
    u = uniform(seed, STREAM_NET_INIT, sum(nw for nw, _, _ in sizes))
    out, k = [], 0
    for layer, (nw, nb, fan_in) in enumerate(sizes):
        lim = 0.0 if (zero_output and layer == len(sizes) - 1) else math.sqrt(6.0 / fan_in)
        out += [(2.0 * u[k:k + nw] - 1.0) * lim, np.zeros(nb)]
        k += nw
    return np.concatenate(out)
