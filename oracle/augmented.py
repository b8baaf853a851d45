"""CPU oracle: a plain, slow, FP64 restatement of the paper's method.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package;
only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline arm of
``bench.py`` may.  It shares no code with the CUDA path: the only common
module is the seeded input generator (``paper_2405_04808_gb300.workloads``),
which contains none of the method's arithmetic.

Paper: Vuchkov, Cyr, Javeed, Ridzal, "A Parallel-in-Time Multigrid
Preconditioner for Optimal Control" (arXiv 2405.04808).  Every function cites
the passage it follows.  The oracle works with assembled sparse matrices and
library primitives (scipy.sparse products, SuperLU factorisations), in the
order the paper states, with no blocking or fusion of its own:

* scaled Jacobian blocks N_k, V_k, Z~_k            Eq. (blocks-aj), Sec. 5.1
* the lifted augmented system in type-major order   Fig. 4, Eq. (augsys-aj)
* the time-major permutation A~ = Q A Q^T           Sec. 5.2, Fig. 5
* interpolation / restriction in time               Sec. 5.3.1
* block-Jacobi smoother                             Eq. (jacobi-aj)
* symmetric block Gauss-Seidel                      Sec. 5.3.4
* right-preconditioned GMRES and flexible GMRES     Sec. 5.3.4, Sec. 6 (Saad 1993)
* two-level cycle generalised to a V-cycle          Alg. 1, Sec. 6 (coarsening 2)

Readings taken where the paper is silent:
* coarse operators are rediscretised at 2 dt with linearisation points taken
  by the injection rule (fine step 2K-1 of the paper's 1-based count);
* linear interpolation at the last coarse step extrapolates the last coarse
  value (``end_rule=0``) or uses a zero neighbour (``end_rule=1``);
* transfers act on the scaled vectors literally, with no sqrt(2) factors;
* the residual is restricted by the variable formulas of Sec. 5.3.1
  (``restrict="inject"``) or by the transpose of the interpolation
  (``restrict="transpose"``); with the transpose and a weighted sweep
  (omega = 2/3) the cycle shows the logarithmic iteration growth of Tables 3
  and 4, with the undamped sweep neither choice does (the sweep's spectrum is
  symmetric about 0, so modes alternating in time are never damped);
* each pre-smoothing starts from y = 0; x0 = 0 for every Krylov solve;
* modified Gram-Schmidt in both Krylov methods.

Parity is pinned by tests/test_oracle_*.py; no function here is "parity
unpinned".
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


# --------------------------------------------------------------------------
# Raw data of one level and its coarsening

@dataclasses.dataclass
class RawLevel:
    """Physical Jacobians of one time grid (0-based step t = paper's k - 1)."""
    kind: str
    n: int
    p: int
    q: int
    dt: float
    theta: float
    gamma: float
    M: np.ndarray
    Ju_cur: np.ndarray
    Ju_prev: np.ndarray
    Jz_cur: np.ndarray
    Jz_prev: np.ndarray
    jz_const: bool

    def jz(self, which: str, t: int) -> np.ndarray:
        arr = self.Jz_cur if which == "cur" else self.Jz_prev
        return arr[0] if self.jz_const else arr[t]


def raw_from_problem(prob) -> RawLevel:
    return RawLevel(kind=prob.kind, n=prob.n, p=prob.p, q=prob.q, dt=1.0 / prob.n,
                    theta=prob.theta, gamma=prob.gamma, M=prob.M,
                    Ju_cur=prob.Ju_cur, Ju_prev=prob.Ju_prev,
                    Jz_cur=prob.Jz_cur, Jz_prev=prob.Jz_prev, jz_const=prob.jz_const)


def coarsen_raw(raw: RawLevel) -> RawLevel:
    """Rediscretise at 2 dt (geometric multigrid, Sec. 5.3; A~^{2dt} in Alg. 1).

    The coarse step K (paper's 1-based K) lives at the fine point 2K - 1, the
    point that injection (Sec. 5.3.1) keeps.  In 0-based indices: the coarse
    current-point Jacobians are the fine ones at 2K, and the coarse
    previous-point Jacobians (taken at v_{K-1}^c = v_{2K-1}^f, 0-based) are the
    fine ones at 2K - 1; coarse step 0 keeps fine step 0 (v_0 is the initial
    state on every grid).
    """
    n = raw.n
    if n % 2:
        raise ValueError("n must be even to coarsen")
    nc = n // 2
    cur = np.arange(nc) * 2
    prev = np.maximum(np.arange(nc) * 2 - 1, 0)
    return RawLevel(kind=raw.kind, n=nc, p=raw.p, q=raw.q, dt=2.0 * raw.dt,
                    theta=raw.theta, gamma=raw.gamma, M=raw.M,
                    Ju_cur=raw.Ju_cur[cur], Ju_prev=raw.Ju_prev[prev],
                    Jz_cur=raw.Jz_cur if raw.jz_const else raw.Jz_cur[cur],
                    Jz_prev=raw.Jz_prev if raw.jz_const else raw.Jz_prev[prev],
                    jz_const=raw.jz_const)


# --------------------------------------------------------------------------
# Scaled blocks (Eq. blocks-aj and Sec. 5.1)

def _as_sparse(kind: str, mat: np.ndarray) -> sp.csr_matrix:
    """A p x p (or p x q) block in the ABI's storage -> scipy sparse."""
    if kind == "tridiag":
        p = mat.shape[-1]
        return sp.diags([mat[0][1:], mat[1], mat[2][:-1]], [-1, 0, 1], shape=(p, p), format="csr")
    return sp.csr_matrix(mat)


def round_bf16(x) -> np.ndarray:
    """Values rounded to FP32 (to nearest) and then to BF16 (to nearest, ties to
    even), returned as FP64.  BF16 keeps the sign, the 8 exponent bits and the
    top 7 stored mantissa bits of the FP32 pattern: rounding adds 0x7FFF plus
    the lowest kept bit to the pattern and clears the low 16 bits.  This is the
    storage the library's MG_PRECISION_BF16_BANDS mode gives the N, V, Z~
    bands of its smoothing levels (finite values only)."""
    f = np.ascontiguousarray(np.asarray(x, dtype=np.float64).astype(np.float32))
    bits = f.view(np.uint32).astype(np.uint64)
    bits = (bits + np.uint64(0x7FFF) + ((bits >> np.uint64(16)) & np.uint64(1))) & np.uint64(0xFFFF0000)
    return bits.astype(np.uint32).view(np.float32).astype(np.float64)


def scaled_blocks(raw: RawLevel):
    """N_k, V_k and Z~_k of Eq. (blocks-aj) with u_{k-1} replaced by v_{k-1} (Sec. 5.1).

    N_k  = dt^-1 [ M - theta dt d_u f(u_k) ]
    V_k  = dt^-1 [-M - (1 - theta) dt d_u f(v_{k-1}) ]
    Z~_k = (gamma dt)^-1 [ -theta dt d_z f(u_k) - (1 - theta) dt d_z f(v_{k-1}) ]

    Returns three lists of scipy sparse matrices indexed by 0-based step.
    """
    dt, th, g = raw.dt, raw.theta, raw.gamma
    M = _as_sparse(raw.kind, raw.M)
    N, V, Z = [], [], []
    for t in range(raw.n):
        Juc = _as_sparse(raw.kind, raw.Ju_cur[t])
        Jup = _as_sparse(raw.kind, raw.Ju_prev[t])
        Jzc = _as_sparse(raw.kind, raw.jz("cur", t))
        Jzp = _as_sparse(raw.kind, raw.jz("prev", t))
        N.append((M - th * dt * Juc) / dt)
        V.append((-M - (1.0 - th) * dt * Jup) / dt)
        Z.append((-th * dt * Jzc - (1.0 - th) * dt * Jzp) / (g * dt))
    return N, V, Z


# --------------------------------------------------------------------------
# The lifted augmented system (Fig. 4) and its time-major permutation (Fig. 5)

def lifted_constraint_jacobian(N, V, Z, n, p, q) -> sp.csr_matrix:
    """B = dF~ of Sec. 5.1: rows (lambda_1..n, mu_1..n), columns (u, v, z).

    lambda_k row:  V_k v_{k-1} + N_k u_k + Z~_k z_k   (v_0 := 0, so V_1 drops)
    mu_k row:      u_k - v_k                          (the scaled u - v, Sec. 5.1)
    """
    Nb = sp.block_diag(N, format="csr")
    Zb = sp.block_diag(Z, format="csr")
    # V_k multiplies v_{k-1}: block row t, block column t - 1
    rows = [[None] * n for _ in range(n)]
    for t in range(n):
        rows[t][t] = sp.csr_matrix((p, p))
    for t in range(1, n):
        rows[t][t - 1] = V[t]
    Vb = sp.bmat(rows, format="csr")
    I = sp.identity(p * n, format="csr")
    return sp.bmat([[Nb, Vb, Zb], [I, -I, None]], format="csr")


def lifted_augmented(N, V, Z, n, p, q) -> sp.csr_matrix:
    """A = [[I, B^T], [B, 0]] in type-major order (u, v, z, lambda, mu): Eq. (augsys-aj), Fig. 4."""
    B = lifted_constraint_jacobian(N, V, Z, n, p, q)
    nx = (2 * p + q) * n
    return sp.bmat([[sp.identity(nx), B.T], [B, None]], format="csr")


def type_major_offsets(n, p, q):
    """Start of each variable type in the type-major vector (Fig. 4)."""
    return {"u": 0, "v": p * n, "z": 2 * p * n, "l": (2 * p + q) * n, "m": (3 * p + q) * n}


def time_major_order(n, p, q):
    """perm with y = x[perm] (y = Q x, Sec. 5.2) and the n + 1 diagonal block bounds (Fig. 5).

    Block 1 = (u_1, z_1, lambda_1); block k = (v_{k-1}, u_k, z_k, lambda_k,
    mu_{k-1}) for k = 2..n; block n + 1 = (v_n, mu_n).
    """
    off = type_major_offsets(n, p, q)

    def seg(kind, t):
        width = q if kind == "z" else p
        start = off[kind] + t * width
        return list(range(start, start + width))

    perm, bounds = [], []
    for j in range(n + 1):
        start = len(perm)
        if j >= 1:
            perm += seg("v", j - 1)
        if j < n:
            perm += seg("u", j) + seg("z", j) + seg("l", j)
        if j >= 1:
            perm += seg("m", j - 1)
        bounds.append((start, len(perm)))
    return np.array(perm), bounds


# --------------------------------------------------------------------------
# Transfers (Sec. 5.3.1), as explicit sparse matrices in type-major order

def _interp_linear(nc: int, end_rule: int) -> sp.csr_matrix:
    """x^f_{2k-1} = x^c_k, x^f_{2k} = (x^c_k + x^c_{k+1}) / 2; last fine point by end_rule."""
    P = sp.lil_matrix((2 * nc, nc))
    for K in range(nc):
        P[2 * K, K] = 1.0
        if K + 1 < nc:
            P[2 * K + 1, K] = 0.5
            P[2 * K + 1, K + 1] = 0.5
        else:
            P[2 * K + 1, K] = 1.0 if end_rule == 0 else 0.5
    return P.tocsr()


def _interp_constant(nc: int) -> sp.csr_matrix:
    """z^f_{2k} = z^f_{2k-1} = z^c_k."""
    P = sp.lil_matrix((2 * nc, nc))
    for K in range(nc):
        P[2 * K, K] = 1.0
        P[2 * K + 1, K] = 1.0
    return P.tocsr()


def _restrict_inject(nc: int) -> sp.csr_matrix:
    """x^c_k = x^f_{2k-1}."""
    R = sp.lil_matrix((nc, 2 * nc))
    for K in range(nc):
        R[K, 2 * K] = 1.0
    return R.tocsr()


def _restrict_average(nc: int) -> sp.csr_matrix:
    """z^c_k = (z^f_{2k} + z^f_{2k-1}) / 2."""
    R = sp.lil_matrix((nc, 2 * nc))
    for K in range(nc):
        R[K, 2 * K] = 0.5
        R[K, 2 * K + 1] = 0.5
    return R.tocsr()


def transfer_type_major(n: int, p: int, q: int, end_rule: int = 0, restrict: str = "inject"):
    """(R, P) between n fine and n/2 coarse steps, type-major, all five variable types.

    restrict = "inject": the residual is restricted with the formulas Sec. 5.3.1
    gives for the variables (injection at fine step 2k-1; average for z).
    restrict = "transpose": the residual, a dual vector (it lives in the rows of
    A~), is restricted by the transpose of the interpolation, R = P^T:
    r^c_k = r_{2k-1} + (r_{2k-2} + r_{2k}) / 2 for u, v, lambda, mu and
    r^c_k = r_{2k-1} + r_{2k} for z (the variational choice of multigrid texts
    such as the tutorial Sec. 5.3 cites).
    """
    nc = n // 2
    Ip, Iq = sp.identity(p), sp.identity(q)
    Pl, Pc = _interp_linear(nc, end_rule), _interp_constant(nc)
    P = sp.block_diag([sp.kron(Pl, Ip), sp.kron(Pl, Ip), sp.kron(Pc, Iq),
                       sp.kron(Pl, Ip), sp.kron(Pl, Ip)], format="csr")
    if restrict == "transpose":
        return P.T.tocsr(), P
    if restrict != "inject":
        raise ValueError(restrict)
    Rl, Ra = _restrict_inject(nc), _restrict_average(nc)
    R = sp.block_diag([sp.kron(Rl, Ip), sp.kron(Rl, Ip), sp.kron(Ra, Iq),
                       sp.kron(Rl, Ip), sp.kron(Rl, Ip)], format="csr")
    return R, P


# --------------------------------------------------------------------------
# One grid level in time-major form

class Level:
    """A~, its block splitting D + L + L^T (Sec. 5.3.2) and factorisations.

    band_round (optional): applied to the entries of every N_k, V_k, Z~_k after
    they are formed (e.g. ``round_bf16``), giving the level whose bands are
    stored in that precision."""

    def __init__(self, raw: RawLevel, band_round=None):
        self.raw = raw
        n, p, q = raw.n, raw.p, raw.q
        self.n, self.p, self.q = n, p, q
        N, V, Z = scaled_blocks(raw)
        if band_round is not None:
            def rnd(m):
                m = m.tocsr(copy=True)
                m.data = band_round(m.data)
                return m
            N, V, Z = [rnd(m) for m in N], [rnd(m) for m in V], [rnd(m) for m in Z]
        self.N, self.V, self.Z = N, V, Z
        self.A = lifted_augmented(N, V, Z, n, p, q)
        self.perm, self.bounds = time_major_order(n, p, q)
        self.At = self.A[self.perm][:, self.perm].tocsr()
        blk = np.empty(self.At.shape[0], dtype=np.int64)
        for j, (a, b) in enumerate(self.bounds):
            blk[a:b] = j
        C = self.At.tocoo()
        br, bc = blk[C.row], blk[C.col]
        shape = self.At.shape

        def part(mask):
            return sp.csr_matrix((C.data[mask], (C.row[mask], C.col[mask])), shape=shape)

        self.D = part(br == bc)
        self.L = part(br > bc)
        self.U = part(br < bc)
        self._D_lu = None
        self._DL_lu = None
        self._DU_lu = None

    @property
    def size(self):
        return self.At.shape[0]

    # factorisations (SuperLU with partial pivoting), built on first use
    def D_solve(self, r):
        if self._D_lu is None:
            self._D_lu = spla.splu(self.D.tocsc())
        return self._D_lu.solve(r)

    def DL_solve(self, r):
        if self._DL_lu is None:
            self._DL_lu = spla.splu((self.D + self.L).tocsc())
        return self._DL_lu.solve(r)

    def DU_solve(self, r):
        if self._DU_lu is None:
            self._DU_lu = spla.splu((self.D + self.U).tocsc())
        return self._DU_lu.solve(r)

    def to_time_major(self, x):
        return x[self.perm]

    def to_type_major(self, y):
        x = np.empty_like(y)
        x[self.perm] = y
        return x


def jacobi_sweep(level: Level, b: np.ndarray, y: np.ndarray, omega: float = 1.0) -> np.ndarray:
    """y^l = D^-1 [ b - (L + L^T) y^{l-1} ]   (Eq. jacobi-aj).

    omega != 1 is a relaxation weight the paper does not use (an option of
    this implementation): y^l = y^{l-1} + omega (D^-1 [...] - y^{l-1}).
    """
    ynew = level.D_solve(b - (level.L @ y + level.U @ y))
    if omega == 1.0:
        return ynew
    return y + omega * (ynew - y)


def sgs_apply(level: Level, r: np.ndarray) -> np.ndarray:
    """[(D + L) D^-1 (D + L^T)]^-1 r = (D + L^T)^-1 D (D + L)^-1 r   (Sec. 5.3.4)."""
    w = level.DL_solve(r)
    return level.DU_solve(level.D @ w)


def jacobi_spectral_radius(level: Level) -> float:
    """rho(I - D^-1 A~) of the block-Jacobi iteration (Table 2), by dense eigenvalues."""
    A = level.At.toarray()
    D = level.D.toarray()
    return float(np.max(np.abs(np.linalg.eigvals(np.eye(A.shape[0]) - np.linalg.solve(D, A)))))


def fixed_point_preconditioner(level: Level, kind: str):
    """The block fixed-point iterations of Sec. 5.3.4 / Table 1 as preconditioners:
    one step from zero of Jacobi D^-1, forward Gauss-Seidel (D + L)^-1,
    backward Gauss-Seidel (D + L^T)^-1, or symmetric Gauss-Seidel."""
    if kind == "sgs":
        return lambda r: sgs_apply(level, r)
    if kind == "jacobi":
        return level.D_solve
    if kind == "fgs":
        return level.DL_solve
    if kind == "bgs":
        return level.DU_solve
    raise ValueError(kind)


# --------------------------------------------------------------------------
# Krylov solvers

@dataclasses.dataclass
class KrylovResult:
    x: np.ndarray
    iters: int
    relres: float           # Arnoldi estimate |g_{j+1}| / ||b||
    history: list


def fgmres(apply_A, apply_M, b: np.ndarray, rtol: float, maxit: int, restart: int = None,
           fixed_iters: int = 0) -> KrylovResult:
    """Flexible GMRES with x0 = 0 (Saad 1993; used in Sec. 6 and Sec. 5.3.4).

    Right-preconditioned Arnoldi that stores z_j = M_j(v_j) and forms
    x = x0 + Z_m y_m, where y_m minimises || beta e_1 - H_m y || (Givens
    rotations on the Hessenberg matrix).  With a fixed linear preconditioner
    this is right-preconditioned GMRES, the coarse solver of Sec. 5.3.4.
    Orthogonalisation: modified Gram-Schmidt.  Stops when the estimate
    |g_{j+1}| <= rtol ||b||, or after ``fixed_iters`` iterations when that is
    positive (then the tolerance is ignored), or at ``maxit``; restarts every
    ``restart`` iterations from the true residual.
    """
    bnorm = float(np.linalg.norm(b))
    x = np.zeros_like(b)
    if bnorm == 0.0:
        return KrylovResult(x, 0, 0.0, [])
    limit = fixed_iters if fixed_iters > 0 else maxit
    m = restart if restart else limit
    total = 0
    history = []
    r = b.copy()
    est = 1.0
    while total < limit:
        beta = float(np.linalg.norm(r))
        if beta == 0.0:
            est = 0.0
            break
        mm = min(m, limit - total)
        Vb = [r / beta]
        Zb = []
        H = np.zeros((mm + 1, mm))
        cs = np.zeros(mm)
        sn = np.zeros(mm)
        g = np.zeros(mm + 1)
        g[0] = beta
        k = 0
        done = False
        for j in range(mm):
            z = apply_M(Vb[j])
            Zb.append(z)
            w = apply_A(z)
            for i in range(j + 1):
                H[i, j] = float(np.dot(w, Vb[i]))
                w = w - H[i, j] * Vb[i]
            H[j + 1, j] = float(np.linalg.norm(w))
            for i in range(j):
                hi, hi1 = H[i, j], H[i + 1, j]
                H[i, j] = cs[i] * hi + sn[i] * hi1
                H[i + 1, j] = -sn[i] * hi + cs[i] * hi1
            hjj, hj1 = H[j, j], H[j + 1, j]
            denom = float(np.hypot(hjj, hj1))
            breakdown = hj1 == 0.0
            if denom == 0.0:
                cs[j], sn[j] = 1.0, 0.0
            else:
                cs[j], sn[j] = hjj / denom, hj1 / denom
            H[j, j] = cs[j] * hjj + sn[j] * hj1
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            k = j + 1
            total += 1
            est = abs(g[j + 1]) / bnorm
            history.append(est)
            if not breakdown:
                Vb.append(w / hj1)
            if breakdown or (fixed_iters <= 0 and est <= rtol):
                done = True
                break
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - float(np.dot(H[i, i + 1:k], y[i + 1:k]))) / H[i, i]
        for i in range(k):
            x = x + y[i] * Zb[i]
        if done or total >= limit:
            break
        r = b - apply_A(x)
    return KrylovResult(x, total, est, history)


# --------------------------------------------------------------------------
# Multigrid hierarchy and V-cycle (Alg. 1)

@dataclasses.dataclass
class MGOptions:
    levels: int = 2
    nu_pre: int = 1
    nu_post: int = 1
    coarse_rtol: float = 1e-3
    coarse_maxit: int = 50
    coarse_fixed_iters: int = 0
    end_rule: int = 0
    omega: float = 1.0
    coarse_precond: str = "sgs"     # the paper's; "jacobi", "fgs", "bgs" are Table 1's alternatives
    restrict: str = "inject"        # residual restriction: "inject" (Sec. 5.3.1 as written) or "transpose" (P^T)
    bands: str = "fp64"             # "bf16": every level but the coarsest with its bands rounded by round_bf16


class Hierarchy:
    def __init__(self, prob, opts: MGOptions):
        self.opts = opts
        raw = raw_from_problem(prob)
        n = raw.n
        if opts.levels < 1 or n % (1 << (opts.levels - 1)):
            raise ValueError("n must be divisible by 2^(levels-1)")
        self.levels = []
        self.R, self.P = [], []
        for lv in range(opts.levels):
            smoothing = lv + 1 < opts.levels
            level = Level(raw, band_round=round_bf16 if (opts.bands == "bf16" and smoothing) else None)
            self.levels.append(level)
            if lv + 1 < opts.levels:
                R, P = transfer_type_major(raw.n, raw.p, raw.q, opts.end_rule, opts.restrict)
                cperm, _ = time_major_order(raw.n // 2, raw.p, raw.q)
                # R~ = Q_c R Q_f^T, P~ = Q_f P Q_c^T
                self.R.append(R[cperm][:, level.perm].tocsr())
                self.P.append(P[level.perm][:, cperm].tocsr())
                raw = coarsen_raw(raw)
        self.coarse_iters = []

    @property
    def fine(self) -> Level:
        return self.levels[0]

    def coarse_solve(self, lv: int, r: np.ndarray) -> np.ndarray:
        """GMRES right-preconditioned by SGS, x0 = 0, relative tolerance 1e-3 (Sec. 5.3.4)."""
        level = self.levels[lv]
        o = self.opts
        res = fgmres(lambda v: level.At @ v, fixed_point_preconditioner(level, o.coarse_precond), r,
                     rtol=o.coarse_rtol, maxit=o.coarse_maxit, fixed_iters=o.coarse_fixed_iters)
        self.coarse_iters.append(res.iters)
        return res.x

    def vcycle(self, lv: int, b: np.ndarray) -> np.ndarray:
        """Alg. 1 generalised to a V-cycle, starting from y = 0 on every level."""
        o = self.opts
        level = self.levels[lv]
        if lv == len(self.levels) - 1:
            return self.coarse_solve(lv, b)
        y = np.zeros_like(b)
        for _ in range(o.nu_pre):
            y = jacobi_sweep(level, b, y, o.omega)
        r = self.R[lv] @ (b - level.At @ y)
        e = self.vcycle(lv + 1, r)
        y = y + self.P[lv] @ e
        for _ in range(o.nu_post):
            y = jacobi_sweep(level, b, y, o.omega)
        return y

    # ABI-shaped entry points (type-major vectors)
    def precondition(self, r_type_major: np.ndarray) -> np.ndarray:
        f = self.fine
        return f.to_type_major(self.vcycle(0, f.to_time_major(r_type_major)))

    def solve(self, b_type_major: np.ndarray, rtol: float, maxit: int = 200, restart: int = 60):
        """FGMRES on A~ y = b~ preconditioned by the V-cycle (Sec. 5.3.4, Sec. 6).  The
        operator is always the fine level's exact A~ (FP64 bands)."""
        f = self.fine if self.opts.bands == "fp64" else Level(self.fine.raw)
        bt = f.to_time_major(b_type_major)
        res = fgmres(lambda v: f.At @ v, lambda v: self.vcycle(0, v), bt,
                     rtol=rtol, maxit=maxit, restart=restart)
        x = f.to_type_major(res.x)
        true_rel = float(np.linalg.norm(b_type_major - f.A @ x) / np.linalg.norm(b_type_major))
        return x, res, true_rel


def direct_solve(prob) -> np.ndarray:
    """x = A^-1 b for the lifted type-major system by SuperLU (library reference)."""
    level = Level(raw_from_problem(prob))
    return spla.spsolve(level.A.tocsc(), prob.b)


def parallel_speedup(n: int, n_ls_ser: float, n_ls_par: float, n_lv: int, n_pre: int, n_post: int) -> float:
    """Modelled speedup of Sec. 6.3: serial units 2 N_ser n over N_par 2 (N_Lv - 1)(N_pre + N_post)."""
    serial = 2.0 * n_ls_ser * n
    parallel = n_ls_par * 2.0 * (n_lv - 1) * (n_pre + n_post)
    return serial / parallel
