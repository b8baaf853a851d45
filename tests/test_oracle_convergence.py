"""Iteration behaviour of the oracle's V-cycle against Tables 2-4 (Sec. 6.1-6.2).

Two readings of the cycle are pinned here.

* The cycle as Alg. 1 and Sec. 5.3.1-5.3.2 write it (undamped block-Jacobi
  sweeps, the variable formulas of Sec. 5.3.1 applied to the residual).  Its
  smoother reproduces Table 2's spectral radii (test_oracle_methods), but its
  FGMRES counts grow linearly in n, unlike Tables 3-4.  The cause is
  structural: A~ is block tridiagonal (Fig. 5), so the block-Jacobi iteration
  matrix S satisfies J S J = -S with J = diag((-1)^k I) and its spectrum is
  symmetric about 0.  The slow eigenvalues form a ring of radius rho(S), and
  the eigenvector at -rho(S) is the one at +rho(S) with every other block
  negated, i.e. it alternates in time.  No coarse space built from linear
  interpolation holds such modes, so a two-level cycle cannot contract
  faster than about rho(S)^(nu_pre + nu_post), whatever the transfers.
* The residual restricted by the transpose of the interpolation and weighted
  sweeps (omega = 2/3): counts grow by about one per doubling of n, the
  logarithmic growth of Tables 3-4, within about 2.5x of their values.
"""
import numpy as np
import pytest

from conftest import read_golden
from oracle import augmented as O
from paper_2405_04808_gb300 import workloads as W

# Table 3 (van der Pol, gamma = 100, V cycle 4/4): n, last level Lv, average FGMRES iterations
TABLE3 = {64: (4, 4.21), 128: (5, 5.16), 256: (6, 5.78)}
# Table 4 (Burgers, gamma = 100, V cycle 4/4): n, Lv, average FGMRES iterations
TABLE4 = {64: (4, 3.58), 128: (5, 4.75), 256: (6, 6.02)}


def _solve_iters(prob, levels, omega=1.0, restrict="inject", b=None, zero_prolongation=False):
    h = O.Hierarchy(prob, O.MGOptions(levels=levels, nu_pre=4, nu_post=4, omega=omega, restrict=restrict))
    if zero_prolongation:
        h.P = [0.0 * P for P in h.P]
    _, res, tr = h.solve(prob.b if b is None else b, rtol=1e-6, maxit=500, restart=500)
    assert tr <= 1.5e-6
    return res.iters


def test_transpose_restriction_worked_example():
    g = {row[0]: np.array([float(v) for v in row[1:]]) for row in read_golden("transfers_n8.txt")}
    f = g["fine"]
    n, p, q = 8, 1, 1
    for end_rule in (0, 1):
        R, _ = O.transfer_type_major(n, p, q, end_rule, restrict="transpose")
        rc = R @ np.tile(f, 5)          # the same fine sequence in each of u, v, z, lambda, mu
        lin = g[f"restrict_transpose_linear_end{end_rule}"]
        assert np.array_equal(rc[0:4], lin) and np.array_equal(rc[4:8], lin)      # u, v
        assert np.array_equal(rc[8:12], g["restrict_transpose_constant"])          # z
        assert np.array_equal(rc[12:16], lin) and np.array_equal(rc[16:20], lin)  # lambda, mu


def test_block_jacobi_spectrum_is_symmetric_ring():
    """J S J = -S for the block-tridiagonal A~; the nonzero spectrum is a ring of radius ~rho."""
    prob = W.vdp_paper(n=32, gamma=100.0)
    lev = O.Level(O.raw_from_problem(prob))
    A, D = lev.At.toarray(), lev.D.toarray()
    S = np.eye(A.shape[0]) - np.linalg.solve(D, A)
    J = np.zeros(A.shape[0])
    for k, (a, b) in enumerate(lev.bounds):
        J[a:b] = (-1.0) ** k
    assert np.allclose(J[:, None] * S * J[None, :], -S, atol=1e-12)
    ev = np.linalg.eigvals(S)
    mags = np.abs(ev)
    rho = mags.max()
    nonzero = mags[mags > 1e-6]
    # every nonzero eigenvalue (4n of them for p = 2) lies within 20 % of the radius: no frequency is damped
    assert nonzero.size == 4 * prob.n * prob.p // 2
    assert nonzero.min() >= 0.8 * rho
    # ... and they are spread all around the circle, alternating-in-time modes included (angle near pi)
    ang = np.angle(ev[mags > 1e-6])
    assert np.max(np.abs(ang)) > 0.97 * np.pi and np.min(np.abs(ang)) < 0.03 * np.pi


@pytest.mark.parametrize("restrict", ["inject", "transpose"])
def test_undamped_two_level_factor_bounded_by_smoother(restrict):
    """With omega = 1 the exact two-level cycle contracts no faster than ~rho(S)^8, for either restriction."""
    prob = W.vdp_paper(n=32, gamma=100.0)
    h = O.Hierarchy(prob, O.MGOptions(levels=2, nu_pre=4, nu_post=4, restrict=restrict))
    f, c = h.levels
    A = f.At.toarray()
    S = np.eye(A.shape[0]) - np.linalg.solve(f.D.toarray(), A)
    C = np.eye(A.shape[0]) - h.P[0].toarray() @ np.linalg.solve(c.At.toarray(), h.R[0].toarray() @ A)
    S4 = np.linalg.matrix_power(S, 4)
    rho_e = np.abs(np.linalg.eigvals(S4 @ C @ S4)).max()
    rho_s = np.abs(np.linalg.eigvals(S)).max()
    assert rho_e >= 0.9 * rho_s ** 8
    # the same bound holds for a Galerkin coarse operator (variational, R = P^T)
    Pm = h.P[0].toarray()
    Cg = np.eye(A.shape[0]) - Pm @ np.linalg.solve(Pm.T @ A @ Pm, Pm.T @ A)
    assert np.abs(np.linalg.eigvals(S4 @ Cg @ S4)).max() >= 0.9 * rho_s ** 8


def test_literal_cycle_counts_grow_linearly():
    """Alg. 1 as written on the paper's van der Pol setting: 30 / 59 / 119 iterations at n = 64 / 128 / 256
    (Table 3: 4.21 / 5.16 / 5.78), and zeroing the coarse correction changes them only to 32 / 62 / 122."""
    counts, counts0 = [], []
    for n, (lv, _) in TABLE3.items():
        prob = W.vdp_paper(n=n, gamma=100.0)
        counts.append(_solve_iters(prob, lv))
        counts0.append(_solve_iters(prob, lv, zero_prolongation=True))
    assert counts == [30, 59, 119]
    assert counts0 == [32, 62, 122]


def test_transpose_restriction_weighted_sweeps_reach_table3_growth():
    counts, counts_chi = [], []
    for n, (lv, paper) in TABLE3.items():
        prob = W.vdp_paper(n=n, gamma=100.0)
        its = _solve_iters(prob, lv, omega=2.0 / 3.0, restrict="transpose")
        counts.append(its)
        # the projection right-hand side (chi, 0) that dominates the SQP's augmented solves (Sec. 6)
        b = prob.b.copy()
        b[prob.n * (2 * prob.p + prob.q):] = 0.0
        its_chi = _solve_iters(prob, lv, omega=2.0 / 3.0, restrict="transpose", b=b)
        counts_chi.append(its_chi)
        assert its <= 2.5 * paper and its_chi <= 2.2 * paper
        # the coarse grid does the work: without it the same cycle needs several times more
        assert _solve_iters(prob, lv, omega=2.0 / 3.0, restrict="transpose", zero_prolongation=True) >= 3 * its
    assert counts == [10, 12, 13] and counts_chi == [9, 9, 11]
    assert all(b - a <= 2 for a, b in zip(counts, counts[1:]))


def test_transpose_restriction_weighted_sweeps_burgers_growth():
    """Burgers (Table 4's setting, P1 in space): about one more iteration per doubling of n."""
    counts = []
    for n, (lv, paper) in TABLE4.items():
        prob = W.burgers(nx=32, n=n, seed=2000)
        its = _solve_iters(prob, lv, omega=2.0 / 3.0, restrict="transpose")
        counts.append(its)
        assert its <= 3.0 * paper
        lit = _solve_iters(prob, lv)
        assert lit >= 2 * its
    assert all(b - a <= 2 for a, b in zip(counts, counts[1:]))


def test_bf16_rounding_closed_forms_and_library():
    """round_bf16 (the storage of MG_PRECISION_BF16_BANDS): ties to even at the 8th significant bit, and
    the same values as torch's float32 -> bfloat16 conversion (round to nearest even) on random data."""
    r = O.round_bf16([1 + 2 ** -8, 1 + 3 * 2 ** -8, 1 + 2 ** -8 + 2 ** -20, -(1 + 3 * 2 ** -8), 3.0, 0.0])
    assert list(r) == [1.0, 1 + 2 ** -6, 1 + 2 ** -7, -(1 + 2 ** -6), 3.0, 0.0]
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(7)
    x = rng.standard_normal(20000) * 10.0 ** rng.uniform(-6, 6, 20000)
    want = torch.tensor(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(O.round_bf16(x), want)


def test_bf16_band_cycle_keeps_the_exact_operator():
    """With BF16 bands on the smoothing levels the V-cycle changes by ~1e-2 but FGMRES, whose operator keeps
    the FP64 bands, still reaches the direct solution of the unrounded system with the same iteration count
    up to one."""
    prob = W.burgers(nx=40, n=32, seed=131)
    opts = dict(levels=2, nu_pre=2, nu_post=2)
    y64 = O.Hierarchy(prob, O.MGOptions(coarse_fixed_iters=2, **opts)).precondition(prob.b)
    yb = O.Hierarchy(prob, O.MGOptions(coarse_fixed_iters=2, bands="bf16", **opts)).precondition(prob.b)
    assert 1e-4 < np.linalg.norm(yb - y64) / np.linalg.norm(y64) < 5e-2
    xb, rb, _ = O.Hierarchy(prob, O.MGOptions(bands="bf16", **opts)).solve(prob.b, rtol=1e-10, maxit=500,
                                                                               restart=200)
    _, r64, _ = O.Hierarchy(prob, O.MGOptions(**opts)).solve(prob.b, rtol=1e-10, maxit=500, restart=200)
    xd = O.direct_solve(prob)
    assert np.linalg.norm(xb - xd) <= 1e-9 * np.linalg.norm(xd)
    assert abs(rb.iters - r64.iters) <= 1
