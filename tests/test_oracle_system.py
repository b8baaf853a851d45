"""Pins of the oracle's lifted augmented system against the paper.

* Fig. 5's block pattern (golden transcription),
* B = dF~ against a complex-step Jacobian of the scaled constraint itself
  (Eq. theta2-aj, the transplant of Sec. 4.1 and the u - v constraint of
  Sec. 5.1),
* symmetry and inertia of the augmented matrix, Theorem 1.
"""
import numpy as np
import pytest

from conftest import read_golden
from oracle import augmented as O
from paper_2405_04808_gb300 import workloads as W


def _tiny_problems():
    return [W.vdp(n=4, seed=11), W.burgers(nx=5, n=4, seed=12),
            W.vdp_paper(n=4, gamma=3.0)]


def _var_index(n, p, q):
    """(type, paper step k) -> slice of the type-major vector."""
    off = O.type_major_offsets(n, p, q)
    out = {}
    for t in "uvzlm":
        wdt = q if t == "z" else p
        for k in range(1, n + 1):
            out[(t, k)] = slice(off[t] + (k - 1) * wdt, off[t] + k * wdt)
    return out


@pytest.mark.parametrize("prob", _tiny_problems(), ids=["vdp", "burgers", "vdp_q2"])
def test_fig5_block_pattern(prob):
    """Every block of A~ (n = 4) is the one Fig. 5 names, every other block is zero."""
    raw = O.raw_from_problem(prob)
    lev = O.Level(raw)
    n, p, q = raw.n, raw.p, raw.q
    A = lev.A.toarray()
    idx = _var_index(n, p, q)
    named = {}
    for k in range(1, n + 1):
        named[f"N{k}"] = lev.N[k - 1].toarray()
        named[f"V{k}"] = lev.V[k - 1].toarray()
        named[f"Z{k}"] = lev.Z[k - 1].toarray()
    expected = {}
    for r, c, blk in read_golden("fig5_pattern.txt"):
        expected[(r, c)] = blk
    seen = 0
    for (rt, rk), rs in idx.items():
        for (ct, ck), cs in idx.items():
            got = A[rs, cs]
            key = (f"{rt}{rk}", f"{ct}{ck}")
            blk = expected.get(key)
            if blk is None:
                assert not np.any(got), key
                continue
            seen += 1
            if blk in ("I", "-I"):
                want = np.eye(got.shape[0]) * (1.0 if blk == "I" else -1.0)
            elif blk.endswith("T"):
                want = named[blk[:-1]].T
            else:
                want = named[blk]
            assert np.array_equal(got, want), key
    assert seen == len(expected)
    # the time-major permutation groups exactly Fig. 5's blocks
    perm, bounds = O.time_major_order(n, p, q)
    assert sorted(perm.tolist()) == list(range(n * (4 * p + q)))
    sizes = [b - a for a, b in bounds]
    assert sizes == [2 * p + q] + [4 * p + q] * (n - 1) + [2 * p]


def _scaled_constraint(prob, u, v, z):
    """F~ of Sec. 5.1 evaluated from f itself, in scaled coordinates.

    lambda_k rows: dt^-1/2 [ M u^_k - M v^_{k-1} - dt (theta f(u^_k + chi, z^_k)
                    + (1 - theta) f(v^_{k-1} + chi, z^_k)) ]
    mu_k rows:     u_k - v_k
    with u^ = dt^-1/2 u, v^ = dt^-1/2 v, z^ = (gamma^2 dt)^-1/2 z, v^_0 = 0
    and chi the initial state (the shift of the footnote to Sec. 1).
    """
    m = prob.model
    n, p, q = prob.n, prob.p, prob.q
    dt, th, g = prob.dt, prob.theta, prob.gamma
    chi = prob.u_phys[0]
    Mm = m.mass()
    dense = prob.kind == "dense"

    def mass(x):
        if dense:
            return Mm @ x
        return W._band_matvec(Mm, x)

    uh = u.reshape(n, p) / np.sqrt(dt)
    vh = v.reshape(n, p) / np.sqrt(dt)
    zh = z.reshape(n, q) / np.sqrt(g * g * dt)
    lam, mu = [], []
    for k in range(n):
        vprev = vh[k - 1] if k > 0 else np.zeros(p, dtype=uh.dtype)
        c = (mass(uh[k]) - mass(vprev)
             - dt * (th * m.f(uh[k] + chi, zh[k]) + (1 - th) * m.f(vprev + chi, zh[k])))
        lam.append(c / np.sqrt(dt))
        mu.append(u.reshape(n, p)[k] - v.reshape(n, p)[k])
    return np.concatenate(lam + mu)


@pytest.mark.parametrize("prob", _tiny_problems(), ids=["vdp", "burgers", "vdp_q2"])
def test_constraint_jacobian_is_dF(prob):
    """The lifted B of the oracle equals dF~ by complex-step differentiation."""
    n, p, q = prob.n, prob.p, prob.q
    dt, g = prob.dt, prob.gamma
    u0 = np.sqrt(dt) * (prob.u_phys[1:] - prob.u_phys[0]).ravel()
    z0 = g * np.sqrt(dt) * prob.z_phys.ravel()
    x0 = np.concatenate([u0, u0.copy(), z0])
    nv = x0.size
    J = np.zeros((2 * p * n, nv))
    h = 1e-30
    for j in range(nv):
        x = x0.astype(complex)
        x[j] += 1j * h
        F = _scaled_constraint(prob, x[:p * n], x[p * n:2 * p * n], x[2 * p * n:])
        J[:, j] = F.imag / h
    raw = O.raw_from_problem(prob)
    N, V, Z = O.scaled_blocks(raw)
    B = O.lifted_constraint_jacobian(N, V, Z, n, p, q).toarray()
    assert np.max(np.abs(B - J)) <= 1e-13 * np.max(np.abs(J))


@pytest.mark.parametrize("prob", _tiny_problems(), ids=["vdp", "burgers", "vdp_q2"])
def test_symmetry_inertia_theorem1(prob):
    """A~ is symmetric with inertia (n(2p+q), 2pn, 0); every D_k is nonsingular (Thm 1)."""
    lev = O.Level(O.raw_from_problem(prob))
    n, p, q = lev.n, lev.p, lev.q
    A = lev.At.toarray()
    assert np.array_equal(A, A.T)
    ev = np.linalg.eigvalsh(A)
    tol = 1e-10 * np.max(np.abs(ev))
    assert np.sum(ev > tol) == n * (2 * p + q)
    assert np.sum(ev < -tol) == 2 * p * n
    for k in range(n):
        assert abs(np.linalg.det(lev.N[k].toarray())) > 0
    for a, b in lev.bounds:
        blk = A[a:b, a:b]
        s = np.linalg.svd(blk, compute_uv=False)
        assert s[-1] > 1e-12 * s[0]


def test_coarsening_reads_injected_points():
    """Coarse Jacobians come from fine steps 2K-1 (current) and 2K-2 (previous), 1-based."""
    prob = W.vdp(n=8, seed=5)
    raw = O.raw_from_problem(prob)
    c = O.coarsen_raw(raw)
    assert c.n == 4 and c.dt == 2 * raw.dt
    for K in range(1, 5):
        assert np.array_equal(c.Ju_cur[K - 1], raw.Ju_cur[2 * K - 2])
        prevk = max(2 * K - 2, 1)
        assert np.array_equal(c.Ju_prev[K - 1], raw.Ju_prev[prevk - 1])
