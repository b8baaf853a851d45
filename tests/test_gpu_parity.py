"""CUDA path (through the C ABI) against the CPU oracle, element by element."""
import numpy as np
import pytest

from oracle import augmented as O
from paper_2405_04808_gb300 import workloads as W
from parity_util import assert_per_type

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# FP64 V-cycle parity: with a fixed coarse iteration count the cycle is a
# deterministic map; oracle (sparse LU, MGS) and GPU (Schur complement,
# affine SGS chains, CGS2) differ only by rounding, amplified by the local
# condition numbers (~1e4 here): 1e-10 relative in the 2-norm.
VCYCLE_RTOL = 1e-10
# The same comparison one variable type at a time: the largest entry error of
# each of u, v, z, lambda, mu against that type's largest entry.
VCYCLE_TYPE_TOL = 1e-9
# FGMRES at a 1e-10 relative residual: the solution differs from the exact one
# by at most cond(A) * 1e-10; the required bar is 1e-9 relative, here asserted
# per variable type (the oracle's own FGMRES at 1e-10 stays below 1e-10 per
# type on these cases).
SOLVE_RTOL = 1e-9


@pytest.fixture(scope="module")
def P():
    from paper_2405_04808_gb300 import pintmg
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pintmg.lib()
    return pintmg


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


CASES = [
    # (problem, levels, nu_pre, nu_post, end_rule[, omega])
    (lambda: W.vdp(n=64, seed=101), 3, 1, 1, 0),
    (lambda: W.vdp(n=48, seed=102), 2, 2, 3, 1),
    (lambda: W.vdp(n=24, seed=103), 1, 0, 0, 0),
    (lambda: W.vdp_paper(n=32, gamma=100.0), 3, 4, 4, 0),
    (lambda: W.burgers(nx=40, n=32, seed=104), 2, 2, 2, 0),      # p = 40: ragged lane chunks
    (lambda: W.burgers(nx=64, n=16, seed=105), 3, 1, 0, 1),
    (lambda: W.burgers(nx=7, n=8, seed=106, theta=0.5), 2, 1, 1, 0),  # theta < 1: V_k varies
    (lambda: W.burgers(nx=130, n=16, seed=107), 2, 4, 4, 0),     # p = 130: 8 per lane, tail lanes empty
    (lambda: W.burgers(nx=40, n=32, seed=108), 3, 3, 2, 0, 0.7),  # relaxed sweeps (option)
    (lambda: W.vdp(n=32, seed=109), 2, 2, 2, 0, 0.6),
    # residual restricted by the transpose of the interpolation (R = P^T), weighted sweeps
    (lambda: W.burgers(nx=40, n=64, seed=110), 3, 4, 4, 0, 2.0 / 3.0, "transpose"),
    (lambda: W.vdp_paper(n=64, gamma=100.0), 4, 4, 4, 1, 2.0 / 3.0, "transpose"),
    (lambda: W.burgers(nx=130, n=16, seed=112), 2, 2, 1, 1, 1.0, "transpose"),  # p = 130, end rule 1
    (lambda: W.vdp(n=48, seed=113), 3, 1, 2, 0, 2.0 / 3.0, "transpose"),
]


def _unpack(case):
    c = CASES[case]
    return (c[0], c[1], c[2], c[3], c[4], (c[5] if len(c) > 5 else 1.0),
            (c[6] if len(c) > 6 else "inject"))


@pytest.mark.parametrize("case", range(len(CASES)))
def test_vcycle_matches_oracle(P, case):
    make, levels, nu_pre, nu_post, end_rule, omega, restrict = _unpack(case)
    prob = make()
    opts = dict(levels=levels, nu_pre=nu_pre, nu_post=nu_post, coarse_fixed_iters=3, end_rule=end_rule,
                omega=omega, restrict=restrict)
    h = P.mg_setup(prob, **opts)
    try:
        rng = np.random.default_rng(case)
        for trial in range(2):
            r = rng.standard_normal(prob.size) if trial else prob.b
            rd = _dev(r)
            yd = torch.empty_like(rd)
            assert P.mg_vcycle(h, rd.data_ptr(), yd.data_ptr(), 0) == P.MG_OK
            torch.cuda.synchronize()
            hier = O.Hierarchy(prob, O.MGOptions(**opts))
            yo = hier.precondition(r)
            err = np.linalg.norm(yd.cpu().numpy() - yo) / np.linalg.norm(yo)
            assert err <= VCYCLE_RTOL, err
            assert_per_type(yd.cpu().numpy(), yo, prob.n, prob.p, prob.q, VCYCLE_TYPE_TOL, "vcycle")
    finally:
        P.mg_destroy(h)


@pytest.mark.parametrize("case", [0, 1, 3, 4, 5, 6, 8, 9, 10, 11, 13])
def test_fgmres_matches_direct_solve(P, case):
    make, levels, nu_pre, nu_post, end_rule, omega, restrict = _unpack(case)
    prob = make()
    h = P.mg_setup(prob, levels=levels, nu_pre=nu_pre, nu_post=nu_post, end_rule=end_rule, omega=omega,
                   restrict=restrict)
    try:
        b = _dev(prob.b)
        x = torch.empty_like(b)
        code, info = P.fgmres_solve(h, b.data_ptr(), x.data_ptr(), 1e-10, 2000, 500)
        assert code == P.MG_OK, P.mg_status_string(code)
        assert info.true_relres <= 2e-10
        xd = O.direct_solve(prob)
        xg = x.cpu().numpy()
        err = np.linalg.norm(xg - xd) / np.linalg.norm(xd)
        assert err <= SOLVE_RTOL, err
        assert_per_type(xg, xd, prob.n, prob.p, prob.q, SOLVE_RTOL, "fgmres vs direct")
        # the oracle's own FGMRES reaches the same solution
        hier = O.Hierarchy(prob, O.MGOptions(levels=levels, nu_pre=nu_pre, nu_post=nu_post, end_rule=end_rule,
                                             omega=omega, restrict=restrict))
        xo, res, tr = hier.solve(prob.b, rtol=1e-10, maxit=2000, restart=500)
        assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= SOLVE_RTOL
        assert_per_type(xg, xo, prob.n, prob.p, prob.q, SOLVE_RTOL, "fgmres vs oracle fgmres")
        # iteration counts may differ by rounding near the threshold only
        assert abs(info.iters - res.iters) <= max(2, res.iters // 20), (info.iters, res.iters)
    finally:
        P.mg_destroy(h)


def test_host_and_device_buffers_agree(P):
    prob = W.vdp(n=32, seed=111)
    h = P.mg_setup(prob, levels=2, nu_pre=1, nu_post=1)
    try:
        b = _dev(prob.b)
        x = torch.empty_like(b)
        code, _ = P.fgmres_solve(h, b.data_ptr(), x.data_ptr(), 1e-10, 1000, 200)
        assert code == P.MG_OK
        bh = np.ascontiguousarray(prob.b)
        xh = np.zeros_like(bh)
        code, _ = P.fgmres_solve(h, bh.ctypes.data, xh.ctypes.data, 1e-10, 1000, 200)
        assert code == P.MG_OK
        assert np.array_equal(xh, x.cpu().numpy())  # same kernels, same order: bitwise
    finally:
        P.mg_destroy(h)


def test_error_paths(P):
    # coarse levels need the separable-control assertion (rediscretised coarse operator); one level does not
    prob = W.vdp(n=16, seed=120)
    with pytest.raises(P.PintmgError) as e:
        P.mg_setup(prob, levels=2, separable=False)
    assert e.value.code == P.MG_ERR_ARG and "separable" in P.mg_last_cuda_error()
    P.mg_destroy(P.mg_setup(prob, levels=1, separable=False))
    # singular N_k (Thm 1 fails): M - theta dt Ju = 0 for one step
    prob = W.vdp(n=16, seed=121)
    prob.Ju_cur[5] = prob.M / (prob.theta * prob.dt)
    with pytest.raises(P.PintmgError) as e:
        P.mg_setup(prob, levels=2)
    assert e.value.code == P.MG_ERR_SINGULAR
    prob = W.vdp(n=16, seed=122)
    h = P.mg_setup(prob, levels=2)
    try:
        b = prob.b.copy()
        b[7] = np.inf
        bd = _dev(b)
        x = torch.empty_like(bd)
        code, _ = P.fgmres_solve(h, bd.data_ptr(), x.data_ptr(), 1e-10, 100, 50)
        assert code == P.MG_ERR_NONFINITE
        bd = _dev(prob.b)
        code, info = P.fgmres_solve(h, bd.data_ptr(), x.data_ptr(), 1e-14, 2, 2)
        assert code == P.MG_NOT_CONVERGED and info.iters == 2
        z = torch.zeros_like(bd)
        code, info = P.fgmres_solve(h, z.data_ptr(), x.data_ptr(), 1e-10, 10, 10)
        assert code == P.MG_OK and info.iters == 0 and float(x.abs().max()) == 0.0
    finally:
        P.mg_destroy(h)


# ---------------------------------------------------------------- mixed precision

def test_fp32_vcycle_close_to_fp64_oracle(P):
    """The FP32 V-cycle (smoother, transfers, SGS) stays within FP32 rounding
    amplified by the local condition numbers of the FP64 oracle's cycle."""
    prob = W.burgers(nx=40, n=32, seed=131)
    opts = dict(levels=2, nu_pre=2, nu_post=2, coarse_fixed_iters=2)
    h = P.mg_setup(prob, precision=P.MG_PRECISION_FP32, **opts)
    try:
        rd = _dev(prob.b)
        yd = torch.empty_like(rd)
        assert P.mg_vcycle(h, rd.data_ptr(), yd.data_ptr(), 0) == P.MG_OK
        torch.cuda.synchronize()
        yo = O.Hierarchy(prob, O.MGOptions(**opts)).precondition(prob.b)
        err = np.linalg.norm(yd.cpu().numpy() - yo) / np.linalg.norm(yo)
        assert err <= 1e-3, err
    finally:
        P.mg_destroy(h)


@pytest.mark.parametrize("case", [0, 4, 7])
def test_fp32_preconditioned_fgmres_reaches_fp64_solution(P, case):
    """FGMRES tolerates the FP32 preconditioner: same solution to 1e-9 at a 1e-10 residual."""
    make, levels, nu_pre, nu_post, end_rule, _, _ = _unpack(case)
    prob = make()
    h = P.mg_setup(prob, levels=levels, nu_pre=nu_pre, nu_post=nu_post, end_rule=end_rule,
                   precision=P.MG_PRECISION_FP32)
    try:
        b = _dev(prob.b)
        x = torch.empty_like(b)
        code, info = P.fgmres_solve(h, b.data_ptr(), x.data_ptr(), 1e-10, 3000, 500)
        assert code == P.MG_OK, P.mg_status_string(code)
        assert info.true_relres <= 2e-10
        xd = O.direct_solve(prob)
        assert np.linalg.norm(x.cpu().numpy() - xd) / np.linalg.norm(xd) <= SOLVE_RTOL
    finally:
        P.mg_destroy(h)


@pytest.mark.parametrize("chain", ["scan", "cluster", "serial", "segmented"])
def test_sgs_chain_variants_full_size_vcycle(P, chain, monkeypatch):
    """Bench-sized coarse grid (257 blocks, p = 128) through each SGS chain
    implementation (parallel scan, 16-SM cluster, one CTA, segments joined by
    their products): the V-cycle agrees with the oracle."""
    monkeypatch.setenv("PINTMG_SGS_CHAIN", chain)
    prob = W.burgers(nx=128, n=256, seed=141)
    opts = dict(levels=2, nu_pre=1, nu_post=1, coarse_fixed_iters=2)
    h = P.mg_setup(prob, **opts)
    try:
        rd = _dev(prob.b)
        yd = torch.empty_like(rd)
        assert P.mg_vcycle(h, rd.data_ptr(), yd.data_ptr(), 0) == P.MG_OK
        torch.cuda.synchronize()
        yo = O.Hierarchy(prob, O.MGOptions(**opts)).precondition(prob.b)
        err = np.linalg.norm(yd.cpu().numpy() - yo) / np.linalg.norm(yo)
        assert err <= VCYCLE_RTOL, err
    finally:
        P.mg_destroy(h)


@pytest.mark.parametrize("chain", ["scan", "serial"])
def test_sgs_chain_variants_dense(P, chain, monkeypatch):
    monkeypatch.setenv("PINTMG_SGS_CHAIN", chain)
    prob = W.vdp(n=64, seed=161)
    opts = dict(levels=2, nu_pre=1, nu_post=1, coarse_fixed_iters=3)
    h = P.mg_setup(prob, **opts)
    try:
        rd = _dev(prob.b)
        yd = torch.empty_like(rd)
        assert P.mg_vcycle(h, rd.data_ptr(), yd.data_ptr(), 0) == P.MG_OK
        torch.cuda.synchronize()
        yo = O.Hierarchy(prob, O.MGOptions(**opts)).precondition(prob.b)
        assert np.linalg.norm(yd.cpu().numpy() - yo) / np.linalg.norm(yo) <= VCYCLE_RTOL
    finally:
        P.mg_destroy(h)


@pytest.mark.parametrize("kind", ["jacobi", "fgs", "bgs", "sgs"])
@pytest.mark.parametrize("levels", [1, 2])
def test_table1_coarse_preconditioners(P, kind, levels):
    """Every coarse preconditioner of Table 1 matches the oracle's inside a V-cycle
    (levels = 2) and as GMRES preconditioner on the whole system (levels = 1)."""
    prob = W.burgers(nx=20, n=16, seed=171)
    opts = dict(levels=levels, nu_pre=2, nu_post=2, coarse_fixed_iters=3)
    h = P.mg_setup(prob, coarse_precond=kind, **opts)
    try:
        rd = _dev(prob.b)
        yd = torch.empty_like(rd)
        assert P.mg_vcycle(h, rd.data_ptr(), yd.data_ptr(), 0) == P.MG_OK
        torch.cuda.synchronize()
        yo = O.Hierarchy(prob, O.MGOptions(coarse_precond=kind, **opts)).precondition(prob.b)
        assert np.linalg.norm(yd.cpu().numpy() - yo) / np.linalg.norm(yo) <= VCYCLE_RTOL
    finally:
        P.mg_destroy(h)


# ---------------------------------------------------------------- device-side loops

@pytest.mark.parametrize("basis", ["pair", "fp64"])
@pytest.mark.parametrize("case,restart", [(0, 7), (4, 9), (8, 7), (9, 5), (10, 7)])
def test_graph_solve_equals_host_loop(P, case, restart, basis):
    """A solve captured as one CUDA graph (FGMRES and coarse GMRES loops as
    conditional nodes) runs the same kernels in the same order as the host-driven
    loop: identical iterations and bitwise-identical solutions, also across a
    restart and on the second launch of the cached graph."""
    make, levels, nu_pre, nu_post, end_rule, omega, _ = _unpack(case)
    prob = make()
    xs, its = [], []
    for loops in (False, True):
        h = P.mg_setup(prob, levels=levels, nu_pre=nu_pre, nu_post=nu_post, end_rule=end_rule, omega=omega,
                       device_loops=loops, krylov_basis=basis)
        try:
            b = _dev(prob.b)
            for rep in range(2):
                x = torch.empty_like(b)
                code, info = P.fgmres_solve(h, b.data_ptr(), x.data_ptr(), 1e-10, 150, restart)
                assert code in (P.MG_OK, P.MG_NOT_CONVERGED), P.mg_status_string(code)
                xs.append(x.cpu().numpy())
                its.append((code, info.iters, info.coarse_iters, info.true_relres))
        finally:
            P.mg_destroy(h)
    assert its[0] == its[1] == its[2] == its[3]
    for k in range(1, 4):
        assert np.array_equal(xs[0], xs[k])


# ---------------------------------------------------------------- batched solves

def test_batched_solves_equal_single_solves(P):
    """Uneven systems (van der Pol and Burgers of different lengths, layouts and
    options) in one graph launch give the same results as one solve at a time."""
    specs = [
        (W.vdp(n=64, seed=201), dict(levels=3, nu_pre=1, nu_post=1)),
        (W.burgers(nx=40, n=32, seed=202), dict(levels=2, nu_pre=2, nu_post=2, omega=0.7)),
        (W.vdp(n=128, seed=203), dict(levels=2, nu_pre=2, nu_post=2, omega=0.7)),
        (W.burgers(nx=24, n=64, seed=204), dict(levels=3, nu_pre=4, nu_post=4, precision=P.MG_PRECISION_FP32)),
        (W.burgers(nx=16, n=16, seed=205), dict(levels=1)),
    ]
    hs, bs, xs, ref = [], [], [], []
    try:
        for prob, opts in specs:
            h = P.mg_setup(prob, **opts)
            hs.append(h)
            b = _dev(prob.b)
            x = torch.empty_like(b)
            code, info = P.fgmres_solve(h, b.data_ptr(), x.data_ptr(), 1e-10, 3000, 400)
            assert code == P.MG_OK
            ref.append((x.cpu().numpy(), info.iters))
            bs.append(b)
            xs.append(torch.empty_like(b))
        for rep in range(2):   # build, then reuse the cached batch graph
            for x in xs:
                x.fill_(float("nan"))
            code, infos = P.fgmres_solve_batched(hs, [b.data_ptr() for b in bs], [x.data_ptr() for x in xs],
                                                 1e-10, 3000, 400)
            assert code == P.MG_OK, P.mg_status_string(code)
            for (xr, it), x, info, (prob, _) in zip(ref, xs, infos, specs):
                assert info.status == P.MG_OK and info.iters == it
                assert np.array_equal(x.cpu().numpy(), xr)
                xd = O.direct_solve(prob)
                assert np.linalg.norm(x.cpu().numpy() - xd) / np.linalg.norm(xd) <= SOLVE_RTOL
        # after the batch, a single solve of one handle still works (recaptured)
        x = torch.empty_like(bs[0])
        code, info = P.fgmres_solve(hs[0], bs[0].data_ptr(), x.data_ptr(), 1e-10, 3000, 400)
        assert code == P.MG_OK and np.array_equal(x.cpu().numpy(), ref[0][0])
    finally:
        for h in hs:
            P.mg_destroy(h)


def test_batched_rejects_shared_handles(P):
    prob = W.vdp(n=16, seed=206)
    h = P.mg_setup(prob, levels=2)
    try:
        b = _dev(prob.b)
        x = torch.empty_like(b)
        code, _ = P.fgmres_solve_batched([h, h], [b.data_ptr()] * 2, [x.data_ptr()] * 2, 1e-8)
        assert code == P.MG_ERR_ARG
    finally:
        P.mg_destroy(h)


def _solve_x(P, prob, settings, restart=60, rtol=1e-10):
    h = P.mg_setup(prob, **settings)
    try:
        b = _dev(prob.b)
        x = torch.empty_like(b)
        st, info = P.fgmres_solve(h, b.data_ptr(), x.data_ptr(), rtol, 1500, restart)
        assert st == P.MG_OK, P.mg_status_string(st)
        return x.cpu().numpy(), info
    finally:
        P.mg_destroy(h)


def test_dot_blocking_is_bitwise_neutral(P, monkeypatch):
    """4, 8 or 16 basis vectors per dot-product CTA: the same partial sums in the same order."""
    prob = W.burgers(nx=40, n=32, seed=151)
    settings = dict(levels=2, nu_pre=2, nu_post=2, krylov_basis="fp64")
    xs = []
    for vb in ("4", "8", "16"):
        monkeypatch.setenv("PINTMG_DOT_VB", vb)
        xs.append(_solve_x(P, prob, settings))
    for x, info in xs[1:]:
        assert info.iters == xs[0][1].iters
        assert np.array_equal(x, xs[0][0])


@pytest.mark.parametrize("case", [0, 1, 3, 4, 5, 7, 8])
def test_pair_basis_reaches_the_direct_solution(P, case):
    """The FGMRES basis as FP32 pairs with compensated dot products and axpys
    (an option) against the FP64 basis (the default): both reach the direct solution to the
    solve tolerance, with iteration counts within one of each other (the basis
    is stored to ~48 bits, the Gram-Schmidt sums to about the same precision)."""
    make, levels, nu_pre, nu_post, end_rule, omega, _ = _unpack(case)
    prob = make()
    assert prob.size % 2 == 0
    xd = O.direct_solve(prob)
    res = {}
    for basis in ("pair", "fp64"):
        x, info = _solve_x(P, prob, dict(levels=levels, nu_pre=nu_pre, nu_post=nu_post, end_rule=end_rule,
                                         omega=omega, krylov_basis=basis))
        assert np.linalg.norm(x - xd) <= SOLVE_RTOL * np.linalg.norm(xd), basis
        assert info.true_relres <= 2e-10, (basis, info.true_relres)
        res[basis] = (x, info.iters)
    assert abs(res["pair"][1] - res["fp64"][1]) <= 1
    assert np.linalg.norm(res["pair"][0] - res["fp64"][0]) <= SOLVE_RTOL * np.linalg.norm(xd)


def test_pair_basis_over_many_multidot_chunks(P):
    """A vector long enough that the streamed multi-dot splits it into many
    chunks of several pipeline stages each, with a ragged last stage
    (n (4p + q) = 64 * 5 * 130 = 41,600 entries), unrestarted and across
    restarts.  The oracle's FGMRES needs 70 iterations at restart 40 and 174
    at restart 25 (at restart 9 it stagnates)."""
    prob = W.burgers(nx=130, n=64, seed=154)
    xd = O.direct_solve(prob)
    for restart, oracle_iters in ((40, 70), (25, 174)):
        x, info = _solve_x(P, prob, dict(levels=3, nu_pre=2, nu_post=2, krylov_basis="pair"), restart=restart)
        assert np.linalg.norm(x - xd) <= SOLVE_RTOL * np.linalg.norm(xd)
        assert abs(info.iters - oracle_iters) <= 3, (restart, info.iters)


@pytest.mark.parametrize("stall", ["1", "2"])
@pytest.mark.parametrize("loops", [True, False])
def test_pair_multidot_wait_runs_out_without_a_fault(P, monkeypatch, loops, stall):
    """Failure detection without a GPU fault.  Hook 1: the streamed multi-dot's
    producer issues no copies, so the consumers' mbarrier waits run out (2 s).
    Hook 2: a consumer warp gives up after its first stage, possibly after the
    producer has issued every copy; the producer still waits for its issued
    copies to land before the CTA exits.  Either way the kernel records the
    failure and returns, later launches of the solve return at once, and
    fgmres_solve reports MG_ERR_TIMEOUT.  The context stays usable: a normal
    solve afterwards reaches the direct solution."""
    import time
    prob = W.burgers(nx=40, n=32, seed=155)
    settings = dict(levels=2, nu_pre=1, nu_post=1, krylov_basis="pair", device_loops=loops)
    monkeypatch.setenv("PINTMG_TEST_PAIR_STALL", stall)
    h = P.mg_setup(prob, **settings)
    monkeypatch.delenv("PINTMG_TEST_PAIR_STALL")
    try:
        b = _dev(prob.b)
        x = torch.empty_like(b)
        t0 = time.time()
        code, info = P.fgmres_solve(h, b.data_ptr(), x.data_ptr(), 1e-10, 6, 6)
        assert code == P.MG_ERR_TIMEOUT, P.mg_status_string(code)
        assert time.time() - t0 < 30.0
    finally:
        P.mg_destroy(h)
    x, info = _solve_x(P, prob, dict(settings, levels=2))
    xd = O.direct_solve(prob)
    assert np.linalg.norm(x - xd) <= SOLVE_RTOL * np.linalg.norm(xd)


@pytest.mark.parametrize("n,levels", [(7, 1), (9, 1), (1, 1)])
def test_odd_lengths_take_the_unpaired_kernels(P, n, levels):
    """n (4p + q) odd (van der Pol, w = 9, n odd): the dot products and axpys run their one-entry-per-step
    variants; n = 1 is the single-block degenerate case.  Against the direct solve."""
    prob = W.vdp(n=n, seed=152 + n)
    assert (prob.size % 2 == 1) == (n % 2 == 1)
    x, info = _solve_x(P, prob, dict(levels=levels, nu_pre=1, nu_post=1))
    xd = O.direct_solve(prob)
    assert np.linalg.norm(x - xd) <= SOLVE_RTOL * np.linalg.norm(xd)


def test_restart_at_its_maximum(P):
    """restart = 512 (the largest the Hessenberg workspace holds) on a case needing a few hundred iterations."""
    prob = W.vdp(n=128, seed=153)
    x, info = _solve_x(P, prob, dict(levels=2, nu_pre=1, nu_post=1), restart=512)
    xd = O.direct_solve(prob)
    assert np.linalg.norm(x - xd) <= SOLVE_RTOL * np.linalg.norm(xd)
    assert info.iters >= 30


@pytest.mark.parametrize("precision", [0, 1])
def test_staged_block_solves_are_bitwise_the_same(P, monkeypatch, precision):
    """Block solves reading their coefficients from shared memory (staged by cp.async) or from global
    memory: the same values in the same arithmetic, so the same solution bit for bit."""
    prob = W.burgers(nx=128, n=64, seed=161)
    settings = dict(levels=3, nu_pre=2, nu_post=2, precision=precision)
    monkeypatch.setenv("PINTMG_TRI_PAIR", "0")      # one warp per block on every level
    xs = []
    for stage in ("1", "0"):
        monkeypatch.setenv("PINTMG_STAGE_TRI", stage)
        xs.append(_solve_x(P, prob, settings))
    assert xs[0][1].iters == xs[1][1].iters
    assert np.array_equal(xs[0][0], xs[1][0])


@pytest.mark.parametrize("nx,n,omega", [(128, 64, 1.0), (40, 32, 1.0), (64, 16, 0.7)])
def test_two_warp_block_solves_match(P, monkeypatch, nx, n, omega):
    """Two warps per time block (N r_u and Z r_z + V v - r_lambda formed in parallel, summed through shared
    memory) against one warp per block: the same solution up to the rounding of that sum's order."""
    prob = W.burgers(nx=nx, n=n, seed=162)
    settings = dict(levels=3 if n >= 32 else 2, nu_pre=2, nu_post=2, omega=omega)
    xs = []
    for pair in ("1", "0"):
        monkeypatch.setenv("PINTMG_TRI_PAIR", pair)
        xs.append(_solve_x(P, prob, settings))
    assert np.linalg.norm(xs[0][0] - xs[1][0]) <= 1e-11 * np.linalg.norm(xs[1][0])
    xd = O.direct_solve(prob)
    assert np.linalg.norm(xs[0][0] - xd) <= SOLVE_RTOL * np.linalg.norm(xd)


@pytest.mark.parametrize("case", [0, 4, 8])
def test_fp32_smoother_fp64_coarse_reaches_fp64_solution(P, case):
    """Smoother and transfers in FP32, coarse GMRES + SGS in FP64: FGMRES (FP64) still reaches the direct solution."""
    make, levels, nu_pre, nu_post, end_rule, omega, _ = _unpack(case)
    prob = make()
    x, info = _solve_x(P, prob, dict(levels=levels, nu_pre=nu_pre, nu_post=nu_post, end_rule=end_rule, omega=omega,
                                     precision=P.MG_PRECISION_FP32_SMOOTH), restart=100)
    xd = O.direct_solve(prob)
    assert np.linalg.norm(x - xd) <= SOLVE_RTOL * np.linalg.norm(xd)


@pytest.mark.parametrize("make,levels", [
    (lambda: W.vdp_paper(n=32, gamma=100.0), 3),
    (lambda: W.vdp_paper(n=32, gamma=1.0), 2),
    (lambda: W.burgers(nx=12, n=16, seed=171), 2),
])
def test_jacobi_spectral_radius_matches_dense_eigenvalues(P, make, levels):
    """mg_jacobi_radius (power iteration on the GPU) against the oracle's dense eigenvalues of I - D^-1 A~ on
    every level (Table 2's quantity)."""
    prob = make()
    h = P.mg_setup(prob, levels=levels)
    try:
        got = [P.mg_jacobi_radius(h, lv, iters=6000) for lv in range(levels)]
    finally:
        P.mg_destroy(h)
    raw = O.raw_from_problem(prob)
    for lv in range(levels):
        want = O.jacobi_spectral_radius(O.Level(raw))
        assert abs(got[lv] - want) <= 5e-3 * want, (lv, got[lv], want)
        raw = O.coarsen_raw(raw)


@pytest.mark.parametrize("nx,n,levels", [(32, 1, 1), (32, 2, 1), (40, 2, 2), (96, 4, 3)])
def test_few_time_blocks(P, nx, n, levels):
    """One to four time steps (the last block j = n carries only v and mu; block 0 has no v): the warp-pair
    and proportional-V block solves on their edge cases, against the direct solve."""
    prob = W.burgers(nx=nx, n=n, seed=181)
    x, info = _solve_x(P, prob, dict(levels=levels, nu_pre=2, nu_post=2))
    xd = O.direct_solve(prob)
    assert np.linalg.norm(x - xd) <= SOLVE_RTOL * np.linalg.norm(xd)


@pytest.mark.parametrize("nx,n,precision", [(64, 64, 0), (64, 100, 0), (64, 64, 1), (40, 48, 0), (512, 32, 0),
                                            (512, 48, 1)])
def test_segmented_sgs_chains_reach_the_solution(P, monkeypatch, nx, n, precision):
    """SGS chains as concurrent segment chains joined by the in-segment products (2 to 6 segments here, the
    last one shorter when n is not a multiple; p = 40 and 512 besides 64), as GMRES + SGS without
    multigrid, against the direct solve."""
    monkeypatch.setenv("PINTMG_SGS_CHAIN", "segmented")
    prob = W.burgers(nx=nx, n=n, seed=191)
    x, info = _solve_x(P, prob, dict(levels=1, precision=precision), restart=60)
    xd = O.direct_solve(prob)
    assert np.linalg.norm(x - xd) <= SOLVE_RTOL * np.linalg.norm(xd)
    h = P.mg_setup(prob, levels=1, precision=precision)
    try:
        assert P.mg_autotune(h)[0] == "segmented"       # a forced chain is kept
    finally:
        P.mg_destroy(h)
