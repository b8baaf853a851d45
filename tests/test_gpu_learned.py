"""Learned coarse correction on the GPU: the network's kernels against the CPU
oracle (forward FP32 and BF16, loss and gradient, Adam), recorded training
pairs against the oracle's coarse operator, FGMRES with the network attached,
and what a trained network gains over the method without it."""
import numpy as np
import pytest

from oracle import augmented as O
from oracle import learned as NL
from paper_2405_04808_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# FP32 forward: 4 layers of <= 672-term FP32 dot products (relative rounding
# ~ sqrt(672) * 2^-24 per layer): 1e-5 relative in the 2-norm.
FWD_FP32_RTOL = 1e-5
# BF16 storage of parameters and activations (8-bit significand, unit
# roundoff 2^-9 ~ 2e-3 per rounding, 5 roundings on a path): 2e-2.
FWD_BF16_RTOL = 2e-2
# FP32 gradient: sums over B*T*X positions of FP32 products: 1e-4 relative.
GRAD_RTOL = 1e-4


@pytest.fixture(scope="module")
def P():
    from paper_2405_04808_gb300 import pintmg
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    pintmg.lib()
    return pintmg


def _params(seed):
    p = W.net_init_params(seed)
    rng = np.random.default_rng(seed)
    p += 0.05 * rng.standard_normal(p.size)           # non-zero biases
    return p.astype(np.float32)


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


# the BF16 path runs the tcgen05 convolutions (128-position tiles of one time row, 4 rows per CTA): shapes
# with partial tiles in both directions, two tiles across, and several samples
@pytest.mark.parametrize("shape", [(1, 4, 5), (2, 9, 11), (3, 17, 40), (2, 13, 130), (1, 64, 256)])
def test_forward_matches_oracle(P, shape):
    B, T, X = shape
    p = _params(11)
    x = np.random.default_rng(5).standard_normal((B, 5, T, X)).astype(np.float32)
    want, _ = NL.forward(p.astype(np.float64), x.astype(np.float64))
    net = P.mg_net_create(p)
    try:
        xd = torch.tensor(x, device="cuda")
        y = torch.empty_like(xd)
        P.mg_net_forward(net, xd.data_ptr(), B, T, X, y.data_ptr(), bf16=False)
        assert _rel(y.cpu().numpy(), want) <= FWD_FP32_RTOL
        P.mg_net_forward(net, xd.data_ptr(), B, T, X, y.data_ptr(), bf16=True)
        assert _rel(y.cpu().numpy(), want) <= FWD_BF16_RTOL
        P.mg_net_forward(net, xd.data_ptr(), B, T, X, xd.data_ptr(), bf16=False)   # in place
        assert _rel(xd.cpu().numpy(), want) <= FWD_FP32_RTOL
    finally:
        P.mg_net_destroy(net)


@pytest.mark.parametrize("shape", [(1, 5, 8), (2, 7, 13), (4, 12, 33)])
def test_loss_and_gradient_match_oracle(P, shape):
    B, T, X = shape
    p = _params(12)
    rng = np.random.default_rng(6)
    x = rng.standard_normal((B, 5, T, X)).astype(np.float32)
    t = rng.standard_normal((B, 5, T, X)).astype(np.float32)
    loss_o, grad_o = NL.loss_and_grad(p.astype(np.float64), x.astype(np.float64), t.astype(np.float64))
    net = P.mg_net_create(p)
    try:
        xd, td = torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda")
        loss = P.mg_net_loss_grad(net, xd.data_ptr(), td.data_ptr(), B, T, X)
        g = P.mg_net_get_grad(net)
    finally:
        P.mg_net_destroy(net)
    assert abs(loss - loss_o) <= 1e-5 * loss_o
    assert _rel(g, grad_o) <= GRAD_RTOL
    # layer by layer too, so a small layer's error is not hidden by a large one's
    k = 0
    for Wt, b in NL.unpack(grad_o):
        for part in (Wt.ravel(), b):
            assert _rel(g[k:k + part.size], part) <= 10 * GRAD_RTOL
            k += part.size


def test_adam_steps_match_oracle(P):
    B, T, X = 2, 6, 10
    p = _params(13)
    rng = np.random.default_rng(7)
    x = rng.standard_normal((B, 5, T, X)).astype(np.float32)
    t = rng.standard_normal((B, 5, T, X)).astype(np.float32)
    net = P.mg_net_create(p)
    po = p.astype(np.float64)
    m = np.zeros_like(po)
    v = np.zeros_like(po)
    try:
        xd, td = torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda")
        for step in (1, 2, 3):
            P.mg_net_loss_grad(net, xd.data_ptr(), td.data_ptr(), B, T, X)
            g = P.mg_net_get_grad(net).astype(np.float64)   # the same gradient on both sides
            P.mg_net_adam_step(net, 1e-3)
            po, m, v = NL.adam_step(po, g, m, v, step, 1e-3)
            got = P.mg_net_get_params(net)
            assert np.max(np.abs(got - po)) <= 1e-6, step
    finally:
        P.mg_net_destroy(net)


@pytest.mark.parametrize("normalize", [False, True])
def test_training_step_matches_oracle(P, normalize):
    """mg_net_train with one minibatch holding every sample: one Adam step as
    the oracle computes it; normalised, the fresh network's parameters are
    the normalised network's, and the scalings are folded in at the end."""
    B, T, X = 3, 6, 9
    p = _params(14)
    x, t = _scaled_data(B, T, X)
    x64, t64 = x.astype(np.float64), t.astype(np.float64)
    p64 = p.astype(np.float64)
    if normalize:
        sx, sy = NL.channel_rms(x64), NL.channel_rms(t64)
        _, g = NL.loss_and_grad(p64, x64 / sx[None, :, None, None], t64 / sy[None, :, None, None])
        pn, _, _ = NL.adam_step(p64, g, np.zeros_like(g), np.zeros_like(g), 1, 1e-3)
        want = NL.fold(pn, sx, sy, -1)
    else:
        _, g = NL.loss_and_grad(p64, x64, t64)
        want, _, _ = NL.adam_step(p64, g, np.zeros_like(g), np.zeros_like(g), 1, 1e-3)
    net = P.mg_net_create(p)
    try:
        xd, td = torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda")
        P.mg_net_train(net, xd.data_ptr(), td.data_ptr(), B, T, X, B, 1, 1e-3, 0, normalize)
        got = P.mg_net_get_params(net).astype(np.float64)
    finally:
        P.mg_net_destroy(net)
    # Adam's first step moves each parameter by lr * g / (|g| + eps), i.e. by about lr * sign(g): where
    # the oracle's gradient is within the FP32 gradient's rounding of zero its sign is not determined
    # by the arithmetic, so those parameters are left out (a few of 49,829)
    decided = np.abs(g) > 1e-6 * np.linalg.norm(g)
    assert decided.mean() > 0.99
    assert np.max((np.abs(got - want) / np.maximum(1.0, np.abs(want)))[decided]) <= 2e-5


def _scaled_data(B, T, X):
    rng = np.random.default_rng(8)
    x = rng.standard_normal((B, 5, T, X)) * np.array([1e-2, 1.0, 20.0, 0.3, 4.0])[None, :, None, None]
    t = rng.standard_normal((B, 5, T, X)) * np.array([5.0, 0.2, 1.0, 60.0, 0.01])[None, :, None, None]
    return x.astype(np.float32), t.astype(np.float32)


def test_normalised_training_of_a_trained_network_keeps_its_function(P):
    """After an optimiser step, a normalised run of zero epochs maps the
    parameters to normalised coordinates and back: the function is unchanged."""
    B, T, X = 2, 5, 7
    x, t = _scaled_data(B, T, X)
    net = P.mg_net_create(_params(15))
    try:
        xd, td = torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda")
        P.mg_net_train(net, xd.data_ptr(), td.data_ptr(), B, T, X, B, 1, 1e-3, 0, False)
        before = P.mg_net_get_params(net)
        P.mg_net_train(net, xd.data_ptr(), td.data_ptr(), B, T, X, B, 0, 1e-3, 0, True)
        after = P.mg_net_get_params(net)
    finally:
        P.mg_net_destroy(net)
    assert np.allclose(after, before, rtol=1e-6, atol=1e-12)


def test_argument_errors(P):
    with pytest.raises(P.PintmgError):
        P.mg_net_create(np.zeros(10, dtype=np.float32))
    net = P.mg_net_create(_params(1))
    try:
        x = torch.zeros((1, 5, 4, 4), device="cuda")
        with pytest.raises(P.PintmgError):
            P.mg_net_forward(net, x.data_ptr(), 0, 4, 4, x.data_ptr())
        with pytest.raises(P.PintmgError):
            P.mg_net_adam_step(net, -1.0)
        prob = W.vdp_paper(n=16)                      # dense, p == q == 2: accepted
        h = P.mg_setup(prob, levels=2)
        try:
            P.mg_attach_coarse_net(h, net, admit=0.5)
            with pytest.raises(P.PintmgError):
                P.mg_attach_coarse_net(h, net, admit=1.5)
            with pytest.raises(P.PintmgError):        # recording needs host-driven loops
                P.mg_record_coarse(h, x.data_ptr(), x.data_ptr(), 1)
            P.mg_attach_coarse_net(h, None)
        finally:
            P.mg_destroy(h)
    finally:
        P.mg_net_destroy(net)


def _small_problem(seed):
    return W.burgers(nx=32, n=64, seed=seed)


SMALL = dict(levels=3, nu_pre=2, nu_post=2)


def test_recorded_pairs_are_coarse_solves(P):
    """Every recorded pair (r, y) has unit mean square, ||r|| = sqrt(N), and
    ||r - A_c y|| <= 1e-3 ||r|| with A_c the oracle's coarse operator (the
    coarse GMRES tolerance), up to FP32 storage."""
    from paper_2405_04808_gb300 import learned as L
    prob = _small_problem(31)
    R, Y = L.collect_pairs([prob], SMALL, max_pairs=40, restart=50)
    assert R.shape[0] == 40
    Ac = O.Hierarchy(prob, O.MGOptions(levels=3, nu_pre=2, nu_post=2)).levels[-1].A
    for k in range(R.shape[0]):
        r = R[k].double().cpu().numpy().ravel()
        y = Y[k].double().cpu().numpy().ravel()
        nr = np.sqrt(r.size)
        assert abs(np.linalg.norm(r) - nr) <= 1e-6 * nr
        assert np.linalg.norm(r - Ac @ y) <= (1e-3 + 1e-5) * nr


@pytest.mark.parametrize("bf16", [True, False])
def test_learned_fgmres_reaches_the_solution(P, bf16):
    """With a network attached (untrained: its proposals are measured and mostly
    rejected; admit 0.9 lets some through) FGMRES still reaches the direct
    solution; the graph and host-loop solves agree bit for bit."""
    prob = _small_problem(32)
    ref = O.direct_solve(prob)
    net = P.mg_net_create(_params(2))
    out = {}
    try:
        for loops in (False, True):
            h = P.mg_setup(prob, device_loops=loops, **SMALL)
            try:
                P.mg_attach_coarse_net(h, net, admit=0.9, bf16=bf16)
                b = torch.tensor(prob.b, dtype=torch.float64, device="cuda")
                x = torch.zeros_like(b)
                st, info = P.fgmres_solve(h, b.data_ptr(), x.data_ptr(), 1e-10, maxit=600, restart=100)
                assert st == P.MG_OK, info.true_relres
                out[loops] = (x.cpu().numpy(), info.iters, info.coarse_learned, info.coarse_iters)
            finally:
                P.mg_destroy(h)
    finally:
        P.mg_net_destroy(net)
    for x, *_ in out.values():
        assert np.linalg.norm(x - ref) <= 1e-9 * np.linalg.norm(ref)
    assert out[False][1:] == out[True][1:]
    assert np.array_equal(out[False][0], out[True][0])


def test_trained_network_gain(P, capsys):
    """Train on the plain method's coarse pairs from seeded runs, then solve
    held-out problems with and without the network.  What the network gains
    is measured and printed; the test asserts what must hold whatever the gain:
    training lowers the loss, the trained network's proposals reduce held-out
    coarse residuals more than the untrained one's, and FGMRES with the
    network converges to the same tolerance."""
    from paper_2405_04808_gb300 import learned as L
    train_probs = [_small_problem(40 + k) for k in range(6)]
    R, Y = L.collect_pairs(train_probs, SMALL, max_pairs=600, restart=50, per_problem=100)
    Rt, Yt = L.collect_pairs([_small_problem(90)], SMALL, max_pairs=50, restart=50)
    count, _, T, X = R.shape
    net0 = L.new_net(5)
    net = L.new_net(5)
    try:
        losses = L.train(net, R, Y, epochs=30, batch=16, lr=2e-3, seed=1)
        assert min(losses[-3:]) < 0.9 * losses[0], losses

        def reduction(nt):
            # rho = ||r - A_c net(r)|| / ||r|| on the held-out pairs, FP64 in the oracle's A_c
            Ac = O.Hierarchy(_small_problem(90), O.MGOptions(levels=3, nu_pre=2, nu_post=2)).levels[-1].A
            y = torch.empty_like(Rt)
            P.mg_net_forward(nt, Rt.data_ptr(), Rt.shape[0], T, X, y.data_ptr(), bf16=True)
            yy = y.double().cpu().numpy().reshape(Rt.shape[0], -1)
            rr = Rt.double().cpu().numpy().reshape(Rt.shape[0], -1)
            return np.array([np.linalg.norm(rr[k] - Ac @ yy[k]) / np.linalg.norm(rr[k]) for k in range(rr.shape[0])])

        rho0, rho = reduction(net0), reduction(net)
        assert np.median(rho) < np.median(rho0)
        stats = {}
        for name, nt in (("plain", None), ("learned", net)):
            its, lrn, crs = [], [], []
            for seed in (91, 92):
                prob = _small_problem(seed)
                h = P.mg_setup(prob, **SMALL)
                try:
                    if nt:
                        P.mg_attach_coarse_net(h, nt, admit=0.5, bf16=True)
                    b = torch.tensor(prob.b, dtype=torch.float64, device="cuda")
                    x = torch.zeros_like(b)
                    st, info = P.fgmres_solve(h, b.data_ptr(), x.data_ptr(), 1e-8, maxit=2000, restart=400)
                    assert st == P.MG_OK
                    assert info.true_relres <= 1e-8 * 1.01
                    its.append(info.iters)
                    lrn.append(info.coarse_learned)
                    crs.append(info.coarse_iters)
                finally:
                    P.mg_destroy(h)
            stats[name] = (its, lrn, crs)
        with capsys.disabled():
            print(f"\nlearned coarse correction (Burgers nx=32 nt=64, {count} pairs, 30 epochs): "
                  f"loss {losses[0]:.3g} -> {losses[-1]:.3g}; held-out median rho {np.median(rho0):.3f} -> "
                  f"{np.median(rho):.3f}; iterations plain {stats['plain'][0]} vs learned {stats['learned'][0]}, "
                  f"admitted coarse solves {stats['learned'][1]} of {stats['learned'][0]}, "
                  f"coarse GMRES iterations {stats['plain'][2]} -> {stats['learned'][2]}")
    finally:
        P.mg_net_destroy(net0)
        P.mg_net_destroy(net)


def _metric_problem(seed):
    return W.burgers(nx=8, n=16, seed=seed)


@pytest.mark.parametrize("B", [1, 3])
def test_metric_loss_and_gradient_match_oracle(P, B):
    """Residual-metric loss mean((A_c (net(x) - t))^2) with the coarse operator of a handle against the
    oracle's, A_c from the oracle's own hierarchy of the same problem."""
    prob = _metric_problem(21)
    h = P.mg_setup(prob, levels=2, nu_pre=1, nu_post=1)
    net = P.mg_net_create(_params(15))
    try:
        T, X = P.mg_coarse_shape(h)
        rng = np.random.default_rng(9)
        x = rng.standard_normal((B, 5, T, X)).astype(np.float32)
        t = rng.standard_normal((B, 5, T, X)).astype(np.float32)
        Ac = O.Hierarchy(prob, O.MGOptions(levels=2, nu_pre=1, nu_post=1)).levels[-1].A
        loss_o, grad_o = NL.metric_loss_and_grad(_params(15).astype(np.float64), x.astype(np.float64),
                                                 t.astype(np.float64), Ac)
        P.mg_net_set_metric(net, h)
        xd, td = torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda")
        loss = P.mg_net_loss_grad(net, xd.data_ptr(), td.data_ptr(), B, T, X)
        g = P.mg_net_get_grad(net)
        with pytest.raises(P.PintmgError):   # samples of another shape than the metric's coarse level
            P.mg_net_loss_grad(net, xd.data_ptr(), td.data_ptr(), 1, T - 1, X)
        P.mg_net_set_metric(net, None)   # back to the mean squared error
        assert abs(P.mg_net_loss_grad(net, xd.data_ptr(), td.data_ptr(), B, T, X) -
                   NL.loss_and_grad(_params(15).astype(np.float64), x.astype(np.float64),
                                    t.astype(np.float64))[0]) <= 1e-5 * loss_o + 1e-5
    finally:
        P.mg_net_destroy(net)
        P.mg_destroy(h)
    assert abs(loss - loss_o) <= 1e-5 * loss_o
    assert _rel(g, grad_o) <= GRAD_RTOL
    k = 0
    for Wt, b in NL.unpack(grad_o):
        for part in (Wt.ravel(), b):
            assert _rel(g[k:k + part.size], part) <= 10 * GRAD_RTOL
            k += part.size


def test_metric_training_step_matches_oracle(P):
    """A normalised mg_net_train step on the residual metric: the loss measures the unnormalised error
    (the targets' channel scales sy inside the metric), one Adam step, the scalings folded back."""
    prob = _metric_problem(22)
    h = P.mg_setup(prob, levels=2, nu_pre=1, nu_post=1)
    net = P.mg_net_create(_params(16))
    try:
        T, X = P.mg_coarse_shape(h)
        B = 3
        x, t = _scaled_data_shape(B, T, X)
        x64, t64, p64 = x.astype(np.float64), t.astype(np.float64), _params(16).astype(np.float64)
        Ac = O.Hierarchy(prob, O.MGOptions(levels=2, nu_pre=1, nu_post=1)).levels[-1].A
        sx, sy = NL.channel_rms(x64), NL.channel_rms(t64)
        _, g = NL.metric_loss_and_grad(p64, x64 / sx[None, :, None, None], t64 / sy[None, :, None, None], Ac, sy)
        pn, _, _ = NL.adam_step(p64, g, np.zeros_like(g), np.zeros_like(g), 1, 1e-3)
        want = NL.fold(pn, sx, sy, -1)
        P.mg_net_set_metric(net, h)
        xd, td = torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda")
        P.mg_net_train(net, xd.data_ptr(), td.data_ptr(), B, T, X, B, 1, 1e-3, 0, True)
        got = P.mg_net_get_params(net).astype(np.float64)
    finally:
        P.mg_net_destroy(net)
        P.mg_destroy(h)
    # as in the mean-squared-error step, parameters whose oracle gradient is within the FP32 gradient's
    # rounding of zero are left out; the metric spreads the gradient's magnitudes wider (A_c weights some
    # error components far more than others), so somewhat more of them (about 1.2 % here)
    decided = np.abs(g) > 1e-6 * np.linalg.norm(g)
    assert decided.mean() > 0.98
    assert np.max((np.abs(got - want) / np.maximum(1.0, np.abs(want)))[decided]) <= 2e-5


def _scaled_data_shape(B, T, X):
    rng = np.random.default_rng(10)
    x = rng.standard_normal((B, 5, T, X)) * np.array([1e-2, 1.0, 20.0, 0.3, 4.0])[None, :, None, None]
    t = rng.standard_normal((B, 5, T, X)) * np.array([5.0, 0.2, 1.0, 60.0, 0.01])[None, :, None, None]
    return x.astype(np.float32), t.astype(np.float32)


ADMIT = dict(levels=4, nu_pre=4, nu_post=4, omega=2.0 / 3.0, restrict="transpose")


def _admit_problem(seed):
    return W.burgers(nx=16, n=512, seed=seed)


def test_metric_trained_network_is_admitted(P, capsys):
    """Trained on the residual metric of one training system's coarse operator, the network's proposals
    pass the admission test (||r - A_c e|| <= 0.5 ||r||) on held-out systems: FGMRES takes them as coarse
    solves and still converges.  The mean-squared-error network of the same data is never admitted."""
    from paper_2405_04808_gb300 import learned as L
    train_probs = [_admit_problem(5001 + k) for k in range(12)]
    R, Y = L.collect_pairs(train_probs, ADMIT, max_pairs=480, rtol=1e-10, restart=60, per_problem=40)
    hm = P.mg_setup(train_probs[0], **ADMIT)
    nets = {}
    try:
        for name, metric in (("mse", None), ("metric", hm)):
            nets[name] = L.new_net(7, zero_output=metric is not None)
            L.train(nets[name], R, Y, epochs=20, batch=8, lr=1e-3, seed=2, metric=metric)
        stats = {}
        for name in ("plain", "mse", "metric"):
            its, lrn = [], []
            for seed in (5000, 4999):
                prob = _admit_problem(seed)
                h = P.mg_setup(prob, **ADMIT)
                try:
                    if name != "plain":
                        P.mg_attach_coarse_net(h, nets[name], admit=0.5, bf16=True)
                    b = torch.tensor(prob.b, dtype=torch.float64, device="cuda")
                    x = torch.zeros_like(b)
                    st, info = P.fgmres_solve(h, b.data_ptr(), x.data_ptr(), 1e-8, maxit=500, restart=60)
                    assert st == P.MG_OK and info.true_relres <= 1e-8 * 1.01
                    its.append(info.iters)
                    lrn.append(info.coarse_learned)
                finally:
                    P.mg_destroy(h)
            stats[name] = (its, lrn)
        with capsys.disabled():
            print(f"\nresidual-metric training (Burgers nx=16 nt=512, {R.shape[0]} pairs, 20 epochs): iterations "
                  f"plain {stats['plain'][0]}, mse {stats['mse'][0]} (admitted {stats['mse'][1]}), metric "
                  f"{stats['metric'][0]} (admitted {stats['metric'][1]})")
        assert sum(stats["metric"][1]) > 0
        assert sum(stats["metric"][1]) > sum(stats["mse"][1])
    finally:
        for nt in nets.values():
            P.mg_net_destroy(nt)
        P.mg_destroy(hm)
