"""Pins of the CPU oracle of the learned coarse correction's network."""
import numpy as np
import pytest

from oracle import learned as NL
from paper_2405_04808_gb300 import workloads as W


def test_parameter_count_is_about_50k():
    assert NL.param_count() == 49829


def test_convolution_is_scipy_correlation():
    """One input and one output channel: zero-padded 'same' correlation."""
    signal = pytest.importorskip("scipy.signal")
    rng = np.random.default_rng(0)
    x = rng.standard_normal((1, 1, 9, 13))
    W = rng.standard_normal((1, 1, 3, 7))
    y = NL.conv_forward(x, W, np.array([0.25]))
    want = signal.correlate2d(x[0, 0], W[0, 0], mode="same", boundary="fill") + 0.25
    assert np.allclose(y[0, 0], want, rtol=0, atol=1e-12)


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    p = W.net_init_params(3)
    p += 0.05 * rng.standard_normal(p.size)          # non-zero biases
    x = rng.standard_normal((2, 5, 6, 9))
    t = rng.standard_normal((2, 5, 6, 9))
    loss, g = NL.loss_and_grad(p, x, t)
    idx = rng.choice(p.size, 40, replace=False)
    for i in idx:
        e = np.zeros_like(p)
        e[i] = 1e-6
        fd = (NL.loss_and_grad(p + e, x, t)[0] - NL.loss_and_grad(p - e, x, t)[0]) / 2e-6
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_adam_two_steps_by_hand():
    """lr 0.1, beta 0.9 / 0.999: the first step moves every parameter by lr * sign(g)."""
    p = np.array([1.0, -2.0])
    g = np.array([0.5, -4.0])
    p1, m, v = NL.adam_step(p, g, np.zeros(2), np.zeros(2), 1, 0.1, eps=0.0)
    assert np.allclose(p1, [0.9, -1.9], atol=1e-15)
    p2, m, v = NL.adam_step(p1, g, m, v, 2, 0.1, eps=0.0)
    assert np.allclose(p2, [0.8, -1.8], atol=1e-12)   # constant gradient: mhat / sqrt(vhat) = sign(g)


def test_seeded_initialisation_layout():
    """The shared generator's layout agrees with the oracle's unpacking: biases zero, weights within He bounds."""
    p = W.net_init_params(7)
    assert p.size == NL.param_count()
    for (Wt, b), (ci, kt, kx) in zip(NL.unpack(p), [(5, 3, 7), (32, 3, 7), (32, 3, 7), (32, 3, 7)]):
        assert np.all(b == 0.0)
        lim = np.sqrt(6.0 / (ci * kt * kx))
        assert np.abs(Wt).max() <= lim and np.abs(Wt).max() > 0.9 * lim
    assert np.array_equal(p, W.net_init_params(7)) and not np.array_equal(p, W.net_init_params(8))


def test_delta_kernels_compose_to_the_activation():
    """Centre-tap identity kernels: the network is leaky^3 elementwise (slope 0.1 -> 1e-3 on negatives)."""
    layers = []
    for ci, co in zip(NL.CHANNELS[:-1], NL.CHANNELS[1:]):
        Wt = np.zeros((co, ci, NL.KT, NL.KX))
        for c in range(min(ci, co)):
            Wt[c, c, NL.KT // 2, NL.KX // 2] = 1.0
        layers += [Wt.ravel(), np.zeros(co)]
    p = np.concatenate(layers)
    x = np.random.default_rng(4).standard_normal((1, 5, 4, 6))
    y, _ = NL.forward(p, x)
    assert np.allclose(y, np.where(x > 0, x, 1e-3 * x), atol=1e-15)


def test_fold_is_the_normalised_network():
    """net'(x / sx) = net(x) / sy per channel, and folding back restores the parameters."""
    rng = np.random.default_rng(9)
    p = W.net_init_params(4) + 0.05 * rng.standard_normal(NL.param_count())
    x = rng.standard_normal((2, 5, 5, 8)) * np.array([1e-3, 2.0, 30.0, 0.5, 7.0])[None, :, None, None]
    sx = NL.channel_rms(x)
    sy = np.array([0.1, 3.0, 50.0, 1e-2, 8.0])
    pn = NL.fold(p, sx, sy, +1)
    y, _ = NL.forward(p, x)
    yn, _ = NL.forward(pn, x / sx[None, :, None, None])
    assert np.allclose(yn, y / sy[None, :, None, None], rtol=1e-12, atol=1e-14)
    assert np.allclose(NL.fold(pn, sx, sy, -1), p, rtol=1e-14, atol=0)
    assert np.allclose(NL.channel_rms(np.ones((3, 5, 2, 2)) * 2.0), 2.0)


def test_batch_workload_mix():
    """The batched workload: 64 systems, half van der Pol (nt 512 ... 16384), half Burgers (nx 64/128/256 x nt 512 ...
    4096), distinct seeds, 4 levels each (every nt divisible by 8).  Built from small counts here (the forward
    solves of the large members take seconds)."""
    from paper_2405_04808_gb300.workloads import _batch_member
    shapes = []
    for k in (0, 1, 2, 3, 22, 23):
        prob, opts = _batch_member(k, 6000)
        assert opts["levels"] == 4 and prob.n % 8 == 0
        shapes.append((prob.kind, prob.n, prob.p))
    assert shapes[0] == ("dense", 512, 2) and shapes[2] == ("dense", 1024, 2)
    assert shapes[1] == ("tridiag", 512, 64) and shapes[3] == ("tridiag", 512, 128)
    assert shapes[4] == ("dense", 16384, 2) and shapes[5] == ("tridiag", 4096, 256)


def test_launch_list_summary(tmp_path):
    from paper_2405_04808_gb300.profile_cases import summarize
    f = tmp_path / "l.csv"
    f.write_text('==PROF== x\n"ID","Kernel Name","Metric Name","Metric Unit","Metric Value"\n'
                 '"0","void k_a<double>(int)","gpu__time_duration.sum","usecond","3"\n'
                 '"1","k_b","gpu__time_duration.sum","nsecond","1,000"\n'
                 '"2","void k_a<double>(int)","gpu__time_duration.sum","usecond","6"\n')
    out = summarize(str(f))
    assert "| k_a<double> | 2 | 0.009 | 90.0 % |" in out and "| k_b | 1 | 0.001 | 10.0 % |" in out


def test_metric_loss_with_identity_is_the_mean_squared_error():
    """A = I and unit scales reduce the residual-metric loss to the plain mean squared error."""
    sp = pytest.importorskip("scipy.sparse")
    rng = np.random.default_rng(5)
    p = W.net_init_params(4) + 0.02 * rng.standard_normal(NL.param_count())
    x = rng.standard_normal((2, 5, 4, 8))
    t = rng.standard_normal((2, 5, 4, 8))
    l0, g0 = NL.loss_and_grad(p, x, t)
    l1, g1 = NL.metric_loss_and_grad(p, x, t, sp.identity(5 * 4 * 8, format="csr"))
    assert abs(l1 - l0) <= 1e-14 * l0 and np.allclose(g1, g0, rtol=0, atol=1e-15 * np.abs(g0).max())


def test_metric_gradients_match_finite_differences():
    """A random sparse non-symmetric A and per-channel scales: central differences of the loss."""
    sp = pytest.importorskip("scipy.sparse")
    rng = np.random.default_rng(6)
    p = W.net_init_params(5) + 0.05 * rng.standard_normal(NL.param_count())
    x = rng.standard_normal((2, 5, 4, 7))
    t = rng.standard_normal((2, 5, 4, 7))
    N = 5 * 4 * 7
    A = sp.random(N, N, density=0.05, random_state=7, format="csr") + sp.identity(N)
    scale = np.array([0.5, 2.0, 1.0, 3.0, 0.25])
    loss, g = NL.metric_loss_and_grad(p, x, t, A, scale)
    for i in rng.choice(p.size, 40, replace=False):
        e = np.zeros_like(p)
        e[i] = 1e-6
        fd = (NL.metric_loss_and_grad(p + e, x, t, A, scale)[0] -
              NL.metric_loss_and_grad(p - e, x, t, A, scale)[0]) / 2e-6
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_metric_loss_is_the_admission_residual():
    """With the coarse operator of a small Burgers hierarchy and targets y = A^-1 r (sparse direct
    solve), the loss is the mean squared residual r - A net(r) of the proposals the admission test
    measures."""
    spla = pytest.importorskip("scipy.sparse.linalg")
    from oracle import augmented as O
    prob = W.burgers(nx=8, n=16, seed=11)
    Lc = O.Hierarchy(prob, O.MGOptions(levels=2)).levels[-1]
    A = Lc.A.tocsc()
    T, X = Lc.n, Lc.p
    rng = np.random.default_rng(8)
    r = rng.standard_normal((3, 5 * T * X))
    y = np.stack([spla.spsolve(A, ri) for ri in r])
    p = W.net_init_params(6) + 0.05 * rng.standard_normal(NL.param_count())
    xr, yr = r.reshape(3, 5, T, X), y.reshape(3, 5, T, X)
    loss, _ = NL.metric_loss_and_grad(p, xr, yr, A)
    e = NL.forward(p, xr)[0].reshape(3, -1)
    res = r - (A @ e.T).T
    assert abs(loss - np.sum(res * res) / r.size) <= 1e-9 * loss
