"""CPU oracle of the learned coarse-grid correction's network (test infrastructure only).

The network maps a coarse residual to a proposed coarse correction.  A coarse
vector in the type-major layout (u, v, z, lambda, mu; each n_c x p) is a
(5, n_c, p) tensor: five channels over (time, space).  The network is four
2-D convolutions over (time, space) with a 3 x 7 kernel and "same" zero
padding, channels 5 -> 32 -> 32 -> 32 -> 5, a leaky rectifier (slope 0.1)
after the first three; 49,829 parameters.  Training minimises, with Adam,
either the mean squared error against the plain method's coarse solutions or
the residual-metric loss mean((A_c (net(x) - y))^2), which measures the error
through the coarse operator A_c as the admission test does.

Everything here is plain numpy in FP64: the reference the GPU kernels'
forward pass, gradients and optimiser step are checked against.  Pins:
tests/test_oracle_learned.py (scipy correlation, finite differences).
"""
from __future__ import annotations

import numpy as np

CHANNELS = (5, 32, 32, 32, 5)
KT, KX = 3, 7
SLOPE = 0.1


def layer_shapes(channels=CHANNELS, kt=KT, kx=KX):
    return [((co, ci, kt, kx), (co,)) for ci, co in zip(channels[:-1], channels[1:])]


def param_count(channels=CHANNELS, kt=KT, kx=KX):
    return sum(int(np.prod(w)) + b[0] for w, b in layer_shapes(channels, kt, kx))


def unpack(params, channels=CHANNELS, kt=KT, kx=KX):
    """Flat parameters -> [(W, b)] (W: co x ci x kt x kx, then b: co), layer by layer."""
    out, k = [], 0
    for wshape, bshape in layer_shapes(channels, kt, kx):
        nw = int(np.prod(wshape))
        W = params[k:k + nw].reshape(wshape)
        k += nw
        b = params[k:k + bshape[0]]
        k += bshape[0]
        out.append((W, b))
    assert k == params.size
    return out


def conv_forward(x, W, b):
    """y[b,o,t,s] = bias[o] + sum_{c,i,j} W[o,c,i,j] x[b,c,t+i-kt//2, s+j-kx//2] (zero outside)."""
    B, C, T, X = x.shape
    O, C2, kt, kx = W.shape
    assert C == C2
    pt, px = kt // 2, kx // 2
    xp = np.zeros((B, C, T + 2 * pt, X + 2 * px))
    xp[:, :, pt:pt + T, px:px + X] = x
    y = np.zeros((B, O, T, X))
    for i in range(kt):
        for j in range(kx):
            y += np.einsum("oc,bctx->botx", W[:, :, i, j], xp[:, :, i:i + T, j:j + X])
    return y + b[None, :, None, None]


def conv_backward(x, W, gy):
    """Gradients of sum(gy * conv_forward(x, W, b)) w.r.t. x, W, b."""
    B, C, T, X = x.shape
    O, _, kt, kx = W.shape
    pt, px = kt // 2, kx // 2
    xp = np.zeros((B, C, T + 2 * pt, X + 2 * px))
    xp[:, :, pt:pt + T, px:px + X] = x
    gxp = np.zeros_like(xp)
    gW = np.zeros_like(W)
    for i in range(kt):
        for j in range(kx):
            gW[:, :, i, j] = np.einsum("botx,bctx->oc", gy, xp[:, :, i:i + T, j:j + X])
            gxp[:, :, i:i + T, j:j + X] += np.einsum("oc,botx->bctx", W[:, :, i, j], gy)
    gb = gy.sum(axis=(0, 2, 3))
    return gxp[:, :, pt:pt + T, px:px + X], gW, gb


def forward(params, x):
    """Network output and the pre-activations of every layer."""
    layers = unpack(params)
    pre, h = [], x
    for k, (W, b) in enumerate(layers):
        z = conv_forward(h, W, b)
        pre.append((h, z))
        h = z if k == len(layers) - 1 else np.where(z > 0, z, SLOPE * z)
    return h, pre


def loss_and_grad(params, x, target):
    """L = mean((net(x) - target)^2) and dL/dparams (flat, same layout)."""
    y, pre = forward(params, x)
    diff = y - target
    loss = float(np.mean(diff * diff))
    return loss, _backward(params, pre, 2.0 * diff / diff.size)


def metric_loss_and_grad(params, x, target, A, scale=None):
    """Residual-metric loss of a coarse correction and dL/dparams.

    A proposal e = net(x) for the coarse system A e = r is admitted by the
    size of its residual, so the loss measures the error e - y (y the plain
    method's coarse solution, A y = r) through the coarse operator:
        d_b = scale * (net(x_b) - target_b)   (scale per channel; 1 if None)
        L = sum_b ||A d_b||^2 / n,            n = number of output entries,
    d_b flattened in the type-major coarse layout (channel = variable type,
    then time, then space).  dL/dnet(x_b) = scale * 2 A^T A d_b / n.  A is
    a scipy sparse (or dense) matrix of the coarse level in that layout."""
    y, pre = forward(params, x)
    B = y.shape[0]
    sc = np.ones(y.shape[1]) if scale is None else np.asarray(scale, dtype=np.float64)
    d = ((y - target) * sc[None, :, None, None]).reshape(B, -1)
    u = np.asarray((A @ d.T)).T
    n = y.size
    loss = float(np.sum(u * u) / n)
    ge = (2.0 / n) * np.asarray(A.T @ u.T).T
    ge = ge.reshape(y.shape) * sc[None, :, None, None]
    return loss, _backward(params, pre, ge)


def _backward(params, pre, g):
    """dL/dparams (flat) from g = dL/d(net output) and the forward pass's pre-activations."""
    layers = unpack(params)
    grads = []
    for k in range(len(layers) - 1, -1, -1):
        h, z = pre[k]
        if k != len(layers) - 1:
            g = np.where(z > 0, g, SLOPE * g)
        gx, gW, gb = conv_backward(h, layers[k][0], g)
        grads.append((gW, gb))
        g = gx
    flat = []
    for gW, gb in reversed(grads):
        flat += [gW.ravel(), gb.ravel()]
    return np.concatenate(flat)


def adam_step(params, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba 2015) with bias correction; returns new (params, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return params - lr * mhat / (np.sqrt(vhat) + eps), m, v


def channel_rms(x):
    """Root mean square of each channel over samples and positions (1 for an all-zero channel)."""
    r = np.sqrt(np.mean(np.asarray(x, dtype=np.float64) ** 2, axis=(0, 2, 3)))
    return np.where(r > 0, r, 1.0)


def fold(params, sx, sy, direction):
    """Parameters of the per-channel normalised network and back.

    direction +1: the network net' with net'(x / sx) = net(x) / sy (first
    layer's weights times sx of their input channel, last layer's weights and
    biases over sy of their output channel); -1 undoes it."""
    layers = [(Wt.copy(), b.copy()) for Wt, b in unpack(params)]
    W0, b0 = layers[0]
    W3, b3 = layers[-1]
    if direction > 0:
        W0 *= sx[None, :, None, None]
        W3 /= sy[:, None, None, None]
        b3 /= sy
    else:
        W0 /= sx[None, :, None, None]
        W3 *= sy[:, None, None, None]
        b3 *= sy
    return np.concatenate([a.ravel() for Wt, b in layers for a in (Wt, b)])
