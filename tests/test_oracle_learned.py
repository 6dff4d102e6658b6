"""Pins of the oracle's learned smoother (oracle/learned.py) against facts of
linear algebra and calculus, independent of its own formulas:

* a convolution whose only non-zero tap is the centre (identity) is the
  identity map; one whose only tap is +x (identity) is the lattice shift;
* the data gradient is the adjoint of the convolution, <conv(W, x), y> =
  <x, conv_backward_data(W, y)>, and the weight gradient its adjoint in W,
  <conv(W, x), y> = <W, conv_backward_weight(x, y)>;
* the back-propagated gradients of the loss agree with central finite
  differences (h = 1e-3 in FP64) to relative 1e-5;
* the first Adam step from zero moments moves every weight by lr sign(G) (up to
  eps), the bias-corrected closed form.
"""
import numpy as np

from oracle import learned as L

DIMS = (3, 3, 3, 4)   # x, y, z, t


def field(rng, c, batch=None):
    lx, ly, lz, lt = DIMS
    shp = (lt, lz, ly, lx, c) if batch is None else (batch, lt, lz, ly, lx, c)
    return rng.normal(size=shp)


def test_centre_and_shift_taps():
    rng = np.random.default_rng(1)
    x = field(rng, 24)
    W = np.zeros((L.NTAP, 24, 24))
    centre = L.taps().index((0, 0, 0, 0))
    W[centre] = np.eye(24)
    assert np.abs(L.conv(W, x) - x).max() == 0
    W[:] = 0
    W[L.taps().index((1, 0, 0, 0))] = np.eye(24)
    assert np.abs(L.conv(W, x) - np.roll(x, -1, axis=-2)).max() == 0


def test_backward_maps_are_adjoints():
    rng = np.random.default_rng(2)
    W = rng.normal(size=(L.NTAP, 32, 24))
    x = field(rng, 24, 2)
    y = field(rng, 32, 2)
    lhs = np.sum(L.conv(W, x) * y)
    assert abs(lhs - np.sum(x * L.conv_backward_data(W, y))) <= 1e-10 * abs(lhs)
    assert abs(lhs - np.sum(W * L.conv_backward_weight(x, y))) <= 1e-10 * abs(lhs)


def test_gradients_match_central_differences():
    rng = np.random.default_rng(3)
    Ws = [0.08 * rng.normal(size=(L.NTAP, co, ci)) for ci, co in zip(L.CHANNELS[:-1], L.CHANNELS[1:])]
    x = field(rng, 24, 2)
    t = 0.1 * field(rng, 24, 2)
    _, G = L.loss_and_grads(Ws, x, t)
    h = 1e-3
    for l in range(3):
        for _ in range(12):
            idx = tuple(rng.integers(0, s) for s in Ws[l].shape)
            w0 = Ws[l][idx]
            Ws[l][idx] = w0 + h
            lp, _ = L.loss_and_grads(Ws, x, t)
            Ws[l][idx] = w0 - h
            lm, _ = L.loss_and_grads(Ws, x, t)
            Ws[l][idx] = w0
            fd = (lp - lm) / (2 * h)
            assert abs(fd - G[l][idx]) <= 1e-5 * np.abs(G[l]).max(), (l, idx, fd, G[l][idx])


def test_gelu_gradient():
    z = np.linspace(-4, 4, 101)
    h = 1e-5
    fd = (L.gelu(z + h) - L.gelu(z - h)) / (2 * h)
    assert np.abs(fd - L.gelu_grad(z)).max() <= 1e-8


def test_first_adam_step():
    rng = np.random.default_rng(4)
    W = rng.normal(size=(5, 7))
    G = rng.normal(size=(5, 7))
    m, v = np.zeros_like(W), np.zeros_like(W)
    W1 = W.copy()
    L.adam_step(W1, G, m, v, 1, 1e-3)
    assert np.abs((W - W1) - 1e-3 * np.sign(G)).max() <= 1e-3 * 1e-8 / np.abs(G).min() + 1e-15
