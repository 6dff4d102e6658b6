"""The learned smoother, FP64 oracle: a three-layer 4D convolutional network
that maps a residual r to an approximation of the SAP correction, and its
training arithmetic (loss, gradients, Adam).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper's two-grid cycle smooths with SAP after the coarse correction (Sec. 2,
the smoother M of Eq. 2.3).  Here a network stands in for that smoother inside
the flexible outer FGMRES (Sec. 2.2), so a poor network changes the iteration
count, never the answer.  The paper has no learned smoother; the network, its
input normalisation and its training loss are this implementation's choices:

  input     x = r / ||r||, the 12 complex spin-colour components of every site
            as 24 real channels (channel 2k = Re r_k, 2k+1 = Im r_k)
  layer l   y(s)[o] = sum_{tap} sum_i W_l[tap][o][i] x(s + tap)[i], tap over the
            3^4 = 81 offsets in {-1, 0, 1}^4 (periodic lattice), no bias;
            tap index ((dt+1)*3 + (dz+1))*9 + (dy+1)*3 + (dx+1)
  network   f(x) = W_3 * g(W_2 * g(W_1 * x)),  24 -> 32 -> 32 -> 24 channels,
            g = GELU in its tanh form (Hendrycks and Gimpel 2016):
            g(z) = z/2 (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3)))
  smoother  M(r) = ||r|| f(r / ||r||)
  loss      L = 1/(2N) sum_n ||f(x_n) - t_n||^2 over N pairs, x_n = r_n/||r_n||,
            t_n = e_n/||r_n|| (e_n the SAP correction of r_n)
  Adam      Kingma and Ba 2015: m = b1 m + (1-b1) G, v = b2 v + (1-b2) G^2,
            W -= lr (m/(1-b1^t)) / (sqrt(v/(1-b2^t)) + eps)

Fields are numpy arrays [T, Z, Y, X, channels] (site order of the spinors).
"""
from __future__ import annotations

import numpy as np

NTAP = 81
CHANNELS = (24, 32, 32, 24)
GELU_C = np.sqrt(2.0 / np.pi)
GELU_A = 0.044715


def taps():
    """The 81 offsets (dx, dy, dz, dt) in tap order."""
    out = []
    for dt in (-1, 0, 1):
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    out.append((dx, dy, dz, dt))
    return out


def shift(x: np.ndarray, off) -> np.ndarray:
    """x(s + off) on the periodic lattice, x of shape [..., T, Z, Y, X, C]."""
    dx, dy, dz, dt = off
    return np.roll(x, shift=(-dt, -dz, -dy, -dx), axis=(-5, -4, -3, -2))


def conv(W: np.ndarray, x: np.ndarray) -> np.ndarray:
    """y(s)[o] = sum_tap sum_i W[tap][o][i] x(s + tap)[i]."""
    y = 0
    for t, off in enumerate(taps()):
        y = y + np.einsum("oi,...i->...o", W[t], shift(x, off))
    return y


def conv_backward_data(W: np.ndarray, dy: np.ndarray) -> np.ndarray:
    """dL/dx for y = conv(W, x): dx(s)[i] = sum_tap sum_o W[tap][o][i] dy(s - tap)[o]."""
    dx = 0
    for t, off in enumerate(taps()):
        back = tuple(-o for o in off)
        dx = dx + np.einsum("oi,...o->...i", W[t], shift(dy, back))
    return dx


def conv_backward_weight(x: np.ndarray, dy: np.ndarray) -> np.ndarray:
    """dL/dW[tap][o][i] = sum_s dy(s)[o] x(s + tap)[i] (summed over leading batch axes)."""
    out = np.zeros((NTAP, dy.shape[-1], x.shape[-1]))
    for t, off in enumerate(taps()):
        xs = shift(x, off)
        out[t] = dy.reshape(-1, dy.shape[-1]).T @ xs.reshape(-1, xs.shape[-1])
    return out


def gelu(z: np.ndarray) -> np.ndarray:
    return 0.5 * z * (1.0 + np.tanh(GELU_C * (z + GELU_A * z ** 3)))


def gelu_grad(z: np.ndarray) -> np.ndarray:
    """d gelu / dz of the tanh form."""
    u = GELU_C * (z + GELU_A * z ** 3)
    th = np.tanh(u)
    du = GELU_C * (1.0 + 3.0 * GELU_A * z * z)
    return 0.5 * (1.0 + th) + 0.5 * z * (1.0 - th * th) * du


def forward(Ws, x):
    """Network output and the intermediate values the gradients need."""
    z1 = conv(Ws[0], x)
    a1 = gelu(z1)
    z2 = conv(Ws[1], a1)
    a2 = gelu(z2)
    y = conv(Ws[2], a2)
    return y, (x, z1, a1, z2, a2)


def loss_and_grads(Ws, x, t):
    """L = 1/(2N) sum ||f(x) - t||^2 over the N samples on the leading axis, and
    its gradients with respect to the three weight tensors (back-propagation)."""
    n = x.shape[0]
    y, (x0, z1, a1, z2, a2) = forward(Ws, x)
    d = y - t
    L = 0.5 * float(np.sum(d * d)) / n
    dy = d / n
    g3 = conv_backward_weight(a2, dy)
    da2 = conv_backward_data(Ws[2], dy)
    dz2 = da2 * gelu_grad(z2)
    g2 = conv_backward_weight(a1, dz2)
    da1 = conv_backward_data(Ws[1], dz2)
    dz1 = da1 * gelu_grad(z1)
    g1 = conv_backward_weight(x0, dz1)
    return L, [g1, g2, g3]


def adam_step(W, G, m, v, step: int, lr: float, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update of W (all arrays updated in place); step counts from 1."""
    m *= b1
    m += (1 - b1) * G
    v *= b2
    v += (1 - b2) * G * G
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    W -= lr * mh / (np.sqrt(vh) + eps)


def spinor_to_channels(psi: np.ndarray) -> np.ndarray:
    """[..., T, Z, Y, X, 4, 3] complex -> [..., T, Z, Y, X, 24] real (Re, Im interleaved)."""
    f = psi.reshape(psi.shape[:-2] + (12,))
    return np.stack([f.real, f.imag], axis=-1).reshape(psi.shape[:-2] + (24,))


def channels_to_spinor(x: np.ndarray) -> np.ndarray:
    f = x.reshape(x.shape[:-1] + (12, 2))
    return (f[..., 0] + 1j * f[..., 1]).reshape(x.shape[:-1] + (4, 3))


def smoother(Ws, r: np.ndarray) -> np.ndarray:
    """M(r) = ||r|| f(r / ||r||) for one spinor field r."""
    nr = float(np.sqrt(np.real(np.vdot(r, r))))
    if nr == 0:
        return np.zeros_like(r)
    y, _ = forward(Ws, spinor_to_channels(r / nr)[None])
    return nr * channels_to_spinor(y[0])
