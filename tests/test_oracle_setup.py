"""Pins of the oracle's setup and Rayleigh-Ritz helpers (Sec. 2.1; Algorithm 1)
on the 4^4 dense-check field against its LAPACK eigendecomposition:
orthonormalisation keeps the span; the Ritz step recovers eigenpairs that are
handed to it mixed by a unitary; the Rayleigh quotient of an eigenvector is its
eigenvalue with zero residual; the setup's test vectors move toward the low
modes of Q (inverse iteration with the two-grid method), far beyond what random
vectors of the same count hold."""
import numpy as np
import pytest

import dense4
import synth
from oracle import mg, rqi

DIMS = dense4.DENSE4["dims"]


def _low(n):
    """The n eigenpairs of smallest |lambda|, ties by lambda."""
    w, v = dense4.q_eigh()
    order = np.lexsort((w, np.abs(w)))[:n]
    return w[order], v[:, order]


def _field(x):
    return x.reshape(synth.gaussian_vectors(DIMS, 1, 0)[0].shape)


def test_orthonormalise_keeps_the_span():
    W0 = synth.gaussian_vectors(DIMS, 5, 21)
    W0[3] = 0.5 * W0[1] - 2.0 * W0[0] + 1e-3 * W0[3]       # a nearly dependent vector
    W = rqi.orthonormalise(W0)
    G, A = W.reshape(5, -1), W0.reshape(5, -1)
    assert np.abs(G @ G.conj().T - np.eye(5)).max() < 1e-13
    proj = (A @ G.conj().T) @ G                            # every W0 vector projected on span(W)
    assert np.abs(proj - A).max() < 1e-12 * np.abs(A).max()


def test_ritz_rotate_recovers_mixed_eigenpairs():
    _, op = dense4.field()
    w, v = _low(5)
    rng = np.random.default_rng(4)
    Umix, _ = np.linalg.qr(rng.standard_normal((5, 5)) + 1j * rng.standard_normal((5, 5)))
    W = np.array([_field(x) for x in (Umix @ v.T)])
    X, th = rqi.ritz_rotate(op, W)
    assert np.abs(th - w).max() < 1e-12
    for i in range(5):
        assert abs(np.vdot(v[:, i], X[i].ravel())) > 1 - 1e-12
    # the Rayleigh quotient of a returned vector: its eigenvalue, zero residual
    lam, res = rqi.rayleigh(op, X[0])
    assert abs(lam - w[0]) < 1e-12 and res < 1e-11


@pytest.mark.parametrize("iters", [0, 3])
def test_setup_moves_the_test_vectors_toward_the_low_modes(iters):
    """SAP smoothing of gamma5 w from zero, then `iters` two-grid inverse
    iterations, make the 8 test vectors hold on average a large part of each of
    the 8 lowest eigenvectors (8 random vectors hold 8 / 3072 of each), more
    after the iterations than before."""
    _, op = dense4.field()
    _, v = _low(8)
    params = dict(mg.DEFAULT_PARAMS, agg=(2, 2, 2, 2), ntv=8, sap_block=(2, 2, 2, 2), setup_iters=iters)
    W, B = rqi.setup(op, synth.uniform_vectors(DIMS, 8, 31), params)
    G = W.reshape(8, -1)
    assert np.abs(G @ G.conj().T - np.eye(8)).max() < 1e-13
    assert np.array_equal(B.W, W)                          # the preconditioner is built on them
    held = np.mean([np.linalg.norm(G.conj() @ v[:, i]) ** 2 for i in range(8)])
    assert held > (0.6 if iters else 0.15), held           # random: 0.0026
    if iters:
        W0, _ = rqi.setup(op, synth.uniform_vectors(DIMS, 8, 31), dict(params, setup_iters=0))
        G0 = W0.reshape(8, -1)
        held0 = np.mean([np.linalg.norm(G0.conj() @ v[:, i]) ** 2 for i in range(8)])
        assert held > 2 * held0
