"""Pins of the oracle's approximate low-mode averaging (oracle/lma.py, Sec. 3.1
and 3.2) on the dense 4^4 field, against facts of linear algebra:

* exact eigenvectors (LAPACK eigh of the dense Q): A is diag(lambda), the
  corrected inverse is Q^-1_low = sum v_i <v_i| / lambda_i of Sec. 3.1, R~ is the
  orthogonal projector 1 - sum |v_i><v_i|, and L_low(t) = sum_i (1/lambda_i)
  sum_{x in t} |v_i(x)|^2;
* approximate vectors (eigenvectors with added noise): R~ is a projector
  (R~^2 = R~), it annihilates every Q v_i, and the trace of Q Q~^-1_low over the
  whole space is N (reading: the paper writes 12 N_eig there; for N orthonormal
  vectors in the full spin-colour space the trace of the rank-N operator
  Q Q~^-1_low = Q V A^-1 V^dag is tr(A^-1 A) = N);
* sum_t L_low(t) = tr(A^-1) (the vectors are orthonormal);
* the cutoff keeps exactly the pairs with eps / |lambda| <= c.
"""
import numpy as np

from oracle import lma
from tests import dense4


def exact(n=6):
    w, v = dense4.q_eigh()
    order = np.lexsort((w, np.abs(w)))[:n]
    lx, ly, lz, lt = dense4.DENSE4["dims"]
    V = v[:, order].T.reshape(n, lt, lz, ly, lx, 4, 3)
    return w[order], V


def test_exact_eigenvectors_give_the_exact_low_mode_objects():
    op = dense4.field()[1]
    w, V = exact()
    lam, eps, QV = lma.approximate_modes(op, V)
    assert np.abs(lam - w).max() <= 1e-12 and eps.max() <= 1e-12
    A = lma.a_matrix(V, QV)
    assert np.abs(A - np.diag(w)).max() <= 1e-12
    Ainv = np.linalg.inv(A)
    x = np.random.default_rng(1).normal(size=V.shape[1:]) + 0j
    want = sum(np.vdot(v, x) / l * v for v, l in zip(V, w))
    assert np.abs(lma.low_inverse_apply(V, Ainv, x) - want).max() <= 1e-10
    proj = x - sum(np.vdot(v, x) * v for v in V)
    assert np.abs(lma.oblique_projector_apply(V, QV, Ainv, x) - proj).max() <= 1e-10
    Lt = lma.low_mode_loop(V, Ainv)
    want_L = [sum((np.abs(v[t]) ** 2).sum() / l for v, l in zip(V, w)) for t in range(V.shape[1])]
    assert np.abs(Lt - np.array(want_L)).max() <= 1e-10


def test_approximate_vectors_projector_identities():
    op = dense4.field()[1]
    w, V0 = exact()
    rng = np.random.default_rng(2)
    V = lma.orthonormalise(V0 + 1e-2 * (rng.normal(size=V0.shape) + 1j * rng.normal(size=V0.shape)))
    lam, eps, QV = lma.approximate_modes(op, V)
    assert eps.max() > 1e-4   # really approximate
    A = lma.a_matrix(V, QV)
    Ainv = np.linalg.inv(A)
    x = rng.normal(size=V.shape[1:]) + 1j * rng.normal(size=V.shape[1:])
    Rx = lma.oblique_projector_apply(V, QV, Ainv, x)
    assert np.linalg.norm(lma.oblique_projector_apply(V, QV, Ainv, Rx) - Rx) <= 1e-10 * np.linalg.norm(x)
    for q in QV:
        assert np.linalg.norm(lma.oblique_projector_apply(V, QV, Ainv, q)) <= 1e-10 * np.linalg.norm(q)
    # tr(Q Q~^-1_low) over the full space with the dense Q
    Qm = dense4.q_matrix()
    Vm = V.reshape(len(V), -1).T
    tr = np.trace(Qm @ Vm @ Ainv @ Vm.conj().T)
    assert abs(tr - len(V)) <= 1e-10
    assert abs(np.sum(lma.low_mode_loop(V, Ainv)) - np.trace(Ainv)) <= 1e-10 * abs(np.trace(Ainv))


def test_cutoff():
    lam = np.array([0.1, -0.2, 0.05, 0.3])
    eps = np.array([0.01, 0.2, 0.04, 0.3])
    # relative accuracies 0.1, 1.0, 0.8, 1.0
    assert list(lma.cutoff(lam, eps, 0.75)) == [0]
    assert list(lma.cutoff(lam, eps, 0.8)) == [0, 2]
    assert list(lma.cutoff(lam, eps, 1.0)) == [0, 1, 2, 3]
