"""Pins of the oracle's completeness check (oracle/chefsi.py: Chebyshev-filtered
subspace iteration on Q^2 for the eigenpairs of smallest |lambda|) against
results fixed by linear algebra alone:

* a Hermitian matrix with a planted spectrum (random unitary basis) holding a
  pair that differs by a relative 1e-8, an exactly degenerate pair +-lambda of
  equal modulus and a threefold eigenvalue: every planted value is found, the
  near-degenerate pair as two pairs, and the eigenvectors span the planted
  eigenspaces;
* the free field on 4^4 (periodic): the 12 lowest |lambda| are the p = 0 modes,
  exactly +-m0, six of each sign (closed form, Sec. 2 operator at U = 1);
* the random 4^4 field of the dense workload: the 8 lowest pairs against LAPACK's
  eigh of the 3072 x 3072 matrix (eigenvalues, residuals, overlaps).
"""
import numpy as np

import synth
from oracle import chefsi, dense, dirac


def planted(n=300, seed=3):
    rng = np.random.default_rng(seed)
    d = np.concatenate([
        [0.02, 0.02 * (1 + 1e-8), -0.03, 0.03, 0.05, 0.05, 0.05, -0.07],
        rng.uniform(0.15, 4.0, n - 8) * rng.choice([-1.0, 1.0], n - 8),
    ])
    G, _ = np.linalg.qr(rng.normal(size=(n, n)) + 1j * rng.normal(size=(n, n)))
    return G @ np.diag(d) @ G.conj().T, d, G


def test_planted_spectrum_with_near_degenerate_pair():
    M, d, G = planted()
    n = M.shape[0]
    apply = lambda X: (X.reshape(X.shape[0], -1) @ M.T).reshape(X.shape)
    rng = np.random.default_rng(11)
    start = rng.normal(size=(14, n)) + 1j * rng.normal(size=(14, n))
    k = 8
    lam, V, res, info = chefsi.lowest_abs_eigenpairs(apply, start, k, 4.0, degree=60, tol=1e-12)
    assert info["converged"]
    want = d[np.lexsort((d, np.abs(d)))][:k]
    assert np.abs(lam - want).max() <= 1e-13
    assert np.all(res <= 1e-12)
    # the near-degenerate pair: two distinct values, and the two vectors span the
    # planted two-dimensional eigenspace
    assert lam[1] - lam[0] > 0.5 * 0.02 * 1e-8
    Pw = G[:, :2] @ G[:, :2].conj().T
    Pg = V[:2].T @ V[:2].conj()
    assert np.linalg.norm(Pw - Pg) <= 1e-9
    # +-0.03 of equal modulus, and the threefold 0.05
    for idx in ([2, 3], [4, 5, 6]):
        Pw = G[:, idx] @ G[:, idx].conj().T
        sel = [i for i in range(k) if abs(abs(lam[i]) - abs(d[idx[0]])) < 1e-9]
        Pg = V[sel].T @ V[sel].conj()
        assert len(sel) == len(idx) and np.linalg.norm(Pw - Pg) <= 1e-9


def test_free_field_p0_modes_twelvefold():
    dims, m0 = (4, 4, 4, 4), -0.4
    op = dirac.WilsonClover(synth.unit_gauge(dims), m0, 1.0)
    start = synth.gaussian_vectors(dims, 16, 21)
    lam, V, res, info = chefsi.lowest_abs_eigenpairs(op.Q, start, 12, chefsi.q_norm_bound(op), degree=30)
    assert info["converged"]
    assert np.abs(np.abs(lam) - abs(m0)).max() <= 1e-12
    assert np.sum(lam > 0) == 6 and np.sum(lam < 0) == 6
    # the rest of the block lies on or above the first momentum shell (Ritz values
    # of Q^2 bound the eigenvalues from above)
    shell = np.sqrt((m0 + 1.0) ** 2 + 1.0)
    assert min(info["block_sqrt_mu"][12:]) >= shell - 1e-9


def test_random_field_against_dense_eigh():
    from tests import dense4
    dims = dense4.DENSE4["dims"]
    op = dense4.field()[1]
    start = synth.gaussian_vectors(dims, 14, 5)
    lam, V, res, info = chefsi.lowest_abs_eigenpairs(op.Q, start, 8, chefsi.q_norm_bound(op), degree=60)
    w_all, v_all = dense4.q_eigh()
    order = np.lexsort((w_all, np.abs(w_all)))[:8]
    w, v = w_all[order], v_all[:, order]
    assert info["converged"]
    assert np.abs(lam - w).max() <= 1e-12 * np.abs(w).max()
    for i in range(8):
        assert abs(np.vdot(v[:, i], V[i].ravel())) >= 1 - 1e-10


def test_norm_bound_holds():
    from tests import dense4
    assert np.abs(dense4.q_eigh()[0]).max() <= chefsi.q_norm_bound(dense4.field()[1])
