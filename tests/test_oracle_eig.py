"""The oracle's Algorithm 1 (setup + Rayleigh quotient iteration with the
two-grid preconditioned FGMRES) against LAPACK's dense eigendecomposition of
the 3072 x 3072 Hermitian Q on the 4^4 lattice (4^4, eps = 0.3, c_sw = 1.0,
m0 = -0.4, 4 lowest pairs, 2^4 aggregates, 8 test vectors)."""
import numpy as np

import synth
from oracle import dense, dirac, mg, rqi

DENSE4 = dict(dims=(4, 4, 4, 4), eps=0.3, seed=1001, m0=-0.4, csw=1.0, n_eig=4)


def test_rqi_matches_dense_eigh():
    from tests import dense4
    c = DENSE4
    op = dense4.field()[1]
    params = dict(mg.DEFAULT_PARAMS, agg=(2, 2, 2, 2), ntv=8, sap_block=(2, 2, 2, 2))
    W0 = synth.uniform_vectors(c["dims"], 8, c["seed"])
    lam, V, res, st = rqi.eigensolve(op, W0, c["n_eig"], 1e-10, params)
    w_all, v_all = dense4.q_eigh()
    order = np.lexsort((w_all, np.abs(w_all)))[:c["n_eig"]]
    w, v = w_all[order], v_all[:, order]
    assert np.all(res <= 1e-10)
    assert np.abs(lam - w).max() <= 1e-10 * np.abs(w).max()
    # gaps to the neighbours are ~1e-3, so the overlap bound (res/gap)^2 is tiny
    for i in range(c["n_eig"]):
        assert abs(np.vdot(v[:, i], V[i].ravel())) >= 1 - 1e-8
    # the residual really is the eigen-residual of the dense matrix
    Qm = dense4.q_matrix()
    for i in range(c["n_eig"]):
        r = Qm @ V[i].ravel() - lam[i] * V[i].ravel()
        assert np.linalg.norm(r) <= 1.01e-10
