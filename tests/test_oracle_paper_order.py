"""Algorithm 1 in the paper's order, every addition of this implementation
switched off (no Ritz rotation of the start vectors, no guard vectors, no
per-sweep Rayleigh-Ritz step or locking, no coarse or fine deflation, no shift
floor, fixed inner tolerance): the oracle against LAPACK's eigh of the dense
3072 x 3072 Q on the 4^4 field (eps = 0.3, c_sw = 1.0, m0 = -0.4, 8 test
vectors, SAP on 2^4 blocks), 4 wanted pairs, 8 sweeps.

What the paper's Algorithm 1 reaches here is pinned as it is:
* v_1 converges to the eigenpair of smallest |lambda| (eigenvalue to relative
  1e-10, residual <= 1e-10, overlap >= 1 - 1e-8);
* every returned vector converges to some eigenpair of Q (residual <= 1e-5,
  and its Rayleigh quotient equals that eigenvalue to within residual^2/gap);
* the returned set is NOT the 4 of smallest |lambda|: the iteration misses
  modes, the failure the paper notes after Algorithm 1.  That check is a strict
  expected failure, so that it reports the miss as a miss (and turns red if the
  oracle ever finds the full set).
"""
import numpy as np
import pytest

import synth
from oracle import dense, dirac, mg, rqi

DENSE4 = dict(dims=(4, 4, 4, 4), eps=0.3, seed=1001, m0=-0.4, csw=1.0, n_eig=4)
PAPER_ORDER = dict(ritz_each_sweep=False, fine_deflate=False, coarse_deflate=False, shift_floor=0.0,
                   adaptive_tol=False, ritz_start=False)


@pytest.fixture(scope="module")
def run():
    from tests import dense4
    c = DENSE4
    op = dense4.field()[1]
    params = dict(mg.DEFAULT_PARAMS, agg=(2, 2, 2, 2), ntv=8, sap_block=(2, 2, 2, 2), **PAPER_ORDER)
    W0 = synth.uniform_vectors(c["dims"], 8, c["seed"])
    lam, V, res, st = rqi.eigensolve(op, W0, c["n_eig"], 1e-10, params, max_sweeps=8, n_guard=0,
                                     seed=c["seed"])
    Qm = dense4.q_matrix()
    w, v = dense4.q_eigh()
    return lam, V, res, Qm, w, v


def test_paper_order_converges_to_eigenpairs(run):
    lam, V, res, Qm, w, v = run
    order = np.lexsort((w, np.abs(w)))
    # the first vector: the eigenpair of smallest |lambda|
    i0 = order[0]
    assert abs(lam[0] - w[i0]) <= 1e-10 * abs(w[i0])
    assert res[0] <= 1e-10
    assert abs(np.vdot(v[:, i0], V[0].ravel())) >= 1 - 1e-8
    # every vector: an eigenpair of the dense Q
    for i in range(len(lam)):
        x = V[i].ravel()
        r = np.linalg.norm(Qm @ x - lam[i] * x)
        assert abs(r - res[i]) <= 1e-12 + 1e-6 * res[i]
        assert res[i] <= 1e-5
        j = np.argmin(np.abs(w - lam[i]))
        gap = np.min(np.abs(np.delete(w, j) - w[j]))
        assert abs(lam[i] - w[j]) <= res[i] ** 2 / gap + 1e-14


@pytest.mark.xfail(strict=True, reason="Algorithm 1 in the paper's order misses wanted modes on this field "
                                       "(the failure noted after Algorithm 1)")
def test_paper_order_finds_the_lowest_set(run):
    lam, V, res, Qm, w, v = run
    want = w[np.lexsort((w, np.abs(w)))][:len(lam)]
    assert np.abs(np.sort(lam) - np.sort(want)).max() <= 1e-8
