"""Algorithm 1 in the paper's order on the GPU (every addition switched off:
ritz_start, n_guard, ritz_each_sweep, coarse and fine deflation, shift floor,
adaptive inner tolerance), the configuration of tests/test_oracle_paper_order.py,
against LAPACK's eigh of the dense 3072 x 3072 Q on the 4^4 field, in FP64 and
mixed precision.  The same properties are checked: v_1 converges to the pair of
smallest |lambda|; every returned vector converges to an eigenpair of Q; and the
full set of the 4 lowest is a strict expected failure, the miss the paper notes
after Algorithm 1, reported as a miss."""
import numpy as np
import pytest

import synth
from oracle import dense, dirac

pytestmark = pytest.mark.gpu

DENSE4 = dict(dims=(4, 4, 4, 4), eps=0.3, seed=1001, m0=-0.4, csw=1.0, n_eig=4)
PAPER_ORDER = dict(ritz_each_sweep=0, fine_deflate=0, coarse_deflate=0, shift_floor=0.0, adaptive_tol=0,
                   ritz_start=0, n_guard=0, max_sweeps=8)


@pytest.fixture(scope="module")
def dense4():
    c = DENSE4
    U = synth.gauge_field(c["dims"], c["eps"], c["seed"])
    op = dirac.WilsonClover(U, c["m0"], c["csw"])
    Qm = dense.operator_matrix(op.Q, c["dims"])
    w, v = np.linalg.eigh(Qm)
    return U, Qm, w, v


@pytest.fixture(scope="module", params=[0, 1], ids=["fp64", "mixed"])
def run(request, dense4):
    from paper_1509_06865_gb300 import Context
    U, Qm, w, v = dense4
    c = DENSE4
    ctx = Context(c["dims"])
    ctx.set_params(m0=c["m0"], csw=c["csw"], agg=(2, 2, 2, 2), n_tv=8, sap_block=(2, 2, 2, 2),
                   precision=request.param, **PAPER_ORDER)
    ctx.load_gauge(U)
    ctx.setup(c["seed"])
    lam, V, res, st = ctx.eigensolve(c["n_eig"], 1e-10)
    ctx.close()
    print("paper order", request.param, lam, res, st)
    return lam, V, res, Qm, w, v


def test_gpu_paper_order_converges_to_eigenpairs(run):
    lam, V, res, Qm, w, v = run
    order = np.lexsort((w, np.abs(w)))
    i0 = order[0]
    assert abs(lam[0] - w[i0]) <= 1e-10 * abs(w[i0])
    assert res[0] <= 1e-10
    assert abs(np.vdot(v[:, i0], V[0].ravel())) >= 1 - 1e-8
    for i in range(len(lam)):
        x = V[i].ravel()
        assert abs(np.linalg.norm(Qm @ x - lam[i] * x) - res[i]) <= 1e-12 + 1e-6 * res[i]
        assert res[i] <= 1e-5
        j = np.argmin(np.abs(w - lam[i]))
        gap = np.min(np.abs(np.delete(w, j) - w[j]))
        assert abs(lam[i] - w[j]) <= res[i] ** 2 / gap + 1e-14


@pytest.mark.xfail(strict=True, reason="Algorithm 1 in the paper's order misses wanted modes on this field "
                                       "(the failure noted after Algorithm 1)")
def test_gpu_paper_order_finds_the_lowest_set(run):
    lam, V, res, Qm, w, v = run
    want = w[np.lexsort((w, np.abs(w)))][:len(lam)]
    assert np.abs(np.sort(lam) - np.sort(want)).max() <= 1e-8
