"""mgeig_solve_batch: every shift and right-hand side of several fields (the
Z2 + iZ2 noise right-hand sides of Sec. 3 and the shifted systems of
Algorithm 1), in both precisions: each solution against numpy.linalg.solve of the
dense (Q - sigma) on two 4^4 fields (different links and masses), and every
residual re-computed with the oracle's stencil, to the requested 1e-10."""
import numpy as np
import pytest

import synth
from oracle import dense, dirac

pytestmark = pytest.mark.gpu

FIELDS = [dict(eps=0.3, seed=1001, m0=-0.4, csw=1.0), dict(eps=0.25, seed=31, m0=-0.3, csw=1.9)]
DIMS = (4, 4, 4, 4)


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_batch_of_shifts_and_noise_rhs(precision):
    from paper_1509_06865_gb300 import Context, solve_batch
    sigmas = [0.0, 0.02, 0.05]
    ctxs, ops, rhs = [], [], []
    for k, f in enumerate(FIELDS):
        U = synth.gauge_field(DIMS, f["eps"], f["seed"])
        ctx = Context(DIMS)
        ctx.set_params(m0=f["m0"], csw=f["csw"], agg=(2, 2, 2, 2), n_tv=8, sap_block=(2, 2, 2, 2),
                       precision=precision)
        ctx.load_gauge(U)
        ctx.setup(f["seed"])
        ctxs.append(ctx)
        ops.append(dirac.WilsonClover(U, f["m0"], f["csw"]))
        rhs.append(synth.z2_noise(DIMS, 3, 100 + k))
    xs, st = solve_batch(ctxs, sigmas, rhs, 1e-10)
    assert st["converged"] and st["solves"] == len(FIELDS) * len(sigmas) * 3, st
    for k, op in enumerate(ops):
        Qm = dense.operator_matrix(op.Q, DIMS)
        for s, sigma in enumerate(sigmas):
            A = Qm - sigma * np.eye(Qm.shape[0])
            for j in range(3):
                b, x = rhs[k][j], xs[k][s, j]
                assert dirac.norm(op.Q_sigma(x, sigma) - b) <= 1.05e-10 * dirac.norm(b)
                xd = np.linalg.solve(A, b.ravel())
                assert np.linalg.norm(x.ravel() - xd) <= 1e-8 * np.linalg.norm(xd)
    for ctx in ctxs:
        ctx.close()
