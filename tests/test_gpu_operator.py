"""GPU fine operator against the oracle on the same seeded inputs: clover term
(four-leaf, FP64) and the Wilson-clover stencil Q - sigma and D - sigma gamma5 in
FP64 (relative 1e-13) and FP32 (relative 1e-6), on the 4^4 lattice, a ragged
lattice with antiperiodic directions, and the full 16^3 x 32 lattice."""
import numpy as np
import pytest

import synth
from oracle import dirac
from tests.gpu_util import norm_rel_err, rel_err

pytestmark = pytest.mark.gpu

CASES = [
    dict(dims=(4, 4, 4, 4), eps=0.3, seed=1001, m0=-0.4, csw=1.0, bc=(1, 1, 1, 1), agg=(2, 2, 2, 2),
         sap=(2, 2, 2, 2)),
    dict(dims=(6, 4, 2, 10), eps=0.5, seed=7, m0=0.1, csw=1.9, bc=(1, -1, 1, -1), agg=(2, 2, 2, 2),
         sap=(3, 2, 1, 5)),
    dict(dims=(16, 16, 16, 32), eps=0.2, seed=1002, m0=-0.05, csw=1.9, bc=(1, 1, 1, 1), agg=(4, 4, 4, 4),
         sap=(4, 4, 4, 4)),
]


@pytest.fixture(scope="module", params=range(len(CASES)), ids=["4x4x4x4", "6x4x2x10_apbc", "16x16x16x32"])
def case(request):
    from paper_1509_06865_gb300 import Context
    c = CASES[request.param]
    U = synth.gauge_field(c["dims"], c["eps"], c["seed"])
    ctx = Context(c["dims"])
    ctx.set_params(m0=c["m0"], csw=c["csw"], bc=c["bc"], agg=c["agg"], sap_block=c["sap"], n_tv=4)
    ctx.load_gauge(U)
    op = dirac.WilsonClover(U, c["m0"], c["csw"], bc=c["bc"])
    yield ctx, op, c
    ctx.close()


def test_clover_term(case):
    ctx, op, c = case
    A = ctx.get_clover()
    Ao = op.A.reshape(-1, 12, 12)
    want = np.stack([Ao[:, :6, :6], Ao[:, 6:, 6:]], axis=1)
    assert np.abs(Ao[:, :6, 6:]).max() == 0
    assert rel_err(A, want) < 1e-13


@pytest.mark.parametrize("sigma", [0.0, 0.137])
def test_stencil_fp64_and_fp32(case, sigma):
    from paper_1509_06865_gb300 import OP_D, OP_Q, PREC_F32, PREC_F64
    ctx, op, c = case
    x = synth.gaussian_vectors(c["dims"], 2, 31)
    yq = ctx.apply(x, sigma, OP_Q, PREC_F64)
    yd = ctx.apply(x, sigma, OP_D, PREC_F64)
    for k in range(2):
        wq = op.Q_sigma(x[k], sigma)
        wd = op.D_sigma(x[k], sigma)
        assert norm_rel_err(yq[k], wq) < 1e-13
        assert norm_rel_err(yd[k], wd) < 1e-13
        assert rel_err(yq[k], wq) < 1e-13
    y32 = ctx.apply(x[:1], sigma, OP_Q, PREC_F32)
    assert norm_rel_err(y32[0], op.Q_sigma(x[0], sigma)) < 1e-6


def test_stencil_device_entry_point(case):
    """mgeig_apply_dev on library-owned device buffers gives the host-call result."""
    from paper_1509_06865_gb300 import OP_Q, PREC_F32, PREC_F64
    ctx, op, c = case
    V = ctx.V
    x = synth.gaussian_vectors(c["dims"], 1, 5)
    want = op.Q_sigma(x[0], 0.05)
    for prec, nbytes, tol in ((PREC_F64, V * 12 * 16, 1e-13), (PREC_F32, V * 12 * 8, 1e-6)):
        px = ctx.alloc_dev(nbytes)
        py = ctx.alloc_dev(nbytes)
        ctx.pack_spinors(x, px, prec)
        ctx.apply_dev(px, py, 0.05, OP_Q, prec)
        got = ctx.unpack_spinors(py, 1, prec)[0]
        assert norm_rel_err(got, want) < tol
