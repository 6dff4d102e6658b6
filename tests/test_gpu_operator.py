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


def test_stencil_double_float(case):
    """The mixed solver's FP64-output stencil in double-float arithmetic (two
    floats per value, links and clover from double-float copies): FP64 input,
    and FP32 input (the outer FGMRES matvec of a preconditioned vector) against
    the oracle applied to the same FP32-rounded input.  Double-float keeps about
    47 bits, so the bound is 1e-12 where FP64 meets 1e-13 and FP32 1e-6."""
    from paper_1509_06865_gb300 import OP_D, OP_Q, PREC_F32, PREC_F32_F64_DS, PREC_F64, PREC_F64_DS
    ctx, op, c = case
    V = ctx.V
    x = synth.gaussian_vectors(c["dims"], 1, 9)
    x32 = x.astype(np.complex64).astype(np.complex128)
    px64, px32 = ctx.alloc_dev(V * 12 * 16), ctx.alloc_dev(V * 12 * 8)
    py = ctx.alloc_dev(V * 12 * 16)
    ctx.pack_spinors(x, px64, PREC_F64)
    ctx.pack_spinors(x, px32, PREC_F32)
    for opn, ref in ((OP_Q, op.Q_sigma), (OP_D, op.D_sigma)):
        for sigma in (0.0, 0.0371):
            ctx.apply_dev(px64, py, sigma, opn, PREC_F64_DS)
            got = ctx.unpack_spinors(py, 1, PREC_F64)[0]
            want = ref(x[0], sigma)
            assert norm_rel_err(got, want) < 1e-12
            assert rel_err(got, want) < 1e-12
            ctx.apply_dev(px32, py, sigma, opn, PREC_F32_F64_DS)
            got = ctx.unpack_spinors(py, 1, PREC_F64)[0]
            want = ref(x32[0], sigma)
            assert norm_rel_err(got, want) < 1e-12
            assert rel_err(got, want) < 1e-12


def _blocks(A12):
    """[..., 12, 12] site matrices -> [site][2][6][6] chirality blocks."""
    A = A12.reshape(-1, 12, 12)
    return np.ascontiguousarray(np.stack([A[:, :6, :6], A[:, 6:, 6:]], axis=1))


def test_load_clover_host_term():
    """mgeig_load_clover: the oracle's clover term loaded from the host gives the
    oracle's stencil; a different Hermitian term (scaled, perturbed) is used as
    given, survives a change of m0, and NULL goes back to the built term."""
    from paper_1509_06865_gb300 import OP_D, OP_Q, PREC_F32, PREC_F64, Context
    c = CASES[1]
    U = synth.gauge_field(c["dims"], c["eps"], c["seed"])
    op = dirac.WilsonClover(U, c["m0"], c["csw"], bc=c["bc"])
    ctx = Context(c["dims"])
    ctx.set_params(m0=c["m0"], csw=c["csw"], bc=c["bc"], agg=c["agg"], sap_block=c["sap"], n_tv=4)
    ctx.load_gauge(U)
    x = synth.gaussian_vectors(c["dims"], 1, 41)
    ctx.load_clover(_blocks(op.A))
    assert rel_err(ctx.get_clover(), _blocks(op.A)) < 1e-15
    assert norm_rel_err(ctx.apply(x, 0.1, OP_Q, PREC_F64)[0], op.Q_sigma(x[0], 0.1)) < 1e-13
    # another Hermitian term, block diagonal in chirality like the clover term
    rng = np.random.default_rng(5)
    H = rng.normal(size=op.A.shape) + 1j * rng.normal(size=op.A.shape)
    H = 0.05 * (H + np.conj(np.swapaxes(H, -1, -2)))
    H[..., :6, 6:] = 0
    H[..., 6:, :6] = 0
    A2 = 0.7 * op.A + H
    ctx.load_clover(_blocks(A2))
    op2 = dirac.WilsonClover(U, c["m0"], c["csw"], bc=c["bc"], A=A2)
    assert norm_rel_err(ctx.apply(x, 0.0, OP_D, PREC_F64)[0], op2.D(x[0])) < 1e-13
    assert norm_rel_err(ctx.apply(x, 0.0, OP_D, PREC_F32)[0], op2.D(x[0])) < 1e-6
    # a new m0 keeps the loaded term and adds the new mass
    ctx.set_params(m0=0.3, csw=c["csw"], bc=c["bc"], agg=c["agg"], sap_block=c["sap"], n_tv=4)
    op3 = dirac.WilsonClover(U, 0.3, c["csw"], bc=c["bc"], A=A2)
    assert norm_rel_err(ctx.apply(x, 0.2, OP_Q, PREC_F64)[0], op3.Q_sigma(x[0], 0.2)) < 1e-13
    # NULL: the term built from the gauge field again
    ctx.load_clover(None)
    op4 = dirac.WilsonClover(U, 0.3, c["csw"], bc=c["bc"])
    assert norm_rel_err(ctx.apply(x, 0.2, OP_Q, PREC_F64)[0], op4.Q_sigma(x[0], 0.2)) < 1e-13
    ctx.close()


@pytest.mark.parametrize("nrhs", [1, 3, 12])
def test_stencil_many_right_hand_sides(case, nrhs):
    """mgeig_apply_dev_nrhs: nrhs fields back to back in one launch, each equal
    to the oracle's stencil on that field (FP64 1e-13, FP32 1e-6)."""
    from paper_1509_06865_gb300 import OP_D, OP_Q, PREC_F32, PREC_F64
    ctx, op, c = case
    V = ctx.V
    x = synth.gaussian_vectors(c["dims"], nrhs, 50 + nrhs)
    ops = ((OP_Q, 0.021), (OP_D, -0.3))
    wants = {o: [op.Q_sigma(x[k], s) if o == OP_Q else op.D_sigma(x[k], s) for k in range(nrhs)] for o, s in ops}
    for prec, per, tol in ((PREC_F64, V * 12 * 16, 1e-13), (PREC_F32, V * 12 * 8, 1e-6)):
        px = ctx.alloc_dev(per * nrhs)
        py = ctx.alloc_dev(per * nrhs)
        ctx.pack_spinors(x, px, prec)
        for opcode, sigma in ops:
            ctx.apply_dev_nrhs(px, py, nrhs, sigma, opcode, prec)
            got = ctx.unpack_spinors(py, nrhs, prec)
            for k in range(nrhs):
                assert norm_rel_err(got[k], wants[opcode][k]) < tol, (prec, opcode, k)
