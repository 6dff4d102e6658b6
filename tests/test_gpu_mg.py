"""GPU two-grid pieces against the oracle on the same seeded test vectors
(4^4 and 8x4x4x8 lattices): interpolation P (Eq. 2.4), restriction and
prolongation, the per-direction coarse operator (Eq. 2.5), the coarse apply
(Q_c - sigma, Eq. 2.6), SAP cycles, one two-grid cycle with a fixed number of
coarse GMRES steps (SAP and GMRES smoothers) and the multigrid setup, in FP64
(relative 1e-10) and in the mixed FP32 level (relative 1e-5)."""
import numpy as np
import pytest

import synth
from oracle import dirac, mg, rqi
from tests.gpu_util import norm_rel_err, rel_err

pytestmark = pytest.mark.gpu

CASES = {
    "4^4": dict(dims=(4, 4, 4, 4), eps=0.3, seed=1001, m0=-0.4, csw=1.0, bc=(1, 1, 1, 1), agg=(2, 2, 2, 2),
                sap=(2, 2, 2, 2), ntv=8),
    "8x4x4x8": dict(dims=(8, 4, 4, 8), eps=0.25, seed=77, m0=-0.2, csw=1.9, bc=(1, 1, 1, -1), agg=(4, 2, 2, 4),
                    sap=(2, 2, 2, 2), ntv=6),
}


def make(c, precision, smoother=0, **extra):
    from paper_1509_06865_gb300 import Context
    ctx = Context(c["dims"])
    kw = dict(m0=c["m0"], csw=c["csw"], bc=c["bc"], agg=c["agg"], sap_block=c["sap"], n_tv=c["ntv"],
              precision=precision, smoother=smoother)
    kw.update(extra)
    ctx.set_params(**kw)
    return ctx


@pytest.fixture(scope="module", params=list(CASES))
def inputs(request):
    c = CASES[request.param]
    U = synth.gauge_field(c["dims"], c["eps"], c["seed"])
    op = dirac.WilsonClover(U, c["m0"], c["csw"], bc=c["bc"])
    W = synth.uniform_vectors(c["dims"], c["ntv"], 99)
    P = mg.Interpolation(W, c["agg"])
    Dc = mg.coarse_operator(op, P)
    return c, U, op, W, P, Dc


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)], ids=["fp64", "mixed"])
def test_interp_restrict_prolong_coarse(inputs, prec, tol):
    c, U, op, W, P, Dc = inputs
    ctx = make(c, prec)
    ctx.load_gauge(U)
    ctx.set_test_vectors(W)
    assert rel_err(ctx.get_interp(), P.vectors()) < (1e-12 if prec == 0 else 2e-6)
    r = synth.gaussian_vectors(c["dims"], 1, 3)[0]
    assert rel_err(ctx.restrict(r), P.restrict(r)) < tol
    ec = P.restrict(synth.gaussian_vectors(c["dims"], 1, 4)[0])
    assert rel_err(ctx.prolong(ec), P.prolong(ec)) < tol
    assert rel_err(ctx.get_coarse_op(), Dc) < tol
    C = mg.CoarseOperator(Dc, P.cdims, P.ntv)
    assert rel_err(ctx.coarse_apply(ec, 0.07), C.apply(ec, 0.07)) < tol
    ctx.close()


@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 2e-5)], ids=["fp64", "mixed"])
def test_sap_cycles(inputs, prec, tol):
    c, U, op, W, P, Dc = inputs
    ctx = make(c, prec, sap_mr_iters=3)
    ctx.load_gauge(U)
    sap = mg.SAP(op, c["sap"])
    b = synth.gaussian_vectors(c["dims"], 1, 8)[0]
    z0 = 0.1 * synth.gaussian_vectors(c["dims"], 1, 9)[0]
    for sigma in (0.0, 0.09):
        got = ctx.sap(b, z0, sigma, cycles=2)
        want = sap.smooth(b, z0, sigma, 2, 3)
        assert norm_rel_err(got, want) < tol
    ctx.close()


@pytest.mark.parametrize("smoother,deflate,restart", [(0, 1, 30), (1, 1, 30), (0, 0, 30), (0, 1, 5)],
                         ids=["sap-deflated", "gmres-deflated", "sap-plain", "sap-deflated-restart5"])
@pytest.mark.parametrize("prec,tol", [(0, 1e-9), (1, 1e-4)], ids=["fp64", "mixed"])
def test_two_grid_cycle(inputs, smoother, deflate, restart, prec, tol):
    """The persistent coarse solve with and without deflation of the test
    vectors' coarse images, both smoothers, with and without restarts."""
    c, U, op, W, P, Dc = inputs
    params = dict(mg.DEFAULT_PARAMS, agg=c["agg"], sap_block=c["sap"], ntv=c["ntv"],
                  smoother="sap" if smoother == 0 else "gmres", coarse_tol=0.0, coarse_maxiter=12,
                  coarse_restart=restart, coarse_deflate=bool(deflate), sap_cycles=2, sap_mr_iters=3,
                  smooth_steps=2, gmres_smooth_k=4)
    B = mg.TwoGrid(op, W, params)
    ctx = make(c, prec, smoother, coarse_tol=0.0, coarse_maxiter=12, coarse_restart=restart,
               coarse_deflate=deflate, sap_cycles=2, sap_mr_iters=3, smooth_steps=2, gmres_smooth_k=4)
    ctx.load_gauge(U)
    ctx.set_test_vectors(W)
    r = synth.gaussian_vectors(c["dims"], 1, 12)[0]
    for sigma in (0.0, 0.11):
        assert norm_rel_err(ctx.mg_cycle(r, sigma), B(r, sigma)) < tol
    ctx.close()


def test_setup_matches_oracle_fp64(inputs):
    """Same Philox start vectors, fixed coarse iterations: identical test vectors."""
    c, U, op, W, P, Dc = inputs
    params = dict(mg.DEFAULT_PARAMS, agg=c["agg"], sap_block=c["sap"], ntv=c["ntv"], coarse_tol=0.0,
                  coarse_maxiter=10, setup_iters=2, setup_smooth=2, sap_cycles=2, sap_mr_iters=3)
    W0 = synth.uniform_vectors(c["dims"], c["ntv"], 4242)
    Wo, _ = rqi.setup(op, W0, params)
    ctx = make(c, 0, coarse_tol=0.0, coarse_maxiter=10, setup_iters=2, setup_smooth=2, sap_cycles=2,
               sap_mr_iters=3)
    ctx.load_gauge(U)
    ctx.setup(4242)
    Wg = ctx.get_test_vectors()
    for j in range(c["ntv"]):
        assert norm_rel_err(Wg[j], Wo[j]) < 1e-8
    ctx.close()


FULL = dict(dims=(8, 8, 8, 16), eps=0.2, seed=1006, m0=-0.0428, csw=1.9, bc=(1, 1, 1, 1), agg=(2, 2, 2, 2),
            sap=(4, 4, 4, 4), ntv=20)


@pytest.fixture(scope="module")
def full_inputs():
    c = FULL
    U = synth.gauge_field(c["dims"], c["eps"], c["seed"])
    op = dirac.WilsonClover(U, c["m0"], c["csw"], bc=c["bc"])
    W = synth.uniform_vectors(c["dims"], c["ntv"], 99)
    return c, U, op, W


@pytest.mark.parametrize("deflate", [1, 0], ids=["deflated", "plain"])
@pytest.mark.parametrize("prec,tol", [(0, 1e-9), (1, 1e-4)], ids=["fp64", "mixed"])
def test_two_grid_cycle_full_size_coarse_solver(full_inputs, deflate, prec, tol):
    """The two-grid cycle on a coarse grid of 512 aggregates x 40 unknowns
    (8^3 x 16 with 2^4 aggregates, 20 test vectors), the size at which the
    persistent coarse GMRES runs on every SM with grid-wide barriers and
    cross-block partial sums; a fixed number of coarse steps with a restart."""
    c, U, op, W = full_inputs
    params = dict(mg.DEFAULT_PARAMS, agg=c["agg"], sap_block=c["sap"], ntv=c["ntv"], smoother="sap",
                  coarse_tol=0.0, coarse_maxiter=16, coarse_restart=10, coarse_deflate=bool(deflate),
                  sap_cycles=2, sap_mr_iters=3)
    B = mg.TwoGrid(op, W, params)
    ctx = make(c, prec, 0, coarse_tol=0.0, coarse_maxiter=16, coarse_restart=10, coarse_deflate=deflate,
               sap_cycles=2, sap_mr_iters=3)
    ctx.load_gauge(U)
    ctx.set_test_vectors(W)
    r = synth.gaussian_vectors(c["dims"], 1, 12)[0]
    for sigma in (0.0, 0.05):
        assert norm_rel_err(ctx.mg_cycle(r, sigma), B(r, sigma)) < tol
    ctx.close()
