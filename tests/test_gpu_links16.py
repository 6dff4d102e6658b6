"""The coarse operator with 16-bit links (BF16 or IEEE half entries, one FP32
scale per 2N_tv x 2N_tv link block, FP32 accumulation) against the oracle's
FP64 coarse operator P^dag D P (Eq. 2.5) applied as Q_c - sigma (Eq. 2.6), on
the same seeded test vectors:

* one right-hand side (the CUDA-core kernel used by the coarse solver's
  deflation data and the coarse apply): relative error within the rounding of
  the links (BF16 8 significant bits: 2e-2 in norm; half: 3e-3);
* 12 right-hand sides in one launch on the tensor cores (BF16 links, right-hand
  sides rounded to BF16 after the link scale): each within 2e-2 of the oracle;
* the two-grid preconditioner and the eigensolver with BF16 links: the FP64
  outer FGMRES still reaches the eigen-residual 1e-10, with the same 20
  eigenvalues as the oracle's independent set on the 8^3 x 16 field.
"""
import json
import os

import numpy as np
import pytest

import synth
from oracle import dirac, mg
from tests.gpu_util import norm_rel_err

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CASE = dict(dims=(8, 8, 8, 16), eps=0.2, seed=1006, m0=-0.0428, csw=1.9, bc=(1, 1, 1, 1), agg=(2, 2, 2, 2),
            sap=(4, 4, 4, 4), ntv=20)


@pytest.fixture(scope="module")
def coarse():
    c = CASE
    U = synth.gauge_field(c["dims"], c["eps"], c["seed"])
    op = dirac.WilsonClover(U, c["m0"], c["csw"], bc=c["bc"])
    W = synth.uniform_vectors(c["dims"], c["ntv"], 99)
    P = mg.Interpolation(W, c["agg"])
    C = mg.CoarseOperator(mg.coarse_operator(op, P), P.cdims, P.ntv)
    X = np.array([P.restrict(x) for x in synth.gaussian_vectors(c["dims"], 12, 17)])
    return c, U, W, C, X


def make(c, links):
    from paper_1509_06865_gb300 import MIXED, Context
    ctx = Context(c["dims"])
    ctx.set_params(m0=c["m0"], csw=c["csw"], bc=c["bc"], agg=c["agg"], sap_block=c["sap"], n_tv=c["ntv"],
                   precision=MIXED, coarse_links=links)
    return ctx


@pytest.mark.parametrize("links,tol", [(1, 2e-2), (2, 3e-3)], ids=["bf16", "f16"])
def test_coarse_apply_16bit_links(coarse, links, tol):
    c, U, W, C, X = coarse
    ctx = make(c, links)
    ctx.load_gauge(U)
    ctx.set_test_vectors(W)
    for sigma in (0.0, 0.07):
        for x in X[:3]:
            assert norm_rel_err(ctx.coarse_apply(x, sigma), C.apply(x, sigma)) < tol
    ctx.close()


@pytest.mark.parametrize("nrhs", [1, 5, 12, 16])
def test_coarse_apply_many_rhs_tensor_cores(coarse, nrhs):
    from paper_1509_06865_gb300 import LINKS_BF16
    c, U, W, C, X = coarse
    ctx = make(c, LINKS_BF16)
    ctx.load_gauge(U)
    ctx.set_test_vectors(W)
    Xn = np.concatenate([X, X[:4] * (1 + 2j)])[:nrhs]
    Y = ctx.coarse_apply_nrhs(Xn, 0.031)
    for r in range(nrhs):
        assert norm_rel_err(Y[r], C.apply(Xn[r], 0.031)) < 2e-2, r
    # the CUDA-core kernel of the same links agrees more closely than either with FP64
    for r in range(min(nrhs, 2)):
        assert norm_rel_err(Y[r], ctx.coarse_apply(Xn[r], 0.031)) < 1e-2
    ctx.close()


def test_eigensolve_with_bf16_links_reaches_1e_10():
    from paper_1509_06865_gb300 import LINKS_BF16, MIXED, Context
    with open(os.path.join(ROOT, "tests", "golden", "lowest_Q_8x8x8x16.json")) as f:
        g = json.load(f)
    with open(os.path.join(ROOT, "workloads.json")) as f:
        cfg = json.load(f)[g["workload"]]
    dims = tuple(cfg["dims"])
    U = synth.gauge_field(dims, cfg["eps"], cfg["seed"])
    ctx = Context(dims)
    ctx.set_params(m0=cfg["m0"], csw=cfg["csw"], bc=cfg["bc"], agg=cfg["agg"], n_tv=cfg["n_tv"],
                   sap_block=cfg["sap_block"], precision=MIXED, coarse_links=LINKS_BF16)
    ctx.load_gauge(U)
    ctx.setup(cfg["seed"])
    lam, V, res, st = ctx.eigensolve(cfg["n_eig"], cfg["tol"])
    ctx.close()
    assert st["converged"] and np.all(res <= 1e-10), (res, st)
    want = np.array(g["eigenvalues"][:cfg["n_eig"]])
    assert np.abs(np.sort(lam) - np.sort(want)).max() <= 1e-10 * np.abs(want).max()
    op = dirac.WilsonClover(U, cfg["m0"], cfg["csw"], tuple(cfg["bc"]))
    for i in range(cfg["n_eig"]):
        assert dirac.norm(op.Q(V[i]) - lam[i] * V[i]) <= 1.05e-10
