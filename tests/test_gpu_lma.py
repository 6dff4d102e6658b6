"""Approximate low-mode averaging on the GPU (Sec. 3.1, 3.2) against the FP64
oracle (oracle/lma.py, pinned in tests/test_oracle_lma.py) on the dense 4^4
field: approximate eigenvectors (exact ones plus noise) give the same Rayleigh
quotients, accuracies, cutoff decisions, A, A^-1, low-mode loop L_low(t),
corrected inverse Q~^-1_low x and oblique projection R~ x to relative 1e-10; the
stochastic high-mode loop with the same Z2 noise equals the oracle's estimator
with dense solves to the solve tolerance.  On the 8^3 x 16 field the setup's
test vectors serve as approximate modes (Sec. 3.3: 30 setup iterations, no
Rayleigh quotient iteration; the Ritz vectors of Q in their span), with the
cutoff 0.75."""
import json
import os

import numpy as np
import pytest

import synth
from oracle import lma
from tests import dense4
from tests.gpu_util import norm_rel_err, rel_err

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def approx():
    op = dense4.field()[1]
    w, v = dense4.q_eigh()
    order = np.lexsort((w, np.abs(w)))[:8]
    lx, ly, lz, lt = dense4.DENSE4["dims"]
    V0 = v[:, order].T.reshape(8, lt, lz, ly, lx, 4, 3)
    rng = np.random.default_rng(3)
    noise = rng.normal(size=V0.shape) + 1j * rng.normal(size=V0.shape)
    scale = np.array([1e-4, 1e-3, 1e-2, 3e-2, 0.1, 0.3, 1e-3, 0.5])[:, None, None, None, None, None, None]
    V = lma.orthonormalise(V0 + scale * noise / np.linalg.norm(noise[0]))
    lam, eps, QV = lma.approximate_modes(op, V)
    keep = lma.cutoff(lam, eps, 0.75)
    A = lma.a_matrix(V[keep], QV[keep])
    return op, V, lam, eps, QV, keep, A, np.linalg.inv(A)


def make_ctx(setup=False):
    from paper_1509_06865_gb300 import Context
    c = dense4.DENSE4
    ctx = Context(c["dims"])
    ctx.set_params(m0=c["m0"], csw=c["csw"], agg=(2, 2, 2, 2), n_tv=8, sap_block=(2, 2, 2, 2))
    ctx.load_gauge(dense4.field()[0])
    if setup:
        ctx.setup(c["seed"])
    return ctx


def test_lma_objects_match_oracle(approx):
    op, V, lam, eps, QV, keep, A, Ainv = approx
    ctx = make_ctx()
    out = ctx.lma_prepare(len(V), V, 0.75)
    assert rel_err(out["lam"], lam) < 1e-10 and rel_err(out["eps"], eps) < 1e-9
    assert list(np.nonzero(out["kept"])[0]) == list(keep) and 0 < len(keep) < len(V)
    assert rel_err(out["A"], A) < 1e-10 and rel_err(out["Ainv"], Ainv) < 1e-9
    assert rel_err(out["Llow"], lma.low_mode_loop(V[keep], Ainv)) < 1e-9
    x = synth.gaussian_vectors(dense4.DENSE4["dims"], 1, 5)[0]
    assert norm_rel_err(ctx.lma_apply(x, 0), lma.low_inverse_apply(V[keep], Ainv, x)) < 1e-10
    assert norm_rel_err(ctx.lma_apply(x, 1), lma.oblique_projector_apply(V[keep], QV[keep], Ainv, x)) < 1e-10
    ctx.close()


def test_high_mode_loop_matches_dense_estimator(approx):
    op, V, lam, eps, QV, keep, A, Ainv = approx
    ctx = make_ctx(setup=True)
    ctx.lma_prepare(len(V), V, 0.75)
    nst, seed = 3, 77
    got, st = ctx.lma_loop_high(nst, seed, 1e-12)
    Qm = dense4.q_matrix()
    eta = synth.z2_noise(dense4.DENSE4["dims"], nst, seed)
    want = 0
    for e in eta:
        b = lma.oblique_projector_apply(V[keep], QV[keep], Ainv, e)
        s = np.linalg.solve(Qm, b.ravel()).reshape(e.shape)
        want = want + np.einsum("tzyxsc,tzyxsc->t", e.conj(), s)
    want = want / nst
    assert rel_err(got, want) < 1e-9, (got, want)
    ctx.close()


def test_setup_test_vectors_as_approximate_modes():
    from paper_1509_06865_gb300 import MIXED, Context
    with open(os.path.join(ROOT, "workloads.json")) as f:
        cfg = json.load(f)["check_8x8x8x16"]
    dims = tuple(cfg["dims"])
    ctx = Context(dims)
    ctx.set_params(m0=cfg["m0"], csw=cfg["csw"], agg=cfg["agg"], n_tv=cfg["n_tv"], sap_block=cfg["sap_block"],
                   precision=MIXED, setup_iters=30)
    ctx.load_gauge(synth.gauge_field(dims, cfg["eps"], cfg["seed"]))
    ctx.setup(cfg["seed"])
    out = ctx.lma_prepare(cfg["n_tv"], None, 0.75)
    rel = out["eps"] / np.abs(out["lam"])
    print("approximate modes after 30 setup iterations: eps", np.round(out["eps"], 5), "eps/|lambda|",
          np.round(rel, 3), "kept", out["n_kept"])
    assert np.array_equal(out["kept"], rel <= 0.75)
    assert out["n_kept"] >= 1
    assert np.allclose(out["A"], out["A"].conj().T, atol=1e-12 * np.abs(out["A"]).max())
    ctx.close()


def test_lma_with_rqi_modes_8x8x8x16():
    """Exact modes from Algorithm 1 (12 lowest pairs of the 8^3 x 16 field): A is
    diagonal to the eigen-residual, L_low(t) equals sum_i (1/lambda_i)
    sum_{x in t} |v_i(x)|^2 computed from the returned vectors, and the deflated
    stochastic loop (Q s = R~ eta) converges for every noise vector."""
    from paper_1509_06865_gb300 import MIXED, Context
    with open(os.path.join(ROOT, "workloads.json")) as f:
        cfg = json.load(f)["check_8x8x8x16"]
    dims = tuple(cfg["dims"])
    ctx = Context(dims)
    ctx.set_params(m0=cfg["m0"], csw=cfg["csw"], agg=cfg["agg"], n_tv=cfg["n_tv"], sap_block=cfg["sap_block"],
                   precision=MIXED)
    ctx.load_gauge(synth.gauge_field(dims, cfg["eps"], cfg["seed"]))
    ctx.setup(cfg["seed"])
    lam, V, res, st = ctx.eigensolve(12, 1e-10)
    assert st["converged"]
    out = ctx.lma_prepare(12, V, 0.75)
    assert out["n_kept"] == 12
    off = out["A"] - np.diag(np.diag(out["A"]))
    assert np.abs(off).max() <= 1e-9 and np.abs(np.diag(out["A"]).real - lam).max() <= 1e-12
    want = [sum((np.abs(V[i][t]) ** 2).sum() / lam[i] for i in range(12)) for t in range(dims[3])]
    assert rel_err(out["Llow"], np.array(want)) < 1e-9
    Lh, sth = ctx.lma_loop_high(2, 5, 1e-8)
    assert np.all(np.isfinite(Lh)) and sth["solves"] == 2
    ctx.close()
