"""GPU multigrid Rayleigh quotient iteration (Algorithm 1) against the oracle:
the 4 lowest eigenpairs of Q on the 4^4 lattice (eps = 0.3, c_sw = 1.0,
m0 = -0.4, 2^4 aggregates, 8 test vectors) compared with the dense FP64
eigendecomposition of the 3072 x 3072 matrix: eigenvalues to relative 1e-10,
eigen-residual <= 1e-10 (re-computed by the oracle's stencil), overlap with
the dense eigenvector >= 1 - 1e-8; and one FGMRES solve against the dense solve."""
import numpy as np
import pytest

import synth
from oracle import dense, dirac

pytestmark = pytest.mark.gpu

DENSE4 = dict(dims=(4, 4, 4, 4), eps=0.3, seed=1001, m0=-0.4, csw=1.0, n_eig=4)


@pytest.fixture(scope="module")
def ref():
    c = DENSE4
    U = synth.gauge_field(c["dims"], c["eps"], c["seed"])
    op = dirac.WilsonClover(U, c["m0"], c["csw"])
    Qm = dense.operator_matrix(op.Q, c["dims"])
    w, v = dense.lowest_eigenpairs(Qm, 8)
    return U, op, Qm, w, v


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("smoother", [0, 1], ids=["sap", "gmres"])
def test_eigensolve_4x4x4x4_vs_dense(ref, precision, smoother):
    from paper_1509_06865_gb300 import Context
    U, op, Qm, w, v = ref
    c = DENSE4
    ctx = Context(c["dims"])
    # the GMRES smoother iterates 16 guard vectors: with the default 8 its FP64
    # path converges to the 5th mode instead of the 3rd on this field (the miss
    # noted after Algorithm 1); 16 give the full set in both precisions
    ctx.set_params(m0=c["m0"], csw=c["csw"], agg=(2, 2, 2, 2), n_tv=8, sap_block=(2, 2, 2, 2),
                   precision=precision, smoother=smoother, n_guard=16 if smoother == 1 else -1)
    ctx.load_gauge(U)
    ctx.setup(c["seed"])
    lam, V, res, st = ctx.eigensolve(c["n_eig"], 1e-10)
    ctx.close()
    print("stats", precision, smoother, st)
    assert st["converged"], st
    assert np.all(res <= 1e-10)
    for i in range(c["n_eig"]):
        x = V[i].ravel()
        assert abs(np.linalg.norm(x) - 1) < 1e-12
        assert np.linalg.norm(Qm @ x - lam[i] * x) <= 1.05e-10
    want = w[:c["n_eig"]]
    # the full set of the 4 lowest, for both smoothers
    assert np.abs(lam - want).max() <= 1e-10 * np.abs(want).max()
    for i in range(c["n_eig"]):
        x = V[i].ravel()
        assert abs(np.vdot(v[:, i], x)) >= 1 - 1e-8
        # phase convention: largest-modulus component real positive
        k = np.argmax(np.abs(x))
        assert abs(x[k].imag) < 1e-14 and x[k].real > 0


def test_fgmres_solve_matches_dense(ref):
    from paper_1509_06865_gb300 import Context
    U, op, Qm, w, v = ref
    c = DENSE4
    ctx = Context(c["dims"])
    ctx.set_params(m0=c["m0"], csw=c["csw"], agg=(2, 2, 2, 2), n_tv=8, sap_block=(2, 2, 2, 2))
    ctx.load_gauge(U)
    ctx.setup(5)
    b = synth.z2_noise(c["dims"], 1, 3)[0]
    sigma = 0.15
    x, st = ctx.solve(b, sigma, 1e-10)
    ctx.close()
    assert st["converged"]
    A = Qm - sigma * np.eye(Qm.shape[0])
    assert np.linalg.norm(A @ x.ravel() - b.ravel()) <= 1.05e-10 * np.linalg.norm(b)
    xs = np.linalg.solve(A, b.ravel())
    assert np.linalg.norm(x.ravel() - xs) <= 1e-8 * np.linalg.norm(xs)


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_non_hermitian_d_solve_matches_dense(ref, precision):
    """(D - sigma gamma5) x = b, sigma = 0 (the Wilson-clover system) and 0.1,
    against numpy.linalg.solve of the dense D_sigma = gamma5 (Q - sigma)."""
    from paper_1509_06865_gb300 import Context
    from oracle import dirac
    U, op, Qm, w, v = ref
    c = DENSE4
    ctx = Context(c["dims"])
    ctx.set_params(m0=c["m0"], csw=c["csw"], agg=(2, 2, 2, 2), n_tv=8, sap_block=(2, 2, 2, 2), precision=precision)
    ctx.load_gauge(U)
    ctx.setup(5)
    b = synth.z2_noise(c["dims"], 1, 4)[0]
    g5 = np.tile(dirac.GAMMA5_DIAG.repeat(3), Qm.shape[0] // 12)
    for sigma in (0.0, 0.1):
        x, st = ctx.solve_d(b, sigma, 1e-10)
        assert st["converged"], st
        Dm = g5[:, None] * (Qm - sigma * np.eye(Qm.shape[0]))
        assert np.linalg.norm(Dm @ x.ravel() - b.ravel()) <= 1.05e-10 * np.linalg.norm(b)
        xs = np.linalg.solve(Dm, b.ravel())
        assert np.linalg.norm(x.ravel() - xs) <= 1e-8 * np.linalg.norm(xs)
        # and the oracle's stencil form of D_sigma
        assert dirac.norm(op.D_sigma(x, sigma) - b) <= 1.05e-10 * dirac.norm(b)
    ctx.close()


def test_p_from_a_subset_of_the_modes(ref):
    """P built from the first 2 iterated vectors and the setup's other 6 test
    vectors (p_modes = 2): the same 4 lowest pairs as dense eigh."""
    from paper_1509_06865_gb300 import Context
    U, op, Qm, w, v = ref
    c = DENSE4
    ctx = Context(c["dims"])
    ctx.set_params(m0=c["m0"], csw=c["csw"], agg=(2, 2, 2, 2), n_tv=8, sap_block=(2, 2, 2, 2), p_modes=2)
    ctx.load_gauge(U)
    ctx.setup(c["seed"])
    lam, V, res, st = ctx.eigensolve(c["n_eig"], 1e-10)
    ctx.close()
    assert st["converged"] and np.all(res <= 1e-10), st
    assert np.abs(lam - w[:c["n_eig"]]).max() <= 1e-10 * np.abs(w[:c["n_eig"]]).max()
