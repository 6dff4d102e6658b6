"""Pins of the oracle's two-grid pieces (Sec. 2, Eqs. 2.3-2.6) and Krylov solvers
against dense linear algebra on small lattices: P^dag P = 1, gamma5 P = P gamma5^c
(Eq. 2.4), the per-direction coarse blocks summed = P^dag D P (Eq. 2.5),
gamma5^c D_c Hermitian (Eq. 2.5), equal coarse corrections for D and Q (Eq. 2.6),
block MR converging to the exact Dirichlet block solve, and GMRES/FGMRES reaching
the dense solution."""
import numpy as np
import pytest

import synth
from oracle import dense, dirac, krylov, mg

DIMS = (4, 4, 4, 4)
AGG = (2, 2, 2, 2)
NTV = 6


@pytest.fixture(scope="module")
def setup4():
    U = synth.gauge_field(DIMS, 0.3, 1001)
    op = dirac.WilsonClover(U, -0.4, 1.0, bc=(1, 1, 1, -1))
    W = synth.uniform_vectors(DIMS, NTV, 77)
    P = mg.Interpolation(W, AGG)
    Dmat = dense.operator_matrix(op.D, DIMS)
    # dense P: columns ordered (coarse site, c, j)
    nc = P.nagg * 2 * NTV
    E = np.eye(nc).reshape(nc, P.nagg, 2, NTV)
    Pmat = np.array([P.prolong(e).ravel() for e in E]).T
    return op, W, P, Dmat, Pmat


def test_interpolation_orthonormal_and_gamma5_compatible(setup4):
    op, W, P, Dmat, Pmat = setup4
    assert np.abs(Pmat.conj().T @ Pmat - np.eye(Pmat.shape[1])).max() < 1e-13
    g5 = np.tile(np.repeat(dirac.GAMMA5_DIAG, 3), Pmat.shape[0] // 12)
    g5c = np.tile(mg.gamma5_coarse(NTV), P.nagg)
    assert np.abs(g5[:, None] * Pmat - Pmat * g5c[None, :]).max() < 1e-14
    # each test vector lies in range(P): P P^dag w = w
    for w in W:
        assert np.abs(P.prolong(P.restrict(w)) - w).max() < 1e-13
    # Gram-Schmidt order: column j of aggregate a only mixes test vectors 0..j
    Wb = [P.restrict(w) for w in W]
    for j in range(NTV):
        if j + 1 < NTV:
            assert np.abs(Wb[j][:, :, j + 1:]).max() < 1e-13
        assert np.all(np.abs(Wb[j][:, :, j].imag) < 1e-13) and np.all(Wb[j][:, :, j].real > 0)


def test_coarse_operator_equals_galerkin_product(setup4):
    op, W, P, Dmat, Pmat = setup4
    Dc = mg.coarse_operator(op, P)
    n2 = 2 * NTV
    dense_c = Pmat.conj().T @ Dmat @ Pmat
    nbr = [np.arange(P.nagg)] + [mg.coarse_neighbor(P.cdims, mu, s) for mu in range(4) for s in (1, -1)]
    asm = np.zeros_like(dense_c)
    for d in range(mg.NDIR):
        for a in range(P.nagg):
            b = nbr[d][a]
            asm[a * n2:(a + 1) * n2, b * n2:(b + 1) * n2] += Dc[d, a]
    assert np.abs(asm - dense_c).max() < 1e-13
    # coarse extent 2: +mu and -mu reach the same site, yet the blocks differ
    assert np.abs(Dc[1] - Dc[2]).max() > 1e-3
    # gamma5^c D_c is Hermitian (Eq. 2.5)
    g5c = np.tile(mg.gamma5_coarse(NTV), P.nagg)
    Qc = g5c[:, None] * dense_c
    assert np.abs(Qc - Qc.conj().T).max() < 1e-13
    # coarse apply with a shift
    C = mg.CoarseOperator(Dc, P.cdims, NTV)
    x = np.random.default_rng(1).standard_normal((P.nagg, 2, NTV)) + 0j
    assert np.abs(C.apply(x, 0.13).ravel() - (Qc @ x.ravel() - 0.13 * x.ravel())).max() < 1e-13


def test_equal_coarse_corrections_for_D_and_Q(setup4):
    """Eq. 2.6: 1 - P Q_c^-1 P^dag Q = 1 - P D_c^-1 P^dag D."""
    op, W, P, Dmat, Pmat = setup4
    g5 = np.tile(np.repeat(dirac.GAMMA5_DIAG, 3), Pmat.shape[0] // 12)
    Qmat = g5[:, None] * Dmat
    Dc = Pmat.conj().T @ Dmat @ Pmat
    Qc = Pmat.conj().T @ Qmat @ Pmat
    v = synth.gaussian_vectors(DIMS, 1, 3)[0].ravel()
    eq = v - Pmat @ np.linalg.solve(Qc, Pmat.conj().T @ (Qmat @ v))
    ed = v - Pmat @ np.linalg.solve(Dc, Pmat.conj().T @ (Dmat @ v))
    assert np.abs(eq - ed).max() < 1e-10 * np.abs(v).max()


def test_block_mr_converges_to_dirichlet_block_solve(setup4):
    op, W, P, Dmat, Pmat = setup4
    sap = mg.SAP(op, (2, 2, 2, 2))
    sigma = 0.05
    r = synth.gaussian_vectors(DIMS, 1, 4)[0]
    e = sap.block_mr(r, 0, sigma, 300)
    g5 = np.tile(np.repeat(dirac.GAMMA5_DIAG, 3), Dmat.shape[0] // 12)
    Ds = Dmat - sigma * np.diag(g5)
    m = np.broadcast_to(sap.mask[0], r.shape).ravel() > 0
    # exact: the colour-0 blocks decouple, so solve the masked system directly
    want = np.zeros(r.size, dtype=complex)
    want[m] = np.linalg.solve(Ds[np.ix_(m, m)], r.ravel()[m])
    assert np.abs(e.ravel() - want).max() < 1e-9


def test_gmres_and_fgmres_reach_dense_solution(setup4):
    op, W, P, Dmat, Pmat = setup4
    sigma = 0.1
    g5 = np.tile(np.repeat(dirac.GAMMA5_DIAG, 3), Dmat.shape[0] // 12)
    A = g5[:, None] * Dmat - sigma * np.eye(Dmat.shape[0])
    b = synth.gaussian_vectors(DIMS, 1, 8)[0]
    want = np.linalg.solve(A, b.ravel())
    x, info = krylov.gmres(lambda v: op.Q_sigma(v, sigma), b, tol=1e-11, restart=40, maxiter=3000)
    assert np.abs(x.ravel() - want).max() < 1e-7 * np.abs(want).max()
    params = dict(mg.DEFAULT_PARAMS, agg=AGG, ntv=NTV, sap_block=(2, 2, 2, 2))
    B = mg.TwoGrid(op, W, params)
    x, info = krylov.fgmres(lambda v: op.Q_sigma(v, sigma), lambda r: B(r, sigma), b,
                            tol=1e-11, restart=20, maxiter=200)
    assert info["resid"] < 1e-11
    assert np.abs(x.ravel() - want).max() < 1e-7 * np.abs(want).max()
    # GMRES with tol = 0 runs exactly maxiter Arnoldi steps
    _, info = krylov.gmres(lambda v: op.Q_sigma(v, sigma), b, tol=0.0, restart=5, maxiter=7)
    assert info["iters"] == 7


def test_deflated_preconditioner_solves_the_deflation_space_exactly(setup4):
    """The fine-grid deflation of the eigensolver's shifted solves:
    z = Z E^-1 Z^dag r + B (r - (Q - sigma) Z E^-1 Z^dag r), E = Z^dag (Q - sigma) Z.
    For r = (Q - sigma) Z c the residual handed to B vanishes and z = Z c
    exactly, for any Z and any B; for r orthogonal to Z the first term vanishes
    and B sees r - (Q - sigma) Z E^-1 Z^dag r = r."""
    from oracle import rqi
    op, W, P, Dmat, Pmat = setup4
    sigma = 0.07
    Z = synth.gaussian_vectors(DIMS, 3, 5)

    class Spy:                       # stands in for the two-grid method B
        def __call__(self, r, s):
            self.seen = r.copy()
            return 2.0 * r

    B = Spy()
    M = rqi.deflated_preconditioner(op, Z, B, sigma)
    coeff = np.array([0.3 - 0.2j, -1.1 + 0.5j, 0.7j])
    zc = np.tensordot(coeff, Z, axes=1)
    r = op.Q_sigma(zc, sigma)
    out = M(r)
    assert np.abs(B.seen).max() < 1e-12 * np.abs(r).max()
    assert np.abs(out - zc).max() < 1e-12 * np.abs(zc).max()
    # r orthogonal to span(Z): no deflation component, B gets r itself
    Zf = Z.reshape(3, -1)
    q, _ = np.linalg.qr(Zf.T)
    r2 = synth.gaussian_vectors(DIMS, 1, 6)[0].ravel()
    r2 = (r2 - q @ (q.conj().T @ r2)).reshape(zc.shape)
    out2 = M(r2)
    assert np.abs(B.seen - r2).max() < 1e-12 * np.abs(r2).max()
    assert np.abs(out2 - 2.0 * r2).max() < 1e-12 * np.abs(r2).max()
