"""Pins of the oracle's two-grid pieces (Sec. 2, Eqs. 2.3-2.6) and Krylov solvers
against dense linear algebra on small lattices: P^dag P = 1, gamma5 P = P gamma5^c
(Eq. 2.4), the per-direction coarse blocks summed = P^dag D P (Eq. 2.5),
gamma5^c D_c Hermitian (Eq. 2.5), equal coarse corrections for D and Q (Eq. 2.6),
block MR converging to the exact Dirichlet block solve, one MR step minimising
each block's residual, SAP with exact blocks = multiplicative Schwarz in the
colour order 0, 1, the two-grid cycle = exact coarse correction followed by the
post-smoother (SAP on D_sigma with right-hand side gamma5 r, or GMRES(k) as the
least-squares minimiser over the Krylov space; deflated and plain coarse solves
alike), and GMRES/FGMRES reaching the dense solution."""
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


def _dense_dsigma(op, Dmat, sigma):
    g5 = np.tile(np.repeat(dirac.GAMMA5_DIAG, 3), Dmat.shape[0] // 12)
    return Dmat - sigma * np.diag(g5), g5


def _masked_solve(Ds, mask, r):
    """The exact Dirichlet solve on every block of one colour (the blocks of a
    colour do not touch, so the masked system is block diagonal)."""
    m = mask.ravel() > 0
    out = np.zeros(r.size, dtype=complex)
    out[m] = np.linalg.solve(Ds[np.ix_(m, m)], r.ravel()[m])
    return out


def test_one_mr_step_minimises_each_block_residual(setup4):
    """One block MR step from e = 0 takes e_B = alpha_B r_B with the alpha_B that
    minimises ||r_B - alpha A_BB r_B|| on every block B of the colour: the
    residual left on B is orthogonal to A_BB r_B, and nudging alpha_B in any
    complex direction raises it."""
    op, W, P, Dmat, Pmat = setup4
    sap = mg.SAP(op, (2, 2, 2, 2))
    sigma = 0.05
    Ds, _ = _dense_dsigma(op, Dmat, sigma)
    r = synth.gaussian_vectors(DIMS, 1, 11)[0]
    for colour in (0, 1):
        mask = np.broadcast_to(sap.mask[colour], r.shape)
        e = sap.block_mr(r, colour, sigma, 1).ravel()
        m = mask.ravel() > 0
        A = Ds[np.ix_(m, m)]                       # block diagonal over the colour's blocks
        rb, eb = r.ravel()[m], e[m]
        assert np.abs(e[~m]).max() == 0.0           # nothing written outside the colour
        blk = _block_index(mask, sap)[m]            # block id of each masked unknown
        for b in np.unique(blk):
            s = blk == b
            Arb = (A @ np.where(s, rb, 0))[s]
            alpha = np.vdot(rb[s], eb[s]) / np.vdot(rb[s], rb[s])
            assert np.abs(eb[s] - alpha * rb[s]).max() < 1e-13 * np.abs(eb[s]).max()
            left = rb[s] - alpha * Arb
            assert abs(np.vdot(Arb, left)) < 1e-12 * np.linalg.norm(Arb) * np.linalg.norm(rb[s])
            for d in (1e-3, 1e-3j, -1e-3, -1e-3j):
                assert np.linalg.norm(rb[s] - alpha * (1 + d) * Arb) > np.linalg.norm(left)


def _block_index(mask, sap):
    """Block index (0 .. nblk-1) of every entry of a (T, Z, Y, X, 4, 3) field."""
    dims = sap.op.dims
    idx = sum(mg.site_coordinate(dims, mu) // sap.block[mu] * int(np.prod([dims[n] // sap.block[n] for n in range(mu)]))
              for mu in range(4))
    return np.broadcast_to(idx, mask.shape).ravel()


def test_sap_cycles_with_exact_blocks_are_multiplicative_schwarz(setup4):
    """With the block MR run to convergence, `cycles` SAP cycles are the
    multiplicative Schwarz iteration on D_sigma: per cycle, colour 0 then colour
    1, x <- x + M_c (b - D_sigma x) with M_c the exact Dirichlet solve on the
    colour's blocks."""
    op, W, P, Dmat, Pmat = setup4
    sap = mg.SAP(op, (2, 2, 2, 2))
    sigma = -0.03
    Ds, _ = _dense_dsigma(op, Dmat, sigma)
    b = synth.gaussian_vectors(DIMS, 1, 12)[0]
    x0 = synth.gaussian_vectors(DIMS, 1, 13)[0]
    got = sap.smooth(b, x0, sigma, 2, 300).ravel()
    x = x0.ravel().astype(complex)
    for _ in range(2):
        for colour in (0, 1):
            mask = np.broadcast_to(sap.mask[colour], b.shape)
            x = x + _masked_solve(Ds, mask, b.ravel() - Ds @ x)
    assert np.abs(got - x).max() < 1e-9 * np.abs(x).max()
    # the colour order matters: the other order gives another result
    y = x0.ravel().astype(complex)
    for colour in (1, 0):
        mask = np.broadcast_to(sap.mask[colour], b.shape)
        y = y + _masked_solve(Ds, mask, b.ravel() - Ds @ y)
    one = sap.smooth(b, x0, sigma, 1, 300).ravel()
    assert np.abs(one - y).max() > 1e-3 * np.abs(y).max()


@pytest.mark.parametrize("deflate", [False, True])
def test_two_grid_is_exact_coarse_correction_then_sap(setup4, deflate):
    """Eq. 2.3 with mu = 0, nu = 1 and exact pieces: B r = S(x) with
    x = P (P^dag (Q - sigma) P)^-1 P^dag r, then one SAP cycle (exact blocks) on
    D_sigma z = gamma5 r from z = x.  With the coarse GMRES run to convergence
    the deflated and the plain coarse solve give the same B r (the deflation
    is exact on span(W))."""
    op, W, P, Dmat, Pmat = setup4
    sigma = 0.04
    Ds, g5 = _dense_dsigma(op, Dmat, sigma)
    Qs = g5[:, None] * Dmat - sigma * np.eye(Dmat.shape[0])
    params = dict(mg.DEFAULT_PARAMS, agg=AGG, ntv=NTV, sap_block=(2, 2, 2, 2), sap_cycles=1, sap_mr_iters=300,
                  coarse_tol=1e-14, coarse_restart=60, coarse_maxiter=600, coarse_deflate=deflate)
    B = mg.TwoGrid(op, W, params)
    r = synth.gaussian_vectors(DIMS, 1, 14)[0]
    got = B(r, sigma).ravel()
    x = Pmat @ np.linalg.solve(Pmat.conj().T @ Qs @ Pmat, Pmat.conj().T @ r.ravel())
    g5r = g5 * r.ravel()
    for colour in (0, 1):
        mask = np.broadcast_to(B.sap.mask[colour], r.shape)
        x = x + _masked_solve(Ds, mask, g5r - Ds @ x)
    assert np.abs(got - x).max() < 1e-9 * np.abs(x).max()


def test_two_grid_gmres_smoother_minimises_over_the_krylov_space(setup4):
    """The GMRES(k) post-smoother: one step from the coarse correction x adds
    the e in K_k(Q - sigma, r - (Q - sigma) x) of least residual, the
    least-squares solution over the Krylov space's monomial basis."""
    op, W, P, Dmat, Pmat = setup4
    sigma = 0.04
    k = 4
    Ds, g5 = _dense_dsigma(op, Dmat, sigma)
    Qs = g5[:, None] * Dmat - sigma * np.eye(Dmat.shape[0])
    params = dict(mg.DEFAULT_PARAMS, agg=AGG, ntv=NTV, smoother="gmres", smooth_steps=1, gmres_smooth_k=k,
                  coarse_tol=1e-14, coarse_restart=60, coarse_maxiter=600, coarse_deflate=False)
    B = mg.TwoGrid(op, W, params)
    rf = synth.gaussian_vectors(DIMS, 1, 15)[0]
    got = B(rf, sigma).ravel()
    r = rf.ravel()
    x = Pmat @ np.linalg.solve(Pmat.conj().T @ Qs @ Pmat, Pmat.conj().T @ r)
    r0 = r - Qs @ x
    K = [r0]
    for _ in range(k - 1):
        K.append(Qs @ K[-1])
    K = np.array(K).T
    y = np.linalg.lstsq(Qs @ K, r0, rcond=None)[0]
    want = x + K @ y
    assert np.abs(got - want).max() < 1e-8 * np.abs(want).max()
