"""Two-grid pieces of the method, FP64, plain numpy (Sec. 2, Eqs. 2.3-2.6).

Aggregation interpolation (Eq. 2.4).  The fine lattice is cut into aggregates of
agg = (ax, ay, az, at) sites.  For aggregate a and chirality c (c = 0: spins 0,1,
gamma5 = +1; c = 1: spins 2,3, gamma5 = -1) the N_tv test vectors restricted to
(a, c) are orthonormalised in Gram-Schmidt order; the columns (a, c, j) of P are
those orthonormal pieces, so P = diag(P1, P2) in the gamma5 spin ordering and
gamma5 P = P gamma5^c with gamma5^c = diag(+1 on c = 0, -1 on c = 1).

Coarse vectors are arrays [coarse site, c, j]; coarse site index
((ct*CZ + cz)*CY + cy)*CX + cx.

The coarse operator is D_c = P^dag D P (Eq. 2.5), stored as nine blocks per coarse
site (2 N_tv x 2 N_tv): direction 0 = self, 1 + 2 mu = +mu, 2 + 2 mu = -mu, so that

    (D_c x)(a) = sum_d D_c[d](a) x(a + d).

The blocks are kept per hop direction (never merged by target site): on a coarse
lattice of extent 2, a+mu and a-mu are the same site.  Q_c = P^dag Q P = gamma5^c D_c
(Eq. 2.6 and the line before it).

Smoothers.  SAP works on D_sigma = D - sigma gamma5 = gamma5 (Q - sigma) with the
right-hand side gamma5 r (the paper reports SAP unsuitable for Q itself, Sec. 2).
GMRES(k) on Q - sigma is the paper's own smoother for Q.
"""
from __future__ import annotations

import numpy as np

from . import dirac, krylov

NDIR = 9


# ----------------------------------------------------------------------------
# geometry helpers


def _blocked(f: np.ndarray, blk, lead: int):
    """Reshape (lead..., T, Z, Y, X, 4, 3) -> (lead..., nblk, sites_per_blk, 4, 3).

    Block index ((bt*BZ + bz)*BY + by)*BX + bx; site order inside a block is
    (t, z, y, x) lexicographic.
    """
    bx, by, bz, bt = blk
    shp = f.shape
    T, Z, Y, X = shp[lead:lead + 4]
    g = f.reshape(shp[:lead] + (T // bt, bt, Z // bz, bz, Y // by, by, X // bx, bx, 4, 3))
    n = lead
    perm = tuple(range(lead)) + (n, n + 2, n + 4, n + 6, n + 1, n + 3, n + 5, n + 7, n + 8, n + 9)
    g = g.transpose(perm)
    return g.reshape(shp[:lead] + ((T // bt) * (Z // bz) * (Y // by) * (X // bx), bt * bz * by * bx, 4, 3))


def _unblocked(g: np.ndarray, blk, dims, lead: int):
    bx, by, bz, bt = blk
    lx, ly, lz, lt = dims
    shp = g.shape
    h = g.reshape(shp[:lead] + (lt // bt, lz // bz, ly // by, lx // bx, bt, bz, by, bx, 4, 3))
    n = lead
    perm = tuple(range(lead)) + (n, n + 4, n + 1, n + 5, n + 2, n + 6, n + 3, n + 7, n + 8, n + 9)
    return h.transpose(perm).reshape(shp[:lead] + (lt, lz, ly, lx, 4, 3))


def coarse_dims(dims, agg):
    return tuple(d // a for d, a in zip(dims, agg))


def coarse_neighbor(cdims, mu: int, sign: int) -> np.ndarray:
    """Index of coarse site a + sign*mu_hat (periodic) for every coarse site a."""
    cx, cy, cz, ct = cdims
    idx = np.arange(cx * cy * cz * ct).reshape(ct, cz, cy, cx)
    ax = {0: 3, 1: 2, 2: 1, 3: 0}[mu]
    return np.roll(idx, -sign, axis=ax).ravel()


def site_coordinate(dims, mu: int) -> np.ndarray:
    """x_mu of every fine site, shaped (T, Z, Y, X, 1, 1) for masking spinors."""
    lx, ly, lz, lt = dims
    t, z, y, x = np.meshgrid(np.arange(lt), np.arange(lz), np.arange(ly), np.arange(lx), indexing="ij")
    return (x, y, z, t)[mu][..., None, None]


# ----------------------------------------------------------------------------
# interpolation P (Eq. 2.4)


class Interpolation:
    """P built from test vectors W[j] (N_tv fine spinors)."""

    def __init__(self, W: np.ndarray, agg):
        self.agg = tuple(agg)
        self.ntv = W.shape[0]
        self.dims = (W.shape[4], W.shape[3], W.shape[2], W.shape[1])
        self.cdims = coarse_dims(self.dims, self.agg)
        Wb = _blocked(W, self.agg, 1)                    # (ntv, nagg, sites, 4, 3)
        nagg, nsite = Wb.shape[1], Wb.shape[2]
        # (nagg, chirality, sites*2 spins*3 colours, ntv)
        M = Wb.reshape(self.ntv, nagg, nsite, 2, 2, 3).transpose(1, 3, 2, 4, 5, 0)
        M = M.reshape(nagg, 2, nsite * 6, self.ntv)
        Qm, R = np.linalg.qr(M)
        d = np.diagonal(R, axis1=-2, axis2=-1)
        ph = d / np.abs(d)
        # Gram-Schmidt order with a real positive R diagonal: Q -> Q diag(ph)
        self.B = Qm * ph[..., None, :]                   # (nagg, 2, nsite*6, ntv)
        self.nagg, self.nsite = nagg, nsite

    def vectors(self) -> np.ndarray:
        """P as N_tv fine spinors (both chiralities of column j stacked)."""
        B = self.B.reshape(self.nagg, 2, self.nsite, 2, 3, self.ntv)
        f = B.transpose(5, 0, 2, 1, 3, 4).reshape(self.ntv, self.nagg, self.nsite, 4, 3)
        return _unblocked(f, self.agg, self.dims, 1)

    def restrict(self, r: np.ndarray) -> np.ndarray:
        """P^dag r -> coarse vector [coarse site, c, j]."""
        rb = _blocked(r[None], self.agg, 1)[0]           # (nagg, nsite, 4, 3)
        rb = rb.reshape(self.nagg, self.nsite, 2, 6).transpose(0, 2, 1, 3).reshape(self.nagg, 2, self.nsite * 6)
        return np.einsum("acij,aci->acj", np.conj(self.B), rb)

    def prolong(self, e: np.ndarray) -> np.ndarray:
        """P e for a coarse vector e [coarse site, c, j]."""
        f = np.einsum("acij,acj->aci", self.B, e)
        f = f.reshape(self.nagg, 2, self.nsite, 6).transpose(0, 2, 1, 3).reshape(self.nagg, self.nsite, 4, 3)
        return _unblocked(f[None], self.agg, self.dims, 1)[0]

    def column(self, c: int, j: int) -> np.ndarray:
        """Fine vector of columns (a, c, j) of P summed over all aggregates a."""
        e = np.zeros((self.nagg, 2, self.ntv), dtype=np.complex128)
        e[:, c, j] = 1.0
        return self.prolong(e)


# ----------------------------------------------------------------------------
# coarse operator (Eqs. 2.5, 2.6)


def coarse_operator(op: dirac.WilsonClover, P: Interpolation) -> np.ndarray:
    """The nine per-direction blocks of D_c = P^dag D P: array [9, nagg, 2N, 2N].

    Column (c', j') of block d at coarse site a is P^dag restricted to a of the
    fine operator's piece that couples a to a + d, applied to column (c', j') of P.
    A fine hop x -> x +- mu belongs to direction +-mu when it leaves the aggregate
    (x_mu at the aggregate's upper / lower face), otherwise to the self block.
    """
    n2 = 2 * P.ntv
    Dc = np.zeros((NDIR, P.nagg, n2, n2), dtype=np.complex128)
    xm = [site_coordinate(op.dims, mu) % P.agg[mu] for mu in range(4)]
    for c in range(2):
        for j in range(P.ntv):
            w = P.column(c, j)
            col = c * P.ntv + j
            self_part = dirac.apply_local(op.A, op.m0, w)
            for mu in range(4):
                fwd = dirac.hop_forward(op.U, w, mu, op.bc)
                bwd = dirac.hop_backward(op.U, w, mu, op.bc)
                leave_up = xm[mu] == P.agg[mu] - 1
                leave_dn = xm[mu] == 0
                self_part = self_part + np.where(leave_up, 0, fwd) + np.where(leave_dn, 0, bwd)
                Dc[1 + 2 * mu, :, :, col] = P.restrict(np.where(leave_up, fwd, 0)).reshape(P.nagg, n2)
                Dc[2 + 2 * mu, :, :, col] = P.restrict(np.where(leave_dn, bwd, 0)).reshape(P.nagg, n2)
            Dc[0, :, :, col] = P.restrict(self_part).reshape(P.nagg, n2)
    return Dc


def gamma5_coarse(ntv: int) -> np.ndarray:
    return np.concatenate([np.ones(ntv), -np.ones(ntv)])


class CoarseOperator:
    """Q_c - sigma = gamma5^c D_c - sigma on coarse vectors [nagg, 2, ntv]."""

    def __init__(self, Dc: np.ndarray, cdims, ntv: int):
        self.Dc = Dc
        self.cdims = tuple(cdims)
        self.ntv = ntv
        self.nbr = [np.arange(Dc.shape[1])]
        for mu in range(4):
            self.nbr.append(coarse_neighbor(self.cdims, mu, +1))
            self.nbr.append(coarse_neighbor(self.cdims, mu, -1))
        self.g5 = gamma5_coarse(ntv)

    def D(self, x: np.ndarray) -> np.ndarray:
        n = x.shape[0]
        xf = x.reshape(n, 2 * self.ntv)
        y = np.zeros_like(xf)
        for d in range(NDIR):
            y += np.einsum("aij,aj->ai", self.Dc[d], xf[self.nbr[d]])
        return y.reshape(x.shape)

    def apply(self, x: np.ndarray, sigma: float) -> np.ndarray:
        y = self.D(x).reshape(x.shape[0], 2 * self.ntv) * self.g5
        return y.reshape(x.shape) - sigma * x

    def gamma5(self, x: np.ndarray) -> np.ndarray:
        return (x.reshape(x.shape[0], 2 * self.ntv) * self.g5).reshape(x.shape)

    def apply_dsigma(self, x: np.ndarray, sigma: float) -> np.ndarray:
        """(D_c - sigma gamma5^c) x = gamma5^c (Q_c - sigma) x."""
        return self.D(x) - sigma * self.gamma5(x)


# ----------------------------------------------------------------------------
# SAP smoother on D_sigma (Schwarz alternating procedure, Sec. 2)


class SAP:
    """Multiplicative red/black block smoother for D_sigma with block-local MR.

    Blocks of sap_block sites; block colour = (bx + by + bz + bt) mod 2.  Every
    direction must hold an even number (>= 2) of blocks, so that no block touches
    a block of its own colour and the Dirichlet block operator of all blocks of
    one colour is mask * D_sigma * mask.
    """

    def __init__(self, op: dirac.WilsonClover, block):
        self.op = op
        self.block = tuple(block)
        nb = [d // b for d, b in zip(op.dims, self.block)]
        for n, d, b in zip(nb, op.dims, self.block):
            if d % b or n < 2 or n % 2:
                raise ValueError("SAP needs an even number (>= 2) of blocks per direction")
        cx = sum(site_coordinate(op.dims, mu) // self.block[mu] for mu in range(4))
        self.mask = [(cx % 2 == col).astype(np.float64) for col in (0, 1)]

    def _block_sum(self, f: np.ndarray) -> np.ndarray:
        """Per-block sums of a site field f (T, Z, Y, X, 4, 3) -> (nblk,)."""
        return _blocked(f[None], self.block, 1)[0].sum(axis=(1, 2, 3))

    def _block_bcast(self, v: np.ndarray) -> np.ndarray:
        nblk = v.shape[0]
        nsite = int(np.prod(self.block))
        g = np.broadcast_to(v[:, None, None, None], (nblk, nsite, 4, 3))
        return _unblocked(g[None], self.block, self.op.dims, 1)[0]

    def block_mr(self, r: np.ndarray, colour: int, sigma: float, iters: int) -> np.ndarray:
        """k steps of minimal residual on every block of one colour, e0 = 0."""
        m = self.mask[colour]
        e = np.zeros_like(r)
        rho = m * r
        for _ in range(iters):
            q = m * self.op.D_sigma(rho, sigma)
            qr = self._block_sum(np.conj(q) * rho)
            qq = self._block_sum(np.real(np.conj(q) * q))
            alpha = np.where(qq > 0, qr / np.where(qq > 0, qq, 1), 0)
            a = self._block_bcast(alpha) * m
            e = e + a * rho
            rho = rho - a * q
        return e

    def smooth(self, b: np.ndarray, x: np.ndarray, sigma: float, cycles: int, mr_iters: int) -> np.ndarray:
        """`cycles` SAP cycles for D_sigma x = b starting from x."""
        x = x.copy()
        for _ in range(cycles):
            for colour in (0, 1):
                r = b - self.op.D_sigma(x, sigma)
                x = x + self.block_mr(r, colour, sigma, mr_iters)
        return x


# ----------------------------------------------------------------------------
# two-grid cycle (Eq. 2.3 with mu = 0 pre- and nu post-smoothing steps)


class TwoGrid:
    """The preconditioner B ~ (Q - sigma)^-1 of one FGMRES step.

    B r = coarse correction x = P (Q_c - sigma)^-1 P^dag r, then nu post-smoothing
    steps on (Q - sigma) z = r from z = x: SAP cycles on D_sigma z = gamma5 r, or
    GMRES(k) restarts on Q - sigma.

    Coarse solve (Q_c - sigma) e = r_c, A = Q_c - sigma.  The test vectors w_j are
    in range(P), so the coarse vectors W = [P^dag w_1 .. P^dag w_N] represent them
    exactly and W^dag A W = (Ritz matrix of Q on span{w_j}) - sigma.  When the w_j
    approximate eigenvectors (the Rayleigh quotient iteration puts its current
    v_i there) and sigma approaches one of their eigenvalues, A is nearly singular
    exactly on span(W).  That part is solved exactly (deflation): with
    E = W^dag A W and Pi = 1 - A W E^-1 W^dag,
        e = W E^-1 W^dag r_c + (1 - W E^-1 W^dag A) y,   Pi A y = Pi r_c,
    and GMRES solves the projected system in the equivalent form
    gamma5^c Pi A y = gamma5^c Pi r_c (gamma5^c A = D_c - sigma gamma5^c has its
    spectrum in the right half plane; Eq. 2.6 with a shift).  With deflate=False
    GMRES runs on (D_c - sigma gamma5^c) e = gamma5^c r_c directly.
    """

    def __init__(self, op: dirac.WilsonClover, W: np.ndarray, params: dict):
        self.op = op
        self.p = dict(params)
        self.set_test_vectors(W)
        self.sap = SAP(op, self.p["sap_block"]) if self.p["smoother"] == "sap" else None

    deflate_active = True     # the setup switches deflation off (its test vectors are no eigenvectors yet)

    def set_test_vectors(self, W: np.ndarray):
        self.W = np.array(W)
        self.P = Interpolation(self.W, self.p["agg"])
        self.Dc = coarse_operator(self.op, self.P)
        self.coarse = CoarseOperator(self.Dc, self.P.cdims, self.P.ntv)
        self._defl = None

    def deflation(self, sigma: float):
        """(W, A W, E^-1) for the current test vectors and shift."""
        if self._defl is None or self._defl[0] != sigma:
            Wc = [self.P.restrict(w) for w in self.W]
            AW = [self.coarse.apply(x, sigma) for x in Wc]
            E = np.array([[np.vdot(Wc[i], AW[j]) for j in range(len(Wc))] for i in range(len(Wc))])
            self._defl = (sigma, Wc, AW, np.linalg.inv(E))
        return self._defl[1:]

    def coarse_solve(self, rc: np.ndarray, sigma: float) -> np.ndarray:
        C = self.coarse
        gm = dict(tol=self.p["coarse_tol"], restart=self.p["coarse_restart"], maxiter=self.p["coarse_maxiter"])
        if not (self.p.get("coarse_deflate", True) and self.deflate_active):
            ec, _ = krylov.gmres(lambda v: C.apply_dsigma(v, sigma), C.gamma5(rc), **gm)
            return ec
        Wc, AW, Einv = self.deflation(sigma)

        def coeff(u):                      # E^-1 W^dag u
            return Einv @ np.array([np.vdot(w, u) for w in Wc])

        def project(u):                    # Pi u = u - A W E^-1 W^dag u
            t = coeff(u)
            return u - sum(ti * awi for ti, awi in zip(t, AW))

        rhs = C.gamma5(project(rc))
        # the tolerance refers to ||r_c||: a right-hand side lying mostly in span(W)
        # leaves a tiny projected system that needs no further reduction
        rn = np.linalg.norm(rhs)
        gm["tol"] = gm["tol"] * np.linalg.norm(rc) / rn if rn > 0 else 0.0
        y = np.zeros_like(rc) if rn == 0 else krylov.gmres(
            lambda v: C.gamma5(project(C.apply(v, sigma))), rhs, **gm)[0]
        t0 = coeff(rc)
        t1 = coeff(C.apply(y, sigma))
        return y + sum((a - b) * w for a, b, w in zip(t0, t1, Wc))

    def __call__(self, r: np.ndarray, sigma: float) -> np.ndarray:
        x = self.P.prolong(self.coarse_solve(self.P.restrict(r), sigma))
        if self.p["smoother"] == "sap":
            x = self.sap.smooth(dirac.gamma5(r), x, sigma, self.p["sap_cycles"], self.p["sap_mr_iters"])
        else:
            A = lambda v: self.op.Q_sigma(v, sigma)
            for _ in range(self.p["smooth_steps"]):
                e, _ = krylov.gmres(A, r - A(x), tol=0.0, restart=self.p["gmres_smooth_k"],
                                    maxiter=self.p["gmres_smooth_k"])
                x = x + e
        return x


DEFAULT_PARAMS = dict(
    agg=(4, 4, 4, 4),
    ntv=20,
    smoother="sap",
    sap_block=(4, 4, 4, 4),
    sap_cycles=3,
    sap_mr_iters=4,
    smooth_steps=2,
    gmres_smooth_k=8,
    coarse_tol=5e-2,
    coarse_restart=30,
    coarse_maxiter=24,
    coarse_deflate=True,
    ritz_each_sweep=True,
    shift_floor=1e-6,
    guard_maxiter=4,
    ritz_keep=1e-6,
    fine_deflate=True,
    fine_deflate_radius=-1.0,
    adaptive_tol=True,
    ritz_start=True,
    outer_restart=20,
    outer_maxiter=50,
    solve_tol=1e-2,
    setup_smooth=3,
    setup_iters=10,
)
