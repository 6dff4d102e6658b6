"""Clover-improved Wilson Dirac operator, FP64, written out site by site (numpy).

Sec. 2 of the paper names D (clover-improved Wilson), Q = gamma5 D and fixes
gamma5 = -g1 g2 g3 g4 = diag(1, 1, -1, -1) in a chiral representation (text
around Eq. 2.1).  The rest of the convention is our reading of the standard
operator (the paper does not print it):

  D psi(x) = (4 + m0) psi(x)
             - 1/2 sum_mu [ (1 - g_mu) U_mu(x) psi(x+mu) + (1 + g_mu) U_mu(x-mu)^dag psi(x-mu) ]
             + c_sw (i/4) sum_{mu,nu} sigma_{mu nu} F_{mu nu}(x) psi(x)

  sigma_{mu nu} = (i/2)[g_mu, g_nu],   F_{mu nu} = (1/8)(Q_{mu nu} - Q_{mu nu}^dag),
  Q_{mu nu}(x) = sum of the four plaquette leaves at x in the (mu, nu) plane, each
  a closed loop from x taken counter-clockwise (mu first, then nu).

  g_k = [[0, i s_k], [-i s_k, 0]] (k = 1, 2, 3), g_4 = [[0, 1], [1, 0]].

Boundary conditions act on the fermion field only: hopping across the lattice
edge in direction mu multiplies by bc[mu] (+1 periodic, -1 antiperiodic).
D_sigma = D - sigma gamma5, so that Q - sigma = gamma5 D_sigma.
"""
from __future__ import annotations

import numpy as np

# spinor axes, counted from the end: (..., t, z, y, x, spin, colour)
_SPINOR_AXIS = {0: -3, 1: -4, 2: -5, 3: -6}
# gauge component U[t, z, y, x, mu, a, b] -> U_mu[t, z, y, x, a, b]
_LINK_AXIS = {0: -3, 1: -4, 2: -5, 3: -6}


def gamma_matrices():
    """The four Euclidean gamma matrices of the chiral basis and gamma5."""
    s = [np.array([[0, 1], [1, 0]], dtype=complex),
         np.array([[0, -1j], [1j, 0]], dtype=complex),
         np.array([[1, 0], [0, -1]], dtype=complex)]
    z = np.zeros((2, 2), dtype=complex)
    one = np.eye(2, dtype=complex)
    g = [np.block([[z, 1j * sk], [-1j * sk, z]]) for sk in s]
    g.append(np.block([[z, one], [one, z]]))
    g5 = -g[0] @ g[1] @ g[2] @ g[3]
    return g, g5


GAMMA, GAMMA5 = gamma_matrices()
GAMMA5_DIAG = np.real(np.diag(GAMMA5))


def sigma_munu(mu: int, nu: int) -> np.ndarray:
    g = GAMMA
    return 0.5j * (g[mu] @ g[nu] - g[nu] @ g[mu])


def shift_spinor(psi: np.ndarray, mu: int, sign: int, bc) -> np.ndarray:
    """psi(x + sign*mu_hat), with the boundary phase bc[mu] on wrapped sites."""
    ax = _SPINOR_AXIS[mu]
    L = psi.shape[ax]
    out = np.roll(psi, -sign, axis=ax)
    idx = [slice(None)] * psi.ndim
    idx[ax] = L - 1 if sign > 0 else 0
    out[tuple(idx)] *= bc[mu]
    return out


def shift_links(f: np.ndarray, mu: int, sign: int) -> np.ndarray:
    """A colour-matrix field f(x) -> f(x + sign*mu_hat), periodic."""
    return np.roll(f, -sign, axis=_LINK_AXIS[mu])


def link(U: np.ndarray, mu: int) -> np.ndarray:
    return U[..., mu, :, :]


def _mm(a, b):
    return np.einsum("...ab,...bc->...ac", a, b)


def _dag(a):
    return np.conj(np.swapaxes(a, -1, -2))


def field_strength(U: np.ndarray, mu: int, nu: int) -> np.ndarray:
    """F_{mu nu}(x) = (Q - Q^dag)/8 from the four counter-clockwise leaves."""
    Umu, Unu = link(U, mu), link(U, nu)
    s = shift_links
    # leaf 1: x -> x+mu -> x+mu+nu -> x+nu -> x
    l1 = _mm(_mm(Umu, s(Unu, mu, +1)), _mm(_dag(s(Umu, nu, +1)), _dag(Unu)))
    # leaf 2: x -> x+nu -> x+nu-mu -> x-mu -> x
    Umu_m = s(Umu, mu, -1)
    l2 = _mm(_mm(Unu, _dag(s(Umu_m, nu, +1))), _mm(_dag(s(Unu, mu, -1)), Umu_m))
    # leaf 3: x -> x-mu -> x-mu-nu -> x-nu -> x
    Umu_mn = s(Umu_m, nu, -1)
    Unu_mn = s(s(Unu, mu, -1), nu, -1)
    Unu_n = s(Unu, nu, -1)
    l3 = _mm(_mm(_dag(Umu_m), _dag(Unu_mn)), _mm(Umu_mn, Unu_n))
    # leaf 4: x -> x-nu -> x-nu+mu -> x+mu -> x
    Umu_n = s(Umu, nu, -1)
    Unu_nm = s(Unu_n, mu, +1)
    l4 = _mm(_mm(_dag(Unu_n), Umu_n), _mm(Unu_nm, _dag(Umu)))
    Q = l1 + l2 + l3 + l4
    return (Q - _dag(Q)) / 8.0


def clover_matrix(U: np.ndarray, csw: float) -> np.ndarray:
    """A(x) = c_sw (i/4) sum_{mu,nu} sigma_{mu nu} (x) F_{mu nu}(x), as 12x12 per site.

    Row/column index = 3*spin + colour.  Returned shape (T, Z, Y, X, 12, 12).
    """
    shape = U.shape[:4]
    A = np.zeros(shape + (12, 12), dtype=np.complex128)
    for mu in range(4):
        for nu in range(4):
            if mu == nu:
                continue
            F = field_strength(U, mu, nu)
            sig = sigma_munu(mu, nu)
            A += np.einsum("st,...ab->...satb", sig, F).reshape(shape + (12, 12))
    return csw * 0.25j * A


def hop_forward(U: np.ndarray, psi: np.ndarray, mu: int, bc) -> np.ndarray:
    """-1/2 (1 - g_mu) U_mu(x) psi(x + mu)."""
    proj = np.eye(4) - GAMMA[mu]
    up = shift_spinor(psi, mu, +1, bc)
    up = np.einsum("...ab,...sb->...sa", link(U, mu), up)
    return -0.5 * np.einsum("st,...tc->...sc", proj, up)


def hop_backward(U: np.ndarray, psi: np.ndarray, mu: int, bc) -> np.ndarray:
    """-1/2 (1 + g_mu) U_mu(x - mu)^dag psi(x - mu)."""
    proj = np.eye(4) + GAMMA[mu]
    dn = shift_spinor(psi, mu, -1, bc)
    Ub = shift_links(link(U, mu), mu, -1)
    dn = np.einsum("...ba,...sb->...sa", np.conj(Ub), dn)
    return -0.5 * np.einsum("st,...tc->...sc", proj, dn)


def apply_local(A: np.ndarray, m0: float, psi: np.ndarray) -> np.ndarray:
    """(4 + m0) psi + A psi  (mass term and clover term, site-diagonal)."""
    shp = psi.shape
    flat = psi.reshape(shp[:-2] + (12,))
    out = (4.0 + m0) * flat + np.einsum("...ij,...j->...i", A, flat)
    return out.reshape(shp)


class WilsonClover:
    """D, Q = gamma5 D and D_sigma on one gauge background (FP64)."""

    def __init__(self, U: np.ndarray, m0: float, csw: float, bc=(1, 1, 1, 1), A=None):
        self.U = np.asarray(U, dtype=np.complex128)
        self.m0 = float(m0)
        self.csw = float(csw)
        self.bc = tuple(int(b) for b in bc)
        self.A = clover_matrix(self.U, self.csw) if A is None else A
        self.dims = (U.shape[3], U.shape[2], U.shape[1], U.shape[0])

    @property
    def volume(self) -> int:
        lx, ly, lz, lt = self.dims
        return lx * ly * lz * lt

    def D(self, psi: np.ndarray) -> np.ndarray:
        out = apply_local(self.A, self.m0, psi)
        for mu in range(4):
            out = out + hop_forward(self.U, psi, mu, self.bc)
            out = out + hop_backward(self.U, psi, mu, self.bc)
        return out

    def D_sigma(self, psi: np.ndarray, sigma: float) -> np.ndarray:
        """D - sigma gamma5."""
        return self.D(psi) - sigma * gamma5(psi)

    def Q(self, psi: np.ndarray) -> np.ndarray:
        return gamma5(self.D(psi))

    def Q_sigma(self, psi: np.ndarray, sigma: float) -> np.ndarray:
        """(Q - sigma) psi."""
        return gamma5(self.D(psi)) - sigma * psi


def gamma5(psi: np.ndarray) -> np.ndarray:
    return psi * GAMMA5_DIAG[:, None]


def dot(a: np.ndarray, b: np.ndarray) -> complex:
    """<a|b> = sum conj(a) b over every index."""
    return complex(np.vdot(a, b))


def norm(a: np.ndarray) -> float:
    return float(np.sqrt(np.real(np.vdot(a, a))))


def apply_at_site(U: np.ndarray, psi: np.ndarray, site, m0: float, csw: float, bc=(1, 1, 1, 1),
                  sigma: float = 0.0, form: str = "Q") -> np.ndarray:
    """One site of (Q - sigma) psi (form "Q") or (D - sigma gamma5) psi (form "D"),
    for lattices too large for the whole-lattice operator above.

    The operator is local: the hopping terms at x read psi(x +- mu) and the
    clover term the links of the leaves around x, all on sites within one step
    of x in every direction.  So the value at x is the whole-lattice operator
    of this module applied to the 3^4 patch of links and spinors around x,
    read at the patch centre; the patch copies psi(x +- mu) with the boundary
    phase bc[mu] already applied where the step crosses the lattice edge (the
    patch itself is never wrapped at its centre).  site = (x, y, z, t); U and psi
    in this module's layout (T, Z, Y, X, ...).  Returns the (4, 3) spinor.
    """
    dims = (U.shape[3], U.shape[2], U.shape[1], U.shape[0])     # (Lx, Ly, Lz, Lt)
    idx, phase = [], []
    for mu in range(4):
        c = np.arange(site[mu] - 1, site[mu] + 2)
        idx.append(c % dims[mu])
        phase.append(np.where((c < 0) | (c >= dims[mu]), bc[mu], 1).astype(float))
    it, iz, iy, ix = idx[3], idx[2], idx[1], idx[0]
    Up = U[np.ix_(it, iz, iy, ix)]
    pp = psi[np.ix_(it, iz, iy, ix)].copy()
    pp *= (phase[3][:, None, None, None] * phase[2][None, :, None, None] * phase[1][None, None, :, None]
           * phase[0][None, None, None, :])[..., None, None]
    op = WilsonClover(Up, m0, csw, bc=(1, 1, 1, 1))
    out = op.Q_sigma(pp, sigma) if form == "Q" else op.D_sigma(pp, sigma)
    return out[1, 1, 1, 1]
