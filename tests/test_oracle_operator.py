"""Pins of the oracle's Wilson-clover operator against facts fixed by the paper
(gamma5 = -g1 g2 g3 g4 = diag(1,-1), Q = gamma5 D Hermitian; Sec. 2) and by the
mathematics (free-field momentum-space spectrum, gauge covariance, a single
deformed link worked out by hand for the clover term)."""
import numpy as np
import pytest

import synth
from oracle import dense, dirac


def test_gamma_algebra():
    g, g5 = dirac.GAMMA, dirac.GAMMA5
    for m in range(4):
        assert np.allclose(g[m], g[m].conj().T)
        for n in range(4):
            assert np.allclose(g[m] @ g[n] + g[n] @ g[m], 2 * (m == n) * np.eye(4))
    assert np.allclose(g5, np.diag([1, 1, -1, -1]))
    for m in range(4):
        for n in range(4):
            s = dirac.sigma_munu(m, n)
            assert np.allclose(s @ g5, g5 @ s)   # clover term is block diagonal in chirality


def _free_spectrum(dims, m0, bc):
    ps = []
    for L, b in zip(dims, bc):
        n = np.arange(L)
        ps.append(2 * np.pi * n / L if b == 1 else (2 * n + 1) * np.pi / L)
    P = np.meshgrid(*ps, indexing="ij")
    M = m0 + sum(1 - np.cos(p) for p in P)
    lam = np.sqrt(M ** 2 + sum(np.sin(p) ** 2 for p in P)).ravel()
    return np.sort(np.concatenate([np.repeat(lam, 6), -np.repeat(lam, 6)]))


@pytest.mark.parametrize("dims,m0,bc", [((4, 4, 4, 4), -0.4, (1, 1, 1, -1)),
                                        ((2, 2, 4, 4), 0.3, (1, 1, 1, 1)),
                                        ((2, 4, 2, 6), -1.1, (1, -1, 1, -1))])
def test_free_field_spectrum_closed_form(dims, m0, bc):
    """U = 1: Q(p) = gamma5 [M(p) + i sum g_mu sin p_mu], eigenvalues +-sqrt(M^2 + sum sin^2 p)."""
    op = dirac.WilsonClover(synth.unit_gauge(dims), m0, 1.9, bc=bc)
    ev = np.linalg.eigvalsh(dense.operator_matrix(op.Q, dims))
    assert np.abs(ev - _free_spectrum(dims, m0, bc)).max() < 1e-12


def test_gamma5_hermiticity_and_hermitian_Q():
    dims = (4, 4, 2, 4)
    op = dirac.WilsonClover(synth.gauge_field(dims, 0.3, 3), -0.4, 1.9, bc=(1, 1, 1, -1))
    x, y = synth.gaussian_vectors(dims, 2, 4)
    lhs = dirac.dot(y, op.D(x))
    rhs = dirac.dot(dirac.gamma5(op.D(dirac.gamma5(y))), x)   # D^dag = gamma5 D gamma5
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    assert abs(dirac.dot(y, op.Q(x)) - dirac.dot(op.Q(y), x)) < 1e-12 * abs(lhs)
    A = op.A.reshape(-1, 12, 12)
    assert np.abs(A - A.conj().transpose(0, 2, 1)).max() < 1e-15
    assert np.abs(A[:, :6, 6:]).max() == 0 and np.abs(A[:, 6:, :6]).max() == 0


def test_gauge_covariance():
    dims = (4, 2, 4, 4)
    U = synth.gauge_field(dims, 0.5, 5)
    g = synth.gauge_field(dims, 1.0, 6)[..., 0, :, :]          # random SU(3) per site
    Ug = np.empty_like(U)
    for mu in range(4):
        gp = dirac.shift_links(g, mu, +1)
        Ug[..., mu, :, :] = np.einsum("...ab,...bc,...dc->...ad", g, U[..., mu, :, :], gp.conj())
    psi = synth.gaussian_vectors(dims, 1, 9)[0]
    gpsi = np.einsum("...ab,...sb->...sa", g, psi)
    for bc in [(1, 1, 1, 1), (1, 1, 1, -1)]:
        op = dirac.WilsonClover(U, -0.3, 1.7, bc=bc)
        opg = dirac.WilsonClover(Ug, -0.3, 1.7, bc=bc)
        lhs = opg.D(gpsi)
        rhs = np.einsum("...ab,...sb->...sa", g, op.D(psi))
        assert np.abs(lhs - rhs).max() < 1e-12


def test_clover_single_deformed_link_by_hand():
    """All links 1 except U_x(0) = diag(e^{i th}, e^{-i th}, 1).

    Only the plaquettes containing that link differ from 1.  Working through the
    four leaves: F_{x nu} = +(i/4) sin(th) T at x0+nu and x0+x+nu, -(i/4) sin(th) T
    at x0-nu and x0+x-nu (T = diag(1,-1,0)), zero at x0 and x0+x (the two leaves
    there cancel) and zero in every other plane, so A = c_sw (i/2) sigma_{x nu} F_{x nu}.
    """
    dims = (4, 4, 4, 4)
    th, csw = 0.7, 1.3
    U = synth.unit_gauge(dims)
    U[0, 0, 0, 0, 0] = np.diag([np.exp(1j * th), np.exp(-1j * th), 1.0])
    A = dirac.clover_matrix(U, csw)
    T = np.diag([1.0, -1.0, 0.0])
    want = np.zeros_like(A)

    def site(x, y, z, t):
        return (t % 4, z % 4, y % 4, x % 4)

    for nu in (1, 2, 3):
        e = [0, 0, 0, 0]
        e[nu] = 1
        blk = np.kron(dirac.sigma_munu(0, nu), T) * (csw / 8) * np.sin(th)
        for dx in (0, 1):
            want[site(dx + e[0], e[1], e[2], e[3])] += -blk
            want[site(dx - e[0], -e[1], -e[2], -e[3])] += blk
    assert np.abs(A - want).max() < 1e-15
    assert np.abs(A).max() > 0.05


def test_clover_vanishes_for_unit_links():
    A = dirac.clover_matrix(synth.unit_gauge((2, 2, 2, 2)), 1.9)
    assert np.abs(A).max() == 0


def test_operator_at_one_site_equals_the_whole_lattice_operator():
    """dirac.apply_at_site (the 3^4 patch around a site, for sampled checks on
    lattices too large for the whole-lattice operator) agrees with the
    whole-lattice Q - sigma and D - sigma gamma5 at every site of an uneven,
    partly antiperiodic lattice, the edge sites included."""
    import itertools
    dims, bc = (4, 6, 4, 4), (-1, 1, 1, -1)
    U = synth.gauge_field(dims, 0.3, 5)
    psi = synth.gaussian_vectors(dims, 1, 6)[0]
    op = dirac.WilsonClover(U, -0.3, 1.7, bc=bc)
    for form, sigma in (("Q", 0.07), ("D", -0.02)):
        full = op.Q_sigma(psi, sigma) if form == "Q" else op.D_sigma(psi, sigma)
        for x, y, z, t in itertools.product(*(range(L) for L in dims)):
            v = dirac.apply_at_site(U, psi, (x, y, z, t), -0.3, 1.7, bc, sigma, form)
            assert np.abs(v - full[t, z, y, x]).max() <= 1e-14 * np.abs(full).max()
