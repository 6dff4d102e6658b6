"""Pins of the oracle's GMRES and flexible GMRES (the solvers of Sec. 2 and
2.2) by the property that defines them, on small dense complex systems: k
steps of GMRES from zero give the vector of least residual in the Krylov space
K_k(A, b); k steps of FGMRES give the vector of least residual in the span of
the preconditioned vectors z_j it formed, whatever the preconditioner does from
step to step; with a fixed preconditioner M that is M times the GMRES solution
of A M y = b.  The residual estimate the solvers report is the true residual."""
import numpy as np
import pytest

from oracle import krylov

N = 60


def _system(seed=2):
    rng = np.random.default_rng(seed)
    A = np.eye(N) * (2.0 + 0.5j) + 0.3 * (rng.standard_normal((N, N)) + 1j * rng.standard_normal((N, N))) / np.sqrt(N)
    b = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    return A, b, rng


def _least_residual(A, b, S):
    """The x in span(columns of S) minimising ||b - A x||."""
    y = np.linalg.lstsq(A @ S, b, rcond=None)[0]
    return S @ y


@pytest.mark.parametrize("k", [1, 3, 6])
def test_gmres_steps_minimise_over_the_krylov_space(k):
    A, b, _ = _system()
    x, info = krylov.gmres(lambda v: A @ v, b, tol=0.0, restart=k, maxiter=k)
    K = np.array([np.linalg.matrix_power(A, i) @ b for i in range(k)]).T
    want = _least_residual(A, b, K)
    assert info["iters"] == k
    assert np.abs(x - want).max() < 1e-10 * np.abs(want).max()
    assert abs(info["resid"] - np.linalg.norm(b - A @ x) / np.linalg.norm(b)) < 1e-12


def test_fgmres_minimises_over_the_span_of_its_preconditioned_vectors():
    A, b, rng = _system(3)
    seen = []

    def varying(v):          # a different preconditioner at every step
        M = np.eye(N) + 0.2 * rng.standard_normal((N, N)) / np.sqrt(N)
        z = M @ v
        seen.append(z)
        return z

    k = 5
    x, info = krylov.fgmres(lambda v: A @ v, varying, b, tol=0.0, restart=k, maxiter=k)
    assert len(seen) == k
    want = _least_residual(A, b, np.array(seen).T)
    assert np.abs(x - want).max() < 1e-10 * np.abs(want).max()
    assert abs(info["resid"] - np.linalg.norm(b - A @ x) / np.linalg.norm(b)) < 1e-12


def test_fgmres_with_a_fixed_preconditioner_is_right_preconditioned_gmres():
    A, b, rng = _system(4)
    M = np.linalg.inv(A) + 0.05 * rng.standard_normal((N, N)) / np.sqrt(N)
    k = 4
    x, _ = krylov.fgmres(lambda v: A @ v, lambda v: M @ v, b, tol=0.0, restart=k, maxiter=k)
    y, _ = krylov.gmres(lambda v: A @ (M @ v), b, tol=0.0, restart=k, maxiter=k)
    assert np.abs(x - M @ y).max() < 1e-10 * np.abs(x).max()


def test_restarts_continue_from_the_last_iterate():
    """GMRES(2) for 4 steps = 2 steps from zero, then 2 steps on the residual."""
    A, b, _ = _system(5)
    x, _ = krylov.gmres(lambda v: A @ v, b, tol=0.0, restart=2, maxiter=4)
    x1 = _least_residual(A, b, np.array([b, A @ b]).T)
    r1 = b - A @ x1
    x2 = x1 + _least_residual(A, r1, np.array([r1, A @ r1]).T)
    assert np.abs(x - x2).max() < 1e-10 * np.abs(x2).max()
