"""Restarted GMRES and flexible GMRES, FP64, textbook form (Saad, Iterative
Methods for Sparse Linear Systems, Alg. 6.9 and 9.6).

The paper solves every shifted system of the Rayleigh quotient iteration with
a double precision flexible GMRES preconditioned by the multigrid method, and
uses restarted GMRES as smoother and coarse-grid solver for Q (Sec. 2 and the
implementation notes of Sec. 2.2).  Vectors are numpy arrays of any shape;
Arnoldi uses modified Gram-Schmidt, the least-squares problem Givens rotations.
"""
from __future__ import annotations

import numpy as np


def _vdot(a, b):
    return complex(np.vdot(a, b))


def _norm(a):
    return float(np.sqrt(np.real(np.vdot(a, a))))


def _givens(a: complex, b: complex):
    """(c, s) with [[c, s], [-conj(s), c]] [a, b]^T = [r, 0]^T, c real."""
    if b == 0:
        return 1.0, 0.0
    if a == 0:
        return 0.0, 1.0
    t = np.hypot(abs(a), abs(b))
    c = abs(a) / t
    s = (a / abs(a)) * np.conj(b) / t
    return c, s


def _arnoldi_cycle(apply_A, precond, r0, beta, m, tol_abs, flexible):
    """One restart cycle; returns (x correction, residual estimate, iterations)."""
    V = [r0 / beta]
    Z = []
    H = np.zeros((m + 1, m), dtype=np.complex128)
    cs = np.zeros(m)
    sn = np.zeros(m, dtype=np.complex128)
    g = np.zeros(m + 1, dtype=np.complex128)
    g[0] = beta
    k = 0
    for j in range(m):
        z = precond(V[j]) if flexible else V[j]
        if flexible:
            Z.append(z)
        w = apply_A(z)
        for i in range(j + 1):
            H[i, j] = _vdot(V[i], w)
            w = w - H[i, j] * V[i]
        H[j + 1, j] = _norm(w)
        for i in range(j):
            hij = H[i, j]
            H[i, j] = cs[i] * hij + sn[i] * H[i + 1, j]
            H[i + 1, j] = -np.conj(sn[i]) * hij + cs[i] * H[i + 1, j]
        cs[j], sn[j] = _givens(H[j, j], H[j + 1, j])
        H[j, j] = cs[j] * H[j, j] + sn[j] * H[j + 1, j]
        H[j + 1, j] = 0.0
        g[j + 1] = -np.conj(sn[j]) * g[j]
        g[j] = cs[j] * g[j]
        k = j + 1
        if abs(g[j + 1]) <= tol_abs or H[j, j] == 0:
            break
        nrm = _norm(w)
        if nrm == 0:
            break
        V.append(w / nrm)
    y = np.zeros(k, dtype=np.complex128)
    for i in range(k - 1, -1, -1):
        y[i] = (g[i] - np.dot(H[i, i + 1:k], y[i + 1:k])) / H[i, i]
    basis = Z if flexible else V
    dx = sum(y[i] * basis[i] for i in range(k))
    return dx, abs(g[k]), k


def gmres(apply_A, b, tol=1e-10, restart=30, maxiter=1000, x0=None):
    """Restarted GMRES(restart) for A x = b.

    Stops when the residual estimate is <= tol*||b|| or after `maxiter` Arnoldi
    steps in total.  tol = 0 runs exactly `maxiter` steps (unless breakdown).
    Returns (x, info) with info = dict(iters, resid) (resid = true relative residual).
    """
    return _restarted(apply_A, None, b, tol, restart, maxiter, x0, flexible=False)


def fgmres(apply_A, precond, b, tol=1e-10, restart=20, maxiter=1000, x0=None):
    """Flexible GMRES(restart), right preconditioning with a variable z_j = precond(v_j)."""
    return _restarted(apply_A, precond, b, tol, restart, maxiter, x0, flexible=True)


def _restarted(apply_A, precond, b, tol, restart, maxiter, x0, flexible):
    bnorm = _norm(b)
    x = np.zeros_like(b) if x0 is None else x0.copy()
    if bnorm == 0:
        return x, dict(iters=0, resid=0.0)
    its = 0
    while its < maxiter:
        r = b - apply_A(x) if its or x0 is not None else b.copy()
        beta = _norm(r)
        if beta <= tol * bnorm:
            break
        m = min(restart, maxiter - its)
        dx, est, k = _arnoldi_cycle(apply_A, precond, r, beta, m, tol * bnorm, flexible)
        x = x + dx
        its += k
        if est <= tol * bnorm:
            break
    res = _norm(b - apply_A(x)) / bnorm
    return x, dict(iters=its, resid=res)
