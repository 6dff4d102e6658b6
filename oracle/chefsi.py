"""Independent check of completeness: the eigenpairs of smallest |lambda| of the
Hermitian Q by Chebyshev-filtered subspace iteration on Q^2, FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper notes after Algorithm 1 that the Rayleigh quotient iteration may
converge to a mode other than the one wanted, so a list of converged eigenpairs
says nothing about whether it holds *the* N_eig modes of smallest |lambda|
(Sec. 2, text after Eq. 2.1: the low modes are those of small modulus).  This
module computes that set by a method that shares nothing with Algorithm 1: no
multigrid, no shifted solves, no start vectors from a setup.

Method (Chebyshev-filtered subspace iteration, Zhou and Saad, "A Chebyshev-
Davidson algorithm for large symmetric eigenproblems", SIAM J. Matrix Anal.
Appl. 29 (2007), and Zhou, Saad, Tiago, Chelikowsky, J. Comput. Phys. 219
(2006)), applied to A = Q^2, whose smallest eigenvalues are the squares of the
eigenvalues of Q of smallest modulus:

    X <- nb random vectors
    repeat
        X <- T_d((A - c) / e) X           Chebyshev polynomial of degree d; it is
                                          bounded by 1 on [a, b] and grows fast
                                          below a, with c = (a+b)/2, e = (b-a)/2
        X <- orthonormal basis of span(X)
        Rayleigh-Ritz of A on span(X):    G = X^dag A X = S diag(mu) S^dag, X <- X S,
                                          mu ascending
        a <- mu_nb                        the filter damps everything above the
                                          block's largest Ritz value of A
        Rayleigh-Ritz of Q on the leading m Ritz vectors of A (m >= k, the first
        index past k whose mu is not within a relative 1e-6 of mu_k, so that no
        eigenspace of A is cut): theta, and ||Q x - theta x||
    until the k pairs of smallest |theta| have ||Q x - theta x|| <= tol

b is a rigorous upper bound of the spectrum of A (``q_norm_bound`` squared), so
no eigenvalue lies above the damped interval.  Because X is a block of nb > k
vectors, degenerate or nearly degenerate eigenvalues are all kept (a single-
vector Krylov method finds one copy of an exactly degenerate eigenvalue only).
The Rayleigh-Ritz step of A = Q^2 (positive semidefinite) orders the block
without the spurious small Ritz values that an indefinite Q produces on a
subspace still holding large components of both ends of its spectrum; the final
Rayleigh-Ritz step with Q itself separates eigenvalues +-lambda of equal modulus
that Q^2 cannot tell apart.

Library primitives used as steps: numpy's QR (orthonormal basis) and eigh
(the nb x nb Hermitian Ritz matrix).
"""
from __future__ import annotations

import concurrent.futures as cf
import multiprocessing as mp

import numpy as np

from . import dirac


def q_norm_bound(op: dirac.WilsonClover) -> float:
    """An upper bound of ||Q|| = ||D|| (gamma5 is unitary).

    D = (4 + m0) + A(x) + sum_mu H_mu with H_mu = -P-_mu U_mu T_+mu - P+_mu U_mu^dag T_-mu,
    P-+_mu = (1 -+ g_mu)/2 complementary orthogonal projectors (g_mu Hermitian,
    g_mu^2 = 1) and U T a unitary link times a unit shift (with a boundary sign).
    The two terms of H_mu map into orthogonal subspaces, so
    ||H_mu x||^2 = ||P- U T x||^2 + ||P+ U^dag T x||^2 <= 2 ||x||^2 and ||H_mu|| <= sqrt 2.
    The clover term is block diagonal: its norm is the largest |eigenvalue| of
    the 12 x 12 site blocks.
    """
    clover = np.abs(np.linalg.eigvalsh(op.A.reshape(-1, 12, 12))).max()
    return abs(4.0 + op.m0) + 4.0 * np.sqrt(2.0) + float(clover)


def chebyshev_filter(apply_A, X: np.ndarray, degree: int, a: float, b: float) -> np.ndarray:
    """T_degree((A - c)/e) X with c = (a + b)/2, e = (b - a)/2 (three-term recurrence
    T_{j+1}(t) = 2 t T_j(t) - T_{j-1}(t)), applied to the block X (leading axis)."""
    e = 0.5 * (b - a)
    c = 0.5 * (b + a)
    prev = X
    cur = (apply_A(X) - c * X) / e
    for _ in range(2, degree + 1):
        nxt = 2.0 * (apply_A(cur) - c * cur) / e - prev
        prev, cur = cur, nxt
    return cur


def orthonormal_basis(X: np.ndarray) -> np.ndarray:
    """Orthonormal basis of the span of the block X (QR of the n x nb matrix)."""
    nb = X.shape[0]
    q, _ = np.linalg.qr(X.reshape(nb, -1).T)
    return q.T.reshape(X.shape)


def rayleigh_ritz(apply_H, X: np.ndarray, key=None):
    """Ritz pairs of the Hermitian H on span(X) (X orthonormal), ordered by
    key(theta) (default: theta ascending, ties by theta); returns (theta, Ritz
    vectors, residual norms ||H x - theta x||)."""
    nb = X.shape[0]
    HX = apply_H(X)
    Xf, HXf = X.reshape(nb, -1), HX.reshape(nb, -1)
    G = Xf.conj() @ HXf.T
    G = 0.5 * (G + G.conj().T)
    theta, S = np.linalg.eigh(G)
    order = np.lexsort((theta, theta if key is None else key(theta)))
    theta, S = theta[order], S[:, order]
    Y = (S.T @ Xf).reshape(X.shape)
    HY = (S.T @ HXf).reshape(X.shape)
    res = np.linalg.norm((HY - theta.reshape((nb,) + (1,) * (X.ndim - 1)) * Y).reshape(nb, -1), axis=1)
    return theta, Y, res


def lowest_abs_eigenpairs(apply_Q, start: np.ndarray, k: int, q_bound: float, degree: int = 40,
                          tol: float = 1e-11, max_iter: int = 60, filter_map=None, log=None):
    """The k eigenpairs of the Hermitian map apply_Q of smallest |lambda|.

    start: nb > k start vectors (leading axis); q_bound >= ||Q||.  filter_map, if
    given, applies the Chebyshev filter to column chunks in parallel (it is called
    as filter_map(X, degree, a, b) and must return the filtered block); the result
    does not depend on it.  Returns (lambda[k], vectors[k], residuals[k], info).
    """
    nb = start.shape[0]
    if nb <= k:
        raise ValueError("the block must be larger than the number of wanted pairs")
    b = q_bound * q_bound

    def apply_A(Y):
        return apply_Q(apply_Q(Y))

    def q_pairs(Y, mu):
        # the leading Ritz vectors of A up to the first index past k outside mu_k's
        # (near-)eigenspace, then Rayleigh-Ritz of Q on them, by |theta|
        m = k
        while m < len(mu) and mu[m] <= mu[k - 1] * (1 + 1e-6) + 1e-300:
            m += 1
        return rayleigh_ritz(apply_Q, Y[:m], key=np.abs)

    X = orthonormal_basis(start)
    mu, X, _ = rayleigh_ritz(apply_A, X)
    theta, V, res = q_pairs(X, mu)
    it = 0
    while it < max_iter and res[:k].max() > tol:
        a = float(mu[-1])
        if filter_map is None:
            Y = chebyshev_filter(apply_A, X, degree, a, b)
        else:
            Y = filter_map(X, degree, a, b)
        mu, X, _ = rayleigh_ritz(apply_A, orthonormal_basis(Y))
        theta, V, res = q_pairs(X, mu)
        it += 1
        if log is not None:
            log(f"chefsi iter {it}: cut a = {a:.4e}, max res (wanted) {res[:k].max():.3e}, "
                f"|theta|_k = {abs(theta[k - 1]):.6e}, sqrt(mu_nb) = {np.sqrt(mu[-1]):.6e}")
    info = dict(iters=it, block=nb, degree=degree, q_bound=q_bound, converged=bool(res[:k].max() <= tol),
                block_sqrt_mu=np.sqrt(np.maximum(mu, 0)).tolist())
    return theta[:k], V[:k], res[:k], info


# ---------------------------------------------------------------------------
# parallel filter for the Wilson-clover Q (plumbing: every worker applies the
# same oracle operator to its own columns; the arithmetic is chebyshev_filter)

_worker_op = None


def _init_worker(U, m0, csw, bc, A):
    global _worker_op
    _worker_op = dirac.WilsonClover(U, m0, csw, bc, A=A)


def _filter_chunk(args):
    X, degree, a, b = args
    op = _worker_op
    return chebyshev_filter(lambda Y: op.Q(op.Q(Y)), X, degree, a, b)


class ParallelFilter:
    """filter_map for lowest_abs_eigenpairs: column chunks of the block filtered
    by `workers` processes (spawned, so that no forked state is shared)."""

    def __init__(self, op: dirac.WilsonClover, workers: int):
        self.workers = workers
        self.ex = cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"),
                                         initializer=_init_worker, initargs=(op.U, op.m0, op.csw, op.bc, op.A))

    def __call__(self, X, degree, a, b):
        chunks = np.array_split(np.arange(X.shape[0]), self.workers)
        parts = self.ex.map(_filter_chunk, [(X[c], degree, a, b) for c in chunks if len(c)])
        return np.concatenate(list(parts))

    def close(self):
        self.ex.shutdown()
