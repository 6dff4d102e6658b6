"""Approximate low-mode averaging, FP64 oracle (Sec. 3.1 and 3.2).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Given N orthonormal approximate eigenvectors v~_i of Q (Sec. 3.2), with
Rayleigh quotients lambda~_i and accuracies eps_i = ||Q v~_i - lambda~_i v~_i||:

  cutoff        keep the pairs with eps_i / |lambda~_i| <= c (Sec. 3.3; c = 0.75
                there): approximate modes that do not respect the mass gap have a
                large relative error
  A_ij          = <v~_i | Q | v~_j>                   (Hermitian, kept pairs only)
  Q~^-1_low     = sum_ij (A^-1)_ij |v~_i><v~_j|       (equals Q^-1_low of Sec. 3.1
                                                       for exact eigenvectors)
  R~            = 1 - sum_ij Q |v~_i> (A^-1)_ij <v~_j|  (oblique projector; the
                                                       orthogonal 1 - sum |v_i><v_i|
                                                       for exact eigenvectors)
  L_low(t)      = sum_{x in timeslice t} tr[(Q~^-1_low)_{x,x}]
                = sum_ij (A^-1)_ij sum_{x in t} <v~_j(x) | v~_i(x)>   (the low-mode
                  part of the disconnected loop, trace over spin and colour)

Spinors are numpy arrays [T, Z, Y, X, 4, 3] (leading axis: the N vectors).
"""
from __future__ import annotations

import numpy as np

from . import dirac


def orthonormalise(V: np.ndarray) -> np.ndarray:
    """Gram-Schmidt (each step twice) of V[0], V[1], ..."""
    out = []
    for v in V:
        w = v.copy()
        for _ in range(2):
            for u in out:
                w = w - np.vdot(u, w) * u
        out.append(w / dirac.norm(w))
    return np.array(out)


def approximate_modes(op: dirac.WilsonClover, V: np.ndarray):
    """Rayleigh quotients and accuracies of orthonormal vectors V."""
    QV = np.array([op.Q(v) for v in V])
    lam = np.array([float(np.real(np.vdot(v, q))) for v, q in zip(V, QV)])
    eps = np.array([dirac.norm(q - l * v) for v, q, l in zip(V, QV, lam)])
    return lam, eps, QV


def cutoff(lam: np.ndarray, eps: np.ndarray, c: float) -> np.ndarray:
    """Indices of the pairs with eps / |lambda| <= c."""
    return np.array([i for i in range(len(lam)) if eps[i] <= c * abs(lam[i])], dtype=int)


def a_matrix(V: np.ndarray, QV: np.ndarray) -> np.ndarray:
    """A_ij = <v_i | Q | v_j>."""
    n = len(V)
    return V.reshape(n, -1).conj() @ QV.reshape(n, -1).T


def low_inverse_apply(V: np.ndarray, Ainv: np.ndarray, x: np.ndarray) -> np.ndarray:
    """Q~^-1_low x = sum_ij (A^-1)_ij v_i <v_j | x>."""
    d = np.array([np.vdot(v, x) for v in V])
    c = Ainv @ d
    return np.tensordot(c, V, axes=1)


def oblique_projector_apply(V: np.ndarray, QV: np.ndarray, Ainv: np.ndarray, x: np.ndarray) -> np.ndarray:
    """R~ x = x - sum_ij Q v_i (A^-1)_ij <v_j | x>."""
    d = np.array([np.vdot(v, x) for v in V])
    c = Ainv @ d
    return x - np.tensordot(c, QV, axes=1)


def low_mode_loop(V: np.ndarray, Ainv: np.ndarray) -> np.ndarray:
    """L_low(t) for every timeslice t (complex array of length T)."""
    n, T = len(V), V.shape[1]
    # M[t][j][i] = sum_{x in t} <v_j(x) | v_i(x)>
    M = np.einsum("jtzyxsc,itzyxsc->tji", V.conj(), V)
    return np.array([np.sum(Ainv * M[t].T) for t in range(T)])
