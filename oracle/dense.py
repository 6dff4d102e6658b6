"""Dense matrices of the fine operators on small lattices (FP64).

The matrix of a linear map is built column by column by applying the map to
unit vectors.  Row/column index = ((((t*Lz + z)*Ly + y)*Lx + x)*4 + spin)*3 + colour,
i.e. the flattened host spinor layout.  Used on the 4^4 lattice (3072 x 3072),
where the eigenpairs of the Hermitian Q come from LAPACK's eigh, the textbook
reference for the Sec. 2 eigenproblem Q v = lambda v (Eq. 2.1).
"""
from __future__ import annotations

import numpy as np


def operator_matrix(apply, dims, batch: int = 384) -> np.ndarray:
    lx, ly, lz, lt = dims
    n = lx * ly * lz * lt * 12
    M = np.empty((n, n), dtype=np.complex128)
    for c0 in range(0, n, batch):
        c1 = min(n, c0 + batch)
        E = np.zeros((c1 - c0, n), dtype=np.complex128)
        E[np.arange(c1 - c0), np.arange(c0, c1)] = 1.0
        cols = apply(E.reshape(c1 - c0, lt, lz, ly, lx, 4, 3))
        M[:, c0:c1] = cols.reshape(c1 - c0, n).T
    return M


def lowest_eigenpairs(Qmat: np.ndarray, n: int):
    """The n eigenpairs of the Hermitian matrix with smallest |lambda|.

    Ordered by |lambda| ascending, ties by lambda ascending (reading of
    "low mode" = small in modulus, text after Eq. 2.1).
    """
    w, v = np.linalg.eigh(Qmat)
    order = np.lexsort((w, np.abs(w)))[:n]
    return w[order], v[:, order]
