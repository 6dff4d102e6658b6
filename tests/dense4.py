"""The 4^4 field of the dense checks (eps = 0.3, seed 1001, c_sw = 1.0,
m0 = -0.4) with its dense 3072 x 3072 Q and LAPACK eigendecomposition, built
once per test session and shared by the tests that need them."""
import functools

import numpy as np

import synth
from oracle import dense, dirac

DENSE4 = dict(dims=(4, 4, 4, 4), eps=0.3, seed=1001, m0=-0.4, csw=1.0)


@functools.lru_cache(maxsize=1)
def field():
    c = DENSE4
    U = synth.gauge_field(c["dims"], c["eps"], c["seed"])
    return U, dirac.WilsonClover(U, c["m0"], c["csw"])


@functools.lru_cache(maxsize=1)
def q_matrix():
    return dense.operator_matrix(field()[1].Q, DENSE4["dims"])


@functools.lru_cache(maxsize=1)
def q_eigh():
    return np.linalg.eigh(q_matrix())
