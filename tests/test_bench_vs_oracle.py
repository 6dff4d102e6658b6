"""The bench's statement of a GPU result's error against the FP64 oracle
(`pairs_vs_oracle`), checked on the CPU with planted eigenpairs: equal sets give
a zero eigenvalue difference and a span overlap of 1 whatever basis a
degenerate eigenspace is given in; a vector from outside the oracle's span (a
missed mode) or a shifted eigenvalue shows in the numbers."""
import numpy as np

import bench


def _planted(n=64, k=4, seed=3):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    lam = np.array([0.1, -0.1, 0.2, 0.2] + list(np.linspace(0.5, 2.0, n - k)))
    return lam, Q.T          # rows are the eigenvectors


def test_equal_sets_in_another_basis_and_order():
    lam, V = _planted()
    # the two vectors of the twofold 0.2 rotated inside their eigenspace, and
    # the pairs listed in another order
    c, s = np.cos(0.7), np.sin(0.7) * np.exp(0.3j)
    W = V[:4].copy()
    W[2], W[3] = c * V[2] + s * V[3], -np.conj(s) * V[2] + c * V[3]
    out = bench.pairs_vs_oracle(lam[[3, 0, 2, 1]], W[[3, 0, 2, 1]] * np.exp(1.1j), lam[:4], V[:4])
    assert out["max_rel_dlambda"] == 0.0
    assert abs(out["min_span_overlap"] - 1) < 1e-13


def test_a_missed_mode_and_a_wrong_eigenvalue_show():
    lam, V = _planted()
    got = V[[0, 1, 2, 5]]                      # the 4th pair replaced by a higher mode
    out = bench.pairs_vs_oracle(lam[[0, 1, 2, 5]], got, lam[:4], V[:4])
    assert out["min_span_overlap"] < 1e-12
    assert out["max_rel_dlambda"] > 1
    # the right vectors with one eigenvalue off by 1e-6 (relative to max |lambda| = 0.2)
    lam_g = lam[:4].copy()
    lam_g[1] += 2e-7
    out = bench.pairs_vs_oracle(lam_g, V[:4], lam[:4], V[:4])
    assert abs(out["max_rel_dlambda"] - 1e-6) < 1e-12


def test_a_count_mismatch_is_reported():
    lam, V = _planted()
    out = bench.pairs_vs_oracle(lam[:3], V[:3], lam[:4], V[:4])
    assert "error" in out
