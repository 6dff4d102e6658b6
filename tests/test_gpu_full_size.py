"""The fine stencil at 32^3 x 64, the lattice of the large eigensolve, against
the oracle on sampled sites: the whole lattice is too large for the oracle's
whole-lattice operator, so each sampled site is checked with
dirac.apply_at_site (that operator on the 3^4 patch around the site, pinned
against the whole-lattice operator at every site of a small lattice).  The
large workload's links and mass, the time direction antiperiodic; FP64 Q - sigma
and D - sigma gamma5 to 1e-13 of the sample's largest value, FP32 Q - sigma to
1e-6 (norm-relative over the sample).  The sample holds random sites and the
lattice's corner and edge sites, where the hops wrap."""
import json
import os

import numpy as np
import pytest

import synth
from oracle import dirac

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def sample_sites(dims, n, seed):
    rng = np.random.default_rng(seed)
    sites = [tuple(int(rng.integers(L)) for L in dims) for _ in range(n)]
    last = tuple(L - 1 for L in dims)
    sites += [(0, 0, 0, 0), last, (last[0], 0, last[2], 0), (0, last[1], 0, last[3])]
    return sites


def test_stencil_32x32x32x64_on_sampled_sites():
    from paper_1509_06865_gb300 import OP_D, OP_Q, PREC_F32, PREC_F64, Context
    w = json.load(open(os.path.join(ROOT, "workloads.json")))["large_32x32x32x64"]
    dims, bc, sigma = tuple(w["dims"]), (1, 1, 1, -1), 0.031
    U = synth.gauge_field(dims, w["eps"], w["seed"])
    x = synth.gaussian_vectors(dims, 1, 41)
    ctx = Context(dims)
    ctx.set_params(m0=w["m0"], csw=w["csw"], bc=bc, agg=w["agg"], n_tv=w["n_tv"], sap_block=w["sap_block"])
    ctx.load_gauge(U)
    sites = sample_sites(dims, 40, 7)

    def at(y, s):                     # y in (T, Z, Y, X, 4, 3); s = (x, y, z, t)
        return y[s[3], s[2], s[1], s[0]]

    for op, form in ((OP_Q, "Q"), (OP_D, "D")):
        y = ctx.apply(x, sigma, op, PREC_F64)[0]
        got = np.array([at(y, s) for s in sites])
        want = np.array([dirac.apply_at_site(U, x[0], s, w["m0"], w["csw"], bc, sigma, form) for s in sites])
        assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max(), form
    y32 = ctx.apply(x, sigma, OP_Q, PREC_F32)[0]
    got = np.array([at(y32, s) for s in sites])
    want = np.array([dirac.apply_at_site(U, x[0], s, w["m0"], w["csw"], bc, sigma, "Q") for s in sites])
    assert np.linalg.norm(got - want) <= 1e-6 * np.linalg.norm(want)
    ctx.close()
