"""Failure paths of the library, each made on the host side, none faulting or
hanging the GPU; after each the same context is used again and works.

* MGEIG_ENOCONV: Algorithm 1 capped at one sweep returns ENOCONV with its
  outputs filled by the current iterates (finite eigenvalues and residuals,
  unit vectors), and the next eigensolve converges.
* MGEIG_EBREAKDOWN: a right-hand side holding a NaN makes the FGMRES norm
  non-finite; a clean solve follows.
* MGEIG_ETIMEOUT: the persistent coarse solver's grid-barrier budget set to a
  nanosecond, so that every block that is not the last to arrive gives up at its
  first barrier (a bounded wait, as every wait of the solver is), raises the
  status word and returns; the host reads it as ETIMEOUT.  With the budget back
  at its default the same context runs the cycle again.
"""
import numpy as np
import pytest

import synth
from tests.gpu_util import norm_rel_err

pytestmark = pytest.mark.gpu

DENSE4 = dict(dims=(4, 4, 4, 4), eps=0.3, seed=1001, m0=-0.4, csw=1.0)


def small_ctx(**kw):
    from paper_1509_06865_gb300 import Context
    c = DENSE4
    ctx = Context(c["dims"])
    ctx.set_params(m0=c["m0"], csw=c["csw"], agg=(2, 2, 2, 2), n_tv=8, sap_block=(2, 2, 2, 2), **kw)
    ctx.load_gauge(synth.gauge_field(c["dims"], c["eps"], c["seed"]))
    ctx.setup(c["seed"])
    return ctx


def test_enoconv_outputs_hold_current_iterates():
    ctx = small_ctx(max_sweeps=1)
    lam, V, res, st = ctx.eigensolve(4, 1e-10)
    assert not st["converged"] and st["sweeps"] == 1
    assert np.all(np.isfinite(lam)) and np.all(np.isfinite(res)) and res.max() > 1e-10
    for i in range(4):
        assert abs(np.linalg.norm(V[i]) - 1) < 1e-12
    ctx.set_params(m0=DENSE4["m0"], csw=DENSE4["csw"], agg=(2, 2, 2, 2), n_tv=8, sap_block=(2, 2, 2, 2))
    ctx.setup(DENSE4["seed"])
    lam2, _, res2, st2 = ctx.eigensolve(4, 1e-10)
    assert st2["converged"] and np.all(res2 <= 1e-10)
    ctx.close()


def test_ebreakdown_on_nan_right_hand_side():
    from paper_1509_06865_gb300 import EBREAKDOWN, MgeigError
    ctx = small_ctx()
    b = synth.z2_noise(DENSE4["dims"], 1, 3)[0]
    bad = b.copy()
    bad[1, 2, 3, 0, 2, 1] = np.nan
    with pytest.raises(MgeigError) as e:
        ctx.solve(bad, 0.1, 1e-10)
    assert e.value.code == EBREAKDOWN
    x, st = ctx.solve(b, 0.1, 1e-10)
    assert st["converged"] and np.all(np.isfinite(x))
    ctx.close()


def test_etimeout_of_a_tiny_barrier_budget():
    from paper_1509_06865_gb300 import ETIMEOUT, MIXED, Context, MgeigError
    dims = (8, 8, 8, 16)   # 2^4 aggregates: 512 coarse sites, the coarse solver on every SM
    kw = dict(m0=-0.0428, csw=1.9, agg=(2, 2, 2, 2), sap_block=(4, 4, 4, 4), n_tv=20, precision=MIXED,
              coarse_tol=0.0, coarse_maxiter=8)
    W = synth.uniform_vectors(dims, 20, 99)
    r = synth.gaussian_vectors(dims, 1, 12)[0]
    ctx = Context(dims)
    ctx.set_params(**kw)
    ctx.load_gauge(synth.gauge_field(dims, 0.2, 1006))
    ctx.set_test_vectors(W)
    want = ctx.mg_cycle(r, 0.0)
    ctx.set_params(barrier_timeout=1e-9, **kw)
    ctx.set_test_vectors(W)
    with pytest.raises(MgeigError) as e:
        ctx.mg_cycle(r, 0.0)
    assert e.value.code == ETIMEOUT
    ctx.set_params(**kw)
    ctx.set_test_vectors(W)
    got = ctx.mg_cycle(r, 0.0)
    assert norm_rel_err(got, want) < 1e-5
    ctx.close()
