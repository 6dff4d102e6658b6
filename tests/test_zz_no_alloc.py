"""mgeig_mg_cycle_dev_noalloc: the two-grid preconditioner for callers that
cannot allocate device memory while they run (a framework whose pool allocator
holds all free GPU memory, or a latency-bound loop that must not take the
driver's allocation lock).  Its scratch is a static 16 MiB device array shared
by every call, so these checks run two calls in a row: the second must not
see anything the first left behind.  The reference is the allocating entry
point mgeig_mg_cycle on the same context; both run the same kernels, so the
two-grid cycle's tolerances apply (FP64 relative 1e-9, mixed 1e-4).

The file name sorts last, so a run that stops at the first failure has run
every other test before this one."""
import numpy as np
import pytest

import synth
from tests.gpu_util import norm_rel_err

pytestmark = pytest.mark.gpu

DIMS = (8, 8, 8, 16)
EPS, SEED, M0, CSW = 0.2, 4242, -0.05, 1.9


def make_ctx(precision, dims=DIMS, agg=(4, 4, 4, 4), setup_iters=2):
    from paper_1509_06865_gb300 import Context
    ctx = Context(dims)
    ctx.set_params(m0=M0, csw=CSW, agg=agg, sap_block=(4, 4, 4, 4), n_tv=20, precision=precision,
                   setup_iters=setup_iters)
    ctx.load_gauge(synth.gauge_field(dims, EPS, SEED))
    ctx.setup(SEED)
    return ctx


def free_device_bytes():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info(0)[0]


# the FP64 case runs first, in a context of its own, so that the first call
# after mgeig_create is the one checked
@pytest.mark.parametrize("prec,tol", [(0, 1e-9), (1, 1e-4)], ids=["fp64", "mixed"])
def test_noalloc_cycle_matches_mg_cycle_twice(prec, tol):
    from paper_1509_06865_gb300 import PREC_F32, PREC_F64
    ctx = make_ctx(prec)
    level = PREC_F32 if prec == 1 else PREC_F64
    V = int(np.prod(DIMS))
    nbytes = V * 12 * (8 if level == PREC_F32 else 16)
    r_dev, z_dev = ctx.alloc_dev(nbytes), ctx.alloc_dev(nbytes)
    rs = synth.gaussian_vectors(DIMS, 2, 11)
    # the references first: mgeig_mg_cycle allocates its own transfer buffers
    wants = [ctx.mg_cycle(r, 0.03) for r in rs]
    for call, r in enumerate(rs):
        ctx.pack_spinors(r, r_dev, level)
        ctx.pack_spinors(np.zeros_like(r), z_dev, level)
        free0 = free_device_bytes()
        ctx.mg_cycle_dev_noalloc(r_dev, z_dev, 0.03)
        free1 = free_device_bytes()
        # no device memory is taken by the call (the second call in particular,
        # after the driver has loaded every kernel it uses)
        if call == 1:
            assert free1 == free0, (free0, free1)
        got = ctx.unpack_spinors(z_dev, 1, level)[0]
        err = norm_rel_err(got, wants[call])
        assert err < tol, (call, err)
    ctx.close()


def test_noalloc_rejects_overlapping_r_and_z():
    from paper_1509_06865_gb300 import MIXED, PREC_F32
    from paper_1509_06865_gb300._lib import EINVAL, MgeigError
    ctx = make_ctx(MIXED, setup_iters=0)
    nbytes = int(np.prod(DIMS)) * 12 * 8
    buf = ctx.alloc_dev(2 * nbytes)
    ctx.pack_spinors(synth.gaussian_vectors(DIMS, 1, 3)[0], buf, PREC_F32)
    for z in (buf, buf + nbytes // 2):
        with pytest.raises(MgeigError) as e:
            ctx.mg_cycle_dev_noalloc(buf, z, 0.0)
        assert e.value.code == EINVAL
    ctx.close()


def test_noalloc_rejects_a_coarse_grid_beyond_its_scratch():
    from paper_1509_06865_gb300 import MIXED, PREC_F32
    from paper_1509_06865_gb300._lib import ESCRATCH, MgeigError
    dims = (16, 16, 16, 16)     # 2^4 aggregates: 4096 x 40 coarse rows need about 45 MB
    ctx = make_ctx(MIXED, dims=dims, agg=(2, 2, 2, 2), setup_iters=0)
    nbytes = int(np.prod(dims)) * 12 * 8
    r_dev, z_dev = ctx.alloc_dev(nbytes), ctx.alloc_dev(nbytes)
    ctx.pack_spinors(synth.gaussian_vectors(dims, 1, 3)[0], r_dev, PREC_F32)
    with pytest.raises(MgeigError) as e:
        ctx.mg_cycle_dev_noalloc(r_dev, z_dev, 0.0)
    assert e.value.code == ESCRATCH
    assert "static scratch" in str(e.value)
    ctx.close()
