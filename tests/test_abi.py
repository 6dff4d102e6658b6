"""The C ABI library loads without a GPU and exports every entry point that
include/mgeig.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mgeig.h")
LIB = os.path.join(ROOT, "paper_1509_06865_gb300", "libmgeig.so")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mgeig_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(LIB):
        from paper_1509_06865_gb300 import build
        build.build()
    return ctypes.CDLL(LIB)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 25
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_calls(lib):
    lib.mgeig_strerror.restype = ctypes.c_char_p
    assert lib.mgeig_strerror(0) == b"ok"
    assert b"invalid" in lib.mgeig_strerror(-1)
    from paper_1509_06865_gb300._lib import Params
    p = Params()
    lib.mgeig_default_params(ctypes.byref(p))
    assert p.n_tv == 20 and list(p.agg) == [4, 4, 4, 4] and p.precision == 1
    # argument checks happen before any device call
    assert lib.mgeig_create(None, None, 0) == -1
    dims = (ctypes.c_int * 4)(1, 4, 4, 4)
    h = ctypes.c_void_p()
    assert lib.mgeig_create(ctypes.byref(h), dims, 0) == -1
    assert lib.mgeig_set_params(None, ctypes.byref(p)) == -1


def test_params_struct_matches_header():
    from paper_1509_06865_gb300._lib import Params
    text = open(HEADER).read()
    body = re.search(r"typedef struct mgeig_params \{(.*?)\} mgeig_params;", text, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"\b(?:double|int)\s+([a-z0-9_]+)", body)
    fields += re.findall(r",\s*([a-z0-9_]+)", body)
    names = [f for f, _ in Params._fields_]
    order = [n for n in re.findall(r"([a-z0-9_]+)(?:\[4\])?\s*[;,]", body)]
    assert order == names


def test_stats_struct_matches_header():
    from paper_1509_06865_gb300._lib import Stats
    text = open(HEADER).read()
    body = re.search(r"typedef struct mgeig_stats \{(.*?)\} mgeig_stats;", text, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    order = re.findall(r"([a-z0-9_]+)\s*;", body)
    assert order == [f for f, _ in Stats._fields_]


def test_parameter_checks_without_a_gpu(lib):
    """mgeig_check_params: the lattice and parameter checks of mgeig_create and
    mgeig_set_params, host only.  The defaults pass on the benchmark lattices;
    every documented rule rejects its violation; the edge values pass."""
    from paper_1509_06865_gb300 import LEARNED, LINKS_BF16, check_params
    ok = [((16, 16, 16, 32), {}), ((32, 32, 32, 64), {}), ((8, 8, 8, 8), {}),
          ((4, 4, 4, 4), dict(agg=(2, 2, 2, 2), sap_block=(2, 2, 2, 2), n_tv=8)),
          ((12, 12, 12, 24), dict(agg=(3, 3, 3, 3), sap_block=(3, 3, 3, 3))),     # SAP: 4 x 4 x 4 x 8 blocks
          ((8, 4, 4, 6), dict(agg=(2, 2, 2, 2), sap_block=(2, 2, 2, 3), n_tv=8)),
          ((6, 8, 8, 8), dict(agg=(3, 4, 4, 4), sap_block=(3, 4, 4, 4))),
          ((16, 16, 16, 32), dict(p_modes=-1, n_guard=-1, barrier_timeout=60.0, blas_blocks=64, n_tv=24)),
          ((16, 16, 16, 32), dict(coarse_links=LINKS_BF16)),
          ((16, 16, 16, 32), dict(smoother=LEARNED)),
          ((16, 16, 16, 32), dict(bc=(1, 1, 1, -1), sap_cycles=0, smooth_steps=0, setup_iters=0))]
    for dims, kw in ok:
        assert check_params(dims, **kw) == 0, (dims, kw)
    bad = [((1, 16, 16, 32), {}),                                        # an extent below 2
           ((1024, 1024, 1024, 2), {}),                                  # 12 V beyond 2^31
           ((12, 12, 12, 24), {}),                                       # 4^4 SAP blocks: 3 per direction, odd
           ((16, 16, 16, 32), dict(agg=(3, 4, 4, 4))),                   # aggregate does not divide
           ((16, 16, 16, 32), dict(sap_block=(16, 4, 4, 4))),            # one SAP block in x
           ((32, 32, 32, 64), dict(agg=(8, 8, 8, 4))),                   # aggregate volume 2048 > 1024
           ((16, 16, 16, 32), dict(n_tv=25)), ((16, 16, 16, 32), dict(n_tv=1)),
           ((16, 16, 16, 32), dict(agg=(1, 1, 1, 2), n_tv=20)),          # n_tv > 6 x aggregate volume
           ((16, 16, 16, 32), dict(bc=(1, 1, 1, 0))),
           ((16, 16, 16, 32), dict(sap_mr_iters=0)), ((16, 16, 16, 32), dict(gmres_smooth_k=0)),
           ((16, 16, 16, 32), dict(outer_restart=0)), ((16, 16, 16, 32), dict(outer_restart=101)),
           ((16, 16, 16, 32), dict(coarse_restart=100000)), ((16, 16, 16, 32), dict(coarse_maxiter=0)),
           ((16, 16, 16, 32), dict(coarse_deflate=2)), ((16, 16, 16, 32), dict(shift_floor=1.0)),
           ((16, 16, 16, 32), dict(ritz_keep=float("nan"))), ((16, 16, 16, 32), dict(fine_deflate_radius=float("inf"))),
           ((16, 16, 16, 32), dict(coarse_links=LINKS_BF16, precision=0)),   # 16-bit links need MIXED
           ((16, 16, 16, 32), dict(smoother=LEARNED, precision=0)),          # the network needs MIXED
           ((6, 8, 8, 8), dict(agg=(3, 4, 4, 4), sap_block=(3, 4, 4, 4), smoother=LEARNED)),  # 6 % 4 != 0
           ((16, 16, 16, 32), dict(barrier_timeout=0.0)), ((16, 16, 16, 32), dict(barrier_timeout=61.0)),
           ((16, 16, 16, 32), dict(p_modes=0)), ((16, 16, 16, 32), dict(blas_blocks=65)),
           ((16, 16, 16, 32), dict(solve_tol=0.0)), ((16, 16, 16, 32), dict(precision=2)),
           ((16, 16, 16, 32), dict(smoother=3)), ((16, 16, 16, 32), dict(max_sweeps=0)),
           ((16, 16, 16, 32), dict(n_guard=-2))]
    for dims, kw in bad:
        assert check_params(dims, **kw) == -1, (dims, kw)
    p = (ctypes.c_int * 4)(16, 16, 16, 32)
    assert lib.mgeig_check_params(None, None) == -1 and lib.mgeig_check_params(p, None) == -1


def test_every_workload_passes_the_library_checks(lib):
    """The synthetic workloads (workloads.json) and the uneven field sizes of
    the batched solves are accepted by the library's own lattice and parameter
    checks, in both precisions, before any GPU sees them."""
    import json
    from paper_1509_06865_gb300 import FP64, MIXED, check_params
    w = json.load(open(os.path.join(ROOT, "workloads.json")))
    for name, cfg in w.items():
        if name.startswith("_"):
            continue
        for prec in (FP64, MIXED):
            kw = dict(m0=cfg["m0"], csw=cfg["csw"], bc=cfg["bc"], agg=cfg["agg"], n_tv=cfg["n_tv"],
                      sap_block=cfg["sap_block"], precision=prec)
            assert check_params(cfg["dims"], **kw) == 0, (name, prec)
    for dims, sap in (((8, 8, 8, 8), (4, 4, 4, 4)), ((12, 12, 12, 24), (3, 3, 3, 3)), ((16, 16, 16, 32), (4, 4, 4, 4))):
        assert check_params(dims, n_tv=20, precision=MIXED, sap_block=sap) == 0, dims
