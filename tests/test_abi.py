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
