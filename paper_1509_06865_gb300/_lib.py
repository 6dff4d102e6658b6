"""ctypes binding of libmgeig (include/mgeig.h): argument marshalling only.

Every step of the method runs in the CUDA library; this module only converts
numpy arrays to pointers and status codes to exceptions.  The library must
have been built (``paper_1509_06865_gb300.build.build()``); importing the
binding without it raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmgeig.so")

OK, EINVAL, ENOTSETUP, ECUDA, ENOCONV, EBREAKDOWN, ENOMEM, ETIMEOUT, ESCRATCH = 0, -1, -2, -3, -4, -5, -6, -7, -8
FP64, MIXED = 0, 1
SAP, GMRES, LEARNED = 0, 1, 2
NET_SHAPE = (3, 81, 32, 32)   # learned smoother weights [layer][tap][out][in]
OP_Q, OP_D = 0, 1
PREC_F64, PREC_F32 = 0, 1
PREC_F64_DS, PREC_F32_F64_DS = 2, 3   # apply_dev only: double-float arithmetic
LINKS_LEVEL, LINKS_BF16, LINKS_F16 = 0, 1, 2


class Params(C.Structure):
    _fields_ = [
        ("m0", C.c_double), ("csw", C.c_double), ("bc", C.c_int * 4), ("agg", C.c_int * 4),
        ("n_tv", C.c_int), ("sap_block", C.c_int * 4), ("sap_cycles", C.c_int), ("sap_mr_iters", C.c_int),
        ("smooth_steps", C.c_int), ("gmres_smooth_k", C.c_int), ("setup_smooth", C.c_int),
        ("setup_iters", C.c_int), ("outer_restart", C.c_int), ("outer_maxiter", C.c_int),
        ("coarse_restart", C.c_int), ("coarse_maxiter", C.c_int), ("coarse_tol", C.c_double),
        ("solve_tol", C.c_double), ("precision", C.c_int), ("smoother", C.c_int), ("max_sweeps", C.c_int),
        ("n_guard", C.c_int), ("coarse_deflate", C.c_int), ("ritz_each_sweep", C.c_int),
        ("shift_floor", C.c_double), ("guard_maxiter", C.c_int), ("ritz_keep", C.c_double),
        ("fine_deflate", C.c_int), ("fine_deflate_radius", C.c_double),
        ("adaptive_tol", C.c_int), ("ritz_start", C.c_int), ("coarse_links", C.c_int), ("p_modes", C.c_int),
        ("barrier_timeout", C.c_double), ("coarse_blocks", C.c_int), ("blas_ds", C.c_int),
        ("stencil_ds", C.c_int), ("blas_blocks", C.c_int),
        ("guard_coarse_maxiter", C.c_int),
    ]


class Stats(C.Structure):
    _fields_ = [
        ("sweeps", C.c_int), ("solves", C.c_int), ("outer_iters", C.c_int), ("mg_cycles", C.c_int),
        ("coarse_iters", C.c_longlong), ("fine_applies", C.c_longlong), ("seconds", C.c_double),
        ("kernel_launches", C.c_longlong),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class MgeigError(RuntimeError):
    def __init__(self, fn: str, code: int, msg: str):
        super().__init__(f"{fn} failed: {msg} ({code})")
        self.code = code


_lib = None


def load():
    """Load libmgeig.so (once).  Raises if the CUDA library was not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libmgeig.so is missing at {LIB_PATH}: run paper_1509_06865_gb300.build.build()")
    lib = C.CDLL(LIB_PATH)
    P, I, D, S = C.c_void_p, C.c_int, C.c_double, C.c_size_t
    sig = {
        "mgeig_default_params": (None, [C.POINTER(Params)]),
        "mgeig_create": (I, [C.POINTER(P), C.POINTER(C.c_int), I]),
        "mgeig_destroy": (None, [P]),
        "mgeig_set_params": (I, [P, C.POINTER(Params)]),
        "mgeig_check_params": (I, [C.POINTER(C.c_int), C.POINTER(Params)]),
        "mgeig_load_gauge": (I, [P, P]),
        "mgeig_load_gauge_dev": (I, [P, P]),
        "mgeig_get_clover": (I, [P, P]),
        "mgeig_load_clover": (I, [P, P]),
        "mgeig_apply": (I, [P, D, I, I, P, P, I]),
        "mgeig_apply_dev": (I, [P, D, I, I, P, P]),
        "mgeig_apply_dev_nrhs": (I, [P, D, I, I, P, P, I]),
        "mgeig_alloc_dev": (I, [P, S, C.POINTER(P)]),
        "mgeig_pack_spinors": (I, [P, I, P, P, I]),
        "mgeig_unpack_spinors": (I, [P, I, P, P, I]),
        "mgeig_setup": (I, [P, C.c_uint64, C.POINTER(Stats)]),
        "mgeig_set_test_vectors": (I, [P, P]),
        "mgeig_get_test_vectors": (I, [P, P]),
        "mgeig_get_interp": (I, [P, P]),
        "mgeig_get_coarse_op": (I, [P, P]),
        "mgeig_restrict": (I, [P, P, P]),
        "mgeig_prolong": (I, [P, P, P]),
        "mgeig_coarse_apply": (I, [P, D, P, P]),
        "mgeig_coarse_apply_nrhs": (I, [P, D, P, P, I]),
        "mgeig_coarse_apply_dev_nrhs": (I, [P, D, P, P, I]),
        "mgeig_sap": (I, [P, D, P, P, I]),
        "mgeig_mg_cycle": (I, [P, D, P, P]),
        "mgeig_solve": (I, [P, D, P, P, D, C.POINTER(Stats)]),
        "mgeig_solve_d": (I, [P, D, P, P, D, C.POINTER(Stats)]),
        "mgeig_solve_batch": (I, [P, I, P, I, P, P, I, D, C.POINTER(Stats)]),
        "mgeig_eigensolve": (I, [P, I, D, P, P, P, C.POINTER(Stats)]),
        "mgeig_set_timing": (I, [P, I]),
        "mgeig_set_timing_classes": (I, [P, C.c_uint]),
        "mgeig_kernel_times": (I, [P, I, P, P, P, P]),
        "mgeig_get_stream": (I, [P, C.POINTER(P)]),
        "mgeig_get_launch_count": (I, [P, C.POINTER(C.c_longlong)]),
        "mgeig_mg_cycle_dev_noalloc": (I, [P, D, P, P]),
        "mgeig_fma_peak": (I, [P, I, I, C.POINTER(D)]),
        "mgeig_multidot_dev": (I, [P, I, I, P, P, C.c_longlong, P]),
        "mgeig_multi_axpy_dev": (I, [P, I, I, P, P, P, C.c_longlong]),
        "mgeig_lma_prepare": (I, [P, I, P, D, P, P, P, P, P, P, P]),
        "mgeig_lma_apply": (I, [P, I, P, P]),
        "mgeig_lma_loop_high": (I, [P, I, C.c_uint64, D, P, C.POINTER(Stats)]),
        "mgeig_net_init": (I, [P, C.c_uint64]),
        "mgeig_net_set_weights": (I, [P, P]),
        "mgeig_net_get_weights": (I, [P, P]),
        "mgeig_net_train": (I, [P, I, I, D, C.c_uint64, P]),
        "mgeig_net_loss_grads": (I, [P, P, P, I, C.POINTER(D), P]),
        "mgeig_net_apply": (I, [P, P, P]),
        "mgeig_strerror": (C.c_char_p, [I]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(a: np.ndarray):
    return C.c_void_p(a.ctypes.data)


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def make_params(**kw) -> Params:
    """The library defaults with the given fields replaced."""
    lib = load()
    p = Params()
    lib.mgeig_default_params(C.byref(p))
    for k, v in kw.items():
        if k in ("bc", "agg", "sap_block"):
            setattr(p, k, (C.c_int * 4)(*v))
        else:
            setattr(p, k, v)
    return p


def check_params(dims, **kw) -> int:
    """mgeig_check_params: 0 if a context of lattice dims (Lx, Ly, Lz, Lt) would
    accept these parameters, else the status code.  Needs no GPU."""
    return load().mgeig_check_params((C.c_int * 4)(*dims), C.byref(make_params(**kw)))


def solve_batch(ctxs, sigmas, rhs, tol=1e-10):
    """(Q - sigma_s) x = b_j for every context (rhs[k]: [nrhs, ...] spinors of context k's
    lattice, the same nrhs for all): list of arrays [nsig, nrhs, ...] and the summed stats."""
    lib = load()
    n = len(ctxs)
    sig = np.ascontiguousarray(sigmas, dtype=np.float64)
    bs = [_c128(b) for b in rhs]
    nrhs = bs[0].shape[0]
    assert all(b.shape[0] == nrhs for b in bs)
    xs = [np.empty((len(sig),) + b.shape, dtype=np.complex128) for b in bs]
    hp = (C.c_void_p * n)(*[c._h.value for c in ctxs])
    bp = (C.c_void_p * n)(*[b.ctypes.data for b in bs])
    xp = (C.c_void_p * n)(*[x.ctypes.data for x in xs])
    st = Stats()
    rc = lib.mgeig_solve_batch(C.cast(hp, C.c_void_p), n, _ptr(sig), len(sig), C.cast(bp, C.c_void_p),
                               C.cast(xp, C.c_void_p), nrhs, float(tol), C.byref(st))
    if rc not in (OK, ENOCONV):
        raise MgeigError("mgeig_solve_batch", rc, lib.mgeig_strerror(rc).decode())
    return xs, dict(st.as_dict(), converged=rc == OK)


class Context:
    """One lattice on one GPU (mgeig_ctx)."""

    def __init__(self, dims, device: int = 0):
        self.lib = load()
        self.dims = tuple(int(d) for d in dims)
        lx, ly, lz, lt = self.dims
        self.V = lx * ly * lz * lt
        self._h = C.c_void_p()
        d = (C.c_int * 4)(*self.dims)
        self._check("mgeig_create", self.lib.mgeig_create(C.byref(self._h), d, int(device)))
        self.params = Params()
        self.lib.mgeig_default_params(C.byref(self.params))

    def _check(self, fn, rc, allow=()):
        if rc != OK and rc not in allow:
            raise MgeigError(fn, rc, self.lib.mgeig_strerror(rc).decode())
        return rc

    def close(self):
        if self._h:
            self.lib.mgeig_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- configuration -------------------------------------------------
    def set_params(self, **kw):
        p = make_params(**kw)
        self._check("mgeig_set_params", self.lib.mgeig_set_params(self._h, C.byref(p)))
        self.params = p

    @property
    def n_tv(self):
        return self.params.n_tv

    @property
    def coarse_sites(self):
        n = 1
        for d, a in zip(self.dims, self.params.agg):
            n *= d // a
        return n

    def _spinor_shape(self, n=None):
        lx, ly, lz, lt = self.dims
        s = (lt, lz, ly, lx, 4, 3)
        return s if n is None else (n,) + s

    def load_gauge(self, U):
        U = _c128(U)
        assert U.size == self.V * 36
        self._check("mgeig_load_gauge", self.lib.mgeig_load_gauge(self._h, _ptr(U)))

    def load_gauge_dev(self, U_dev_ptr: int):
        self._check("mgeig_load_gauge_dev", self.lib.mgeig_load_gauge_dev(self._h, C.c_void_p(U_dev_ptr)))

    def load_clover(self, A=None):
        """Use the clover term A ([site][2][6][6] complex128, no mass term) instead of
        the one built from the gauge field; None goes back to the built one."""
        if A is None:
            self._check("mgeig_load_clover", self.lib.mgeig_load_clover(self._h, None))
            return
        A = _c128(A)
        assert A.size == self.V * 72
        self._check("mgeig_load_clover", self.lib.mgeig_load_clover(self._h, _ptr(A)))

    def get_clover(self):
        out = np.empty((self.V, 2, 6, 6), dtype=np.complex128)
        self._check("mgeig_get_clover", self.lib.mgeig_get_clover(self._h, _ptr(out)))
        return out

    # ---- fine operator ---------------------------------------------------
    def apply(self, x, sigma=0.0, op=OP_Q, prec=PREC_F64):
        x = _c128(x)
        nrhs = x.size // (self.V * 12)
        y = np.empty_like(x)
        self._check("mgeig_apply", self.lib.mgeig_apply(self._h, float(sigma), op, prec, _ptr(x), _ptr(y), nrhs))
        return y

    def apply_dev(self, x_ptr: int, y_ptr: int, sigma=0.0, op=OP_Q, prec=PREC_F64):
        self._check("mgeig_apply_dev", self.lib.mgeig_apply_dev(self._h, float(sigma), op, prec,
                                                                C.c_void_p(x_ptr), C.c_void_p(y_ptr)))

    def apply_dev_nrhs(self, x_ptr: int, y_ptr: int, nrhs: int, sigma=0.0, op=OP_Q, prec=PREC_F64):
        self._check("mgeig_apply_dev_nrhs", self.lib.mgeig_apply_dev_nrhs(self._h, float(sigma), op, prec,
                                                                          C.c_void_p(x_ptr), C.c_void_p(y_ptr),
                                                                          int(nrhs)))

    def alloc_dev(self, nbytes: int) -> int:
        p = C.c_void_p()
        self._check("mgeig_alloc_dev", self.lib.mgeig_alloc_dev(self._h, C.c_size_t(nbytes), C.byref(p)))
        return p.value

    def pack_spinors(self, host, dev_ptr: int, prec=PREC_F64):
        host = _c128(host)
        n = host.size // (self.V * 12)
        self._check("mgeig_pack_spinors", self.lib.mgeig_pack_spinors(self._h, prec, _ptr(host), C.c_void_p(dev_ptr), n))

    def unpack_spinors(self, dev_ptr: int, n: int = 1, prec=PREC_F64):
        host = np.empty(self._spinor_shape(n), dtype=np.complex128)
        self._check("mgeig_unpack_spinors", self.lib.mgeig_unpack_spinors(self._h, prec, C.c_void_p(dev_ptr),
                                                                          _ptr(host), n))
        return host

    # ---- multigrid -------------------------------------------------------
    def setup(self, seed: int):
        st = Stats()
        self._check("mgeig_setup", self.lib.mgeig_setup(self._h, C.c_uint64(seed), C.byref(st)))
        return st.as_dict()

    def set_test_vectors(self, W):
        W = _c128(W)
        assert W.size == self.n_tv * self.V * 12
        self._check("mgeig_set_test_vectors", self.lib.mgeig_set_test_vectors(self._h, _ptr(W)))

    def get_test_vectors(self):
        W = np.empty(self._spinor_shape(self.n_tv), dtype=np.complex128)
        self._check("mgeig_get_test_vectors", self.lib.mgeig_get_test_vectors(self._h, _ptr(W)))
        return W

    def get_interp(self):
        P = np.empty(self._spinor_shape(self.n_tv), dtype=np.complex128)
        self._check("mgeig_get_interp", self.lib.mgeig_get_interp(self._h, _ptr(P)))
        return P

    def get_coarse_op(self):
        n2 = 2 * self.n_tv
        D = np.empty((9, self.coarse_sites, n2, n2), dtype=np.complex128)
        self._check("mgeig_get_coarse_op", self.lib.mgeig_get_coarse_op(self._h, _ptr(D)))
        return D

    def restrict(self, r):
        r = _c128(r)
        rc = np.empty((self.coarse_sites, 2, self.n_tv), dtype=np.complex128)
        self._check("mgeig_restrict", self.lib.mgeig_restrict(self._h, _ptr(r), _ptr(rc)))
        return rc

    def prolong(self, ec):
        ec = _c128(ec)
        e = np.empty(self._spinor_shape(), dtype=np.complex128)
        self._check("mgeig_prolong", self.lib.mgeig_prolong(self._h, _ptr(ec), _ptr(e)))
        return e

    def coarse_apply(self, xc, sigma=0.0):
        xc = _c128(xc)
        yc = np.empty_like(xc)
        self._check("mgeig_coarse_apply", self.lib.mgeig_coarse_apply(self._h, float(sigma), _ptr(xc), _ptr(yc)))
        return yc

    def coarse_apply_nrhs(self, xc, sigma=0.0):
        """(Q_c - sigma) on nrhs coarse vectors xc[nrhs, sites, 2, n_tv] in one call."""
        xc = _c128(xc)
        yc = np.empty_like(xc)
        self._check("mgeig_coarse_apply_nrhs", self.lib.mgeig_coarse_apply_nrhs(self._h, float(sigma), _ptr(xc),
                                                                                _ptr(yc), xc.shape[0]))
        return yc

    def coarse_apply_dev_nrhs(self, x_ptr: int, y_ptr: int, nrhs: int, sigma=0.0):
        self._check("mgeig_coarse_apply_dev_nrhs", self.lib.mgeig_coarse_apply_dev_nrhs(
            self._h, float(sigma), C.c_void_p(x_ptr), C.c_void_p(y_ptr), int(nrhs)))

    def sap(self, b, z, sigma=0.0, cycles=1):
        b = _c128(b)
        z = _c128(z).copy()
        self._check("mgeig_sap", self.lib.mgeig_sap(self._h, float(sigma), _ptr(b), _ptr(z), int(cycles)))
        return z

    def mg_cycle(self, r, sigma=0.0):
        r = _c128(r)
        z = np.empty_like(r)
        self._check("mgeig_mg_cycle", self.lib.mgeig_mg_cycle(self._h, float(sigma), _ptr(r), _ptr(z)))
        return z

    def mg_cycle_dev_noalloc(self, r_dev: int, z_dev: int, sigma=0.0):
        """z = B r on device spinors of the level precision (see the C header):
        for callers that cannot allocate device memory during the call; the
        scratch is a static 16 MiB device array shared by all calls."""
        self._check("mgeig_mg_cycle_dev_noalloc",
                    self.lib.mgeig_mg_cycle_dev_noalloc(self._h, float(sigma), C.c_void_p(r_dev), C.c_void_p(z_dev)))

    def solve(self, b, sigma=0.0, tol=1e-10):
        b = _c128(b)
        x = np.empty_like(b)
        st = Stats()
        rc = self._check("mgeig_solve", self.lib.mgeig_solve(self._h, float(sigma), _ptr(b), _ptr(x), float(tol),
                                                             C.byref(st)), allow=(ENOCONV,))
        return x, dict(st.as_dict(), converged=rc == OK)

    def solve_d(self, b, sigma=0.0, tol=1e-10):
        """(D - sigma gamma5) x = b (non-Hermitian), FGMRES with the two-grid preconditioner."""
        b = _c128(b)
        x = np.empty_like(b)
        st = Stats()
        rc = self._check("mgeig_solve_d", self.lib.mgeig_solve_d(self._h, float(sigma), _ptr(b), _ptr(x),
                                                                 float(tol), C.byref(st)), allow=(ENOCONV,))
        return x, dict(st.as_dict(), converged=rc == OK)

    def eigensolve(self, n_eig: int, tol: float, want_vectors: bool = True):
        evals = np.empty(n_eig)
        resid = np.empty(n_eig)
        evecs = np.empty(self._spinor_shape(n_eig), dtype=np.complex128) if want_vectors else None
        st = Stats()
        rc = self._check("mgeig_eigensolve",
                         self.lib.mgeig_eigensolve(self._h, int(n_eig), float(tol), _ptr(evals),
                                                   _ptr(evecs) if want_vectors else None, _ptr(resid), C.byref(st)),
                         allow=(ENOCONV,))
        return evals, evecs, resid, dict(st.as_dict(), converged=rc == OK)

    # ---- instrumentation -------------------------------------------------
    def stream(self) -> int:
        s = C.c_void_p()
        self._check("mgeig_get_stream", self.lib.mgeig_get_stream(self._h, C.byref(s)))
        return s.value or 0

    # ---- approximate low-mode averaging -------------------------------------
    def lma_prepare(self, n: int, V=None, cutoff: float = 0.75):
        """Approximate modes V (n host spinors, None: the setup's first n test
        vectors): dict of lam, eps, kept, A, Ainv (kept x kept), Llow[Lt]."""
        lam, eps = np.empty(n), np.empty(n)
        kept = np.empty(n, dtype=np.int32)
        nk = C.c_int()
        A = np.empty((n, n), dtype=np.complex128)
        Ai = np.empty((n, n), dtype=np.complex128)
        Llow = np.empty(self.dims[3], dtype=np.complex128)
        Vp = None
        if V is not None:
            V = _c128(V)
            assert V.size == n * self.V * 12
            Vp = _ptr(V)
        self._check("mgeig_lma_prepare", self.lib.mgeig_lma_prepare(self._h, int(n), Vp, float(cutoff), _ptr(lam),
                                                                    _ptr(eps), _ptr(kept), C.byref(nk), _ptr(A),
                                                                    _ptr(Ai), _ptr(Llow)))
        k = nk.value
        return dict(lam=lam, eps=eps, kept=kept.astype(bool), n_kept=k,
                    A=A.reshape(-1)[:k * k].reshape(k, k).copy(), Ainv=Ai.reshape(-1)[:k * k].reshape(k, k).copy(),
                    Llow=Llow)

    def lma_apply(self, x, mode: int):
        x = _c128(x)
        y = np.empty_like(x)
        self._check("mgeig_lma_apply", self.lib.mgeig_lma_apply(self._h, int(mode), _ptr(x), _ptr(y)))
        return y

    def lma_loop_high(self, nstoch: int, seed: int, tol: float = 1e-10):
        L = np.empty(self.dims[3], dtype=np.complex128)
        st = Stats()
        self._check("mgeig_lma_loop_high", self.lib.mgeig_lma_loop_high(self._h, int(nstoch), C.c_uint64(seed),
                                                                        float(tol), _ptr(L), C.byref(st)))
        return L, st.as_dict()

    # ---- learned smoother ------------------------------------------------
    def net_init(self, seed: int):
        self._check("mgeig_net_init", self.lib.mgeig_net_init(self._h, C.c_uint64(seed)))

    def net_set_weights(self, W):
        W = np.ascontiguousarray(W, dtype=np.float32)
        assert W.shape == NET_SHAPE
        self._check("mgeig_net_set_weights", self.lib.mgeig_net_set_weights(self._h, _ptr(W)))

    def net_get_weights(self):
        W = np.empty(NET_SHAPE, dtype=np.float32)
        self._check("mgeig_net_get_weights", self.lib.mgeig_net_get_weights(self._h, _ptr(W)))
        return W

    def net_train(self, steps: int, batch: int, lr: float, seed: int):
        losses = np.empty(steps)
        self._check("mgeig_net_train", self.lib.mgeig_net_train(self._h, int(steps), int(batch), float(lr),
                                                                C.c_uint64(seed), _ptr(losses)))
        return losses

    def net_loss_grads(self, x, t):
        """x, t: FP64 channel fields [batch, T, Z, Y, X, 24] -> (loss, gradients [3, 81, 32, 32])."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        t = np.ascontiguousarray(t, dtype=np.float64)
        G = np.empty(NET_SHAPE, dtype=np.float32)
        L = C.c_double()
        self._check("mgeig_net_loss_grads", self.lib.mgeig_net_loss_grads(self._h, _ptr(x), _ptr(t), x.shape[0],
                                                                          C.byref(L), _ptr(G)))
        return L.value, G

    def net_apply(self, r):
        r = _c128(r)
        e = np.empty_like(r)
        self._check("mgeig_net_apply", self.lib.mgeig_net_apply(self._h, _ptr(r), _ptr(e)))
        return e

    def fma_peak(self, prec=PREC_F64, reps: int = 5) -> float:
        """FMA throughput of the device in FLOP/s (FP64 or FP32), own kernel."""
        f = C.c_double()
        self._check("mgeig_fma_peak", self.lib.mgeig_fma_peak(self._h, prec, int(reps), C.byref(f)))
        return f.value

    def multidot_dev(self, X_ptrs, y_ptr: int, n: int, prec=PREC_F64) -> np.ndarray:
        """<X_j, y> for device vectors of n complex values (FP64 or FP32)."""
        k = len(X_ptrs)
        arr = (C.c_void_p * k)(*X_ptrs)
        d = np.zeros(2 * k)
        self._check("mgeig_multidot_dev",
                    self.lib.mgeig_multidot_dev(self._h, prec, k, arr, C.c_void_p(y_ptr), n, _ptr(d)))
        return d[0::2] + 1j * d[1::2]

    def multi_axpy_dev(self, X_ptrs, coef, y_ptr: int, n: int, prec=PREC_F64):
        """y += sum_j coef[j] X_j for device vectors of n complex values (FP64 or FP32)."""
        k = len(X_ptrs)
        arr = (C.c_void_p * k)(*X_ptrs)
        cf = np.ascontiguousarray(np.stack([np.real(coef), np.imag(coef)], axis=1).ravel(), dtype=np.float64)
        self._check("mgeig_multi_axpy_dev",
                    self.lib.mgeig_multi_axpy_dev(self._h, prec, k, arr, _ptr(cf), C.c_void_p(y_ptr), n))

    def launch_count(self) -> int:
        n = C.c_longlong()
        self._check("mgeig_get_launch_count", self.lib.mgeig_get_launch_count(self._h, C.byref(n)))
        return int(n.value)

    def set_timing(self, on: bool):
        self._check("mgeig_set_timing", self.lib.mgeig_set_timing(self._h, 1 if on else 0))

    def set_timing_classes(self, names):
        """Time only the named kernel classes (names as in kernel_times())."""
        order = list(self.kernel_times())
        mask = 0
        for n in names:
            mask |= 1 << order.index(n)
        self._check("mgeig_set_timing_classes", self.lib.mgeig_set_timing_classes(self._h, C.c_uint(mask)))

    def kernel_times(self):
        n = 16
        launches = np.zeros(n, dtype=np.int64)
        ms = np.zeros(n)
        nbytes = np.zeros(n)
        names = (C.c_char_p * n)()
        k = self.lib.mgeig_kernel_times(self._h, n, _ptr(launches), _ptr(ms), _ptr(nbytes), C.cast(names, C.c_void_p))
        self._check("mgeig_kernel_times", 0 if k > 0 else k)
        return {names[i].decode(): dict(launches=int(launches[i]), ms=float(ms[i]), bytes=float(nbytes[i]))
                for i in range(k)}
