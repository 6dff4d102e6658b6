"""The Gram-Schmidt building blocks on FP64 vectors: the inner products
<X_j, y> (the projection coefficients of Algorithm 1's Gram-Schmidt step and of
the FGMRES Arnoldi process, Sec. 2.1) and the update y += sum_j c_j X_j, in the
double-float arithmetic of the mixed path (blas_ds = 1) and in FP64.

The double-float kernels split every double into two floats (24 + 23
significant bits) and sum the products with error-free transformations
(TwoProduct by FMA, Knuth's TwoSum: the compensated dot product of Ogita, Rump
and Oishi), so the error is a few 2^-46 of sum |a_i b_i|, where an FP32 sum
would be off by about 2^-24 of it.  The bound below, 2^-40 sum |a_i b_i|, is
met by both FP64 and double-float arithmetic and missed by any FP32 shortcut by
five orders of magnitude.  The reference is numpy's FP64 vdot; its own error
(about 2^-53 sqrt(n) sum |a_i b_i|) is far below the bound."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

BOUND = 2.0 ** -40


def ctx_for(blas_ds, precision):
    from paper_1509_06865_gb300 import Context
    ctx = Context((4, 4, 4, 4))
    ctx.set_params(m0=-0.1, csw=1.0, n_tv=8, agg=(2, 2, 2, 2), sap_block=(2, 2, 2, 2), precision=precision,
                   blas_ds=blas_ds)
    return ctx


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).to("cuda:0")


def random_vectors(rng, k, n, spread=False):
    X = rng.standard_normal((k, n)) + 1j * rng.standard_normal((k, n))
    if spread:
        # magnitudes from 1e-30 to 1e10, exact zeros, signed zeros
        X *= 10.0 ** rng.uniform(-30, 10, size=(k, n))
        X[:, 3::97] = 0.0
        X[:, 5::101] = -0.0
    return X / np.linalg.norm(X, axis=1, keepdims=True)


ARITH = [(1, 1, "double-float"), (0, 1, "fp64-mixed"), (1, 0, "fp64")]


@pytest.mark.parametrize("blas_ds,precision,name", ARITH, ids=[a[2] for a in ARITH])
@pytest.mark.parametrize("n", [1, 255, 1000003])
@pytest.mark.parametrize("k", [1, 8, 13])
def test_multidot(blas_ds, precision, name, n, k):
    import torch
    rng = np.random.default_rng(1000 * k + n % 1000)
    X = random_vectors(rng, k, n)
    y = random_vectors(rng, 1, n)[0]
    ctx = ctx_for(blas_ds, precision)
    Xd = [dev(x) for x in X]
    yd = dev(y)
    torch.cuda.synchronize()
    d = ctx.multidot_dev([t.data_ptr() for t in Xd], yd.data_ptr(), n)
    want = np.array([np.vdot(x, y) for x in X])
    scale = np.abs(X) @ np.abs(y)
    err = np.abs(d - want)
    assert np.all(err <= BOUND * scale), (name, err / scale)
    ctx.close()


BOUND32 = 2.0 ** -18   # FP32 products and per-thread FP32 sums of at most a few hundred terms


@pytest.mark.parametrize("n", [1, 255, 1000003])
@pytest.mark.parametrize("k", [1, 16, 21])
def test_multidot_fp32(n, k):
    """The FP32 vectors of the fine-grid deflation (level precision)."""
    import torch
    from paper_1509_06865_gb300 import PREC_F32
    rng = np.random.default_rng(77 * k + n % 1000)
    X = random_vectors(rng, k, n).astype(np.complex64)
    y = random_vectors(rng, 1, n)[0].astype(np.complex64)
    ctx = ctx_for(1, 1)
    Xd = [torch.from_numpy(x).to("cuda:0") for x in X]
    yd = torch.from_numpy(y).to("cuda:0")
    torch.cuda.synchronize()
    d = ctx.multidot_dev([t.data_ptr() for t in Xd], yd.data_ptr(), n, prec=PREC_F32)
    X64, y64 = X.astype(np.complex128), y.astype(np.complex128)
    want = np.array([np.vdot(x, y64) for x in X64])
    scale = np.abs(X64) @ np.abs(y64)
    assert np.all(np.abs(d - want) <= BOUND32 * scale)
    ctx.close()


@pytest.mark.parametrize("n", [1, 1000003])
@pytest.mark.parametrize("k", [1, 16, 19])
def test_multi_axpy_fp32(n, k):
    import torch
    from paper_1509_06865_gb300 import PREC_F32
    rng = np.random.default_rng(91 * k + n % 1000)
    X = random_vectors(rng, k, n).astype(np.complex64)
    y = random_vectors(rng, 1, n)[0].astype(np.complex64)
    c = rng.standard_normal(k) + 1j * rng.standard_normal(k)
    ctx = ctx_for(1, 1)
    Xd = [torch.from_numpy(x).to("cuda:0") for x in X]
    yd = torch.from_numpy(y.copy()).to("cuda:0")
    torch.cuda.synchronize()
    ctx.multi_axpy_dev([t.data_ptr() for t in Xd], c, yd.data_ptr(), n, prec=PREC_F32)
    got = yd.cpu().numpy().astype(np.complex128)
    X64, y64 = X.astype(np.complex128), y.astype(np.complex128)
    c32 = c.astype(np.complex64).astype(np.complex128)   # the kernel's coefficients are FP32
    want = y64 + c32 @ X64
    scale = np.abs(y64) + np.abs(c32) @ np.abs(X64)
    assert np.all(np.abs(got - want) <= 2.0 ** -20 * scale)
    ctx.close()


@pytest.mark.parametrize("blas_ds,precision,name", ARITH, ids=[a[2] for a in ARITH])
def test_multidot_cancellation_and_range(blas_ds, precision, name):
    """y orthogonal to X up to rounding (the case Gram-Schmidt produces), and
    elements spread over 40 decades with exact and signed zeros."""
    import torch
    rng = np.random.default_rng(7)
    n, k = 300001, 9
    X = random_vectors(rng, k, n, spread=True)
    Q, _ = np.linalg.qr(X.T)
    z = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    y = z - Q @ (Q.conj().T @ z)
    y /= np.linalg.norm(y)
    ctx = ctx_for(blas_ds, precision)
    Xd = [dev(x) for x in X]
    yd = dev(y)
    torch.cuda.synchronize()
    d = ctx.multidot_dev([t.data_ptr() for t in Xd], yd.data_ptr(), n)
    want = np.array([np.vdot(x, y) for x in X])
    scale = np.abs(X) @ np.abs(y)
    assert np.all(np.abs(d - want) <= BOUND * scale)
    # and the squared norm <y, y> = 1 through the same kernel
    d1 = ctx.multidot_dev([yd.data_ptr()], yd.data_ptr(), n)
    assert abs(d1[0] - 1.0) <= 4 * BOUND
    ctx.close()


@pytest.mark.parametrize("blas_ds,precision,name", ARITH, ids=[a[2] for a in ARITH])
@pytest.mark.parametrize("n", [1, 1000003])
@pytest.mark.parametrize("k", [1, 8, 11])
def test_multi_axpy(blas_ds, precision, name, n, k):
    import torch
    rng = np.random.default_rng(31 * k + n % 1000)
    X = random_vectors(rng, k, n, spread=(k == 11))
    y = random_vectors(rng, 1, n)[0]
    c = rng.standard_normal(k) + 1j * rng.standard_normal(k)
    ctx = ctx_for(blas_ds, precision)
    Xd = [dev(x) for x in X]
    yd = dev(y)
    torch.cuda.synchronize()
    ctx.multi_axpy_dev([t.data_ptr() for t in Xd], c, yd.data_ptr(), n)
    got = yd.cpu().numpy()
    want = y + c @ X
    scale = np.abs(y) + np.abs(c) @ np.abs(X)
    err = np.abs(got - want)
    assert np.all(err <= BOUND * scale), (name, np.max(err / np.where(scale > 0, scale, 1)))
    # the inputs are untouched
    for t, x in zip(Xd, X):
        assert np.array_equal(t.cpu().numpy(), x)
    ctx.close()


def test_blas_entry_argument_checks():
    import torch
    from paper_1509_06865_gb300 import MgeigError
    ctx = ctx_for(1, 1)
    a = dev(np.ones(16))
    with pytest.raises(MgeigError):
        ctx.multidot_dev([], a.data_ptr(), 16)
    with pytest.raises(MgeigError):
        ctx.multidot_dev([a.data_ptr()] * 33, a.data_ptr(), 16)
    with pytest.raises(MgeigError):
        ctx.multi_axpy_dev([a.data_ptr()], np.ones(1), a.data_ptr(), 16)   # y is one of the X_j
    torch.cuda.synchronize()
    ctx.close()
