// BLAS-1 on flat complex arrays (fine spinors of one precision share one
// layout, so element-wise operations ignore it; coarse vectors are flat).
//
// Reductions are deterministic two-pass trees: a fixed grid of 256-thread
// blocks accumulates grid-stride partial sums (per thread in the array's own
// precision, then in FP64 across the block with warp shuffles), writes one
// partial per block, and a second kernel adds the partials in a fixed order.
// Inner products of up to 16 vectors against one vector share one read of that
// vector (the Arnoldi / Gram-Schmidt steps of GMRES, FGMRES and Algorithm 1).
#include <algorithm>

#include "ds.cuh"
#include "internal.h"

namespace mgeig {

constexpr int RED_THREADS = 256;
constexpr int RED_MAXBLOCKS = 1024;
constexpr int CHUNK = 16;   // pointer slots per launch
// vectors per launch: 16 in FP32 (bandwidth bound, fewer passes over y); 8 in
// FP64, where the FP64 pipe bounds the kernel and 16 accumulators cost occupancy
template <typename R> struct Chunk { static constexpr int n = sizeof(R) == 4 ? 16 : 8; };

template <typename R> struct V2;
template <> struct V2<double> { typedef double2 T; };
template <> struct V2<float> { typedef float2 T; };

struct PtrPack { const void *p[CHUNK]; };

// FP32 arrays of an even number of complex values on 16-byte boundaries are
// processed two values per float4 access
template <typename R>
static bool vec4_ok(const PtrPack &pk, int k, const void *y, size_t n) {
    if (sizeof(R) != 4 || (n & 1)) return false;
    if (reinterpret_cast<uintptr_t>(y) & 15) return false;
    for (int j = 0; j < k; ++j)
        if (reinterpret_cast<uintptr_t>(pk.p[j]) & 15) return false;
    return true;
}

// reduction grids: one block per 4 * 256 elements, at most 4 blocks per SM (or
// blas_blocks per SM when the context sets it) and 1024 in all.  Measured on
// GB300 (16 FP32 or 8 double-float vectors per launch): 4 per SM beat 1024
// blocks by 1.1-1.35x at 16^3 x 32 and 32^3 x 64 (fewer block epilogues and
// partial sums)
static int red_grid(const Ctx &c, size_t n, int per_sm = 4) {
    size_t b = (n + RED_THREADS * 4 - 1) / (RED_THREADS * 4);
    b = std::min<size_t>(b, (size_t)c.sms * (c.prm.blas_blocks > 0 ? c.prm.blas_blocks : per_sm));
    if (b < 1) b = 1;
    if (b > RED_MAXBLOCKS) b = RED_MAXBLOCKS;
    return (int)b;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// block-reduce `cnt` complex values held by every thread; thread 0 writes them
template <int MAXV>
__device__ __forceinline__ void block_reduce_store(double (&re)[MAXV], double (&im)[MAXV], int cnt, double2 *out,
                                                   size_t out_stride) {
    __shared__ double sh[RED_THREADS / 32][2 * MAXV];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < MAXV; ++k) {
        if (k < cnt) {
            double a = warp_sum(re[k]), b = warp_sum(im[k]);
            if (lane == 0) { sh[w][2 * k] = a; sh[w][2 * k + 1] = b; }
        }
    }
    __syncthreads();
    if (threadIdx.x < cnt) {
        double a = 0, b = 0;
        for (int i = 0; i < RED_THREADS / 32; ++i) { a += sh[i][2 * threadIdx.x]; b += sh[i][2 * threadIdx.x + 1]; }
        out[(size_t)threadIdx.x * out_stride + blockIdx.x] = make_double2(a, b);
    }
}

template <typename R>
__global__ void __launch_bounds__(RED_THREADS) multidot_kernel(PtrPack X, int k, const void *__restrict__ yv, size_t n,
                                                               double2 *__restrict__ partial, size_t pstride, bool vec4) {
    typedef typename V2<R>::T T;
    const T *y = static_cast<const T *>(yv);
    constexpr int C = Chunk<R>::n;
    R ar[C], ai[C];
#pragma unroll
    for (int j = 0; j < C; ++j) { ar[j] = 0; ai[j] = 0; }
    if constexpr (sizeof(R) == 4) {
        if (vec4) {   // two complex values per 16-byte load (n even, 16-byte aligned arrays)
            const float4 *y4 = static_cast<const float4 *>(yv);
            for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n / 2; i += (size_t)gridDim.x * blockDim.x) {
                const float4 b = y4[i];
#pragma unroll
                for (int j = 0; j < C; ++j) {
                    if (j < k) {
                        const float4 a = static_cast<const float4 *>(X.p[j])[i];
                        ar[j] = fmaf(a.x, b.x, ar[j]); ar[j] = fmaf(a.y, b.y, ar[j]);
                        ar[j] = fmaf(a.z, b.z, ar[j]); ar[j] = fmaf(a.w, b.w, ar[j]);
                        ai[j] = fmaf(a.x, b.y, ai[j]); ai[j] = fmaf(-a.y, b.x, ai[j]);
                        ai[j] = fmaf(a.z, b.w, ai[j]); ai[j] = fmaf(-a.w, b.z, ai[j]);
                    }
                }
            }
            n = 0;   // the scalar loop below has nothing left to do
        }
    }
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        T b = y[i];
#pragma unroll
        for (int j = 0; j < C; ++j) {
            if (j < k) {
                T a = static_cast<const T *>(X.p[j])[i];
                ar[j] = fma(a.x, b.x, ar[j]); ar[j] = fma(a.y, b.y, ar[j]);
                ai[j] = fma(a.x, b.y, ai[j]); ai[j] = fma(-a.y, b.x, ai[j]);
            }
        }
    }
    double re[C], im[C];
#pragma unroll
    for (int j = 0; j < C; ++j) { re[j] = ar[j]; im[j] = ai[j]; }
    block_reduce_store<C>(re, im, k, partial, pstride);
}

template <typename R>
__global__ void __launch_bounds__(RED_THREADS) norm2_kernel(const void *__restrict__ xv, size_t n,
                                                            double2 *__restrict__ partial) {
    typedef typename V2<R>::T T;
    const T *x = static_cast<const T *>(xv);
    R acc = 0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        T a = x[i];
        acc = fma(a.x, a.x, acc); acc = fma(a.y, a.y, acc);
    }
    double re[1] = {(double)acc}, im[1] = {0.0};
    block_reduce_store<1>(re, im, 1, partial, 1);
}

__global__ void resid_norm2_kernel(const double2 *__restrict__ qv, const double2 *__restrict__ v,
                                   const double2 *__restrict__ lam, size_t n, double2 *__restrict__ partial) {
    const double l = lam[0].x;
    double acc = 0;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        double2 a = qv[i], b = v[i];
        double rx = fma(-l, b.x, a.x), ry = fma(-l, b.y, a.y);
        acc = fma(rx, rx, acc); acc = fma(ry, ry, acc);
    }
    double re[1] = {acc}, im[1] = {0.0};
    block_reduce_store<1>(re, im, 1, partial, 1);
}

// out[j] = sum of partial[j][0..nb)
__global__ void finalize_kernel(const double2 *__restrict__ partial, size_t pstride, int nb, double2 *__restrict__ out) {
    const int j = blockIdx.x;
    double a = 0, b = 0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) { double2 t = partial[(size_t)j * pstride + i]; a += t.x; b += t.y; }
    a = warp_sum(a); b = warp_sum(b);
    __shared__ double sh[2][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) { sh[0][w] = a; sh[1][w] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0, y = 0;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { x += sh[0][i]; y += sh[1][i]; }
        out[j] = make_double2(x, y);
    }
}

// ---------------------------------------------------------------------------
// FP64 arrays, FP32 arithmetic: the double-float dot product and axpy.
//
// The FP64 pipe of this GPU issues about 1/64 of the FP32 rate, so the FP64
// multidot / multi_axpy (4 FP64 FMAs per complex element and vector) are bound
// by it at about a third of the memory rate.  These kernels read the same FP64
// arrays and compute in FP32 with error-free transformations:
//  * each double d becomes the unevaluated sum hi + lo of two floats by bit
//    manipulation only (hi: sign, exponent and the leading 24 significant bits;
//    lo: the next 23 bits), so |d - hi - lo| < 2^-46 |d| (Dekker's double-length
//    representation, built here by truncation instead of rounding);
//  * a product of two such numbers is hi*hi exactly as p + e (TwoProduct with
//    one FMA) plus the cross terms hi*lo + lo*hi in FP32 (lo*lo < 2^-46 of the
//    product is dropped);
//  * p is added to the running high word by Knuth's TwoSum (exact: s + err), err,
//    e and the cross terms to the low word.
// This is the compensated dot product Dot2 of Ogita, Rump and Oishi (SIAM J.
// Sci. Comput. 26, 2005) on double-float inputs: the result is as accurate as a
// sum in 47-bit arithmetic, i.e. within a few 2^-46 sum|a_i b_i| of the exact
// value (FP64 arithmetic: 2^-53 per operation).  The per-thread sums go to FP64
// for the block and grid reductions.
//
// Range: elements with |d| < 2^-126 count as 0 and the low word is dropped below
// 2^-80 (absolute errors below 2^-103 |d|-units); |d| >= 2^128 becomes +-inf (the
// orthonormal vectors, Krylov vectors and iterates these kernels serve stay far
// inside the range).  Every addition and multiplication below uses the _rn
// intrinsics, which the compiler never contracts into an FMA.

// (h, l) += (uh + ul)(vh + vl)
__device__ __forceinline__ void ds_mac(float &h, float &l, float uh, float ul, float vh, float vl) {
    const float p = __fmul_rn(uh, vh);
    float e = fmaf(uh, vh, -p);
    e = fmaf(uh, vl, e);
    e = fmaf(ul, vh, e);
    const float s = __fadd_rn(h, p);
    const float bv = __fsub_rn(s, h);
    const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bv)), __fsub_rn(p, bv));
    h = s;
    l = __fadd_rn(l, __fadd_rn(err, e));
}

constexpr int DS_CHUNK = 8;

__global__ void __launch_bounds__(RED_THREADS) multidot_ds_kernel(PtrPack X, int k, const double2 *__restrict__ y,
                                                                  size_t n, double2 *__restrict__ partial,
                                                                  size_t pstride) {
    float rh[DS_CHUNK], rl[DS_CHUNK], ih[DS_CHUNK], il[DS_CHUNK];
#pragma unroll
    for (int j = 0; j < DS_CHUNK; ++j) { rh[j] = rl[j] = ih[j] = il[j] = 0.0f; }
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double2 b = y[i];
        float brh, brl, bih, bil;
        ds_split(b.x, brh, brl);
        ds_split(b.y, bih, bil);
#pragma unroll
        for (int j = 0; j < DS_CHUNK; ++j) {
            if (j < k) {
                const double2 a = static_cast<const double2 *>(X.p[j])[i];
                float arh, arl, aih, ail;
                ds_split(a.x, arh, arl);
                ds_split(a.y, aih, ail);
                // conj(a) b = (ar br + ai bi) + i (ar bi - ai br)
                ds_mac(rh[j], rl[j], arh, arl, brh, brl);
                ds_mac(rh[j], rl[j], aih, ail, bih, bil);
                ds_mac(ih[j], il[j], arh, arl, bih, bil);
                ds_mac(ih[j], il[j], -aih, -ail, brh, brl);
            }
        }
    }
    double re[DS_CHUNK], im[DS_CHUNK];
#pragma unroll
    for (int j = 0; j < DS_CHUNK; ++j) {
        re[j] = f2d_exact(rh[j]) + f2d_exact(rl[j]);
        im[j] = f2d_exact(ih[j]) + f2d_exact(il[j]);
    }
    block_reduce_store<DS_CHUNK>(re, im, k, partial, pstride);
}

// y += sign * sum_j coef[j] X_j, y and X_j FP64, double-float arithmetic
__global__ void __launch_bounds__(256) multi_axpy_ds_kernel(double2 *__restrict__ y, PtrPack X, int k,
                                                            const double2 *__restrict__ coef, double sign, size_t n) {
    float crh[DS_CHUNK], crl[DS_CHUNK], cih[DS_CHUNK], cil[DS_CHUNK];
#pragma unroll
    for (int j = 0; j < DS_CHUNK; ++j) {
        if (j < k) {
            const double2 t = coef[j];
            ds_split(sign * t.x, crh[j], crl[j]);
            ds_split(sign * t.y, cih[j], cil[j]);
        } else {
            crh[j] = crl[j] = cih[j] = cil[j] = 0.0f;
        }
    }
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double2 t = y[i];
        float rh, rl, ih, il;
        ds_split(t.x, rh, rl);
        ds_split(t.y, ih, il);
#pragma unroll
        for (int j = 0; j < DS_CHUNK; ++j) {
            if (j < k) {
                const double2 a = static_cast<const double2 *>(X.p[j])[i];
                float arh, arl, aih, ail;
                ds_split(a.x, arh, arl);
                ds_split(a.y, aih, ail);
                // c a = (cr ar - ci ai) + i (cr ai + ci ar)
                ds_mac(rh, rl, crh[j], crl[j], arh, arl);
                ds_mac(rh, rl, -cih[j], -cil[j], aih, ail);
                ds_mac(ih, il, crh[j], crl[j], aih, ail);
                ds_mac(ih, il, cih[j], cil[j], arh, arl);
            }
        }
        y[i] = make_double2(f2d_exact(rh) + f2d_exact(rl), f2d_exact(ih) + f2d_exact(il));
    }
}

static double2 *partial_ptr(Ctx &c) { return c.red_partial.as<double2>(); }

template <typename R>
void blas_multidot(Ctx &c, const void *const *X, int k, const void *y, size_t n, cpx<double> *d_out) {
    // FP32 vectors below 8 M complex values (a 16^3 x 32 spinor is 1.6 M): 2 blocks
    // per SM, 1.3x faster there than 4 (measured); the longer ones and the
    // double-float kernels run best at 4
    const int nb = red_grid(c, n, (sizeof(R) == 4 && n < ((size_t)8 << 20)) ? 2 : 4);
    const size_t pstride = RED_MAXBLOCKS;
    TimeScope ts(c.timer, sizeof(R) == 8 ? K_BLAS_F64 : K_BLAS_LOW, (double)(k + 1) * n * 2 * sizeof(R));
    const bool ds = sizeof(R) == 8 && c.ds_blas();
    const int C = ds ? DS_CHUNK : Chunk<R>::n;
    for (int j0 = 0; j0 < k; j0 += C) {
        PtrPack pk{};
        const int kk = k - j0 < C ? k - j0 : C;
        for (int j = 0; j < kk; ++j) pk.p[j] = X[j0 + j];
        if (ds)
            multidot_ds_kernel<<<nb, RED_THREADS, 0, c.stream>>>(pk, kk, static_cast<const double2 *>(y), n,
                                                                  partial_ptr(c) + (size_t)j0 * pstride, pstride);
        else
            multidot_kernel<R><<<nb, RED_THREADS, 0, c.stream>>>(pk, kk, y, n, partial_ptr(c) + (size_t)j0 * pstride,
                                                                 pstride, vec4_ok<R>(pk, kk, y, n));
        MG_CHECK_LAUNCH();
    }
    finalize_kernel<<<k, 128, 0, c.stream>>>(partial_ptr(c), pstride, nb, reinterpret_cast<double2 *>(d_out));
    MG_CHECK_LAUNCH();
}

template <typename R>
void blas_norm2(Ctx &c, const void *x, size_t n, cpx<double> *d_out) {
    const int nb = red_grid(c, n);
    TimeScope ts(c.timer, sizeof(R) == 8 ? K_BLAS_F64 : K_BLAS_LOW, (double)n * 2 * sizeof(R));
    norm2_kernel<R><<<nb, RED_THREADS, 0, c.stream>>>(x, n, partial_ptr(c));
    MG_CHECK_LAUNCH();
    finalize_kernel<<<1, 128, 0, c.stream>>>(partial_ptr(c), RED_MAXBLOCKS, nb, reinterpret_cast<double2 *>(d_out));
    MG_CHECK_LAUNCH();
}

void blas_resid_norm2(Ctx &c, const void *qv, const void *v, const cpx<double> *d_lambda, size_t n, cpx<double> *d_out) {
    const int nb = red_grid(c, n);
    TimeScope ts(c.timer, K_BLAS_F64, (double)n * 32);
    resid_norm2_kernel<<<nb, RED_THREADS, 0, c.stream>>>(static_cast<const double2 *>(qv), static_cast<const double2 *>(v),
                                                         reinterpret_cast<const double2 *>(d_lambda), n, partial_ptr(c));
    MG_CHECK_LAUNCH();
    finalize_kernel<<<1, 128, 0, c.stream>>>(partial_ptr(c), RED_MAXBLOCKS, nb, reinterpret_cast<double2 *>(d_out));
    MG_CHECK_LAUNCH();
}

// y += sign * sum_j coef[j] X_j
template <typename R>
__global__ void multi_axpy_kernel(void *__restrict__ yv, PtrPack X, int k, const double2 *__restrict__ coef, double sign,
                                  size_t n, bool vec4) {
    typedef typename V2<R>::T T;
    T *y = static_cast<T *>(yv);
    constexpr int C = Chunk<R>::n;
    R cr[C], ci[C];
#pragma unroll
    for (int j = 0; j < C; ++j) {
        if (j < k) { double2 t = coef[j]; cr[j] = (R)(sign * t.x); ci[j] = (R)(sign * t.y); }
        else { cr[j] = 0; ci[j] = 0; }
    }
    if constexpr (sizeof(R) == 4) {
        if (vec4) {   // two complex values per 16-byte access
            float4 *y4 = static_cast<float4 *>(yv);
            for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n / 2; i += (size_t)gridDim.x * blockDim.x) {
                float4 acc = y4[i];
#pragma unroll
                for (int j = 0; j < C; ++j) {
                    if (j < k) {
                        const float4 a = static_cast<const float4 *>(X.p[j])[i];
                        acc.x = fmaf(cr[j], a.x, acc.x); acc.x = fmaf(-ci[j], a.y, acc.x);
                        acc.y = fmaf(cr[j], a.y, acc.y); acc.y = fmaf(ci[j], a.x, acc.y);
                        acc.z = fmaf(cr[j], a.z, acc.z); acc.z = fmaf(-ci[j], a.w, acc.z);
                        acc.w = fmaf(cr[j], a.w, acc.w); acc.w = fmaf(ci[j], a.z, acc.w);
                    }
                }
                y4[i] = acc;
            }
            return;
        }
    }
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        T acc = y[i];
#pragma unroll
        for (int j = 0; j < C; ++j) {
            if (j < k) {
                T a = static_cast<const T *>(X.p[j])[i];
                acc.x = fma(cr[j], a.x, acc.x); acc.x = fma(-ci[j], a.y, acc.x);
                acc.y = fma(cr[j], a.y, acc.y); acc.y = fma(ci[j], a.x, acc.y);
            }
        }
        y[i] = acc;
    }
}

// element-wise grids: one thread per element up to per_sm blocks per SM (or
// blas_blocks per SM when the context sets it).  The FP32 multi-vector update
// runs best at 4 per SM (1.5x over 16 at 16^3 x 32), the double-float one,
// bound by its FP32 arithmetic, at 16
static int ew_grid(const Ctx &c, size_t n, int per_sm = 16) {
    size_t b = (n + 255) / 256;
    const size_t cap = (size_t)c.sms * (c.prm.blas_blocks > 0 ? c.prm.blas_blocks : per_sm);
    return (int)(b < cap ? (b < 1 ? 1 : b) : cap);
}

template <typename R>
void blas_multi_axpy(Ctx &c, void *y, const void *const *X, int k, const cpx<double> *d_coef, double sign, size_t n) {
    TimeScope ts(c.timer, sizeof(R) == 8 ? K_BLAS_F64 : K_BLAS_LOW, (double)(k + 2) * n * 2 * sizeof(R));
    const bool ds = sizeof(R) == 8 && c.ds_blas();
    const int C = ds ? DS_CHUNK : Chunk<R>::n;
    for (int j0 = 0; j0 < k; j0 += C) {
        PtrPack pk{};
        const int kk = k - j0 < C ? k - j0 : C;
        for (int j = 0; j < kk; ++j) pk.p[j] = X[j0 + j];
        if (ds) {
            multi_axpy_ds_kernel<<<ew_grid(c, n), 256, 0, c.stream>>>(
                static_cast<double2 *>(y), pk, kk, reinterpret_cast<const double2 *>(d_coef + j0), sign, n);
        } else {
            const bool v4 = vec4_ok<R>(pk, kk, y, n);
            multi_axpy_kernel<R><<<ew_grid(c, v4 ? n / 2 : n, sizeof(R) == 4 ? 4 : 16), 256, 0, c.stream>>>(
                y, pk, kk, reinterpret_cast<const double2 *>(d_coef + j0), sign, n, v4);
        }
        MG_CHECK_LAUNCH();
    }
}

template <typename R>
__global__ void axpy_kernel(double ar, double ai, const void *__restrict__ xv, void *__restrict__ yv, size_t n) {
    typedef typename V2<R>::T T;
    const T *x = static_cast<const T *>(xv);
    T *y = static_cast<T *>(yv);
    const R a = (R)ar, b = (R)ai;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        T u = x[i], v = y[i];
        v.x = fma(a, u.x, v.x); v.x = fma(-b, u.y, v.x);
        v.y = fma(a, u.y, v.y); v.y = fma(b, u.x, v.y);
        y[i] = v;
    }
}

template <typename R>
__global__ void scale_kernel(double ar, double ai, void *__restrict__ xv, size_t n) {
    typedef typename V2<R>::T T;
    T *x = static_cast<T *>(xv);
    const R a = (R)ar, b = (R)ai;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        T u = x[i];
        T v;
        v.x = a * u.x - b * u.y;
        v.y = a * u.y + b * u.x;
        x[i] = v;
    }
}

template <typename R>
void blas_axpy(Ctx &c, cpx<double> a, const void *x, void *y, size_t n) {
    TimeScope ts(c.timer, sizeof(R) == 8 ? K_BLAS_F64 : K_BLAS_LOW, 3.0 * n * 2 * sizeof(R));
    axpy_kernel<R><<<ew_grid(c, n), 256, 0, c.stream>>>(a.re, a.im, x, y, n);
    MG_CHECK_LAUNCH();
}

template <typename R>
void blas_scale(Ctx &c, cpx<double> a, void *x, size_t n) {
    TimeScope ts(c.timer, sizeof(R) == 8 ? K_BLAS_F64 : K_BLAS_LOW, 2.0 * n * 2 * sizeof(R));
    scale_kernel<R><<<ew_grid(c, n), 256, 0, c.stream>>>(a.re, a.im, x, n);
    MG_CHECK_LAUNCH();
}

template <typename R>
void blas_copy(Ctx &c, const void *x, void *y, size_t n) {
    MG_CUDA(cudaMemcpyAsync(y, x, n * 2 * sizeof(R), cudaMemcpyDeviceToDevice, c.stream));
}

template <typename R>
void blas_zero(Ctx &c, void *x, size_t n) {
    MG_CUDA(cudaMemsetAsync(x, 0, n * 2 * sizeof(R), c.stream));
}

// y (FP64 fine layout) += a * x (fine layout of precision R)
template <typename R>
__global__ void axpy_to_f64_fine_kernel(int V, double ar, double ai, const void *__restrict__ x, double2 *__restrict__ y) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
    cpx<R> v[12];
    Spinor<R>::load(x, V, s, v);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        double2 t = y[(size_t)k * V + s];
        double xr = v[k].re, xi = v[k].im;
        t.x = fma(ar, xr, t.x); t.x = fma(-ai, xi, t.x);
        t.y = fma(ar, xi, t.y); t.y = fma(ai, xr, t.y);
        y[(size_t)k * V + s] = t;
    }
}

template <typename R>
void blas_axpy_to_f64(Ctx &c, cpx<double> a, const void *x, void *y64, size_t n) {
    const int V = (int)(n / 12);
    TimeScope ts(c.timer, K_BLAS_F64, (double)n * (2 * sizeof(R) + 32));
    axpy_to_f64_fine_kernel<R><<<grid_for(V, 256), 256, 0, c.stream>>>(V, a.re, a.im, x, static_cast<double2 *>(y64));
    MG_CHECK_LAUNCH();
}

// y = A x and ys = s * y for a small row-major k x k matrix A (k <= 64), one
// thread per row; A, x, y and ys live on the device (no host round trip)
__global__ void small_gemv_kernel(const double2 *__restrict__ A, int k, const double2 *__restrict__ x, double s,
                                  double2 *__restrict__ y, double2 *__restrict__ ys) {
    const int i = threadIdx.x;
    if (i >= k) return;
    double re = 0, im = 0;
    for (int l = 0; l < k; ++l) {
        const double2 a = A[(size_t)i * k + l], b = x[l];
        re = fma(a.x, b.x, re); re = fma(-a.y, b.y, re);
        im = fma(a.x, b.y, im); im = fma(a.y, b.x, im);
    }
    y[i] = make_double2(re, im);
    ys[i] = make_double2(s * re, s * im);
}

void small_gemv(Ctx &c, const cpx<double> *A, int k, const cpx<double> *x, double s, cpx<double> *y, cpx<double> *ys) {
    MG_REQUIRE(k >= 1 && k <= 64, MGEIG_EINVAL);
    TimeScope ts(c.timer, K_BLAS_F64, (double)k * (k + 3) * 16);
    small_gemv_kernel<<<1, 64, 0, c.stream>>>(reinterpret_cast<const double2 *>(A), k, reinterpret_cast<const double2 *>(x),
                                              s, reinterpret_cast<double2 *>(y), reinterpret_cast<double2 *>(ys));
    MG_CHECK_LAUNCH();
}

#define INST(R)                                                                                             \
    template void blas_multidot<R>(Ctx &, const void *const *, int, const void *, size_t, cpx<double> *);    \
    template void blas_multi_axpy<R>(Ctx &, void *, const void *const *, int, const cpx<double> *, double, size_t); \
    template void blas_norm2<R>(Ctx &, const void *, size_t, cpx<double> *);                                     \
    template void blas_axpy<R>(Ctx &, cpx<double>, const void *, void *, size_t);                          \
    template void blas_scale<R>(Ctx &, cpx<double>, void *, size_t);                                       \
    template void blas_copy<R>(Ctx &, const void *, void *, size_t);                                       \
    template void blas_zero<R>(Ctx &, void *, size_t);                                                     \
    template void blas_axpy_to_f64<R>(Ctx &, cpx<double>, const void *, void *, size_t);
INST(double)
INST(float)
#undef INST

}  // namespace mgeig
