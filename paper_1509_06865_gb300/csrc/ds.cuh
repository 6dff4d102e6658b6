// Double-float ("double-single") arithmetic: a value is the unevaluated sum
// h + l of two floats with |l| <= ulp(h) / 2, about 48 significant bits, kept on
// the FP32 pipe.  The FP64 pipe of this GPU issues about 1/64 of the FP32 rate,
// so the FP64-class operations of the mixed path (the outer FGMRES matvec,
// Gram-Schmidt, Rayleigh quotients) run faster in this form than in FP64.
//
// The building blocks are the error-free transformations of Dekker (Numer.
// Math. 18, 1971) and Knuth (TAOCP vol. 2): TwoSum (s + e = a + b exactly, six
// additions), TwoProduct by one FMA (p + e = a * b exactly), and the Fast2Sum
// renormalisation (|a| >= |b|).  Every addition and multiplication uses the
// _rn intrinsics, which the compiler never contracts into an FMA.
//
// Range: FP32 exponents (|x| < 2^128; the low word underflows below about
// 2^-102), far wider than the normalised vectors these kernels see need.
#pragma once

#include "common.cuh"

namespace mgeig {

#ifdef __CUDA_ARCH__
#define DS_ADD(a, b) __fadd_rn(a, b)
#define DS_SUB(a, b) __fsub_rn(a, b)
#define DS_MUL(a, b) __fmul_rn(a, b)
#else
#define DS_ADD(a, b) ((a) + (b))
#define DS_SUB(a, b) ((a) - (b))
#define DS_MUL(a, b) ((a) * (b))
#endif

// float -> double by bit manipulation (exact; no FP64 conversion instruction):
// the exponent rebiased by 1023 - 127, the 23 mantissa bits moved up by 29.
// Zeros, subnormals, infinities and NaN take the conversion instruction.
__device__ __forceinline__ double f2d_exact(float f) {
    const unsigned b = __float_as_uint(f);
    const unsigned e = (b >> 23) & 0xffu;
    if (e == 0u || e == 255u) return (double)f;
    const unsigned hw = (b & 0x80000000u) | (((b & 0x7fffffffu) >> 3) + (896u << 20));
    return __hiloint2double((int)hw, (int)(b << 29));
}

struct dsf {
    float h, l;
    __host__ __device__ dsf() : h(0.0f), l(0.0f) {}
    __host__ __device__ dsf(int i) : h((float)i), l(0.0f) {}
    __host__ __device__ dsf(float f) : h(f), l(0.0f) {}
    // round to nearest twice: h = fl(d), l = fl(d - h)
    __host__ __device__ dsf(double d) : h((float)d), l((float)(d - (double)(float)d)) {}
    __host__ __device__ static dsf raw(float hh, float ll) { dsf r; r.h = hh; r.l = ll; return r; }
    // h + l rounded once to FP64
#ifdef __CUDA_ARCH__
    __device__ double to_double() const { return f2d_exact(h) + f2d_exact(l); }
#else
    double to_double() const { return (double)h + (double)l; }
#endif
};

// Fast2Sum: h + l = a + b exactly when |a| >= |b|
__host__ __device__ __forceinline__ dsf ds_fast2sum(float a, float b) {
    const float s = DS_ADD(a, b);
    return dsf::raw(s, DS_SUB(b, DS_SUB(s, a)));
}

__host__ __device__ __forceinline__ dsf operator+(dsf a, dsf b) {
    const float s = DS_ADD(a.h, b.h);                                        // TwoSum(a.h, b.h)
    const float v = DS_SUB(s, a.h);
    const float e = DS_ADD(DS_SUB(a.h, DS_SUB(s, v)), DS_SUB(b.h, v));
    return ds_fast2sum(s, DS_ADD(e, DS_ADD(a.l, b.l)));
}
__host__ __device__ __forceinline__ dsf operator-(dsf a) { return dsf::raw(-a.h, -a.l); }
__host__ __device__ __forceinline__ dsf operator-(dsf a, dsf b) { return a + (-b); }
__host__ __device__ __forceinline__ dsf operator*(dsf a, dsf b) {
    const float p = DS_MUL(a.h, b.h);
    float e = fmaf(a.h, b.h, -p);                                             // TwoProduct(a.h, b.h)
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);                                                    // a.l * b.l dropped (2^-48)
    return ds_fast2sum(p, e);
}
// a * b + c (the overload joins the FP32 / FP64 fma of the global namespace)
using ::fma;
__host__ __device__ __forceinline__ dsf fma(dsf a, dsf b, dsf c) { return a * b + c; }

#undef DS_ADD
#undef DS_SUB
#undef DS_MUL

// A double as the unevaluated sum of two floats by bit manipulation only (no
// FP64 instruction): hi = sign, exponent and the leading 24 significant bits,
// lo = the next 23 bits, so |d - hi - lo| < 2^-46 |d|.  |d| < 2^-126 gives 0,
// the low word is dropped below 2^-80, |d| >= 2^128 gives +-inf.
__device__ __forceinline__ void ds_split(double d, float &hi, float &lo) {
    const unsigned hw = (unsigned)__double2hiint(d), lw = (unsigned)__double2loint(d);
    const unsigned sgn = hw & 0x80000000u;
    const unsigned e = (hw >> 20) & 0x7ffu;   // biased FP64 exponent
    // FP32 exponent field e - 896; the top 23 mantissa bits: 20 of hw, 3 of lw
    unsigned hb = __funnelshift_l(lw, (hw & 0x7fffffffu) - (896u << 20), 3) | sgn;
    hb = e < 897u ? sgn : hb;
    hb = e > 1150u ? (sgn | 0x7f800000u) : hb;
    hi = __uint_as_float(hb);
    // lo = m * 2^(e - 1023 - 46) for the next 23 mantissa bits m = lw[28:6]:
    // x = 2^23 + m exactly (the mantissa field of 2^23), lo = x s - 2^23 s
    const float x = __uint_as_float(0x4B000000u | ((lw >> 6) & 0x7fffffu));
    const float sc = (e >= 943u && e <= 1150u) ? __uint_as_float(sgn | ((e - 942u) << 23)) : 0.0f;
    lo = fmaf(x, sc, -__fmul_rn(sc, 8388608.0f));
}

__device__ __forceinline__ dsf ds_from_double(double d) {
    float h, l;
    ds_split(d, h, l);
    return dsf::raw(h, l);   // |l| < 2^-23 |h|: a valid (unnormalised by at most one ulp) pair
}

// field access in double-float form: spinors stay FP64 in memory (the FP64
// layout double2 [12][V]); links and clover come from double-float copies of
// the FP64 arrays, one float2 (h, l) per double at the same index.
template <> struct Spinor<dsf> {
    __device__ __forceinline__ static void load(const void *base, int V, int s, cpx<dsf> v[12]) {
        const double2 *p = static_cast<const double2 *>(base);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const double2 t = p[(size_t)k * V + s];
            v[k] = cpx<dsf>(ds_from_double(t.x), ds_from_double(t.y));
        }
    }
    __device__ __forceinline__ static void store(void *base, int V, int s, const cpx<dsf> v[12]) {
        double2 *p = static_cast<double2 *>(base);
#pragma unroll
        for (int k = 0; k < 12; ++k) p[(size_t)k * V + s] = make_double2(v[k].re.to_double(), v[k].im.to_double());
    }
};

template <> struct Gauge<dsf> {
    __device__ __forceinline__ static void load(const void *base, int V, int mu, int s, cpx<dsf> u[9]) {
        const float4 *p = static_cast<const float4 *>(base) + (size_t)mu * 9 * V;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const float4 t = p[(size_t)k * V + s];
            u[k] = cpx<dsf>(dsf::raw(t.x, t.y), dsf::raw(t.z, t.w));
        }
    }
};

template <> struct Clover<dsf> {
    __device__ __forceinline__ static void load_block(const void *base, int V, int blk, int s, dsf r[36]) {
        const float4 *p = static_cast<const float4 *>(base) + (size_t)blk * 18 * V;
#pragma unroll
        for (int e = 0; e < 18; ++e) {
            const float4 t = p[(size_t)e * V + s];
            r[2 * e] = dsf::raw(t.x, t.y);
            r[2 * e + 1] = dsf::raw(t.z, t.w);
        }
    }
};

}  // namespace mgeig
