// Shared device types of libmgeig: complex arithmetic, lattice geometry and
// the internal field layouts.
//
// Internal layouts (structure of arrays, one component array after another, so
// that a warp of consecutive sites reads consecutive 16-byte words):
//   spinor FP64  double2 [12][V]          component k = 3*spin + colour
//   spinor FP32  float4  [6][V]           float4 q = components 2q, 2q+1
//   gauge  FP64  double2 [4][9][V]        U_mu(x)[a][b] at [mu][3a+b][x]
//   gauge  FP32  float4  [4][3][V]        two rows (u00,u01),(u02,u10),(u11,u12);
//                                         row 2 = conj(row0 x row1) (SU(3))
//   clover FP64  double2 [36][V]          per chirality block 36 reals: 6 diagonal,
//   clover FP32  float4  [18][V]          then the 15 upper off-diagonals (re, im)
//                                         in row-major order; (4 + m0) included
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mgeig {

template <typename R>
struct cpx {
    R re, im;
    __host__ __device__ cpx() : re(0), im(0) {}
    __host__ __device__ cpx(R r, R i = R(0)) : re(r), im(i) {}
};

template <typename R> __host__ __device__ __forceinline__ cpx<R> operator+(cpx<R> a, cpx<R> b) { return cpx<R>(a.re + b.re, a.im + b.im); }
template <typename R> __host__ __device__ __forceinline__ cpx<R> operator-(cpx<R> a, cpx<R> b) { return cpx<R>(a.re - b.re, a.im - b.im); }
template <typename R> __host__ __device__ __forceinline__ cpx<R> operator-(cpx<R> a) { return cpx<R>(-a.re, -a.im); }
template <typename R> __host__ __device__ __forceinline__ cpx<R> operator*(cpx<R> a, cpx<R> b) {
    return cpx<R>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename R> __host__ __device__ __forceinline__ cpx<R> operator*(R s, cpx<R> a) { return cpx<R>(s * a.re, s * a.im); }
template <typename R> __host__ __device__ __forceinline__ cpx<R> conj(cpx<R> a) { return cpx<R>(a.re, -a.im); }
template <typename R> __host__ __device__ __forceinline__ cpx<R> times_i(cpx<R> a) { return cpx<R>(-a.im, a.re); }
template <typename R> __host__ __device__ __forceinline__ cpx<R> times_mi(cpx<R> a) { return cpx<R>(a.im, -a.re); }
// a += b * c
template <typename R> __host__ __device__ __forceinline__ void cmac(cpx<R> &a, cpx<R> b, cpx<R> c) {
    a.re = fma(b.re, c.re, a.re); a.re = fma(-b.im, c.im, a.re);
    a.im = fma(b.re, c.im, a.im); a.im = fma(b.im, c.re, a.im);
}
// a += conj(b) * c
template <typename R> __host__ __device__ __forceinline__ void cmac_conj(cpx<R> &a, cpx<R> b, cpx<R> c) {
    a.re = fma(b.re, c.re, a.re); a.re = fma(b.im, c.im, a.re);
    a.im = fma(b.re, c.im, a.im); a.im = fma(-b.im, c.re, a.im);
}

// ---------------------------------------------------------------------------
// geometry

struct Geom {
    int L[4];        // Lx, Ly, Lz, Lt
    int stride[4];   // 1, Lx, Lx*Ly, Lx*Ly*Lz
    int bc[4];       // +1 / -1
    int V;           // number of sites (< 2^31)
};

__device__ __forceinline__ void site_coords(const Geom &g, int s, int c[4]) {
    c[0] = s % g.L[0]; s /= g.L[0];
    c[1] = s % g.L[1]; s /= g.L[1];
    c[2] = s % g.L[2];
    c[3] = s / g.L[2];
}

// neighbour of site s (coords c) in direction mu, forward (+1) or backward;
// *phase = boundary factor of the hop.
__device__ __forceinline__ int neighbor(const Geom &g, int s, const int c[4], int mu, bool fwd, int *phase) {
    if (fwd) {
        if (c[mu] == g.L[mu] - 1) { *phase = g.bc[mu]; return s - (g.L[mu] - 1) * g.stride[mu]; }
        *phase = 1; return s + g.stride[mu];
    }
    if (c[mu] == 0) { *phase = g.bc[mu]; return s + (g.L[mu] - 1) * g.stride[mu]; }
    *phase = 1; return s - g.stride[mu];
}

// ---------------------------------------------------------------------------
// field access

template <typename R> struct Spinor;

// Spinor<R>::comp(p, V, k, s): component k of site s as a complex lvalue
// (FP64 [12][V] complex; FP32 [6][V] float4 = [6][V][2] complex).
template <> struct Spinor<double> {
    __device__ __forceinline__ static cpx<double> &comp(const cpx<double> *p, int V, int k, int s) {
        return const_cast<cpx<double> *>(p)[(size_t)k * V + s];
    }
    __device__ __forceinline__ static void load(const void *base, int V, int s, cpx<double> v[12]) {
        const double2 *p = static_cast<const double2 *>(base);
#pragma unroll
        for (int k = 0; k < 12; ++k) { double2 t = p[(size_t)k * V + s]; v[k] = cpx<double>(t.x, t.y); }
    }
    __device__ __forceinline__ static void store(void *base, int V, int s, const cpx<double> v[12]) {
        double2 *p = static_cast<double2 *>(base);
#pragma unroll
        for (int k = 0; k < 12; ++k) p[(size_t)k * V + s] = make_double2(v[k].re, v[k].im);
    }
};

template <> struct Spinor<float> {
    __device__ __forceinline__ static cpx<float> &comp(const cpx<float> *p, int V, int k, int s) {
        return const_cast<cpx<float> *>(p)[((size_t)(k >> 1) * V + s) * 2 + (k & 1)];
    }
    __device__ __forceinline__ static void load(const void *base, int V, int s, cpx<float> v[12]) {
        const float4 *p = static_cast<const float4 *>(base);
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            float4 t = p[(size_t)q * V + s];
            v[2 * q] = cpx<float>(t.x, t.y); v[2 * q + 1] = cpx<float>(t.z, t.w);
        }
    }
    __device__ __forceinline__ static void store(void *base, int V, int s, const cpx<float> v[12]) {
        float4 *p = static_cast<float4 *>(base);
#pragma unroll
        for (int q = 0; q < 6; ++q) p[(size_t)q * V + s] = make_float4(v[2 * q].re, v[2 * q].im, v[2 * q + 1].re, v[2 * q + 1].im);
    }
};

template <typename R> struct Gauge;

template <> struct Gauge<double> {
    __device__ __forceinline__ static void load(const void *base, int V, int mu, int s, cpx<double> u[9]) {
        const double2 *p = static_cast<const double2 *>(base) + (size_t)mu * 9 * V;
#pragma unroll
        for (int k = 0; k < 9; ++k) { double2 t = p[(size_t)k * V + s]; u[k] = cpx<double>(t.x, t.y); }
    }
};

template <> struct Gauge<float> {
    __device__ __forceinline__ static void load(const void *base, int V, int mu, int s, cpx<float> u[9]) {
        const float4 *p = static_cast<const float4 *>(base) + (size_t)mu * 3 * V;
        float4 a = p[s], b = p[(size_t)V + s], c = p[(size_t)2 * V + s];
        u[0] = cpx<float>(a.x, a.y); u[1] = cpx<float>(a.z, a.w); u[2] = cpx<float>(b.x, b.y);
        u[3] = cpx<float>(b.z, b.w); u[4] = cpx<float>(c.x, c.y); u[5] = cpx<float>(c.z, c.w);
        // third row of an SU(3) matrix: conj of the cross product of rows 0 and 1
        u[6] = conj(u[1] * u[5] - u[2] * u[4]);
        u[7] = conj(u[2] * u[3] - u[0] * u[5]);
        u[8] = conj(u[0] * u[4] - u[1] * u[3]);
    }
};

template <typename R> struct Clover;

template <> struct Clover<double> {
    __device__ __forceinline__ static void load_block(const void *base, int V, int blk, int s, double r[36]) {
        const double2 *p = static_cast<const double2 *>(base) + (size_t)blk * 18 * V;
#pragma unroll
        for (int e = 0; e < 18; ++e) { double2 t = p[(size_t)e * V + s]; r[2 * e] = t.x; r[2 * e + 1] = t.y; }
    }
};

template <> struct Clover<float> {
    __device__ __forceinline__ static void load_block(const void *base, int V, int blk, int s, float r[36]) {
        const float4 *p = static_cast<const float4 *>(base) + (size_t)blk * 9 * V;
#pragma unroll
        for (int e = 0; e < 9; ++e) { float4 t = p[(size_t)e * V + s]; r[4 * e] = t.x; r[4 * e + 1] = t.y; r[4 * e + 2] = t.z; r[4 * e + 3] = t.w; }
    }
};

// index of the upper off-diagonal (i < j) of a 6x6 Hermitian block
__host__ __device__ __forceinline__ int offdiag_index(int i, int j) {
    // rows 0..4 hold 5,4,3,2,1 entries
    return i * 5 - (i * (i - 1)) / 2 + (j - i - 1);
}

// out[0..5] = H in[0..5] for the packed Hermitian block r[36]
template <typename R>
__device__ __forceinline__ void hermitian6_apply(const R r[36], const cpx<R> in[6], cpx<R> out[6]) {
#pragma unroll
    for (int i = 0; i < 6; ++i) out[i] = r[i] * in[i];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
#pragma unroll
        for (int j = i + 1; j < 6; ++j) {
            const int o = offdiag_index(i, j);
            cpx<R> h(r[6 + 2 * o], r[7 + 2 * o]);
            cmac(out[i], h, in[j]);        // H_ij x_j
            cmac_conj(out[j], h, in[i]);   // H_ji x_i = conj(H_ij) x_i
        }
    }
}

template <typename R>
__device__ __forceinline__ void clover_apply(const void *clov, int V, int s, const cpx<R> in[12], cpx<R> out[12]) {
    R r[36];
    Clover<R>::load_block(clov, V, 0, s, r);
    hermitian6_apply<R>(r, in, out);
    Clover<R>::load_block(clov, V, 1, s, r);
    hermitian6_apply<R>(r, in + 6, out + 6);
}

// ---------------------------------------------------------------------------
// spin projection in the chiral basis: g_mu = [[0, B_mu], [B_mu^dag, 0]] with
// B_k = i sigma_k (k = 1, 2, 3) and B_4 = 1.  Two-component spin vectors of
// colour triplets: a[s*3 + c].

template <typename R>
__device__ __forceinline__ void spin_B(int mu, const cpx<R> l[6], cpx<R> out[6]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        cpx<R> l0 = l[c], l1 = l[3 + c];
        switch (mu) {
            case 0: out[c] = times_i(l1); out[3 + c] = times_i(l0); break;      // i s_1
            case 1: out[c] = l1; out[3 + c] = -l0; break;                     // i s_2
            case 2: out[c] = times_i(l0); out[3 + c] = times_mi(l1); break;   // i s_3
            default: out[c] = l0; out[3 + c] = l1; break;                     // 1
        }
    }
}

template <typename R>
__device__ __forceinline__ void spin_Bdag(int mu, const cpx<R> a[6], cpx<R> out[6]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        cpx<R> a0 = a[c], a1 = a[3 + c];
        switch (mu) {
            case 0: out[c] = times_mi(a1); out[3 + c] = times_mi(a0); break;
            case 1: out[c] = -a1; out[3 + c] = a0; break;
            case 2: out[c] = times_mi(a0); out[3 + c] = times_i(a1); break;
            default: out[c] = a0; out[3 + c] = a1; break;
        }
    }
}

// y[0..2] = U x,  U row-major 3x3
template <typename R>
__device__ __forceinline__ void su3_mul(const cpx<R> u[9], const cpx<R> *x, cpx<R> *y) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        cpx<R> acc = u[3 * a] * x[0];
        cmac(acc, u[3 * a + 1], x[1]);
        cmac(acc, u[3 * a + 2], x[2]);
        y[a] = acc;
    }
}

// y[0..2] = U^dag x
template <typename R>
__device__ __forceinline__ void su3_dag_mul(const cpx<R> u[9], const cpx<R> *x, cpx<R> *y) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        cpx<R> acc = conj(u[a]) * x[0];
        cmac_conj(acc, u[3 + a], x[1]);
        cmac_conj(acc, u[6 + a], x[2]);
        y[a] = acc;
    }
}

// Hopping contributions at one site in direction mu, accumulated into the
// upper (spins 0,1) and lower (spins 2,3) halves:
//   forward:  -1/2 (1 - g_mu) U psi   = -1/2 (U h, -B^dag U h),   h = psi_u - B psi_l
//   backward: -1/2 (1 + g_mu) U^dag psi = -1/2 (U^dag h', B^dag U^dag h'), h' = psi_u + B psi_l
// The -1/2 is applied by the caller.  `phase` is the boundary factor.
template <typename R>
__device__ __forceinline__ void hop_accumulate(int mu, bool fwd, const cpx<R> u[9], const cpx<R> psi[12], R phase,
                                               cpx<R> up[6], cpx<R> lo[6]) {
    cpx<R> bl[6], h[6], uh[6], bd[6];
    spin_B<R>(mu, psi + 6, bl);
#pragma unroll
    for (int k = 0; k < 6; ++k) h[k] = fwd ? (psi[k] - bl[k]) : (psi[k] + bl[k]);
    if (fwd) { su3_mul<R>(u, h, uh); su3_mul<R>(u, h + 3, uh + 3); }
    else { su3_dag_mul<R>(u, h, uh); su3_dag_mul<R>(u, h + 3, uh + 3); }
#pragma unroll
    for (int k = 0; k < 6; ++k) uh[k] = phase * uh[k];
    spin_Bdag<R>(mu, uh, bd);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        up[k] = up[k] + uh[k];
        lo[k] = fwd ? (lo[k] - bd[k]) : (lo[k] + bd[k]);
    }
}

// ---------------------------------------------------------------------------
// fine operator modes
enum OpMode { MODE_D = 0, MODE_DSIGMA = 1, MODE_QSIGMA = 2 };

}  // namespace mgeig
