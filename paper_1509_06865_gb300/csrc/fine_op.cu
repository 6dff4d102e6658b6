// Fine-grid fields and the clover-improved Wilson stencil (Sec. 2 of
// arXiv:1509.06865: D, Q = gamma5 D and the shifted forms Q - sigma and
// D_sigma = D - sigma gamma5 used by the Rayleigh quotient iteration).
//
// One thread per site.  The stencil reads the site's spinor and clover, the
// eight neighbour spinors and the eight links (forward links of the site,
// backward links of the lower neighbours), uses the chiral-basis half-spinor
// projection (two SU(3) products per hop) and writes one spinor.  Counting
// every field once (neighbour spinors and backward links are re-reads of data
// other sites also need), that is 672 bytes per site in FP32 (x 96, y 96,
// two-row links 192, clover 288) and 1536 bytes in FP64 (x 192, y 192, full
// links 576, clover 576).
#include "ds.cuh"
#include "internal.h"

namespace mgeig {

int grid_for(size_t n, int threads) { return (int)((n + threads - 1) / threads); }

// ---------------------------------------------------------------------------
// gauge packing

__global__ void pack_gauge_kernel(int V, const double2 *__restrict__ in, double2 *__restrict__ u64,
                                  float4 *__restrict__ u32) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
    for (int mu = 0; mu < 4; ++mu) {
        const double2 *src = in + ((size_t)s * 4 + mu) * 9;
        double2 e[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            e[k] = src[k];
            u64[((size_t)mu * 9 + k) * V + s] = e[k];
        }
        float4 *d = u32 + (size_t)mu * 3 * V;
        d[s] = make_float4((float)e[0].x, (float)e[0].y, (float)e[1].x, (float)e[1].y);
        d[(size_t)V + s] = make_float4((float)e[2].x, (float)e[2].y, (float)e[3].x, (float)e[3].y);
        d[(size_t)2 * V + s] = make_float4((float)e[4].x, (float)e[4].y, (float)e[5].x, (float)e[5].y);
    }
}

void pack_gauge(Ctx &c, const double *dev_in) {
    const int V = c.g.V;
    c.ds_fields_valid = false;
    TimeScope ts(c.timer, K_OTHER, 0);
    pack_gauge_kernel<<<grid_for(V, 128), 128, 0, c.stream>>>(V, reinterpret_cast<const double2 *>(dev_in),
                                                            c.U64.as<double2>(), c.U32.as<float4>());
    MG_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------
// clover term

// sigma_{mu nu} restricted to chirality block c, for the planes
// (0,1) (0,2) (0,3) (1,2) (1,3) (2,3): [c][plane][2x2]
__constant__ double c_sigma[2][6][4][2];

static void host_sigma_blocks(double out[2][6][4][2]) {
    // B_mu in the chiral basis (g_mu = [[0, B], [B^dag, 0]])
    typedef cpx<double> C;
    C B[4][2][2] = {
        {{C(0, 0), C(0, 1)}, {C(0, 1), C(0, 0)}},     // i s_1
        {{C(0, 0), C(1, 0)}, {C(-1, 0), C(0, 0)}},    // i s_2
        {{C(0, 1), C(0, 0)}, {C(0, 0), C(0, -1)}},    // i s_3
        {{C(1, 0), C(0, 0)}, {C(0, 0), C(1, 0)}},     // 1
    };
    auto mul = [](const C a[2][2], const C b[2][2], bool adag_a, bool adag_b, C r[2][2]) {
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) {
                C acc(0, 0);
                for (int k = 0; k < 2; ++k) {
                    C x = adag_a ? conj(a[k][i]) : a[i][k];
                    C y = adag_b ? conj(b[j][k]) : b[k][j];
                    acc = acc + x * y;
                }
                r[i][j] = acc;
            }
    };
    const int planes[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
    for (int p = 0; p < 6; ++p) {
        int mu = planes[p][0], nu = planes[p][1];
        C t1[2][2], t2[2][2];
        // g_mu g_nu = diag(B_mu B_nu^dag, B_mu^dag B_nu);  sigma = (i/2)(g_mu g_nu - g_nu g_mu)
        mul(B[mu], B[nu], false, true, t1);
        mul(B[nu], B[mu], false, true, t2);
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) {
                C d = t1[i][j] - t2[i][j];
                C s = C(0, 0.5) * d;
                out[0][p][2 * i + j][0] = s.re;
                out[0][p][2 * i + j][1] = s.im;
            }
        mul(B[mu], B[nu], true, false, t1);
        mul(B[nu], B[mu], true, false, t2);
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) {
                C d = t1[i][j] - t2[i][j];
                C s = C(0, 0.5) * d;
                out[1][p][2 * i + j][0] = s.re;
                out[1][p][2 * i + j][1] = s.im;
            }
    }
}

__device__ __forceinline__ void mat3_mul(const cpx<double> *a, const cpx<double> *b, cpx<double> *r, bool da, bool db) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            cpx<double> acc;
            for (int k = 0; k < 3; ++k) {
                cpx<double> x = da ? conj(a[3 * k + i]) : a[3 * i + k];
                cpx<double> y = db ? conj(b[3 * j + k]) : b[3 * k + j];
                cmac(acc, x, y);
            }
            r[3 * i + j] = acc;
        }
}

__device__ void load_link64(const double2 *u64, int V, int mu, int s, cpx<double> *u) {
    for (int k = 0; k < 9; ++k) {
        double2 t = u64[((size_t)mu * 9 + k) * V + s];
        u[k] = cpx<double>(t.x, t.y);
    }
}

// product of four links, each optionally daggered
__device__ void leaf(const double2 *u64, int V, int m0, int s0, bool d0, int m1, int s1, bool d1, int m2, int s2,
                     bool d2, int m3, int s3, bool d3, cpx<double> *out) {
    cpx<double> a[9], b[9], t[9], t2[9];
    load_link64(u64, V, m0, s0, a);
    load_link64(u64, V, m1, s1, b);
    mat3_mul(a, b, t, d0, d1);
    load_link64(u64, V, m2, s2, a);
    load_link64(u64, V, m3, s3, b);
    mat3_mul(a, b, t2, d2, d3);
    mat3_mul(t, t2, out, false, false);
}

__global__ void clover_build_kernel(Geom g, const double2 *__restrict__ u64, double csw, double mass,
                                    double2 *__restrict__ clov64, float4 *__restrict__ clov32) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    const int V = g.V;
    int c[4];
    site_coords(g, s, c);
    // packed accumulators: per block 6 diagonal reals + 15 upper complex
    double diag[2][6];
    cpx<double> off[2][15];
    for (int b = 0; b < 2; ++b) {
        for (int i = 0; i < 6; ++i) diag[b][i] = 0;
        for (int i = 0; i < 15; ++i) off[b][i] = cpx<double>();
    }
    const int planes[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
    for (int p = 0; p < 6; ++p) {
        const int mu = planes[p][0], nu = planes[p][1];
        int ph, cc[4];
        const int xpm = neighbor(g, s, c, mu, true, &ph);
        const int xmm = neighbor(g, s, c, mu, false, &ph);
        const int xpn = neighbor(g, s, c, nu, true, &ph);
        const int xmn = neighbor(g, s, c, nu, false, &ph);
        for (int k = 0; k < 4; ++k) cc[k] = c[k];
        cc[mu] = (c[mu] + g.L[mu] - 1) % g.L[mu];
        const int xmm_pn = neighbor(g, xmm, cc, nu, true, &ph);   // x - mu + nu
        const int xmm_mn = neighbor(g, xmm, cc, nu, false, &ph);  // x - mu - nu
        for (int k = 0; k < 4; ++k) cc[k] = c[k];
        cc[nu] = (c[nu] + g.L[nu] - 1) % g.L[nu];
        const int xmn_pm = neighbor(g, xmn, cc, mu, true, &ph);   // x - nu + mu
        cpx<double> Q[9], l[9];
        // x -> x+mu -> x+mu+nu -> x+nu -> x
        leaf(u64, V, mu, s, false, nu, xpm, false, mu, xpn, true, nu, s, true, Q);
        // x -> x+nu -> x+nu-mu -> x-mu -> x
        leaf(u64, V, nu, s, false, mu, xmm_pn, true, nu, xmm, true, mu, xmm, false, l);
        for (int k = 0; k < 9; ++k) Q[k] = Q[k] + l[k];
        // x -> x-mu -> x-mu-nu -> x-nu -> x
        leaf(u64, V, mu, xmm, true, nu, xmm_mn, true, mu, xmm_mn, false, nu, xmn, false, l);
        for (int k = 0; k < 9; ++k) Q[k] = Q[k] + l[k];
        // x -> x-nu -> x-nu+mu -> x+mu -> x
        leaf(u64, V, nu, xmn, true, mu, xmn, false, nu, xmn_pm, false, mu, s, true, l);
        for (int k = 0; k < 9; ++k) Q[k] = Q[k] + l[k];
        // F = (Q - Q^dag) / 8 ; the plane contributes c_sw (i/2) sigma (x) F
        cpx<double> F[9];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) F[3 * a + b] = 0.125 * (Q[3 * a + b] - conj(Q[3 * b + a]));
        for (int blk = 0; blk < 2; ++blk) {
            for (int i = 0; i < 6; ++i) {
                const int si = i / 3, ai = i % 3;
                for (int j = i; j < 6; ++j) {
                    const int sj = j / 3, aj = j % 3;
                    cpx<double> sg(c_sigma[blk][p][2 * si + sj][0], c_sigma[blk][p][2 * si + sj][1]);
                    cpx<double> v = cpx<double>(0, 0.5 * csw) * (sg * F[3 * ai + aj]);
                    if (i == j) diag[blk][i] += v.re;
                    else off[blk][offdiag_index(i, j)] = off[blk][offdiag_index(i, j)] + v;
                }
            }
        }
    }
    for (int blk = 0; blk < 2; ++blk) {
        double r[36];
        for (int i = 0; i < 6; ++i) r[i] = diag[blk][i] + mass;
        for (int o = 0; o < 15; ++o) { r[6 + 2 * o] = off[blk][o].re; r[7 + 2 * o] = off[blk][o].im; }
        for (int e = 0; e < 18; ++e) clov64[((size_t)blk * 18 + e) * V + s] = make_double2(r[2 * e], r[2 * e + 1]);
        for (int e = 0; e < 9; ++e)
            clov32[((size_t)blk * 9 + e) * V + s] =
                make_float4((float)r[4 * e], (float)r[4 * e + 1], (float)r[4 * e + 2], (float)r[4 * e + 3]);
    }
}

void build_clover(Ctx &c) {
    c.ds_fields_valid = false;
    double sig[2][6][4][2];
    host_sigma_blocks(sig);
    MG_CUDA(cudaMemcpyToSymbolAsync(c_sigma, sig, sizeof(sig), 0, cudaMemcpyHostToDevice, c.stream));
    TimeScope ts(c.timer, K_OTHER, 0);
    clover_build_kernel<<<grid_for(c.g.V, 64), 64, 0, c.stream>>>(c.g, c.U64.as<double2>(), c.prm.csw,
                                                                  4.0 + c.prm.m0, c.clov64.as<double2>(),
                                                                  c.clov32.as<float4>());
    MG_CHECK_LAUNCH();
}

// A caller's clover term [site][blk][6][6] complex (without the mass term) ->
// the packed layouts, with (4 + m0) added on the diagonal.  Only the real part
// of the diagonal and the upper triangle are read (the blocks are Hermitian).
__global__ void pack_clover_kernel(int V, const double2 *__restrict__ in, double mass, double2 *__restrict__ clov64,
                                   float4 *__restrict__ clov32) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
    for (int blk = 0; blk < 2; ++blk) {
        const double2 *b = in + ((size_t)s * 2 + blk) * 36;
        double r[36];
        for (int i = 0; i < 6; ++i) r[i] = b[i * 6 + i].x + mass;
        for (int i = 0; i < 6; ++i)
            for (int j = i + 1; j < 6; ++j) {
                const int o = offdiag_index(i, j);
                r[6 + 2 * o] = b[i * 6 + j].x;
                r[7 + 2 * o] = b[i * 6 + j].y;
            }
        for (int e = 0; e < 18; ++e) clov64[((size_t)blk * 18 + e) * V + s] = make_double2(r[2 * e], r[2 * e + 1]);
        for (int e = 0; e < 9; ++e)
            clov32[((size_t)blk * 9 + e) * V + s] =
                make_float4((float)r[4 * e], (float)r[4 * e + 1], (float)r[4 * e + 2], (float)r[4 * e + 3]);
    }
}

void pack_clover(Ctx &c, const double *dev_in) {
    c.ds_fields_valid = false;
    TimeScope ts(c.timer, K_OTHER, 0);
    pack_clover_kernel<<<grid_for(c.g.V, 128), 128, 0, c.stream>>>(c.g.V, reinterpret_cast<const double2 *>(dev_in),
                                                                   4.0 + c.prm.m0, c.clov64.as<double2>(),
                                                                   c.clov32.as<float4>());
    MG_CHECK_LAUNCH();
}

// [site][blk][6][6] complex, without the mass term
__global__ void unpack_clover_kernel(int V, const double2 *__restrict__ clov64, double mass, double2 *__restrict__ out) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
    for (int blk = 0; blk < 2; ++blk) {
        double r[36];
        for (int e = 0; e < 18; ++e) {
            double2 t = clov64[((size_t)blk * 18 + e) * V + s];
            r[2 * e] = t.x;
            r[2 * e + 1] = t.y;
        }
        double2 *o = out + ((size_t)s * 2 + blk) * 36;
        for (int i = 0; i < 6; ++i)
            for (int j = 0; j < 6; ++j) {
                double2 v;
                if (i == j) v = make_double2(r[i] - mass, 0.0);
                else if (i < j) { int k = offdiag_index(i, j); v = make_double2(r[6 + 2 * k], r[7 + 2 * k]); }
                else { int k = offdiag_index(j, i); v = make_double2(r[6 + 2 * k], -r[7 + 2 * k]); }
                o[i * 6 + j] = v;
            }
    }
}

void unpack_clover(Ctx &c, double *dev_out) {
    unpack_clover_kernel<<<grid_for(c.g.V, 128), 128, 0, c.stream>>>(c.g.V, c.clov64.as<double2>(), 4.0 + c.prm.m0,
                                                                     reinterpret_cast<double2 *>(dev_out));
    MG_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------
// the stencil

template <typename R, typename Rin>
struct InLoad {
    __device__ __forceinline__ static void load(const void *base, int V, int s, cpx<R> v[12]) {
        Spinor<R>::load(base, V, s, v);
    }
};
template <>
struct InLoad<double, float> {
    __device__ __forceinline__ static void load(const void *base, int V, int s, cpx<double> v[12]) {
        cpx<float> t[12];
        Spinor<float>::load(base, V, s, t);
#pragma unroll
        for (int k = 0; k < 12; ++k) v[k] = cpx<double>(t[k].re, t[k].im);
    }
};

template <>
struct InLoad<dsf, float> {
    __device__ __forceinline__ static void load(const void *base, int V, int s, cpx<dsf> v[12]) {
        cpx<float> t[12];
        Spinor<float>::load(base, V, s, t);
#pragma unroll
        for (int k = 0; k < 12; ++k) v[k] = cpx<dsf>(dsf(t[k].re), dsf(t[k].im));
    }
};

// Where a site's links and clover come from: the global arrays, or (FP32, many
// fields per launch) the CTA's copy in shared memory of its own sites' forward
// links and clover, in the global layout with V = the CTA's site count, so the
// same loaders read it.  A backward hop's link is the forward link of the lower
// neighbour: from the copy when that neighbour is one of the CTA's sites.
template <typename R>
struct GlobalFields {
    const void *U, *clov;
    int V;
    // the forward link of the site itself, the backward link (forward link of the lower neighbour)
    __device__ __forceinline__ void link_fwd(int mu, int site, cpx<R> u[9]) const { Gauge<R>::load(U, V, mu, site, u); }
    __device__ __forceinline__ void link_bwd(int mu, int site, cpx<R> u[9]) const { Gauge<R>::load(U, V, mu, site, u); }
    __device__ __forceinline__ void clover(int s, const cpx<R> in[12], cpx<R> out[12]) const {
        clover_apply<R>(clov, V, s, in, out);
    }
};

struct StagedFields {
    const float4 *sU, *sC;   // [4*3][stride] and [18][stride] float4 planes of the CTA's sites
    const void *U;           // the global FP32 links, for neighbours outside the CTA
    int s0, n, stride, V;    // first site, sites staged, plane stride, lattice volume
    __device__ __forceinline__ void link_fwd(int mu, int site, cpx<float> u[9]) const {
        Gauge<float>::load(sU, stride, mu, site - s0, u);   // always one of the CTA's sites
    }
    __device__ __forceinline__ void link_bwd(int mu, int site, cpx<float> u[9]) const {
        const int l = site - s0;
        if (l >= 0 && l < n) Gauge<float>::load(sU, stride, mu, l, u);
        else Gauge<float>::load(U, V, mu, site, u);
    }
    __device__ __forceinline__ void clover(int s, const cpx<float> in[12], cpx<float> out[12]) const {
        clover_apply<float>(sC, stride, s - s0, in, out);
    }
};

// y(s) = op(x)(s) for one site s: the eight hops, the clover term and the shift
template <typename R, typename Rin, int MODE, typename F>
__device__ __forceinline__ void wilson_clover_site_f(const Geom &g, const F &fields, const void *__restrict__ x,
                                                     void *__restrict__ y, R sigma, int s) {
    const int V = g.V;
    int c[4];
    site_coords(g, s, c);
    cpx<R> up[6], lo[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) { up[k] = cpx<R>(); lo[k] = cpx<R>(); }
    // unrolled: the coordinates, strides and gamma structure of each direction are
    // compile-time, nothing is indexed at run time (no local-memory frame)
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        int ph;
        cpx<R> u[9], psi[12];
        int n = neighbor(g, s, c, mu, true, &ph);
        fields.link_fwd(mu, s, u);
        InLoad<R, Rin>::load(x, V, n, psi);
        hop_accumulate<R>(mu, true, u, psi, (R)ph, up, lo);
        n = neighbor(g, s, c, mu, false, &ph);
        fields.link_bwd(mu, n, u);
        InLoad<R, Rin>::load(x, V, n, psi);
        hop_accumulate<R>(mu, false, u, psi, (R)ph, up, lo);
    }
    cpx<R> psi[12], out[12];
    InLoad<R, Rin>::load(x, V, s, psi);
    fields.clover(s, psi, out);
    const R half = R(0.5);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        out[k] = out[k] - half * up[k];
        out[6 + k] = out[6 + k] - half * lo[k];
    }
    if (MODE == MODE_DSIGMA) {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            out[k] = out[k] - sigma * psi[k];
            out[6 + k] = out[6 + k] + sigma * psi[6 + k];
        }
    } else if (MODE == MODE_QSIGMA) {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            out[k] = out[k] - sigma * psi[k];
            out[6 + k] = -out[6 + k] - sigma * psi[6 + k];
        }
    }
    Spinor<R>::store(y, V, s, out);
}

template <typename R, typename Rin, int MODE>
__device__ __forceinline__ void wilson_clover_site(const Geom &g, const void *__restrict__ U,
                                                   const void *__restrict__ clov, const void *__restrict__ x,
                                                   void *__restrict__ y, R sigma, int s) {
    wilson_clover_site_f<R, Rin, MODE>(g, GlobalFields<R>{U, clov, g.V}, x, y, sigma, s);
}

template <typename R, typename Rin, int MODE>
__global__ void __launch_bounds__(128) wilson_clover_kernel(Geom g, const void *__restrict__ U,
                                                            const void *__restrict__ clov,
                                                            const void *__restrict__ x, void *__restrict__ y,
                                                            R sigma) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    wilson_clover_site<R, Rin, MODE>(g, U, clov, x, y, sigma, s);
}

// nrhs fields stored back to back (field k at byte offset k * field_bytes).  CTA b
// takes field b % nrhs on the site range b / nrhs: the nrhs CTAs of one site range
// are scheduled back to back, so the range's links and clover come from HBM once
// and from L2 for the other nrhs - 1 fields.
template <typename R, int MODE>
__global__ void __launch_bounds__(128) wilson_clover_nrhs_kernel(Geom g, const void *__restrict__ U,
                                                                 const void *__restrict__ clov,
                                                                 const char *__restrict__ x, char *__restrict__ y,
                                                                 R sigma, int nrhs, size_t field_bytes) {
    const int rhs = blockIdx.x % nrhs;
    const int s = (blockIdx.x / nrhs) * blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    wilson_clover_site<R, R, MODE>(g, U, clov, x + rhs * field_bytes, y + rhs * field_bytes, sigma, s);
}

// FP32, several fields per launch: a CTA of NR_SITES consecutive sites copies
// its sites' forward links (two rows, 12 float4 planes) and clover (18 planes)
// into shared memory once, with coalesced loads, and applies the stencil to
// every field from there; only the spinors (and the backward links of hops that
// leave the CTA) stream from memory for each field.
constexpr int NR_SITES = 128;
constexpr size_t NR_SMEM = (size_t)(12 + 18) * NR_SITES * sizeof(float4);

template <int MODE>
__global__ void __launch_bounds__(NR_SITES, 3) wilson_clover_nrhs_staged_kernel(
    Geom g, const float4 *__restrict__ U, const float4 *__restrict__ clov, const char *__restrict__ x,
    char *__restrict__ y, float sigma, int nrhs, size_t field_bytes) {
    extern __shared__ float4 nr_smem[];
    float4 *sU = nr_smem, *sC = nr_smem + 12 * NR_SITES;
    const int s0 = blockIdx.x * NR_SITES;
    const int n = min(NR_SITES, g.V - s0);
    const int t = threadIdx.x;
    if (t < n) {
#pragma unroll
        for (int q = 0; q < 12; ++q) sU[q * NR_SITES + t] = U[(size_t)q * g.V + s0 + t];
#pragma unroll
        for (int q = 0; q < 18; ++q) sC[q * NR_SITES + t] = clov[(size_t)q * g.V + s0 + t];
    }
    __syncthreads();
    if (t >= n) return;
    const StagedFields f{sU, sC, U, s0, n, NR_SITES, g.V};
#pragma unroll 1
    for (int r = 0; r < nrhs; ++r) {
        // re-read the staged links and clover for every field instead of holding
        // all of them in registers across fields (168 of them: occupancy)
        asm volatile("" ::: "memory");
        wilson_clover_site_f<float, float, MODE>(g, f, x + r * field_bytes, y + r * field_bytes, sigma, s0 + t);
    }
}

template <typename R, typename Rin>
static void launch_fine(Ctx &c, int mode, double sigma, const void *x, void *y) {
    const int threads = 128;
    const int blocks = grid_for(c.g.V, threads);
    const void *U = sizeof(R) == 8 ? c.U64.p : c.U32.p;
    const void *C = sizeof(R) == 8 ? c.clov64.p : c.clov32.p;
    // algorithmic bytes per site, every field counted once: x, y, links, clover
    const double spin = 12 * 2 * sizeof(Rin), spout = 12 * 2 * sizeof(R);
    const double links = sizeof(R) == 8 ? 4 * 9 * 16 : 4 * 12 * 4;
    const double clov = 72 * sizeof(R);
    TimeScope ts(c.timer, sizeof(R) == 8 ? K_STENCIL_F64 : K_STENCIL_F32, (spin + spout + links + clov) * c.g.V);
    c.st.fine_applies += 1;
    switch (mode) {
        case MODE_D: wilson_clover_kernel<R, Rin, MODE_D><<<blocks, threads, 0, c.stream>>>(c.g, U, C, x, y, (R)sigma); break;
        case MODE_DSIGMA: wilson_clover_kernel<R, Rin, MODE_DSIGMA><<<blocks, threads, 0, c.stream>>>(c.g, U, C, x, y, (R)sigma); break;
        default: wilson_clover_kernel<R, Rin, MODE_QSIGMA><<<blocks, threads, 0, c.stream>>>(c.g, U, C, x, y, (R)sigma); break;
    }
    MG_CHECK_LAUNCH();
}

// double-float copies of the FP64 links and clover: (h, l) = (fl(d), fl(d - h))
// for every double, a float2 at the double's index
__global__ void ds_copy_kernel(size_t n, const double *__restrict__ in, float2 *__restrict__ out) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const double d = in[i];
        const float h = __double2float_rn(d);
        out[i] = make_float2(h, __double2float_rn(d - (double)h));
    }
}

static void ensure_ds_fields(Ctx &c) {
    if (c.ds_fields_valid) return;
    const size_t nu = (size_t)c.g.V * 4 * 9 * 2, nc = (size_t)c.g.V * 36 * 2;   // doubles
    if (!c.Uds.p) c.Uds.alloc(nu * sizeof(float2));
    if (!c.clovds.p) c.clovds.alloc(nc * sizeof(float2));
    TimeScope ts(c.timer, K_OTHER, 0);
    ds_copy_kernel<<<152 * 8, 256, 0, c.stream>>>(nu, c.U64.as<double>(), c.Uds.as<float2>());
    MG_CHECK_LAUNCH();
    ds_copy_kernel<<<152 * 8, 256, 0, c.stream>>>(nc, c.clov64.as<double>(), c.clovds.as<float2>());
    MG_CHECK_LAUNCH();
    c.ds_fields_valid = true;
}

// the FP64-output stencil in double-float arithmetic: FP64 (Rin = dsf) or FP32
// (Rin = float) input, FP64 output, links and clover from the double-float copies
template <typename Rin>
static void launch_fine_ds(Ctx &c, int mode, double sigma, const void *x, void *y) {
    ensure_ds_fields(c);
    const int threads = 128;
    const int blocks = grid_for(c.g.V, threads);
    const void *U = c.Uds.p, *C = c.clovds.p;
    const double spin = 12 * 2 * (sizeof(Rin) == 4 ? 4 : 8), spout = 12 * 2 * 8;
    TimeScope ts(c.timer, K_STENCIL_F64, (spin + spout + 4 * 9 * 16 + 72 * 8) * c.g.V);
    c.st.fine_applies += 1;
    const dsf sg(sigma);
    switch (mode) {
        case MODE_D: wilson_clover_kernel<dsf, Rin, MODE_D><<<blocks, threads, 0, c.stream>>>(c.g, U, C, x, y, sg); break;
        case MODE_DSIGMA: wilson_clover_kernel<dsf, Rin, MODE_DSIGMA><<<blocks, threads, 0, c.stream>>>(c.g, U, C, x, y, sg); break;
        default: wilson_clover_kernel<dsf, Rin, MODE_QSIGMA><<<blocks, threads, 0, c.stream>>>(c.g, U, C, x, y, sg); break;
    }
    MG_CHECK_LAUNCH();
}

template <typename R>
void apply_fine_nrhs(Ctx &c, int mode, double sigma, const void *x, void *y, int nrhs) {
    const int threads = 128;
    const long long blocks = (long long)grid_for(c.g.V, threads) * nrhs;
    MG_REQUIRE(nrhs >= 1 && blocks < (1LL << 31), MGEIG_EINVAL);
    const void *U = sizeof(R) == 8 ? c.U64.p : c.U32.p;
    const void *C = sizeof(R) == 8 ? c.clov64.p : c.clov32.p;
    const size_t fb = (size_t)c.g.V * 24 * sizeof(R);
    const double links = sizeof(R) == 8 ? 4 * 9 * 16 : 4 * 12 * 4;
    // algorithmic bytes: every field read or written once, links and clover once for all fields
    TimeScope ts(c.timer, sizeof(R) == 8 ? K_STENCIL_F64 : K_STENCIL_F32,
                 ((double)nrhs * 2 * 24 * sizeof(R) + links + 72 * sizeof(R)) * c.g.V);
    c.st.fine_applies += nrhs;
    const char *xb = static_cast<const char *>(x);
    char *yb = static_cast<char *>(y);
    if (sizeof(R) == 4 && nrhs > 1) {
        const int nb = grid_for(c.g.V, NR_SITES);
        const float4 *U4 = c.U32.as<float4>(), *C4 = c.clov32.as<float4>();
        const float sg = (float)sigma;
        switch (mode) {
            case MODE_D:
                MG_CUDA(cudaFuncSetAttribute(wilson_clover_nrhs_staged_kernel<MODE_D>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)NR_SMEM));
                wilson_clover_nrhs_staged_kernel<MODE_D><<<nb, NR_SITES, NR_SMEM, c.stream>>>(c.g, U4, C4, xb, yb, sg, nrhs, fb);
                break;
            case MODE_DSIGMA:
                MG_CUDA(cudaFuncSetAttribute(wilson_clover_nrhs_staged_kernel<MODE_DSIGMA>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)NR_SMEM));
                wilson_clover_nrhs_staged_kernel<MODE_DSIGMA><<<nb, NR_SITES, NR_SMEM, c.stream>>>(c.g, U4, C4, xb, yb, sg, nrhs, fb);
                break;
            default:
                MG_CUDA(cudaFuncSetAttribute(wilson_clover_nrhs_staged_kernel<MODE_QSIGMA>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)NR_SMEM));
                wilson_clover_nrhs_staged_kernel<MODE_QSIGMA><<<nb, NR_SITES, NR_SMEM, c.stream>>>(c.g, U4, C4, xb, yb, sg, nrhs, fb);
                break;
        }
        MG_CHECK_LAUNCH();
        return;
    }
    switch (mode) {
        case MODE_D: wilson_clover_nrhs_kernel<R, MODE_D><<<(int)blocks, threads, 0, c.stream>>>(c.g, U, C, xb, yb, (R)sigma, nrhs, fb); break;
        case MODE_DSIGMA: wilson_clover_nrhs_kernel<R, MODE_DSIGMA><<<(int)blocks, threads, 0, c.stream>>>(c.g, U, C, xb, yb, (R)sigma, nrhs, fb); break;
        default: wilson_clover_nrhs_kernel<R, MODE_QSIGMA><<<(int)blocks, threads, 0, c.stream>>>(c.g, U, C, xb, yb, (R)sigma, nrhs, fb); break;
    }
    MG_CHECK_LAUNCH();
}
template void apply_fine_nrhs<double>(Ctx &, int, double, const void *, void *, int);
template void apply_fine_nrhs<float>(Ctx &, int, double, const void *, void *, int);

// the solver's stencil: FP64 output in double-float arithmetic when the context
// asks for it (mixed precision), else in R
template <typename R>
void apply_fine(Ctx &c, int mode, double sigma, const void *x, void *y) {
    if (sizeof(R) == 8 && c.ds_stencil()) launch_fine_ds<dsf>(c, mode, sigma, x, y);
    else launch_fine<R, R>(c, mode, sigma, x, y);
}
template void apply_fine<double>(Ctx &, int, double, const void *, void *);
template void apply_fine<float>(Ctx &, int, double, const void *, void *);

// double-float arithmetic whatever the context asks (the ABI's double-float apply)
void apply_fine_ds(Ctx &c, int mode, double sigma, const void *x, void *y, bool x_fp32) {
    if (x_fp32) launch_fine_ds<float>(c, mode, sigma, x, y);
    else launch_fine_ds<dsf>(c, mode, sigma, x, y);
}

// always FP64 arithmetic (the ABI's FP64 apply, the final eigen-residual check)
void apply_fine_fp64(Ctx &c, int mode, double sigma, const void *x, void *y) {
    launch_fine<double, double>(c, mode, sigma, x, y);
}

void apply_fine_f64_from_f32(Ctx &c, int mode, double sigma, const void *x32, void *y64) {
    if (c.ds_stencil()) launch_fine_ds<float>(c, mode, sigma, x32, y64);
    else launch_fine<double, float>(c, mode, sigma, x32, y64);
}

// ---------------------------------------------------------------------------
// layout conversions

__global__ void pack_spinor_kernel(int V, int n, const double2 *__restrict__ in, double2 *__restrict__ out) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)V * n) return;
    int f = (int)(i / V), s = (int)(i % V);
    const double2 *src = in + ((size_t)f * V + s) * 12;
    double2 *dst = out + (size_t)f * 12 * V;
#pragma unroll
    for (int k = 0; k < 12; ++k) dst[(size_t)k * V + s] = src[k];
}

__global__ void unpack_spinor_kernel(int V, int n, const double2 *__restrict__ in, double2 *__restrict__ out) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)V * n) return;
    int f = (int)(i / V), s = (int)(i % V);
    const double2 *src = in + (size_t)f * 12 * V;
    double2 *dst = out + ((size_t)f * V + s) * 12;
#pragma unroll
    for (int k = 0; k < 12; ++k) dst[k] = src[(size_t)k * V + s];
}

void pack_spinor_f64(Ctx &c, const double *in, void *out, int n) {
    size_t tot = (size_t)c.g.V * n;
    pack_spinor_kernel<<<grid_for(tot, 256), 256, 0, c.stream>>>(c.g.V, n, reinterpret_cast<const double2 *>(in),
                                                                 static_cast<double2 *>(out));
    MG_CHECK_LAUNCH();
}

void unpack_spinor_f64(Ctx &c, const void *in, double *out, int n) {
    size_t tot = (size_t)c.g.V * n;
    unpack_spinor_kernel<<<grid_for(tot, 256), 256, 0, c.stream>>>(c.g.V, n, static_cast<const double2 *>(in),
                                                                   reinterpret_cast<double2 *>(out));
    MG_CHECK_LAUNCH();
}

// fine spinor FP64 [12][V] <-> FP32 [6][V] float4 (site based); for the
// coarse / flat arrays the same kernels run with V = n/12 only when the layout
// is the fine one, so the flat variants below are used elsewhere.
__global__ void f64_to_f32_fine(int V, const double2 *__restrict__ in, float4 *__restrict__ out) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        double2 a = in[(size_t)(2 * q) * V + s], b = in[(size_t)(2 * q + 1) * V + s];
        out[(size_t)q * V + s] = make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
    }
}

__global__ void f32_to_f64_fine(int V, const float4 *__restrict__ in, double2 *__restrict__ out) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= V) return;
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        float4 a = in[(size_t)q * V + s];
        out[(size_t)(2 * q) * V + s] = make_double2(a.x, a.y);
        out[(size_t)(2 * q + 1) * V + s] = make_double2(a.z, a.w);
    }
}

void convert_f64_to_f32(Ctx &c, const void *in64, void *out32, size_t ncomplex) {
    const int V = (int)(ncomplex / 12);
    TimeScope ts(c.timer, K_BLAS_LOW, ncomplex * 24.0);
    f64_to_f32_fine<<<grid_for(V, 256), 256, 0, c.stream>>>(V, static_cast<const double2 *>(in64), static_cast<float4 *>(out32));
    MG_CHECK_LAUNCH();
}

void convert_f32_to_f64(Ctx &c, const void *in32, void *out64, size_t ncomplex) {
    const int V = (int)(ncomplex / 12);
    TimeScope ts(c.timer, K_BLAS_LOW, ncomplex * 24.0);
    f32_to_f64_fine<<<grid_for(V, 256), 256, 0, c.stream>>>(V, static_cast<const float4 *>(in32), static_cast<double2 *>(out64));
    MG_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------
// random test vectors: Philox4x32-10 (Salmon et al., SC'11), uniforms int32(w) * 2^-31

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t hi0 = __umulhi(M0, c[0]), lo0 = M0 * c[0];
        uint32_t hi1 = __umulhi(M1, c[2]), lo1 = M1 * c[2];
        uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
        k0 += W0; k1 += W1;
    }
}

__global__ void random_spinor_kernel(int V, int n, uint32_t k0, uint32_t k1, uint32_t tag, double2 *__restrict__ out) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)V * n * 6) return;
    const int q = (int)(i % 6);
    const int s = (int)((i / 6) % V);
    const int j = (int)(i / ((size_t)6 * V));
    uint32_t ctr[4] = {(uint32_t)s, (uint32_t)q, (uint32_t)j, tag};
    philox4x32_10(ctr, k0, k1);
    const double sc = 1.0 / 2147483648.0;
    double2 *o = out + (size_t)j * 12 * V;
    o[(size_t)(2 * q) * V + s] = make_double2((double)(int32_t)ctr[0] * sc, (double)(int32_t)ctr[1] * sc);
    o[(size_t)(2 * q + 1) * V + s] = make_double2((double)(int32_t)ctr[2] * sc, (double)(int32_t)ctr[3] * sc);
}

void random_spinors(Ctx &c, uint64_t seed, void *out64, int n, uint32_t tag) {
    size_t tot = (size_t)c.g.V * n * 6;
    random_spinor_kernel<<<grid_for(tot, 256), 256, 0, c.stream>>>(c.g.V, n, (uint32_t)(seed & 0xFFFFFFFFu),
                                                                   (uint32_t)(seed >> 32), tag, static_cast<double2 *>(out64));
    MG_CHECK_LAUNCH();
}

}  // namespace mgeig
