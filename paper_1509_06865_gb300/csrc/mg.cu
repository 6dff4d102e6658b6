// Two-grid kernels (Sec. 2 of arXiv:1509.06865, Eqs. 2.3-2.6):
//   build_interp   aggregation interpolation P (Eq. 2.4): per aggregate and
//                  chirality, Gram-Schmidt (twice) of the N_tv test vectors, FP64
//   restrict_vec   r_c = P^dag r          (one CTA per aggregate)
//   prolong_vec    e = P e_c              (one thread per fine site)
//   build_coarse   D_c = P^dag D P as nine per-direction blocks (Eq. 2.5)
//   coarse_apply   y = gamma5^c D_c x - sigma x = (Q_c - sigma) x (Eq. 2.6)
//   sap_sweep      one colour of the Schwarz alternating procedure on
//                  D_sigma = D - sigma gamma5: block-local minimal residual with
//                  Dirichlet block boundaries, block vector staged in shared memory
//
// P is stored as N_tv fine spinors in the internal spinor layout (column (a, c, j)
// of P = spinor j restricted to aggregate a and chirality c).  Coarse vectors are
// [coarse site][c][j] complex; coarse blocks are column-major:
// Dc[d][a][col][row], d = 0 self, 1 + 2 mu = +mu, 2 + 2 mu = -mu.
#include "internal.h"

namespace mgeig {

struct AggGeom {
    int agg[4];     // aggregate (or SAP block) extent
    int cdims[4];   // number of aggregates per direction
    int vol;        // sites per aggregate
    int n;          // number of aggregates
};

static AggGeom make_agg(const Ctx &c, const int *blk) {
    AggGeom a;
    a.vol = 1;
    a.n = 1;
    for (int mu = 0; mu < 4; ++mu) {
        a.agg[mu] = blk[mu];
        a.cdims[mu] = c.dims[mu] / blk[mu];
        a.vol *= blk[mu];
        a.n *= a.cdims[mu];
    }
    return a;
}

// fine site of local site l in aggregate a; local coords in lc
__device__ __forceinline__ int agg_site(const Geom &g, const AggGeom &A, int a, int l, int lc[4]) {
    int ac[4];
    ac[0] = a % A.cdims[0]; a /= A.cdims[0];
    ac[1] = a % A.cdims[1]; a /= A.cdims[1];
    ac[2] = a % A.cdims[2];
    ac[3] = a / A.cdims[2];
    lc[0] = l % A.agg[0]; l /= A.agg[0];
    lc[1] = l % A.agg[1]; l /= A.agg[1];
    lc[2] = l % A.agg[2];
    lc[3] = l / A.agg[2];
    int s = 0;
    for (int mu = 3; mu >= 0; --mu) s = s * g.L[mu] + ac[mu] * A.agg[mu] + lc[mu];
    return s;
}

__device__ __forceinline__ int agg_of_site(const Geom &g, const AggGeom &A, const int c[4]) {
    int a = 0;
    for (int mu = 3; mu >= 0; --mu) a = a * A.cdims[mu] + c[mu] / A.agg[mu];
    return a;
}

struct PtrList { const void *p[24]; };
struct MutPtrList { void *p[24]; };

// ---------------------------------------------------------------------------
// interpolation: classical Gram-Schmidt (twice) per (aggregate, chirality),
// arithmetic in precision R (FP64 for the all-FP64 path; FP32 for the mixed
// path, whose P is stored in FP32).  Test vectors are read in FP64.  One CTA per
// (aggregate, chirality); all <q_i, w> of one pass share one block reduction.

constexpr int PB_THREADS = 256;
constexpr int PB_MAXS = 4;    // sites per thread (aggregates of up to 1024 sites)
constexpr int PB_MAXN = 24;   // test vectors

// Block Gram-Schmidt of the test vectors on one aggregate and chirality, two
// passes per vector.  Sums run in the level precision R: in the mixed path the
// FP64 warp reductions of an earlier form (1/64 of the FP32 rate here) took
// half of the kernel's time, and P is stored in FP32 anyway.
template <typename R>
__global__ void __launch_bounds__(PB_THREADS) interp_kernel(Geom g, AggGeom A, PtrList W, int ntv, MutPtrList P) {
    __shared__ R sh[PB_THREADS / 32][2 * PB_MAXN];
    __shared__ R hs[2 * PB_MAXN];
    const int a = blockIdx.x >> 1, chir = blockIdx.x & 1;
    const int V = g.V;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    int sites[PB_MAXS];
    int ns = 0;
    for (int l = threadIdx.x; l < A.vol && ns < PB_MAXS; l += blockDim.x) {
        int lc[4];
        sites[ns++] = agg_site(g, A, a, l, lc);
    }
    // block-reduce cnt complex values parked per warp in sh -> hs (all threads)
    auto reduce = [&](int cnt) {
        __syncthreads();
        for (int i = threadIdx.x; i < 2 * cnt; i += blockDim.x) {
            R s = 0;
            for (int w = 0; w < nw; ++w) s += sh[w][i];
            hs[i] = s;
        }
        __syncthreads();
    };
    auto warp_sum = [&](R v) {
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        return v;
    };
    for (int j = 0; j < ntv; ++j) {
        cpx<R> w[PB_MAXS][6];
        const double2 *src = static_cast<const double2 *>(W.p[j]);
        for (int i = 0; i < PB_MAXS; ++i)
            for (int k = 0; k < 6; ++k) {
                if (i < ns) { double2 t = src[(size_t)(chir * 6 + k) * V + sites[i]]; w[i][k] = cpx<R>((R)t.x, (R)t.y); }
                else w[i][k] = cpx<R>();
            }
        for (int pass = 0; pass < 2 && j > 0; ++pass) {
#pragma unroll 4
            for (int q = 0; q < j; ++q) {
                const cpx<R> *pq = static_cast<const cpx<R> *>(P.p[q]);
                cpx<R> d;
                for (int i = 0; i < ns; ++i)
                    for (int k = 0; k < 6; ++k) cmac_conj(d, Spinor<R>::comp(pq, V, chir * 6 + k, sites[i]), w[i][k]);
                const R re = warp_sum(d.re), im = warp_sum(d.im);
                if (lane == 0) { sh[wp][2 * q] = re; sh[wp][2 * q + 1] = im; }
            }
            reduce(j);
            for (int q = 0; q < j; ++q) {
                const cpx<R> *pq = static_cast<const cpx<R> *>(P.p[q]);
                const cpx<R> hc((R)hs[2 * q], (R)hs[2 * q + 1]);
                for (int i = 0; i < ns; ++i)
                    for (int k = 0; k < 6; ++k) w[i][k] = w[i][k] - hc * Spinor<R>::comp(pq, V, chir * 6 + k, sites[i]);
            }
        }
        R nn = 0;
        for (int i = 0; i < ns; ++i)
            for (int k = 0; k < 6; ++k) nn += w[i][k].re * w[i][k].re + w[i][k].im * w[i][k].im;
        nn = warp_sum(nn);
        if (lane == 0) { sh[wp][0] = nn; sh[wp][1] = 0; }
        reduce(1);
        const R inv = hs[0] > 0 ? R(1) / sqrt(hs[0]) : R(0);
        cpx<R> *dst = static_cast<cpx<R> *>(P.p[j]);
        for (int i = 0; i < ns; ++i)
            for (int k = 0; k < 6; ++k) Spinor<R>::comp(dst, V, chir * 6 + k, sites[i]) = inv * w[i][k];
    }
}

// P (ntv spinors of precision R) from the FP64 test vectors W64
template <typename R>
void build_interp(Ctx &c, const void *const *W64, int ntv, void *const *P) {
    AggGeom A = make_agg(c, c.prm.agg);
    MG_REQUIRE(A.vol <= PB_THREADS * PB_MAXS && ntv <= PB_MAXN, MGEIG_EINVAL);
    PtrList w{};
    MutPtrList p{};
    for (int j = 0; j < ntv; ++j) { w.p[j] = W64[j]; p.p[j] = P[j]; }
    const int threads = A.vol < PB_THREADS ? ((A.vol + 31) / 32) * 32 : PB_THREADS;
    TimeScope ts(c.timer, K_PBUILD, (double)ntv * c.g.V * 12 * (16 + 2 * sizeof(R)));
    interp_kernel<R><<<A.n * 2, threads, 0, c.stream>>>(c.g, A, w, ntv, p);
    MG_CHECK_LAUNCH();
}
template void build_interp<double>(Ctx &, const void *const *, int, void *const *);
template void build_interp<float>(Ctx &, const void *const *, int, void *const *);

// ---------------------------------------------------------------------------
// restriction r_c = P^dag r

template <typename R>
__global__ void restrict_kernel(Geom g, AggGeom A, PtrList P, int ntv, const void *__restrict__ r,
                                cpx<R> *__restrict__ rc) {
    extern __shared__ unsigned char smem_raw[];
    R *sh = reinterpret_cast<R *>(smem_raw);   // [nwarps][2*ntv][2]
    const int a = blockIdx.x;
    const int V = g.V;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int n2 = 2 * ntv;
    // one site per thread (aggregates of at most blockDim sites, the usual case):
    // r is loaded once and kept in registers for all test vectors; otherwise each
    // thread visits its sites once per j
    const bool one = A.vol <= (int)blockDim.x;
    int s1 = -1;
    cpx<R> x1[12];
    if (one && (int)threadIdx.x < A.vol) {
        int lc[4];
        s1 = agg_site(g, A, a, threadIdx.x, lc);
        Spinor<R>::load(r, V, s1, x1);
    }
#pragma unroll 2
    for (int j = 0; j < ntv; ++j) {
        cpx<R> d0, d1;
        if (one) {
            if (s1 >= 0) {
                cpx<R> p[12];
                Spinor<R>::load(P.p[j], V, s1, p);
#pragma unroll
                for (int k = 0; k < 6; ++k) { cmac_conj(d0, p[k], x1[k]); cmac_conj(d1, p[6 + k], x1[6 + k]); }
            }
        } else {
            for (int l = threadIdx.x; l < A.vol; l += blockDim.x) {
                int lc[4];
                const int s = agg_site(g, A, a, l, lc);
                cpx<R> x[12], p[12];
                Spinor<R>::load(r, V, s, x);
                Spinor<R>::load(P.p[j], V, s, p);
#pragma unroll
                for (int k = 0; k < 6; ++k) { cmac_conj(d0, p[k], x[k]); cmac_conj(d1, p[6 + k], x[6 + k]); }
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            d0.re += __shfl_xor_sync(0xffffffffu, d0.re, o); d0.im += __shfl_xor_sync(0xffffffffu, d0.im, o);
            d1.re += __shfl_xor_sync(0xffffffffu, d1.re, o); d1.im += __shfl_xor_sync(0xffffffffu, d1.im, o);
        }
        if (lane == 0) {
            sh[(w * n2 + j) * 2] = d0.re; sh[(w * n2 + j) * 2 + 1] = d0.im;
            sh[(w * n2 + ntv + j) * 2] = d1.re; sh[(w * n2 + ntv + j) * 2 + 1] = d1.im;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n2; i += blockDim.x) {
        cpx<R> t;
        for (int q = 0; q < nw; ++q) { t.re += sh[(q * n2 + i) * 2]; t.im += sh[(q * n2 + i) * 2 + 1]; }
        rc[(size_t)a * n2 + i] = t;
    }
}

static int agg_threads(int vol) {
    if (vol >= 256) return 256;
    return ((vol + 31) / 32) * 32;
}

template <typename R>
void restrict_vec(Ctx &c, const void *const *P, const void *r, void *rc) {
    AggGeom A = make_agg(c, c.prm.agg);
    const int ntv = c.prm.n_tv;
    PtrList p{};
    for (int j = 0; j < ntv; ++j) p.p[j] = P[j];
    const int threads = agg_threads(A.vol);
    const size_t smem = (size_t)(threads / 32) * 2 * ntv * 2 * sizeof(R);
    TimeScope ts(c.timer, K_RESTRICT, (double)(ntv + 1) * c.g.V * 24 * sizeof(R));
    restrict_kernel<R><<<A.n, threads, smem, c.stream>>>(c.g, A, p, ntv, r, static_cast<cpx<R> *>(rc));
    MG_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------
// prolongation e = P e_c

template <typename R>
__global__ void prolong_kernel(Geom g, AggGeom A, PtrList P, int ntv, const cpx<R> *__restrict__ ec, void *__restrict__ e) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= g.V) return;
    const int V = g.V;
    int c[4];
    site_coords(g, s, c);
    const int a = agg_of_site(g, A, c);
    const cpx<R> *ea = ec + (size_t)a * 2 * ntv;
    cpx<R> out[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) out[k] = cpx<R>();
    for (int j = 0; j < ntv; ++j) {
        cpx<R> p[12];
        Spinor<R>::load(P.p[j], V, s, p);
        const cpx<R> e0 = ea[j], e1 = ea[ntv + j];
#pragma unroll
        for (int k = 0; k < 6; ++k) { cmac(out[k], p[k], e0); cmac(out[6 + k], p[6 + k], e1); }
    }
    Spinor<R>::store(e, V, s, out);
}

template <typename R>
void prolong_vec(Ctx &c, const void *const *P, const void *ec, void *e) {
    AggGeom A = make_agg(c, c.prm.agg);
    const int ntv = c.prm.n_tv;
    PtrList p{};
    for (int j = 0; j < ntv; ++j) p.p[j] = P[j];
    TimeScope ts(c.timer, K_PROLONG, (double)(ntv + 1) * c.g.V * 24 * sizeof(R));
    prolong_kernel<R><<<grid_for(c.g.V, 128), 128, 0, c.stream>>>(c.g, A, p, ntv, static_cast<const cpx<R> *>(ec), e);
    MG_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------
// coarse operator build: one CTA per (aggregate, direction)

constexpr int CB_THREADS = 256;
constexpr int CB_CHUNK = 8;   // fine sites staged per step
constexpr int CB_MAXO = 9;    // outputs per thread: (2*24)^2 / 256

// keeps chirality cp of a spinor (components 6 cp .. 6 cp + 5) and zeroes the
// other, with compile-time indices only
template <typename R>
__device__ __forceinline__ void zero_other_chirality(cpx<R> psi[12], int cp) {
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        if (cp == 0) psi[6 + k] = cpx<R>();
        else psi[k] = cpx<R>();
    }
}

// directional fine operator applied to column (cp, jp) of P at fine site s:
// d = 0: local term + hops that stay inside the aggregate; d = 1 + 2mu / 2 + 2mu:
// the single hop leaving the aggregate through its upper / lower mu face.
template <typename R>
__device__ void directional_column(const Geom &g, const AggGeom &A, const void *U, const void *clov, const void *Pj,
                                   int cp, int d, int s, const int c[4], cpx<R> out[12]) {
    const int V = g.V;
    cpx<R> up[6], lo[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) { up[k] = cpx<R>(); lo[k] = cpx<R>(); }
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
#pragma unroll
        for (int f = 0; f < 2; ++f) {
            const bool fwd = f == 0;
            const int lm = c[mu] % A.agg[mu];
            const bool leaves = fwd ? (lm == A.agg[mu] - 1) : (lm == 0);
            const int want = fwd ? 1 + 2 * mu : 2 + 2 * mu;
            if (d == 0 ? leaves : (d != want)) continue;
            int ph;
            const int n = neighbor(g, s, c, mu, fwd, &ph);
            cpx<R> u[9], psi[12];
            Gauge<R>::load(U, V, mu, fwd ? s : n, u);
            Spinor<R>::load(Pj, V, n, psi);
            zero_other_chirality(psi, cp);
            hop_accumulate<R>(mu, fwd, u, psi, (R)ph, up, lo);
        }
    }
    const R half = R(0.5);
    if (d == 0) {
        cpx<R> psi[12];
        Spinor<R>::load(Pj, V, s, psi);
        zero_other_chirality(psi, cp);
        clover_apply<R>(clov, V, s, psi, out);
    } else {
#pragma unroll
        for (int k = 0; k < 12; ++k) out[k] = cpx<R>();
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) { out[k] = out[k] - half * up[k]; out[6 + k] = out[6 + k] - half * lo[k]; }
}

template <typename R>
__global__ void __launch_bounds__(CB_THREADS) coarse_build_kernel(Geom g, AggGeom A, const void *__restrict__ U,
                                                                  const void *__restrict__ clov, PtrList P, int ntv,
                                                                  cpx<R> *__restrict__ Dc) {
    extern __shared__ unsigned char smem_raw[];
    const int a = blockIdx.x / 9, d = blockIdx.x % 9;
    const int n2 = 2 * ntv;
    // component-major within a staged site ([CHUNK][12][ntv]): the threads of a warp
    // take consecutive rows, i.e. consecutive test vectors, so their reads of sP are
    // consecutive words (a [CHUNK][ntv][12] layout had 4-way bank conflicts)
    cpx<R> *sP = reinterpret_cast<cpx<R> *>(smem_raw);           // [CHUNK][12][ntv]
    cpx<R> *sH = sP + (size_t)CB_CHUNK * ntv * 12;               // [CHUNK][n2][12]
    const int V = g.V;
    // sites of this direction: all sites (d = 0) or the face l_mu = agg-1 / 0
    const int mu = d == 0 ? -1 : (d - 1) / 2;
    const int nsite = d == 0 ? A.vol : A.vol / A.agg[mu];
    cpx<R> acc[CB_MAXO];
#pragma unroll
    for (int q = 0; q < CB_MAXO; ++q) acc[q] = cpx<R>();
    for (int base = 0; base < nsite; base += CB_CHUNK) {
        const int cnt = nsite - base < CB_CHUNK ? nsite - base : CB_CHUNK;
        // stage P(x) rows and H(x) columns
        for (int t = threadIdx.x; t < cnt * (ntv + n2); t += blockDim.x) {
            const int sl = t % cnt, item = t / cnt;
            // face site enumeration: local index over the face, expanded to the aggregate
            int l = base + sl;
            if (d != 0) {
                // local coordinates with l_mu fixed (no run-time indexed arrays)
                int rem = l, ln = 0, st = 1;
#pragma unroll
                for (int nu = 0; nu < 4; ++nu) {
                    int x;
                    if (nu == mu) {
                        x = (d & 1) ? A.agg[nu] - 1 : 0;
                    } else {
                        x = rem % A.agg[nu];
                        rem /= A.agg[nu];
                    }
                    ln += x * st;
                    st *= A.agg[nu];
                }
                l = ln;
            }
            int lc[4], c[4];
            const int s = agg_site(g, A, a, l, lc);
            site_coords(g, s, c);
            cpx<R> v[12];
            if (item < ntv) {
                Spinor<R>::load(P.p[item], V, s, v);
                for (int k = 0; k < 12; ++k) sP[((size_t)sl * 12 + k) * ntv + item] = v[k];
            } else {
                const int col = item - ntv, cp = col / ntv, jp = col % ntv;
                directional_column<R>(g, A, U, clov, P.p[jp], cp, d, s, c, v);
                for (int k = 0; k < 12; ++k) sH[((size_t)sl * n2 + col) * 12 + k] = v[k];
            }
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < CB_MAXO; ++q) {
            const int o = threadIdx.x + q * blockDim.x;
            if (o < n2 * n2) {
                const int row = o % n2, col = o / n2;
                const int cr = row / ntv, jr = row % ntv;
                cpx<R> t = acc[q];
                for (int sl = 0; sl < cnt; ++sl) {
                    const cpx<R> *pr = sP + ((size_t)sl * 12 + cr * 6) * ntv + jr;   // component k at pr[k * ntv]
                    const cpx<R> *hc = sH + ((size_t)sl * n2 + col) * 12 + cr * 6;
#pragma unroll
                    for (int k = 0; k < 6; ++k) cmac_conj(t, pr[(size_t)k * ntv], hc[k]);
                }
                acc[q] = t;
            }
        }
        __syncthreads();
    }
    cpx<R> *out = Dc + ((size_t)d * A.n + a) * n2 * n2;
#pragma unroll
    for (int q = 0; q < CB_MAXO; ++q) {
        const int o = threadIdx.x + q * blockDim.x;
        if (o < n2 * n2) out[o] = acc[q];   // o = col*n2 + row: column-major block
    }
}

template <typename R>
void build_coarse(Ctx &c, const void *const *P, void *Dc) {
    AggGeom A = make_agg(c, c.prm.agg);
    const int ntv = c.prm.n_tv;
    MG_REQUIRE(4 * ntv * ntv <= CB_THREADS * CB_MAXO, MGEIG_EINVAL);
    PtrList p{};
    for (int j = 0; j < ntv; ++j) p.p[j] = P[j];
    const size_t smem = (size_t)CB_CHUNK * (ntv + 2 * ntv) * 12 * sizeof(cpx<R>);
    MG_CUDA(cudaFuncSetAttribute(coarse_build_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const void *U = sizeof(R) == 8 ? c.U64.p : c.U32.p;
    const void *C = sizeof(R) == 8 ? c.clov64.p : c.clov32.p;
    TimeScope ts(c.timer, K_COARSE_BUILD, (double)ntv * c.g.V * 24 * sizeof(R) * 2);
    coarse_build_kernel<R><<<A.n * 9, CB_THREADS, smem, c.stream>>>(c.g, A, U, C, p, ntv, static_cast<cpx<R> *>(Dc));
    MG_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------
// coarse apply: thread per (coarse site, row)

// dform = 0: y = (gamma5^c D_c - sigma) x = (Q_c - sigma) x
// dform = 1: y = (D_c - sigma gamma5^c) x = gamma5^c (Q_c - sigma) x
template <typename R>
__global__ void coarse_apply_kernel(AggGeom A, int ntv, const cpx<R> *__restrict__ Dc, const int *__restrict__ nbr,
                                    R sigma, const cpx<R> *__restrict__ x, cpx<R> *__restrict__ y, int dform) {
    const int n2 = 2 * ntv;
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)A.n * n2) return;
    const int a = (int)(t / n2), row = (int)(t % n2);
    cpx<R> acc;
    for (int d = 0; d < 9; ++d) {
        const int b = __ldg(nbr + (size_t)d * A.n + a);   // neighbour aggregate in direction d
        const cpx<R> *blk = Dc + ((size_t)d * A.n + a) * n2 * n2 + row;
        const cpx<R> *xb = x + (size_t)b * n2;
        for (int j = 0; j < n2; ++j) cmac(acc, blk[(size_t)j * n2], xb[j]);
    }
    if (dform) {
        y[t] = acc - (row >= ntv ? -sigma : sigma) * x[t];
    } else {
        if (row >= ntv) acc = -acc;
        y[t] = acc - sigma * x[t];
    }
}

// y = gamma5^c x on coarse vectors
template <typename R>
__global__ void coarse_gamma5_kernel(size_t n, int ntv, const cpx<R> *__restrict__ x, cpx<R> *__restrict__ y) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int row = (int)(t % (2 * ntv));
    y[t] = row >= ntv ? -x[t] : x[t];
}

template <typename R>
void coarse_gamma5(Ctx &c, const void *x, void *y) {
    const size_t n = c.coarse_ncpx();
    coarse_gamma5_kernel<R><<<grid_for(n, 256), 256, 0, c.stream>>>(n, c.prm.n_tv, static_cast<const cpx<R> *>(x),
                                                                    static_cast<cpx<R> *>(y));
    MG_CHECK_LAUNCH();
}

template <typename R>
void coarse_apply(Ctx &c, const void *Dc, double sigma, const void *x, void *y, bool dform) {
    AggGeom A = make_agg(c, c.prm.agg);
    const int ntv = c.prm.n_tv;
    const size_t n = (size_t)A.n * 2 * ntv;
    if (sizeof(R) == 4 && c.prm.coarse_links != MGEIG_LINKS_LEVEL) {
        coarse_apply_links16(c, sigma, x, y, dform);   // the operator in its 16-bit form
        return;
    }
    TimeScope ts(c.timer, K_COARSE_APPLY, (double)A.n * (9.0 * 4 * ntv * ntv + 20.0 * ntv) * sizeof(cpx<R>));
    MG_REQUIRE(c.cnbr.p != nullptr, MGEIG_ENOTSETUP);
    coarse_apply_kernel<R><<<grid_for(n, 128), 128, 0, c.stream>>>(A, ntv, static_cast<const cpx<R> *>(Dc),
                                                                   c.cnbr.as<int>(), (R)sigma,
                                                                   static_cast<const cpx<R> *>(x), static_cast<cpx<R> *>(y),
                                                                   dform ? 1 : 0);
    MG_CHECK_LAUNCH();
}

// ---------------------------------------------------------------------------
// SAP: one colour of blocks; CTA = one block, thread = one site

// FP32: the block's forward links (two rows, 3 float4 per link) are staged in
// shared memory once and serve every MR step (the backward link of an in-block
// hop is the forward link of the in-block neighbour); two CTAs fit an SM.
template <typename R> struct SapBounds { static constexpr int minb = 1; };
template <> struct SapBounds<float> { static constexpr int minb = 2; };

template <typename R>
__global__ void __launch_bounds__(256, SapBounds<R>::minb)
sap_kernel(Geom g, AggGeom B, int colour, R sigma, const void *__restrict__ U,
           const void *__restrict__ clov, const void *__restrict__ rhs, int rhs_g5, void *z, int mr_iters) {
    extern __shared__ unsigned char smem_raw[];
    // component-major (rho[k][vol], slink[mu][3][vol]): consecutive threads read
    // consecutive words, without the 4-way bank conflicts of a site-major layout
    cpx<R> *rho = reinterpret_cast<cpx<R> *>(smem_raw);       // [12][vol]
    float4 *slink = reinterpret_cast<float4 *>(smem_raw + (size_t)B.vol * 12 * sizeof(cpx<R>));   // [4][3][vol]
    const int bv = B.vol;
    constexpr bool stage = sizeof(R) == 4;
    __shared__ R red[3 * 32];   // MR step sums, in the kernel's precision
    // the grid covers the blocks of one colour: blocks 2i and 2i + 1 differ in
    // colour (an even number of blocks per direction), CTA i takes the one of
    // this sweep's colour
    int b = 2 * blockIdx.x;
    {
        int r = b, bsum = 0;
        for (int mu = 0; mu < 4; ++mu) { bsum += r % B.cdims[mu]; r /= B.cdims[mu]; }
        if ((bsum & 1) != colour) b += 1;
    }
    const int V = g.V;
    const int l = threadIdx.x;
    const bool active = l < B.vol;
    int lc[4] = {0, 0, 0, 0}, c[4] = {0, 0, 0, 0}, s = 0;
    if (active) {
        s = agg_site(g, B, b, l, lc);
        site_coords(g, s, c);
    }
    cpx<R> e[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) e[k] = cpx<R>();
    if (stage && active) {
        const float4 *ug = static_cast<const float4 *>(U);
        for (int mu = 0; mu < 4; ++mu)
            for (int e = 0; e < 3; ++e) slink[(mu * 3 + e) * bv + l] = ug[((size_t)mu * 3 + e) * V + s];
    }
    // residual of D_sigma z = rhs on this block (z read with its global neighbours)
    if (active) {
        cpx<R> up[6], lo[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) { up[k] = cpx<R>(); lo[k] = cpx<R>(); }
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            int ph;
            cpx<R> u[9], psi[12];
            int n = neighbor(g, s, c, mu, true, &ph);
            Gauge<R>::load(U, V, mu, s, u);
            Spinor<R>::load(z, V, n, psi);
            hop_accumulate<R>(mu, true, u, psi, (R)ph, up, lo);
            n = neighbor(g, s, c, mu, false, &ph);
            Gauge<R>::load(U, V, mu, n, u);
            Spinor<R>::load(z, V, n, psi);
            hop_accumulate<R>(mu, false, u, psi, (R)ph, up, lo);
        }
        cpx<R> zs[12], dz[12], bb[12];
        Spinor<R>::load(z, V, s, zs);
        clover_apply<R>(clov, V, s, zs, dz);
        Spinor<R>::load(rhs, V, s, bb);
        const R half = R(0.5);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            cpx<R> du = dz[k] - half * up[k] - sigma * zs[k];
            cpx<R> dl = dz[6 + k] - half * lo[k] + sigma * zs[6 + k];
            cpx<R> bu = bb[k], bl = rhs_g5 ? -bb[6 + k] : bb[6 + k];
            rho[k * bv + l] = bu - du;
            rho[(6 + k) * bv + l] = bl - dl;
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    for (int it = 0; it < mr_iters; ++it) {
        // q = D_sigma restricted to the block (Dirichlet) applied to rho
        cpx<R> q[12], rl[12];
        R qr_re = 0, qr_im = 0, qq = 0;
        if (active) {
            cpx<R> up[6], lo[6];
#pragma unroll
            for (int k = 0; k < 6; ++k) { up[k] = cpx<R>(); lo[k] = cpx<R>(); }
#pragma unroll
            for (int mu = 0; mu < 4; ++mu) {
#pragma unroll
                for (int f = 0; f < 2; ++f) {
                    const bool fwd = f == 0;
                    const int lm = lc[mu] + (fwd ? 1 : -1);
                    if (lm < 0 || lm >= B.agg[mu]) continue;
                    int ln = l + (fwd ? 1 : -1) * (mu == 0 ? 1 : mu == 1 ? B.agg[0] : mu == 2 ? B.agg[0] * B.agg[1]
                                                                                              : B.agg[0] * B.agg[1] * B.agg[2]);
                    cpx<R> u[9], psi[12];
                    if constexpr (stage) {
                        const float4 *q = slink + (size_t)mu * 3 * bv + (fwd ? l : ln);
                        const float4 a = q[0], b = q[bv], cc = q[2 * bv];
                        u[0] = cpx<R>(a.x, a.y); u[1] = cpx<R>(a.z, a.w); u[2] = cpx<R>(b.x, b.y);
                        u[3] = cpx<R>(b.z, b.w); u[4] = cpx<R>(cc.x, cc.y); u[5] = cpx<R>(cc.z, cc.w);
                        u[6] = conj(u[1] * u[5] - u[2] * u[4]);
                        u[7] = conj(u[2] * u[3] - u[0] * u[5]);
                        u[8] = conj(u[0] * u[4] - u[1] * u[3]);
                    } else {
                        int ph;
                        const int n = neighbor(g, s, c, mu, fwd, &ph);
                        Gauge<R>::load(U, V, mu, fwd ? s : n, u);
                    }
#pragma unroll
                    for (int k = 0; k < 12; ++k) psi[k] = rho[k * bv + ln];
                    hop_accumulate<R>(mu, fwd, u, psi, (R)1, up, lo);
                }
            }
#pragma unroll
            for (int k = 0; k < 12; ++k) rl[k] = rho[k * bv + l];
            clover_apply<R>(clov, V, s, rl, q);
            const R half = R(0.5);
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                q[k] = q[k] - half * up[k] - sigma * rl[k];
                q[6 + k] = q[6 + k] - half * lo[k] + sigma * rl[6 + k];
            }
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                qr_re += q[k].re * rl[k].re + q[k].im * rl[k].im;
                qr_im += q[k].re * rl[k].im - q[k].im * rl[k].re;
                qq += q[k].re * q[k].re + q[k].im * q[k].im;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            qr_re += __shfl_xor_sync(0xffffffffu, qr_re, o);
            qr_im += __shfl_xor_sync(0xffffffffu, qr_im, o);
            qq += __shfl_xor_sync(0xffffffffu, qq, o);
        }
        if (lane == 0) { red[3 * w] = qr_re; red[3 * w + 1] = qr_im; red[3 * w + 2] = qq; }
        __syncthreads();   // all reads of rho for this step are done, partials visible
        R A_re = 0, A_im = 0, A_qq = 0;
        for (int i = 0; i < nw; ++i) { A_re += red[3 * i]; A_im += red[3 * i + 1]; A_qq += red[3 * i + 2]; }
        const cpx<R> alpha = A_qq > 0 ? cpx<R>(A_re / A_qq, A_im / A_qq) : cpx<R>();
        if (active) {
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                cmac(e[k], alpha, rl[k]);
                rho[k * bv + l] = rl[k] - alpha * q[k];
            }
        }
        __syncthreads();
    }
    if (active) {
        cpx<R> zs[12];
        Spinor<R>::load(z, V, s, zs);
#pragma unroll
        for (int k = 0; k < 12; ++k) zs[k] = zs[k] + e[k];
        Spinor<R>::store(z, V, s, zs);
    }
}

template <typename R>
void sap_sweep(Ctx &c, int colour, double sigma, const void *rhs, bool rhs_gamma5, void *z) {
    AggGeom B = make_agg(c, c.prm.sap_block);
    MG_REQUIRE(B.vol <= 1024, MGEIG_EINVAL);
    const int threads = ((B.vol + 31) / 32) * 32;
    const size_t smem = (size_t)B.vol * 12 * sizeof(cpx<R>) + (sizeof(R) == 4 ? (size_t)B.vol * 12 * sizeof(float4) : 0);
    MG_CUDA(cudaFuncSetAttribute(sap_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const void *U = sizeof(R) == 8 ? c.U64.p : c.U32.p;
    const void *C = sizeof(R) == 8 ? c.clov64.p : c.clov32.p;
    // half the sites: z read+write, rhs, links, clover (from HBM once per sweep)
    const double site_bytes = 12 * 2 * sizeof(R) * 3 + (sizeof(R) == 8 ? 576 : 192) + 72 * sizeof(R);
    TimeScope ts(c.timer, sizeof(R) == 8 ? K_SAP_F64 : K_SAP_F32, site_bytes * c.g.V / 2);
    MG_REQUIRE(B.cdims[0] % 2 == 0, MGEIG_EINVAL);
    sap_kernel<R><<<B.n / 2, threads, smem, c.stream>>>(c.g, B, colour, (R)sigma, U, C, rhs, rhs_gamma5 ? 1 : 0, z,
                                                        c.prm.sap_mr_iters);
    MG_CHECK_LAUNCH();
}

#define INST(R)                                                                              \
    template void restrict_vec<R>(Ctx &, const void *const *, const void *, void *);         \
    template void prolong_vec<R>(Ctx &, const void *const *, const void *, void *);          \
    template void build_coarse<R>(Ctx &, const void *const *, void *);                       \
    template void coarse_apply<R>(Ctx &, const void *, double, const void *, void *, bool);  \
    template void coarse_gamma5<R>(Ctx &, const void *, void *);                             \
    template void sap_sweep<R>(Ctx &, int, double, const void *, bool, void *);
INST(double)
INST(float)
#undef INST

}  // namespace mgeig
