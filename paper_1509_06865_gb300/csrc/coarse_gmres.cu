// Coarse-grid solve of the two-grid cycle (Sec. 2: restarted GMRES as the
// coarse solver for Q_c) as ONE persistent cooperative launch: every Arnoldi
// step runs on the device, with no host round trip.
//
// It solves (Q_c - sigma) e = r_c, A = Q_c - sigma = gamma5^c D_c - sigma.
//  * Deflation (k > 0): W = [P^dag w_1 .. P^dag w_k] are the coarse images of the
//    test vectors (the current eigenvector approximations of Algorithm 1), the
//    directions on which A becomes nearly singular when sigma approaches their
//    eigenvalues.  With E^-1 = (W^dag A W)^-1 (host-computed) and
//    Pi = 1 - A W E^-1 W^dag:  e = W E^-1 W^dag r_c + (1 - W E^-1 W^dag A) y,
//    where Pi A y = Pi r_c.
//  * GMRES runs on gamma5^c Pi A y = gamma5^c Pi r_c, i.e. on the D_c form
//    (gamma5^c A = D_c - sigma gamma5^c, Eq. 2.6 with a shift), whose spectrum
//    lies in the right half plane instead of around the origin.
//
// Grid: G co-resident blocks; block b owns a contiguous slice of rb coarse rows.
// Every vector the block only ever reads or writes on its own rows (the Krylov
// basis V_i, the raw products U_i = A s_i V_i, the right-hand side, the iterate,
// a work vector, and when room is left the deflation vectors W, A W) lives in
// the block's shared memory (in a per-block slice of global scratch when the
// coarse grid is too large for that); only the vector being multiplied goes to
// global memory (`pub`), where the matvecs of the neighbouring blocks read it.
//
// One Arnoldi step, classical Gram-Schmidt with a second pass, two grid-wide
// reductions:
//   u     = A s_j V_j                          (matvec of pub, see below)
//   R1:   a_l = <W_l, u>, b_i = <g5 s_i V_i, u>, f_l = <g5 s_j V_j, A W_l>
//   t     = E^-1 a;  h1_i = b_i - sum_l F_il t_l   (F_il = <g5 s_i V_i, A W_l>)
//   w1    = g5 (u - A W t) - sum_i h1_i s_i V_i;  pub <- w1
//   R2:   h2_i = <s_i V_i, w1>, ||w1||^2  (||w2||^2 = ||w1||^2 - ||h2||^2)
//   V_j+1 = w1 - sum_i h2_i s_i V_i  (own rows only)
// The next matvec reads w1 from pub, complete on every block after the R2
// barrier, and corrects it on its own rows with the stored products:
// A s_j+1 V_j+1 = s_j+1 (A w1 - sum_i h2_i U_i).  So no block ever reads a
// vector that another block is still writing, with two grid barriers per step.
// Partial sums go to a [G][slots] buffer (consecutive reductions use disjoint
// slots); after each barrier every block adds the G partials in the same
// order, so all blocks hold bit-identical scalars and run the Givens rotations
// and the triangular solve redundantly.  Basis vectors stay unnormalised with
// one scale factor each.
//
// The grid barrier spins on a generation counter with a clock64() budget; on
// expiry it raises a sticky error word (the kernel then returns without further
// waits) that the host reads at its next synchronisation (MGEIG_ETIMEOUT).
#include <array>
#include <map>
#include <mutex>

#include "half16.cuh"
#include "internal.h"

namespace mgeig {

constexpr int CG_THREADS = 1024;
constexpr int CG_GATHER = 8;                      // partial sums per lane: up to 256 blocks
constexpr int CG_NBR_SITES = 64;                  // coarse sites of a block's staged neighbour table
constexpr int CG_MAXM = COARSE_PERSISTENT_MAXM;   // restart length limit
constexpr int CG_MAXK = 24;                       // deflation vectors (= max N_tv)
// partial-sum regions of consecutive reductions never overlap
constexpr int WS = 2 * CG_MAXK + CG_MAXM + 2;     // values of one reduction
constexpr int OFF_S1 = 0, OFF_S2 = WS, OFF_N = 2 * WS, OFF_P = 2 * WS + 2;
constexpr int CG_SLOTS = OFF_P + CG_MAXK;
// shared memory a block may use in all (static + dynamic), with a reserve
constexpr size_t CG_SMEM_LIMIT = 227 * 1024 - 1024;

struct CGState {
    unsigned int count;   // barrier arrivals (returns to 0 after every barrier)
    unsigned int gen;     // barrier generation
    int status;           // sticky: 0 ok, 1 barrier timeout, 2 breakdown
    int iters;            // accumulated Arnoldi steps of all solves
};
static_assert(sizeof(CGState) == 16, "CGState lives in one reduction slot");

template <typename R> struct Pod2;
template <> struct Pod2<float> { using T = float2; };
template <> struct Pod2<double> { using T = double2; };

template <typename R>
struct CGArgs {
    int nagg, ntv, n;              // coarse sites, test vectors, rows = nagg * 2 ntv
    int rb;                        // rows per block (the last block may own fewer)
    int nslice;                    // owned-row vectors per block: V (m+1), U (m+1), rhs, x, w
    int smem_slices, smem_defl;    // 1: the slices / copies of W, A W live in shared memory
    const cpx<R> *Dc;              // [9][nagg][col][row]
    const void *L16;               // 16-bit links [9][nagg][re|im][row][col] (16-bit kernels)
    const float *Ls;               // their scales [9][nagg]
    const int *nbr;                // [9][nagg] neighbour aggregates
    R sigma;
    const cpx<R> *b;               // r_c
    cpx<R> *x;                     // e (output)
    cpx<R> *pub;                   // the vector being multiplied (n)
    cpx<R> *gslices;               // G x nslice x rb, when the slices are not in shared memory
    int k;                         // deflation vectors (0: none)
    const cpx<R> *W, *AW;          // k x n each
    const double2 *Einv;           // k x k, row-major
    typename Pod2<R>::T *partial;  // [G][CG_SLOTS]
    CGState *st;
    int m, maxiter;
    double tol;
    long long timeout;
};

__device__ __forceinline__ bool grid_sync(CGState *st, unsigned int nblocks, long long timeout) {
    __syncthreads();
    __shared__ int ok;
    if (threadIdx.x == 0) {
        volatile unsigned int *vgen = &st->gen;
        const unsigned int g0 = *vgen;
        __threadfence();
        const unsigned int arrived = atomicAdd(&st->count, 1u);
        if (arrived == nblocks - 1) {
            atomicExch(&st->count, 0u);
            __threadfence();
            atomicAdd(&st->gen, 1u);
        } else {
            const long long t0 = clock64();
            while (*vgen == g0) {
                if (clock64() - t0 > timeout) { atomicExch(&st->status, 1); break; }
                __nanosleep(32);
            }
        }
        __threadfence();
        ok = *((volatile int *)&st->status) == 0;
    }
    __syncthreads();
    return ok;
}

// Loads of data other blocks wrote before the last grid barrier bypass the
// (non-coherent) L1: ld.global.cg.
__device__ __forceinline__ cpx<float> ldcg(const cpx<float> *p) {
    float2 v = __ldcg(reinterpret_cast<const float2 *>(p));
    return cpx<float>(v.x, v.y);
}
__device__ __forceinline__ cpx<double> ldcg(const cpx<double> *p) {
    double2 v = __ldcg(reinterpret_cast<const double2 *>(p));
    return cpx<double>(v.x, v.y);
}

// out[t - r0] = ((Q_c - sigma)(s v))[t] = ((gamma5^c D_c - sigma)(s v))[t] for the
// owned rows t in [r0, r1), v = the published vector; a group of TPR consecutive
// threads shares one row: lane q takes the columns j = q (mod TPR) of all nine
// hop blocks, and the group reduces with shuffles.
constexpr int TPR = 8;

// The neighbour aggregate of hop d of site `site`: from the block's staged table
// (sites s0 .. s0 + CG_NBR_SITES - 1) when there is one, else from global memory.
template <typename R>
__device__ __forceinline__ int hop_nbr(const CGArgs<R> &a, const int *snb, int s0, int d, int site) {
    return snb ? snb[d * CG_NBR_SITES + site - s0] : __ldg(a.nbr + (size_t)d * a.nagg + site);
}

template <typename R>
__device__ __forceinline__ void qmatvec(const CGArgs<R> &a, const cpx<R> *v, R s, cpx<R> *out, int r0, int r1,
                                        const int *snb, int s0) {
    const int n2 = 2 * a.ntv;
    const int grp = threadIdx.x / TPR, q = threadIdx.x % TPR, ngrp = blockDim.x / TPR;
    for (int tb = r0; tb < r1; tb += ngrp) {
        const int t = tb + grp;
        cpx<R> acc0, acc1;
        if (t < r1) {
            const int site = t / n2, row = t % n2;
            if constexpr (sizeof(R) == 4) {
                // n2 <= 2 * CG_MAXK = 48: a lane's (at most 6) columns of one block are
                // loaded before they are used, so their L2 latencies overlap
                constexpr int U = (2 * CG_MAXK + TPR - 1) / TPR;
                for (int d = 0; d < 9; ++d) {
                    const int nb = hop_nbr(a, snb, s0, d, site);
                    const cpx<R> *blk = a.Dc + ((size_t)d * a.nagg + site) * n2 * n2 + row;
                    const cpx<R> *xb = v + (size_t)nb * n2;
                    cpx<R> bv[U], xv[U];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int j = q + u * TPR;
                        if (j < n2) { bv[u] = blk[(size_t)j * n2]; xv[u] = ldcg(xb + j); }
                    }
#pragma unroll
                    for (int u = 0; u < U; ++u)
                        if (q + u * TPR < n2) cmac((u & 1) ? acc1 : acc0, bv[u], xv[u]);
                }
            } else {
#pragma unroll 3
                for (int d = 0; d < 9; ++d) {
                    const int nb = hop_nbr(a, snb, s0, d, site);
                    const cpx<R> *blk = a.Dc + ((size_t)d * a.nagg + site) * n2 * n2 + row;
                    const cpx<R> *xb = v + (size_t)nb * n2;
                    int j = q;
                    for (; j + TPR < n2; j += 2 * TPR) {
                        cmac(acc0, blk[(size_t)j * n2], ldcg(xb + j));
                        cmac(acc1, blk[(size_t)(j + TPR) * n2], ldcg(xb + j + TPR));
                    }
                    if (j < n2) cmac(acc0, blk[(size_t)j * n2], ldcg(xb + j));
                }
            }
        }
        cpx<R> acc = acc0 + acc1;
        for (int o = 1; o < TPR; o <<= 1) {
            acc.re += __shfl_xor_sync(0xffffffffu, acc.re, o);
            acc.im += __shfl_xor_sync(0xffffffffu, acc.im, o);
        }
        if (t < r1 && q == 0) {
            if ((t % n2) >= a.ntv) acc = -acc;
            out[t - r0] = s * acc - (a.sigma * s) * ldcg(v + t);
        }
    }
}

// The same product with 16-bit links (FP32 vectors and arithmetic): lane q takes
// the column pairs p = q (mod TPR) of the real and imaginary planes, and every
// hop block's sum is multiplied by the block's scale.
template <typename H>
__device__ __forceinline__ void qmatvec16(const CGArgs<float> &a, const cpx<float> *v, float s, cpx<float> *out,
                                          int r0, int r1, const int *snb, int s0) {
    using HP = typename H16<H>::P;
    const int n2 = 2 * a.ntv, np = a.ntv;
    const int grp = threadIdx.x / TPR, q = threadIdx.x % TPR, ngrp = blockDim.x / TPR;
    constexpr int U = (CG_MAXK + TPR - 1) / TPR;   // pairs per lane (n2 / 2 <= CG_MAXK)
    const H *L = static_cast<const H *>(a.L16);
    for (int tb = r0; tb < r1; tb += ngrp) {
        const int t = tb + grp;
        float ar = 0.f, ai = 0.f;
        if (t < r1) {
            const int site = t / n2, row = t % n2;
            for (int d = 0; d < 9; ++d) {
                const size_t blk = (size_t)d * a.nagg + site;
                const int nb = hop_nbr(a, snb, s0, d, site);
                const HP *pr = reinterpret_cast<const HP *>(L + blk * 2 * n2 * n2 + (size_t)row * n2);
                const HP *pi = pr + (size_t)n2 * n2 / 2;
                const float4 *xb = reinterpret_cast<const float4 *>(v + (size_t)nb * n2);
                HP rv[U], iv[U];
                float4 xv[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int p = q + u * TPR;
                    if (p < np) { rv[u] = pr[p]; iv[u] = pi[p]; xv[u] = __ldcg(xb + p); }
                }
                float dr = 0.f, di = 0.f;
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if (q + u * TPR < np) {
                        const float2 r = H16<H>::pair(rv[u]), im = H16<H>::pair(iv[u]);
                        const float4 x = xv[u];
                        dr = fmaf(r.x, x.x, dr); dr = fmaf(-im.x, x.y, dr);
                        di = fmaf(r.x, x.y, di); di = fmaf(im.x, x.x, di);
                        dr = fmaf(r.y, x.z, dr); dr = fmaf(-im.y, x.w, dr);
                        di = fmaf(r.y, x.w, di); di = fmaf(im.y, x.z, di);
                    }
                }
                const float sc = __ldg(a.Ls + blk);
                ar = fmaf(sc, dr, ar);
                ai = fmaf(sc, di, ai);
            }
        }
        for (int o = 1; o < TPR; o <<= 1) {
            ar += __shfl_xor_sync(0xffffffffu, ar, o);
            ai += __shfl_xor_sync(0xffffffffu, ai, o);
        }
        if (t < r1 && q == 0) {
            cpx<float> acc(ar, ai);
            if ((t % n2) >= a.ntv) acc = -acc;
            out[t - r0] = s * acc - (a.sigma * s) * ldcg(v + t);
        }
    }
}

// the product of the kernel's link format LK (0: level precision, 1: BF16, 2: FP16)
template <typename R, int LK>
__device__ __forceinline__ void matvec(const CGArgs<R> &a, const cpx<R> *v, R s, cpx<R> *out, int r0, int r1,
                                       const int *snb, int s0) {
    if constexpr (LK == 0) qmatvec<R>(a, v, s, out, r0, r1, snb, s0);
    else if constexpr (LK == 1) qmatvec16<__nv_bfloat16>(a, v, s, out, r0, r1, snb, s0);
    else qmatvec16<__half>(a, v, s, out, r0, r1, snb, s0);
}

// Scalars (partial sums, Hessenberg matrix, Givens rotations, E^-1) are kept in
// the solver's own precision R: FP32 in the mixed-precision preconditioner,
// where FP64 arithmetic (1/64 of the FP32 rate on this part) held most warps at
// block barriers, FP64 in the all-FP64 path.
template <typename R, int LK>
__global__ void __launch_bounds__(CG_THREADS, 1) coarse_gmres_kernel(CGArgs<R> a) {
    using P = typename Pod2<R>::T;
    auto P2 = [](R x, R y) { return P{x, y}; };
    extern __shared__ __align__(16) unsigned char cg_dyn[];
    __shared__ P wpart[WS];                    // this block's partial sums
    __shared__ P h[WS];                        // grid-wide sums after a gather
    __shared__ P F[CG_MAXM * CG_MAXK];         // F_il = <g5 s_i V_i, A W_l>
    __shared__ P h1[CG_MAXM];
    __shared__ P h2s[CG_MAXM];                 // second-pass coefficients of the last step
    __shared__ R nsum[CG_THREADS / 32];
    __shared__ R nrm2s;
    __shared__ P Rm[(CG_MAXM + 1) * CG_MAXM];  // rotated Hessenberg, column-major
    __shared__ R cs[CG_MAXM];
    __shared__ P sn[CG_MAXM], g[CG_MAXM + 1], y[CG_MAXM];
    __shared__ R scale[CG_MAXM + 1];
    __shared__ P Ei[CG_MAXK * CG_MAXK], t0[CG_MAXK], tc[CG_MAXK];
    __shared__ R bnorm, beta;
    __shared__ int stop;
    const unsigned int G = gridDim.x;
    const int nw = CG_THREADS / 32;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int rb = a.rb;
    const int r0 = min(a.n, (int)blockIdx.x * rb);
    const int r1 = min(a.n, r0 + rb);
    const int nr = r1 - r0;
    const int m = a.m, k = a.k, n2 = 2 * a.ntv;
    P *mypart = a.partial + (size_t)blockIdx.x * CG_SLOTS;

    // owned-row slices: V_0..V_m, U_0..U_m, rhs, x, w
    cpx<R> *S = a.smem_slices ? reinterpret_cast<cpx<R> *>(cg_dyn)
                              : a.gslices + (size_t)blockIdx.x * a.nslice * rb;
    auto Vv = [&](int i) { return S + (size_t)i * rb; };
    auto Uv = [&](int i) { return S + (size_t)(m + 1 + i) * rb; };
    cpx<R> *rhs = S + (size_t)(2 * m + 2) * rb;
    cpx<R> *xs = rhs + rb;
    cpx<R> *ws = xs + rb;
    cpx<R> *Dl = a.smem_defl ? reinterpret_cast<cpx<R> *>(cg_dyn) + (size_t)a.nslice * rb : nullptr;
    auto Wv = [&](int l) -> const cpx<R> * { return Dl ? Dl + (size_t)l * rb : a.W + (size_t)l * a.n + r0; };
    auto AWv = [&](int l) -> const cpx<R> * { return Dl ? Dl + (size_t)(k + l) * rb : a.AW + (size_t)l * a.n + r0; };
    auto g5 = [&](int i, cpx<R> v) { return ((r0 + i) % n2) >= a.ntv ? -v : v; };

    // the neighbour table of the block's coarse sites, staged once (the matvec's
    // block loads then wait on one L2 round trip per hop instead of two)
    __shared__ int snb[9 * CG_NBR_SITES];
    const int s0 = nr > 0 ? r0 / n2 : 0;
    const int nsites = nr > 0 ? (r1 - 1) / n2 - s0 + 1 : 0;
    const int *snb_p = nsites <= CG_NBR_SITES ? snb : nullptr;
    if (snb_p)
        for (int e = threadIdx.x; e < 9 * nsites; e += blockDim.x) {
            const int d = e / nsites, sl = e % nsites;
            snb[d * CG_NBR_SITES + sl] = __ldg(a.nbr + (size_t)d * a.nagg + s0 + sl);
        }
    for (int i = threadIdx.x; i < k * k; i += blockDim.x) Ei[i] = P2((R)a.Einv[i].x, (R)a.Einv[i].y);
    if (threadIdx.x < CG_MAXK) { tc[threadIdx.x] = P2(0, 0); t0[threadIdx.x] = P2(0, 0); }
    if (Dl)
        for (int e = threadIdx.x; e < k * nr; e += blockDim.x) {
            const int l = e / nr, i = e % nr;
            Dl[(size_t)l * rb + i] = a.W[(size_t)l * a.n + r0 + i];
            Dl[(size_t)(k + l) * rb + i] = a.AW[(size_t)l * a.n + r0 + i];
        }
    __syncthreads();

    // wpart[i] = sc_i <X_i, u> over the owned rows, i < cnt: warp i takes value i,
    // its lanes stride over the rows
    auto dots = [&](int cnt, int base, auto vec, auto sc, const cpx<R> *u, bool g5x) {
        for (int i = wp; i < cnt; i += nw) {
            const cpx<R> *xi = vec(i);
            R sr = 0, si = 0;
            for (int t = lane; t < nr; t += 32) {
                cpx<R> p = xi[t], q = u[t];
                if (g5x) p = g5(t, p);
                sr += p.re * q.re + p.im * q.im;
                si += p.re * q.im - p.im * q.re;
            }
            for (int o = 16; o > 0; o >>= 1) {
                sr += __shfl_xor_sync(0xffffffffu, sr, o);
                si += __shfl_xor_sync(0xffffffffu, si, o);
            }
            if (lane == 0) wpart[base + i] = P2(sr * sc(i), si * sc(i));
        }
    };
    // wpart[slot] = ||v||^2 over the owned rows
    auto norm_part = [&](const cpx<R> *v, int slot) {
        R acc = 0;
        for (int t = threadIdx.x; t < nr; t += blockDim.x) {
            cpx<R> q = v[t];
            acc += q.re * q.re + q.im * q.im;
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) nsum[wp] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            R s2 = 0;
            for (int w = 0; w < nw; ++w) s2 += nsum[w];
            wpart[slot] = P2(s2, 0);
        }
    };
    // publish wpart[0..cnt) to this block's partial slots, barrier, h = grid sums
    auto reduce = [&](int off, int cnt) -> bool {
        __syncthreads();
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) mypart[off + i] = wpart[i];
        if (!grid_sync(a.st, G, a.timeout)) return false;
        for (int i = wp; i < cnt; i += nw) {
            // all of a lane's partials are loaded before they are added (G <= 32 *
            // CG_GATHER), so their L2 latencies overlap; the order of the sums is
            // the same in every block
            P pv[CG_GATHER];
#pragma unroll
            for (int u = 0; u < CG_GATHER; ++u) {
                const unsigned int q = lane + 32u * u;
                pv[u] = q < G ? __ldcg(a.partial + (size_t)q * CG_SLOTS + off + i) : P{0, 0};
            }
            R sr = 0, si = 0;
#pragma unroll
            for (int u = 0; u < CG_GATHER; ++u) { sr += pv[u].x; si += pv[u].y; }
            for (int o = 16; o > 0; o >>= 1) {
                sr += __shfl_xor_sync(0xffffffffu, sr, o);
                si += __shfl_xor_sync(0xffffffffu, si, o);
            }
            if (lane == 0) h[i] = P2(sr, si);
        }
        __syncthreads();
        return true;
    };
    // u[i] = f(i, u[i], sum_l coef_l X_l[i]) on the owned rows; TPR lanes share a row
    auto combine = [&](int cnt, auto vec, auto coef, cpx<R> *u, auto f) {
        const int grp = threadIdx.x / TPR, q = threadIdx.x % TPR, ngrp = blockDim.x / TPR;
        for (int ib = 0; ib < nr; ib += ngrp) {
            const int i = ib + grp;
            cpx<R> acc0, acc1;
            if (i < nr) {
                int l = q;
                for (; l + TPR < cnt; l += 2 * TPR) {
                    cmac(acc0, coef(l), vec(l)[i]);
                    cmac(acc1, coef(l + TPR), vec(l + TPR)[i]);
                }
                if (l < cnt) cmac(acc0, coef(l), vec(l)[i]);
            }
            cpx<R> acc = acc0 + acc1;
            for (int o = 1; o < TPR; o <<= 1) {
                acc.re += __shfl_xor_sync(0xffffffffu, acc.re, o);
                acc.im += __shfl_xor_sync(0xffffffffu, acc.im, o);
            }
            if (i < nr && q == 0) u[i] = f(i, u[i], acc);
        }
        __syncthreads();
    };
    // u[i] = f(i, u[i], sum_l coef1_l X1_l[i], sum_l coef2_l X2_l[i]): two combines
    // in one pass over the rows and one block barrier
    auto combine2 = [&](int cnt1, auto vec1, auto coef1, int cnt2, auto vec2, auto coef2, cpx<R> *u, auto f) {
        const int grp = threadIdx.x / TPR, q = threadIdx.x % TPR, ngrp = blockDim.x / TPR;
        for (int ib = 0; ib < nr; ib += ngrp) {
            const int i = ib + grp;
            cpx<R> a1, a2;
            if (i < nr) {
                for (int l = q; l < cnt1; l += TPR) cmac(a1, coef1(l), vec1(l)[i]);
                for (int l = q; l < cnt2; l += TPR) cmac(a2, coef2(l), vec2(l)[i]);
            }
            for (int o = 1; o < TPR; o <<= 1) {
                a1.re += __shfl_xor_sync(0xffffffffu, a1.re, o);
                a1.im += __shfl_xor_sync(0xffffffffu, a1.im, o);
                a2.re += __shfl_xor_sync(0xffffffffu, a2.re, o);
                a2.im += __shfl_xor_sync(0xffffffffu, a2.im, o);
            }
            if (i < nr && q == 0) u[i] = f(i, u[i], a1, a2);
        }
        __syncthreads();
    };
    auto publish = [&](const cpx<R> *v) {
        for (int i = threadIdx.x; i < nr; i += blockDim.x) a.pub[r0 + i] = v[i];
    };
    auto one = [](int) { return R(1); };
    auto tcoef = [&](int l) { return cpx<R>((R)tc[l].x, (R)tc[l].y); };

    // tc = E^-1 W^dag u
    auto deflation_coeffs = [&](const cpx<R> *u) -> bool {
        dots(k, 0, Wv, one, u, false);
        if (!reduce(OFF_P, k)) return false;
        for (int i = threadIdx.x; i < k; i += blockDim.x) {
            R sr = 0, si = 0;
            for (int l = 0; l < k; ++l) {
                P e = Ei[i * k + l], d = h[l];
                sr += e.x * d.x - e.y * d.y;
                si += e.x * d.y + e.y * d.x;
            }
            tc[i] = P2(sr, si);
        }
        __syncthreads();
        return true;
    };
    // u <- gamma5^c (u - A W tc)
    auto project_g5 = [&](cpx<R> *u) {
        combine(k, AWv, tcoef, u, [&](int i, cpx<R> ui, cpx<R> s) { return g5(i, ui - s); });
    };

    // rhs = gamma5^c Pi r_c, t0 = E^-1 W^dag r_c, x = 0.  The tolerance refers
    // to ||r_c||: when r_c lies mostly in span(W) the projected right-hand side
    // is small and needs no further reduction.
    for (int i = threadIdx.x; i < nr; i += blockDim.x) { rhs[i] = a.b[r0 + i]; xs[i] = cpx<R>(); }
    __syncthreads();
    norm_part(rhs, 0);
    if (!reduce(OFF_N, 1)) return;
    if (threadIdx.x == 0) bnorm = sqrt(h[0].x);
    __syncthreads();
    if (k > 0) {
        if (!deflation_coeffs(rhs)) return;
        for (int i = threadIdx.x; i < k; i += blockDim.x) t0[i] = tc[i];
        __syncthreads();
    }
    project_g5(rhs);
    if (threadIdx.x == 0) stop = !(bnorm > 0) || !isfinite(bnorm);
    __syncthreads();
    const R tol_abs = (R)a.tol * bnorm;
    int its = 0;
    bool have_x = false;
    while (!stop && its < a.maxiter) {
        cpx<R> *v0 = Vv(0);
        // V0 = rhs - op(x)  (or rhs)
        if (have_x) {
            publish(xs);
            if (!grid_sync(a.st, G, a.timeout)) return;       // x complete everywhere
            matvec<R, LK>(a, a.pub, R(1), v0, r0, r1, snb_p, s0);
            __syncthreads();
            if (k > 0) {
                if (!deflation_coeffs(v0)) return;             // its barrier also ends the reads of pub
            } else if (!grid_sync(a.st, G, a.timeout)) {
                return;                                        // every matvec done before pub changes
            }
            combine(k, AWv, tcoef, v0, [&](int i, cpx<R> vi, cpx<R> s) { return rhs[i] - g5(i, vi - s); });
        } else {
            for (int i = threadIdx.x; i < nr; i += blockDim.x) v0[i] = rhs[i];
            __syncthreads();
        }
        publish(v0);
        norm_part(v0, 0);
        if (!reduce(OFF_N, 1)) return;                         // also makes V0 visible in pub
        if (threadIdx.x == 0) {
            beta = sqrt(h[0].x);
            stop = !(beta > tol_abs) || !isfinite(beta);
            if (!isfinite(beta)) atomicExch(&a.st->status, 2);
            scale[0] = beta > 0 ? R(1) / beta : R(0);
            g[0] = P2(beta, 0);
            for (int i = 1; i <= CG_MAXM; ++i) g[i] = P2(0, 0);
        }
        __syncthreads();
        if (stop) break;
        const int mm = min(m, a.maxiter - its);
        int kk = 0;
        bool conv = false;
        for (int j = 0; j < mm; ++j) {
            cpx<R> *uj = Uv(j);
            const cpx<R> *vj = Vv(j);
            // U_j = A s_j V_j: the matvec of pub (= V_j before its second pass),
            // corrected by the second-pass coefficients of the last step
            matvec<R, LK>(a, a.pub, (R)scale[j], uj, r0, r1, snb_p, s0);
            __syncthreads();
            if (j > 0)
                combine(j, Uv, [&](int i) { return cpx<R>((R)(h2s[i].x * scale[j]), (R)(h2s[i].y * scale[j])); },
                        uj, [](int, cpx<R> ui, cpx<R> s) { return ui - s; });
            // reduction 1: a_l = <W_l, u>, b_i = <g5 s_i V_i, u>, f_l = <g5 s_j V_j, A W_l>
            dots(k, 0, Wv, one, uj, false);
            dots(j + 1, k, Vv, [&](int i) { return scale[i]; }, uj, true);
            for (int l = wp; l < k; l += nw) {
                const cpx<R> *awl = AWv(l);
                R sr = 0, si = 0;
                for (int t = lane; t < nr; t += 32) {
                    cpx<R> pv = g5(t, vj[t]), q = awl[t];
                    sr += pv.re * q.re + pv.im * q.im;
                    si += pv.re * q.im - pv.im * q.re;
                }
                for (int o = 16; o > 0; o >>= 1) {
                    sr += __shfl_xor_sync(0xffffffffu, sr, o);
                    si += __shfl_xor_sync(0xffffffffu, si, o);
                }
                if (lane == 0) wpart[k + j + 1 + l] = P2(sr * scale[j], si * scale[j]);
            }
            if (!reduce(OFF_S1, 2 * k + j + 1)) return;
            // t = E^-1 a ; F row j ; h1_i = b_i - sum_l F_il t_l
            for (int l = threadIdx.x; l < k; l += blockDim.x) F[j * CG_MAXK + l] = h[k + j + 1 + l];
            for (int i = threadIdx.x; i < k; i += blockDim.x) {
                R sr = 0, si = 0;
                for (int l = 0; l < k; ++l) {
                    P e = Ei[i * k + l], d = h[l];
                    sr += e.x * d.x - e.y * d.y;
                    si += e.x * d.y + e.y * d.x;
                }
                tc[i] = P2(sr, si);
            }
            __syncthreads();
            for (int i = threadIdx.x; i <= j; i += blockDim.x) {
                P b = h[k + i];
                for (int l = 0; l < k; ++l) {
                    P f = F[i * CG_MAXK + l], t = tc[l];
                    b.x -= f.x * t.x - f.y * t.y;
                    b.y -= f.x * t.y + f.y * t.x;
                }
                h1[i] = b;
                Rm[j * (CG_MAXM + 1) + i] = b;
            }
            __syncthreads();
            // w1 = g5 (u - A W t) - sum_i h1_i s_i V_i, published for the next matvec
            combine2(k, AWv, tcoef, j + 1, Vv,
                     [&](int i) { return cpx<R>((R)(h1[i].x * scale[i]), (R)(h1[i].y * scale[i])); }, ws,
                     [&](int i, cpx<R>, cpx<R> s1, cpx<R> s2) { return g5(i, uj[i] - s1) - s2; });
            publish(ws);
            // reduction 2: h2_i = <s_i V_i, w1>, ||w1||^2
            dots(j + 1, 0, Vv, [&](int i) { return scale[i]; }, ws, false);
            // ||w1||^2 as one more inner product (no extra block barrier)
            dots(1, j + 1, [&](int) -> const cpx<R> * { return ws; }, one, ws, false);
            if (!reduce(OFF_S2, j + 2)) return;
            if (threadIdx.x == 0) {
                R n2s = h[j + 1].x;
                for (int i = 0; i <= j; ++i) {
                    P &col = Rm[j * (CG_MAXM + 1) + i];
                    col = P2(col.x + h[i].x, col.y + h[i].y);
                    n2s -= h[i].x * h[i].x + h[i].y * h[i].y;
                }
                nrm2s = n2s > 0 ? n2s : R(0);
            }
            for (int i = threadIdx.x; i <= j; i += blockDim.x) h2s[i] = h[i];
            __syncthreads();
            // V_j+1 = w1 - sum_i h2_i s_i V_i on the owned rows
            cpx<R> *vn = Vv(j + 1);
            combine(j + 1, Vv, [&](int i) { return cpx<R>((R)(h2s[i].x * scale[i]), (R)(h2s[i].y * scale[i])); },
                    vn, [&](int i, cpx<R>, cpx<R> s) { return ws[i] - s; });
            if (threadIdx.x == 0) {
                const R nrm = sqrt(nrm2s);
                P *col = Rm + j * (CG_MAXM + 1);
                col[j + 1] = P2(nrm, 0);
                for (int i = 0; i < j; ++i) {   // previous rotations
                    P p = col[i], q = col[i + 1], sv = sn[i];
                    col[i] = P2(cs[i] * p.x + (sv.x * q.x - sv.y * q.y), cs[i] * p.y + (sv.x * q.y + sv.y * q.x));
                    col[i + 1] = P2(cs[i] * q.x - (sv.x * p.x + sv.y * p.y), cs[i] * q.y - (sv.x * p.y - sv.y * p.x));
                }
                P p = col[j], q = col[j + 1];
                R ap = hypot(p.x, p.y), aq = hypot(q.x, q.y);
                R c, sr, si;
                if (aq == 0) { c = 1; sr = 0; si = 0; }
                else if (ap == 0) { c = 0; sr = 1; si = 0; }
                else {
                    R tt = hypot(ap, aq);
                    c = ap / tt;
                    R ur = p.x / ap, ui = p.y / ap;          // s = (p/|p|) conj(q) / t
                    sr = (ur * q.x + ui * q.y) / tt;
                    si = (ui * q.x - ur * q.y) / tt;
                }
                cs[j] = c;
                sn[j] = P2(sr, si);
                col[j] = P2(c * p.x + (sr * q.x - si * q.y), c * p.y + (sr * q.y + si * q.x));
                col[j + 1] = P2(0, 0);
                P gj = g[j];
                g[j + 1] = P2(-(sr * gj.x + si * gj.y), -(sr * gj.y - si * gj.x));
                g[j] = P2(c * gj.x, c * gj.y);
                const R est = hypot(g[j + 1].x, g[j + 1].y);
                if (!isfinite(nrm) || !isfinite(est)) atomicExch(&a.st->status, 2);
                scale[j + 1] = nrm > 0 ? R(1) / nrm : R(0);
                stop = (est <= tol_abs) || nrm == 0 || !isfinite(est);
            }
            __syncthreads();
            kk = j + 1;
            if (stop) { conv = true; break; }
        }
        if (threadIdx.x == 0) {   // y = R^-1 g
            for (int i = kk - 1; i >= 0; --i) {
                P sacc = g[i];
                for (int l = i + 1; l < kk; ++l) {
                    P r = Rm[l * (CG_MAXM + 1) + i], yl = y[l];
                    sacc.x -= r.x * yl.x - r.y * yl.y;
                    sacc.y -= r.x * yl.y + r.y * yl.x;
                }
                P d = Rm[i * (CG_MAXM + 1) + i];
                R dd = d.x * d.x + d.y * d.y;
                y[i] = dd > 0 ? P2((sacc.x * d.x + sacc.y * d.y) / dd, (sacc.y * d.x - sacc.x * d.y) / dd)
                              : P2(0, 0);
            }
        }
        __syncthreads();
        combine(kk, Vv, [&](int i) { return cpx<R>((R)(y[i].x * scale[i]), (R)(y[i].y * scale[i])); }, xs,
                [](int, cpx<R> xi, cpx<R> s) { return xi + s; });
        have_x = true;
        its += kk;
        if (conv) break;
        if (threadIdx.x == 0) stop = 0;
        __syncthreads();
    }
    // e = y + W (t0 - E^-1 W^dag A y)
    if (k > 0) {
        publish(xs);
        if (!grid_sync(a.st, G, a.timeout)) return;
        matvec<R, LK>(a, a.pub, R(1), ws, r0, r1, snb_p, s0);
        __syncthreads();
        if (!deflation_coeffs(ws)) return;
        combine(k, Wv, [&](int i) { return cpx<R>((R)(t0[i].x - tc[i].x), (R)(t0[i].y - tc[i].y)); }, xs,
                [](int, cpx<R> xi, cpx<R> s) { return xi + s; });
    }
    for (int i = threadIdx.x; i < nr; i += blockDim.x) a.x[r0 + i] = xs[i];
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&a.st->iters, its);
}

// ---------------------------------------------------------------------------
// host side: the launch plan (grid, slices in shared or global memory) and the
// global scratch it needs

namespace {

struct CGPlan {
    int G, rb, nslice, m;
    bool smem_slices, smem_defl;
    size_t dyn_smem;          // dynamic shared memory per block
    size_t off_slices, off_partial, scratch_bytes;   // global scratch layout
};

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

// the kernel instance for the context's precision and link format
template <typename R>
const void *kernel_for(Ctx &c) {
    if constexpr (sizeof(R) == 8) {
        return (const void *)coarse_gmres_kernel<double, 0>;
    } else {
        switch (c.prm.coarse_links) {
            case MGEIG_LINKS_BF16: return (const void *)coarse_gmres_kernel<float, 1>;
            case MGEIG_LINKS_F16: return (const void *)coarse_gmres_kernel<float, 2>;
            default: return (const void *)coarse_gmres_kernel<float, 0>;
        }
    }
}

template <typename R>
CGPlan compute_plan(Ctx &c, int k) {
    CGPlan p;
    const int n = c.nagg * 2 * c.prm.n_tv;
    p.m = std::min(c.prm.coarse_restart, CG_MAXM);
    int dev_sms = 0;
    MG_CUDA(cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, c.device));
    cudaFuncAttributes fa;
    const void *kern = kernel_for<R>(c);
    MG_CUDA(cudaFuncGetAttributes(&fa, kern));
    const size_t elem = sizeof(cpx<R>);
    int G = std::max(1, std::min((n * TPR + CG_THREADS - 1) / CG_THREADS, dev_sms));
    if (c.prm.coarse_blocks > 0) G = std::min(G, c.prm.coarse_blocks);
    G = std::min(G, 32 * CG_GATHER);
    p.rb = (n + G - 1) / G;
    p.G = (n + p.rb - 1) / p.rb;   // every block owns at least one row
    p.nslice = 2 * (p.m + 1) + 3;
    const size_t budget = CG_SMEM_LIMIT > fa.sharedSizeBytes ? CG_SMEM_LIMIT - fa.sharedSizeBytes : 0;
    const size_t slice_b = (size_t)p.nslice * p.rb * elem, defl_b = (size_t)2 * k * p.rb * elem;
    p.smem_slices = slice_b <= budget;
    p.smem_defl = p.smem_slices && k > 0 && slice_b + defl_b <= budget;
    p.dyn_smem = p.smem_slices ? slice_b + (p.smem_defl ? defl_b : 0) : 0;
    // global scratch: pub | slices (when not in shared memory) | partial sums
    p.off_slices = align256((size_t)n * elem);
    p.off_partial = p.off_slices + (p.smem_slices ? 0 : align256((size_t)p.G * slice_b));
    p.scratch_bytes = p.off_partial + align256((size_t)p.G * CG_SLOTS * sizeof(typename Pod2<R>::T));
    MG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)p.dyn_smem));
    int per_sm = 0;
    MG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, CG_THREADS, p.dyn_smem));
    MG_REQUIRE(per_sm >= 1 && p.G <= dev_sms * per_sm, MGEIG_ECUDA);
    return p;
}

// plans depend only on the device and the problem shape: computed once each
template <typename R>
CGPlan make_plan(Ctx &c, int k) {
    static std::mutex mu;
    static std::map<std::array<int, 8>, CGPlan> cache;
    const std::array<int, 8> key{c.device, c.nagg, c.prm.n_tv, std::min(c.prm.coarse_restart, CG_MAXM), k,
                                 (int)sizeof(R), sizeof(R) == 4 ? c.prm.coarse_links : 0, c.prm.coarse_blocks};
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    const CGPlan p = compute_plan<R>(c, k);
    cache.emplace(key, p);
    return p;
}

}  // namespace

// the barrier budget in SM clock cycles
long long barrier_cycles(Ctx &c) {
    int khz = 0;
    MG_CUDA(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, c.device));
    if (khz <= 0) khz = 2000000;
    return std::max(1LL, (long long)(c.prm.barrier_timeout * khz * 1e3));
}

size_t coarse_gmres_scratch_bytes(Ctx &c, int k) {
    return c.mixed() ? make_plan<float>(c, k).scratch_bytes : make_plan<double>(c, k).scratch_bytes;
}

// The persistent coarse solve with its global scratch (coarse_gmres_scratch_bytes)
// at a caller-given device address and the CGState word block (16 bytes, zero on
// entry) at `state`.
template <typename R>
void coarse_gmres_at(Ctx &c, double sigma, const void *rc, void *ec, void *scratch, void *state, int k,
                     const void *W, const void *AW, const void *Einv) {
    MG_REQUIRE(k <= CG_MAXK && k <= c.prm.n_tv, MGEIG_EINVAL);
    const CGPlan p = make_plan<R>(c, k);
    char *sc = static_cast<char *>(scratch);
    CGArgs<R> a;
    a.nagg = c.nagg; a.ntv = c.prm.n_tv; a.n = c.nagg * 2 * c.prm.n_tv;
    a.rb = p.rb; a.nslice = p.nslice;
    a.smem_slices = p.smem_slices; a.smem_defl = p.smem_defl;
    a.Dc = static_cast<const cpx<R> *>(c.Dc.p);
    a.L16 = c.Dc16.p;
    a.Ls = c.Dcs.as<float>();
    MG_REQUIRE(sizeof(R) == 8 || c.prm.coarse_links == MGEIG_LINKS_LEVEL || c.Dc16.p, MGEIG_ENOTSETUP);
    a.nbr = c.cnbr.as<int>();
    a.sigma = (R)sigma;
    a.b = static_cast<const cpx<R> *>(rc);
    a.x = static_cast<cpx<R> *>(ec);
    a.pub = reinterpret_cast<cpx<R> *>(sc);
    a.gslices = p.smem_slices ? nullptr : reinterpret_cast<cpx<R> *>(sc + p.off_slices);
    a.k = k;
    a.W = static_cast<const cpx<R> *>(W);
    a.AW = static_cast<const cpx<R> *>(AW);
    a.Einv = static_cast<const double2 *>(Einv);
    a.partial = reinterpret_cast<typename Pod2<R>::T *>(sc + p.off_partial);
    a.st = static_cast<CGState *>(state);
    a.m = p.m;
    a.maxiter = c.prm.coarse_maxiter;
    a.tol = c.prm.coarse_tol;
    a.timeout = barrier_cycles(c);
    void *args[] = {&a};
    // the dynamic shared-memory limit is an attribute of the kernel, not of the
    // plan: plans of other problem shapes may have changed it since
    const void *kern = kernel_for<R>(c);
    MG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.dyn_smem));
    TimeScope ts(c.timer, K_COARSE_SOLVE, 0);
    MG_CUDA(cudaLaunchCooperativeKernel(kern, dim3(p.G), dim3(CG_THREADS), args,
                                        p.dyn_smem, c.stream));
    ++c.launches;
}

template void coarse_gmres_at<float>(Ctx &, double, const void *, void *, void *, void *, int, const void *,
                                     const void *, const void *);
template void coarse_gmres_at<double>(Ctx &, double, const void *, void *, void *, void *, int, const void *,
                                      const void *, const void *);

// Launch the persistent coarse solve for (Q_c - sigma) e_c = r_c with scratch
// owned by the context.
template <typename R>
void coarse_gmres_persistent(Ctx &c, const CoarseSolveBufs &B, double sigma, const void *rc, void *ec) {
    B.scratch->alloc(coarse_gmres_scratch_bytes(c, B.k));
    coarse_gmres_at<R>(c, sigma, rc, ec, B.scratch->p, B.state, B.k, B.W, B.AW, B.Einv);
}

template void coarse_gmres_persistent<float>(Ctx &, const CoarseSolveBufs &, double, const void *, void *);
template void coarse_gmres_persistent<double>(Ctx &, const CoarseSolveBufs &, double, const void *, void *);

}  // namespace mgeig
