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
// Grid: G co-resident blocks; block b owns a contiguous slice of coarse rows.
// One Arnoldi step = the coarse matvec on the owned rows (reading neighbour rows
// written before the last grid barrier), the deflation projection, two classical
// Gram-Schmidt passes and a norm in TWO grid-wide reductions: the deflation
// coefficients W^dag u and the first pass are reduced together, since
// <v_i, g5 (u - A W t)> = <g5 v_i, u> - sum_l t_l F_il with F_il = <g5 v_i, A W_l>
// (row i reduced when v_i is made); the second pass and the norm go together,
// ||w2||^2 = ||w1||^2 - ||h2||^2.  Partial sums go to
// a [G][slots] buffer; after each barrier every block adds the G partials in the
// same order, so all blocks hold bit-identical scalars and run the Givens
// rotations and the triangular solve redundantly (deterministic, no extra
// barrier).  Basis vectors stay unnormalised with one scale factor each.
//
// The grid barrier spins on a generation counter with a clock64() budget; on
// expiry it raises a sticky error word (the kernel then returns without further
// waits) that the host reads at its next synchronisation (MGEIG_ETIMEOUT).
#include "internal.h"

namespace mgeig {

constexpr int CG_THREADS = 1024;
constexpr int CG_MAXM = COARSE_PERSISTENT_MAXM;   // restart length limit
constexpr int CG_MAXK = 24;                       // deflation vectors (= max N_tv)
// partial-sum regions of consecutive reductions never overlap
constexpr int WS = 2 * CG_MAXK + CG_MAXM + 2;     // values of one reduction
constexpr int OFF_S1 = 0, OFF_S2 = WS, OFF_N = 2 * WS, OFF_P = 2 * WS + 2;
constexpr int CG_SLOTS = OFF_P + CG_MAXK;

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
    int cd[4];                     // coarse lattice extents
    const cpx<R> *Dc;              // [9][nagg][col][row]
    const int *nbr;                // [9][nagg] neighbour aggregates
    R sigma;
    const cpx<R> *b;               // r_c
    cpx<R> *x;                     // e (output); holds y during the iteration
    cpx<R> *rhs;                   // gamma5^c Pi r_c (scratch, n)
    cpx<R> *V;                     // (m + 1) x n
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

// u[t] = ((Q_c - sigma)(s v))[t] = ((gamma5^c D_c - sigma)(s v))[t] for the rows
// t in [r0, r1); a group of TPR consecutive threads shares one row: lane q takes
// the columns j = q (mod TPR) of all nine hop blocks, and the group reduces with
// shuffles.
constexpr int TPR = 8;

template <typename R>
__device__ __forceinline__ void qmatvec(const CGArgs<R> &a, const cpx<R> *v, R s, cpx<R> *u, int r0, int r1) {
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
                    const int nb = __ldg(a.nbr + (size_t)d * a.nagg + site);
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
                    const int nb = __ldg(a.nbr + (size_t)d * a.nagg + site);
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
            u[t] = s * acc - (a.sigma * s) * ldcg(v + t);
        }
    }
}

template <typename R>
__device__ __forceinline__ cpx<R> g5c(const CGArgs<R> &a, int t, cpx<R> v) {
    return (t % (2 * a.ntv)) >= a.ntv ? -v : v;
}

// Scalars (partial sums, Hessenberg matrix, Givens rotations, E^-1) are kept in
// the solver's own precision R: FP32 in the mixed-precision preconditioner,
// where FP64 arithmetic (1/64 of the FP32 rate on this part) held most warps at
// block barriers, FP64 in the all-FP64 path.
template <typename R>
__global__ void __launch_bounds__(CG_THREADS, 1) coarse_gmres_kernel(CGArgs<R> a) {
    using P = typename Pod2<R>::T;
    auto P2 = [](R x, R y) { return P{x, y}; };
    __shared__ P wpart[WS];                    // this block's partial sums
    __shared__ P h[WS];                        // grid-wide sums after a gather
    __shared__ P F[CG_MAXM * CG_MAXK];         // F_il = <g5 s_i V_i, A W_l>
    __shared__ P h1[CG_MAXM];
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
    const int rows_per_block = (a.n + G - 1) / G;
    const int r0 = blockIdx.x * rows_per_block;
    const int r1 = min(a.n, r0 + rows_per_block);
    P *mypart = a.partial + (size_t)blockIdx.x * CG_SLOTS;
    const int k = a.k;

    for (int i = threadIdx.x; i < k * k; i += blockDim.x) Ei[i] = P2((R)a.Einv[i].x, (R)a.Einv[i].y);
    if (threadIdx.x < CG_MAXK) { tc[threadIdx.x] = P2(0, 0); t0[threadIdx.x] = P2(0, 0); }
    __syncthreads();

    // wpart[i] = sc_i <X_i, u> over the owned rows, i < cnt: warp i takes value i,
    // its lanes stride over the rows (u complete on the owned rows)
    auto dots = [&](int cnt, auto vec, auto sc, const cpx<R> *u) {
        for (int i = wp; i < cnt; i += nw) {
            const cpx<R> *xi = vec(i);
            R sr = 0, si = 0;
            for (int t = r0 + lane; t < r1; t += 32) {
                cpx<R> p = xi[t], q = u[t];
                sr += p.re * q.re + p.im * q.im;
                si += p.re * q.im - p.im * q.re;
            }
            for (int o = 16; o > 0; o >>= 1) {
                sr += __shfl_xor_sync(0xffffffffu, sr, o);
                si += __shfl_xor_sync(0xffffffffu, si, o);
            }
            if (lane == 0) wpart[i] = P2(sr * sc(i), si * sc(i));
        }
    };
    // publish wpart[0..cnt) to this block's partial slots, barrier, h = grid sums
    auto reduce = [&](int off, int cnt) -> bool {
        __syncthreads();
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) mypart[off + i] = wpart[i];
        if (!grid_sync(a.st, G, a.timeout)) return false;
        for (int i = wp; i < cnt; i += nw) {
            R sr = 0, si = 0;
            for (unsigned int q = lane; q < G; q += 32) {
                P p = __ldcg(a.partial + (size_t)q * CG_SLOTS + off + i);
                sr += p.x; si += p.y;
            }
            for (int o = 16; o > 0; o >>= 1) {
                sr += __shfl_xor_sync(0xffffffffu, sr, o);
                si += __shfl_xor_sync(0xffffffffu, si, o);
            }
            if (lane == 0) h[i] = P2(sr, si);
        }
        __syncthreads();
        return true;
    };
    // u[t] = f(t, u[t], sum_i coef_i X_i[t]) on the owned rows; TPR lanes share a row
    auto combine = [&](int cnt, auto vec, auto coef, cpx<R> *u, auto f) {
        const int grp = threadIdx.x / TPR, q = threadIdx.x % TPR, ngrp = blockDim.x / TPR;
        for (int tb = r0; tb < r1; tb += ngrp) {
            const int t = tb + grp;
            cpx<R> acc0, acc1;
            if (t < r1) {
                int i = q;
                for (; i + TPR < cnt; i += 2 * TPR) {
                    cmac(acc0, coef(i), vec(i)[t]);
                    cmac(acc1, coef(i + TPR), vec(i + TPR)[t]);
                }
                if (i < cnt) cmac(acc0, coef(i), vec(i)[t]);
            }
            cpx<R> acc = acc0 + acc1;
            for (int o = 1; o < TPR; o <<= 1) {
                acc.re += __shfl_xor_sync(0xffffffffu, acc.re, o);
                acc.im += __shfl_xor_sync(0xffffffffu, acc.im, o);
            }
            if (t < r1 && q == 0) u[t] = f(t, u[t], acc);
        }
        __syncthreads();
    };
    auto one = [](int) { return R(1); };
    auto Wvec = [&](int i) { return a.W + (size_t)i * a.n; };
    auto AWvec = [&](int i) { return a.AW + (size_t)i * a.n; };
    auto Vvec = [&](int i) { return a.V + (size_t)i * a.n; };

    // tc = E^-1 W^dag u
    auto deflation_coeffs = [&](const cpx<R> *u) -> bool {
        dots(k, Wvec, one, u);
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
        combine(k, AWvec, [&](int i) { return cpx<R>((R)tc[i].x, (R)tc[i].y); }, u,
                [&](int t, cpx<R> ut, cpx<R> s) { return g5c(a, t, ut - s); });
    };
    // u = gamma5^c Pi (Q_c - sigma)(s v) on the owned rows
    auto apply_op = [&](const cpx<R> *v, R s, cpx<R> *u) -> bool {
        qmatvec<R>(a, v, s, u, r0, r1);
        __syncthreads();
        if (k > 0 && !deflation_coeffs(u)) return false;
        project_g5(u);
        return true;
    };
    // h[0] = ||v||^2 over the grid
    auto grid_norm2 = [&](const cpx<R> *v) -> bool {
        R acc = 0;
        for (int t = r0 + threadIdx.x; t < r1; t += blockDim.x) {
            cpx<R> q = v[t];
            acc += q.re * q.re + q.im * q.im;
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) nsum[wp] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            R s2 = 0;
            for (int w = 0; w < nw; ++w) s2 += nsum[w];
            wpart[0] = P2(s2, 0);
        }
        return reduce(OFF_N, 1);
    };

    // rhs = gamma5^c Pi r_c, t0 = E^-1 W^dag r_c, x = 0.  The tolerance refers
    // to ||r_c||: when r_c lies mostly in span(W) the projected right-hand side
    // is small and needs no further reduction.
    for (int t = r0 + threadIdx.x; t < r1; t += blockDim.x) { a.rhs[t] = a.b[t]; a.x[t] = cpx<R>(); }
    __syncthreads();
    if (!grid_norm2(a.rhs)) return;
    if (threadIdx.x == 0) bnorm = sqrt(h[0].x);
    __syncthreads();
    if (k > 0) {
        if (!deflation_coeffs(a.rhs)) return;
        for (int i = threadIdx.x; i < k; i += blockDim.x) t0[i] = tc[i];
        __syncthreads();
    }
    project_g5(a.rhs);
    if (threadIdx.x == 0) stop = !(bnorm > 0) || !isfinite(bnorm);
    __syncthreads();
    const R tol_abs = (R)a.tol * bnorm;
    int its = 0;
    bool have_x = false;
    while (!stop && its < a.maxiter) {
        // V0 = rhs - op(x)  (or rhs)
        if (have_x) {
            if (!apply_op(a.x, R(1), a.V)) return;
            for (int t = r0 + threadIdx.x; t < r1; t += blockDim.x) a.V[t] = a.rhs[t] - a.V[t];
        } else {
            for (int t = r0 + threadIdx.x; t < r1; t += blockDim.x) a.V[t] = a.rhs[t];
        }
        __syncthreads();
        if (!grid_norm2(a.V)) return;
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
        const int mm = min(a.m, a.maxiter - its);
        int kk = 0;
        bool conv = false;
        for (int j = 0; j < mm; ++j) {
            cpx<R> *w = a.V + (size_t)(j + 1) * a.n;
            const cpx<R> *vj = Vvec(j);
            // u = (Q_c - sigma) s_j V_j on the owned rows
            qmatvec<R>(a, vj, (R)scale[j], w, r0, r1);
            __syncthreads();
            // reduction 1: a_l = <W_l, u>, b_i = <g5 s_i V_i, u>, f_l = <g5 s_j V_j, A W_l>
            dots(k, Wvec, one, w);
            for (int i = wp; i <= j; i += nw) {
                const cpx<R> *vi = Vvec(i);
                R sr = 0, si = 0;
                for (int t = r0 + lane; t < r1; t += 32) {
                    cpx<R> pv = g5c(a, t, vi[t]), q = w[t];
                    sr += pv.re * q.re + pv.im * q.im;
                    si += pv.re * q.im - pv.im * q.re;
                }
                for (int o = 16; o > 0; o >>= 1) {
                    sr += __shfl_xor_sync(0xffffffffu, sr, o);
                    si += __shfl_xor_sync(0xffffffffu, si, o);
                }
                if (lane == 0) wpart[k + i] = P2(sr * scale[i], si * scale[i]);
            }
            for (int l = wp; l < k; l += nw) {
                const cpx<R> *awl = AWvec(l);
                R sr = 0, si = 0;
                for (int t = r0 + lane; t < r1; t += 32) {
                    cpx<R> pv = g5c(a, t, vj[t]), q = awl[t];
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
            // w1 = g5 (u - A W t) - sum_i h1_i s_i V_i
            combine(k, AWvec, [&](int i) { return cpx<R>((R)tc[i].x, (R)tc[i].y); }, w,
                    [&](int t, cpx<R> ut, cpx<R> sm) { return g5c(a, t, ut - sm); });
            combine(j + 1, Vvec, [&](int i) { return cpx<R>((R)(h1[i].x * scale[i]), (R)(h1[i].y * scale[i])); }, w,
                    [](int, cpx<R> ut, cpx<R> sm) { return ut - sm; });
            // reduction 2: h2_i = <s_i V_i, w1>, ||w1||^2
            dots(j + 1, Vvec, [&](int i) { return scale[i]; }, w);
            {
                R acc = 0;
                for (int t = r0 + threadIdx.x; t < r1; t += blockDim.x) {
                    cpx<R> q = w[t];
                    acc += q.re * q.re + q.im * q.im;
                }
                for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                if (lane == 0) nsum[wp] = acc;
                __syncthreads();
                if (threadIdx.x == 0) {
                    R s2 = 0;
                    for (int ww = 0; ww < nw; ++ww) s2 += nsum[ww];
                    wpart[j + 1] = P2(s2, 0);
                }
            }
            if (!reduce(OFF_S2, j + 2)) return;
            if (threadIdx.x == 0) {
                R n2 = h[j + 1].x;
                for (int i = 0; i <= j; ++i) {
                    P &col = Rm[j * (CG_MAXM + 1) + i];
                    col = P2(col.x + h[i].x, col.y + h[i].y);
                    n2 -= h[i].x * h[i].x + h[i].y * h[i].y;
                }
                nrm2s = n2 > 0 ? n2 : R(0);
            }
            combine(j + 1, Vvec, [&](int i) { return cpx<R>((R)(h[i].x * scale[i]), (R)(h[i].y * scale[i])); }, w,
                    [](int, cpx<R> ut, cpx<R> sm) { return ut - sm; });
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
        combine(kk, Vvec, [&](int i) { return cpx<R>((R)(y[i].x * scale[i]), (R)(y[i].y * scale[i])); }, a.x,
                [](int, cpx<R> ut, cpx<R> s) { return ut + s; });
        have_x = true;
        its += kk;
        if (!grid_sync(a.st, G, a.timeout)) return;   // x complete before any matvec on it
        if (conv) break;
        if (threadIdx.x == 0) stop = 0;
        __syncthreads();
    }
    // e = y + W (t0 - E^-1 W^dag A y)
    if (k > 0) {
        cpx<R> *u = a.V;   // scratch
        qmatvec<R>(a, a.x, R(1), u, r0, r1);
        __syncthreads();
        if (!deflation_coeffs(u)) return;
        combine(k, Wvec, [&](int i) { return cpx<R>((R)(t0[i].x - tc[i].x), (R)(t0[i].y - tc[i].y)); }, a.x,
                [](int, cpx<R> ut, cpx<R> s) { return ut + s; });
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&a.st->iters, its);
}

// Launch the persistent coarse solve for (Q_c - sigma) e_c = r_c.
template <typename R>
void coarse_gmres_persistent(Ctx &c, const CoarseSolveBufs &B, double sigma, const void *rc, void *ec) {
    const int ntv = c.prm.n_tv;
    const int n = c.nagg * 2 * ntv;
    const int m = std::min(c.prm.coarse_restart, CG_MAXM);
    int dev_sms = 0;
    MG_CUDA(cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, c.device));
    int per_sm = 0;
    MG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, coarse_gmres_kernel<R>, CG_THREADS, 0));
    MG_REQUIRE(per_sm >= 1, MGEIG_ECUDA);
    int G = (n * TPR + CG_THREADS - 1) / CG_THREADS;
    G = std::max(1, std::min(G, std::min(dev_sms * per_sm, dev_sms)));
    B.V->alloc((size_t)(m + 1) * n * sizeof(cpx<R>));
    B.rhs->alloc((size_t)n * sizeof(cpx<R>));
    B.partial->alloc((size_t)G * CG_SLOTS * sizeof(double2));
    CGArgs<R> a;
    a.nagg = c.nagg; a.ntv = ntv; a.n = n;
    for (int mu = 0; mu < 4; ++mu) a.cd[mu] = c.cdims[mu];
    a.Dc = static_cast<const cpx<R> *>(c.Dc.p);
    a.nbr = c.cnbr.as<int>();
    a.sigma = (R)sigma;
    a.b = static_cast<const cpx<R> *>(rc);
    a.x = static_cast<cpx<R> *>(ec);
    a.rhs = B.rhs->as<cpx<R>>();
    a.V = B.V->as<cpx<R>>();
    a.k = B.k;
    MG_REQUIRE(a.k <= CG_MAXK, MGEIG_EINVAL);
    a.W = static_cast<const cpx<R> *>(B.W);
    a.AW = static_cast<const cpx<R> *>(B.AW);
    a.Einv = static_cast<const double2 *>(B.Einv);
    a.partial = B.partial->as<typename Pod2<R>::T>();
    a.st = static_cast<CGState *>(B.state);
    a.m = m;
    a.maxiter = c.prm.coarse_maxiter;
    a.tol = c.prm.coarse_tol;
    a.timeout = 4000000000LL;   // about 2 s of SM clock per barrier wait
    void *args[] = {&a};
    TimeScope ts(c.timer, K_COARSE_SOLVE, 0);
    MG_CUDA(cudaLaunchCooperativeKernel((void *)coarse_gmres_kernel<R>, dim3(G), dim3(CG_THREADS), args, 0, c.stream));
    ++c.launches;
}

template void coarse_gmres_persistent<float>(Ctx &, const CoarseSolveBufs &, double, const void *, void *);
template void coarse_gmres_persistent<double>(Ctx &, const CoarseSolveBufs &, double, const void *, void *);

// The same persistent coarse solve, with its scratch at caller-given device
// addresses instead of context buffers: the Krylov basis V ((m + 1) n level
// complex values), the projected right-hand side rhs (n), the per-block
// partial sums (coarse_gmres_partial_bytes) and the CGState word block
// (16 bytes, zero on entry).  Grid size and restart length are those of
// coarse_gmres_persistent, so both give the same result.
int coarse_gmres_grid(Ctx &c) {
    const int n = c.nagg * 2 * c.prm.n_tv;
    int dev_sms = 0;
    MG_CUDA(cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, c.device));
    int per_sm = 0;
    if (c.mixed())
        MG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, coarse_gmres_kernel<float>, CG_THREADS, 0));
    else
        MG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, coarse_gmres_kernel<double>, CG_THREADS, 0));
    MG_REQUIRE(per_sm >= 1, MGEIG_ECUDA);
    int G = (n * TPR + CG_THREADS - 1) / CG_THREADS;
    return std::max(1, std::min(G, std::min(dev_sms * per_sm, dev_sms)));
}

size_t coarse_gmres_partial_bytes(Ctx &c, int G) {
    return (size_t)G * CG_SLOTS * (c.mixed() ? sizeof(float2) : sizeof(double2));
}

template <typename R>
void coarse_gmres_at(Ctx &c, int G, double sigma, const void *rc, void *ec, void *V, void *rhs, void *partial,
                     void *state, int k, const void *W, const void *AW, const void *Einv) {
    const int ntv = c.prm.n_tv;
    MG_REQUIRE(k <= CG_MAXK, MGEIG_EINVAL);
    CGArgs<R> a;
    a.nagg = c.nagg; a.ntv = ntv; a.n = c.nagg * 2 * ntv;
    for (int mu = 0; mu < 4; ++mu) a.cd[mu] = c.cdims[mu];
    a.Dc = static_cast<const cpx<R> *>(c.Dc.p);
    a.nbr = c.cnbr.as<int>();
    a.sigma = (R)sigma;
    a.b = static_cast<const cpx<R> *>(rc);
    a.x = static_cast<cpx<R> *>(ec);
    a.rhs = static_cast<cpx<R> *>(rhs);
    a.V = static_cast<cpx<R> *>(V);
    a.k = k;
    a.W = static_cast<const cpx<R> *>(W);
    a.AW = static_cast<const cpx<R> *>(AW);
    a.Einv = static_cast<const double2 *>(Einv);
    a.partial = static_cast<typename Pod2<R>::T *>(partial);
    a.st = static_cast<CGState *>(state);
    a.m = std::min(c.prm.coarse_restart, CG_MAXM);
    a.maxiter = c.prm.coarse_maxiter;
    a.tol = c.prm.coarse_tol;
    a.timeout = 4000000000LL;   // about 2 s of SM clock per barrier wait
    void *args[] = {&a};
    TimeScope ts(c.timer, K_COARSE_SOLVE, 0);
    MG_CUDA(cudaLaunchCooperativeKernel((void *)coarse_gmres_kernel<R>, dim3(G), dim3(CG_THREADS), args, 0, c.stream));
    ++c.launches;
}

template void coarse_gmres_at<float>(Ctx &, int, double, const void *, void *, void *, void *, void *, void *, int,
                                     const void *, const void *, const void *);
template void coarse_gmres_at<double>(Ctx &, int, double, const void *, void *, void *, void *, void *, void *, int,
                                      const void *, const void *, const void *);

}  // namespace mgeig
