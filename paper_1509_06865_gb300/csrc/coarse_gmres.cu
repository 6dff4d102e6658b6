// Coarse-grid GMRES (the coarse solver of Sec. 2) as ONE persistent
// cooperative launch: every Arnoldi step runs on the device, with no host round
// trip.  It solves (Q_c - sigma) e = r_c in the equivalent form
// (D_c - sigma gamma5^c) e = gamma5^c r_c (Q_c - sigma = gamma5^c (D_c - sigma
// gamma5^c), Eq. 2.6 with a shift).
//
// Grid: G co-resident blocks (cooperative launch); block b owns a contiguous
// slice of coarse rows.  One Arnoldi step = the coarse matvec on the owned rows
// (reading the neighbours' rows written before the last grid barrier), two
// classical Gram-Schmidt passes and a norm, i.e. three grid-wide reductions.
// Partial sums go to a [G][slots] buffer; after each barrier every block adds
// the G partials in the same order, so all blocks hold bit-identical Hessenberg
// columns and run the Givens rotations and the final triangular solve
// redundantly (no extra barrier, deterministic).  Basis vectors are kept
// unnormalised with a scale factor each, so no barrier is needed between a
// norm and the next matvec.
//
// The grid barrier spins on a generation counter with a clock64() budget; on
// expiry it raises a sticky error word (the kernel then returns without further
// waits) that the host reads at its next synchronisation and reports as
// MGEIG_ETIMEOUT.  The same state block accumulates the iteration count.
#include "internal.h"

namespace mgeig {

constexpr int CG_THREADS = 256;
constexpr int CG_MAXM = 32;                  // restart length limit of this kernel
constexpr int CG_SLOTS = 2 * (CG_MAXM + 2) + 2;

struct CGState {
    unsigned int count;   // barrier arrivals (returns to 0 after every barrier)
    unsigned int gen;     // barrier generation
    int status;           // sticky: 0 ok, 1 barrier timeout, 2 breakdown
    int iters;            // accumulated Arnoldi steps of all solves
};
static_assert(sizeof(CGState) == 16, "CGState lives in one reduction slot");

template <typename R>
struct CGArgs {
    int nagg, ntv, n;              // coarse sites, test vectors, rows = nagg * 2 ntv
    int cd[4];                     // coarse lattice extents
    const cpx<R> *Dc;              // [9][nagg][col][row]
    R sigma;
    const cpx<R> *b;
    cpx<R> *x;
    cpx<R> *V;                     // (m + 1) x n
    double2 *partial;              // [G][CG_SLOTS]
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
                __nanosleep(40);
            }
        }
        __threadfence();
        ok = *((volatile int *)&st->status) == 0;
    }
    __syncthreads();
    return ok;
}

// Loads of data that other blocks wrote before the last grid barrier bypass
// the (non-coherent) L1: ld.global.cg.
__device__ __forceinline__ cpx<float> ldcg(const cpx<float> *p) {
    float2 v = __ldcg(reinterpret_cast<const float2 *>(p));
    return cpx<float>(v.x, v.y);
}
__device__ __forceinline__ cpx<double> ldcg(const cpx<double> *p) {
    double2 v = __ldcg(reinterpret_cast<const double2 *>(p));
    return cpx<double>(v.x, v.y);
}

// y[row] = (D_c - sigma gamma5^c) v (v scaled by s) for one row
template <typename R>
__device__ __forceinline__ cpx<R> coarse_row(const CGArgs<R> &a, const cpx<R> *v, R s, int t) {
    const int n2 = 2 * a.ntv;
    const int site = t / n2, row = t % n2;
    int ac[4], rem = site;
    for (int mu = 0; mu < 4; ++mu) { ac[mu] = rem % a.cd[mu]; rem /= a.cd[mu]; }
    cpx<R> acc;
    for (int d = 0; d < 9; ++d) {
        int nb = site;
        if (d > 0) {
            const int mu = (d - 1) / 2, step = (d & 1) ? 1 : -1;
            int bc[4] = {ac[0], ac[1], ac[2], ac[3]};
            bc[mu] = (bc[mu] + step + a.cd[mu]) % a.cd[mu];
            nb = ((bc[3] * a.cd[2] + bc[2]) * a.cd[1] + bc[1]) * a.cd[0] + bc[0];
        }
        const cpx<R> *blk = a.Dc + ((size_t)d * a.nagg + site) * n2 * n2 + row;
        const cpx<R> *xb = v + (size_t)nb * n2;
#pragma unroll 4
        for (int j = 0; j < n2; ++j) cmac(acc, blk[(size_t)j * n2], ldcg(xb + j));
    }
    const R sg = row >= a.ntv ? -a.sigma : a.sigma;
    return s * acc - (sg * s) * ldcg(v + t);
}

// block-reduce `cnt` complex partials (one per thread-local value array) into
// partial[blockIdx][off + i]
__device__ __forceinline__ void block_partial(double re, double im, int i, double2 *sh, double2 *out) {
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sh[w * (CG_MAXM + 2) + i] = make_double2(re, im);
    (void)out;
}

template <typename R>
__global__ void __launch_bounds__(CG_THREADS) coarse_gmres_kernel(CGArgs<R> a) {
    __shared__ double2 wsum[(CG_THREADS / 32) * (CG_MAXM + 2)];
    __shared__ double2 h[CG_MAXM + 2];
    __shared__ double2 Rm[(CG_MAXM + 1) * CG_MAXM];   // rotated Hessenberg, column-major
    __shared__ double cs[CG_MAXM];
    __shared__ double2 sn[CG_MAXM], g[CG_MAXM + 1], y[CG_MAXM];
    __shared__ double scale[CG_MAXM + 1];
    __shared__ double bnorm, beta;
    __shared__ int stop, kcols;
    const unsigned int G = gridDim.x;
    const int nw = CG_THREADS / 32;
    const int rows_per_block = (a.n + G - 1) / G;
    const int r0 = blockIdx.x * rows_per_block;
    const int r1 = min(a.n, r0 + rows_per_block);
    double2 *mypart = a.partial + (size_t)blockIdx.x * CG_SLOTS;

    // sum partial[0..G)[off + i] for i < cnt into h[i] (all blocks, same order)
    auto gather = [&](int off, int cnt) {
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
            double sr = 0, si = 0;
            for (unsigned int q = 0; q < G; ++q) {
                double2 p = __ldcg(a.partial + (size_t)q * CG_SLOTS + off + i);
                sr += p.x; si += p.y;
            }
            h[i] = make_double2(sr, si);
        }
        __syncthreads();
    };
    // reduce per-thread values in wsum[w][i] (i < cnt) to mypart[off + i]
    auto flush = [&](int off, int cnt) {
        __syncthreads();
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
            double sr = 0, si = 0;
            for (int w = 0; w < nw; ++w) { double2 p = wsum[w * (CG_MAXM + 2) + i]; sr += p.x; si += p.y; }
            mypart[off + i] = make_double2(sr, si);
        }
    };

    // ||b||
    {
        double acc = 0;
        for (int t = r0 + threadIdx.x; t < r1; t += blockDim.x) {
            cpx<R> v = a.b[t];   // |gamma5^c b| = |b|
            acc += (double)v.re * v.re + (double)v.im * v.im;
            a.x[t] = cpx<R>();
        }
        block_partial(acc, 0.0, 0, wsum, nullptr);
        flush(2 * (CG_MAXM + 2), 1);
        if (!grid_sync(a.st, G, a.timeout)) return;
        gather(2 * (CG_MAXM + 2), 1);
        if (threadIdx.x == 0) { bnorm = sqrt(h[0].x); stop = !(bnorm > 0); }
        __syncthreads();
        if (stop) return;
    }
    const double tol_abs = a.tol * bnorm;
    int its = 0;
    bool have_x = false;
    while (its < a.maxiter) {
        // V0 = b - A x  (or b), beta = ||V0||
        {
            double acc = 0;
            for (int t = r0 + threadIdx.x; t < r1; t += blockDim.x) {
                cpx<R> r = a.b[t];
                if ((t % (2 * a.ntv)) >= a.ntv) r = -r;    // gamma5^c r_c
                if (have_x) r = r - coarse_row<R>(a, a.x, R(1), t);
                a.V[t] = r;
                acc += (double)r.re * r.re + (double)r.im * r.im;
            }
            block_partial(acc, 0.0, 0, wsum, nullptr);
            flush(2 * (CG_MAXM + 2), 1);
            if (!grid_sync(a.st, G, a.timeout)) return;
            gather(2 * (CG_MAXM + 2), 1);
            if (threadIdx.x == 0) {
                beta = sqrt(h[0].x);
                stop = !(beta > tol_abs) || !isfinite(beta);
                if (!isfinite(beta)) atomicExch(&a.st->status, 2);
                scale[0] = beta > 0 ? 1.0 / beta : 0.0;
                g[0] = make_double2(beta, 0);
                for (int i = 1; i <= CG_MAXM; ++i) g[i] = make_double2(0, 0);
            }
            __syncthreads();
            if (stop) break;
        }
        const int mm = min(a.m, a.maxiter - its);
        int k = 0;
        bool conv = false;
        for (int j = 0; j < mm; ++j) {
            cpx<R> *vj = a.V + (size_t)j * a.n;
            cpx<R> *w = a.V + (size_t)(j + 1) * a.n;
            // w = A (s_j V_j) on owned rows; first Gram-Schmidt partials
            for (int t = r0 + threadIdx.x; t < r1; t += blockDim.x) w[t] = coarse_row<R>(a, vj, (R)scale[j], t);
            for (int pass = 0; pass < 2; ++pass) {
                for (int i = 0; i <= j; ++i) {
                    const cpx<R> *vi = a.V + (size_t)i * a.n;
                    double sr = 0, si = 0;
                    for (int t = r0 + threadIdx.x; t < r1; t += blockDim.x) {
                        cpx<R> p = vi[t], q = w[t];
                        sr += (double)p.re * q.re + (double)p.im * q.im;
                        si += (double)p.re * q.im - (double)p.im * q.re;
                    }
                    block_partial(sr * scale[i], si * scale[i], i, wsum, nullptr);
                }
                flush(pass * (CG_MAXM + 2), j + 1);
                if (!grid_sync(a.st, G, a.timeout)) return;
                gather(pass * (CG_MAXM + 2), j + 1);
                if (threadIdx.x == 0) {
                    for (int i = 0; i <= j; ++i) {
                        double2 &col = Rm[j * (CG_MAXM + 1) + i];
                        if (pass == 0) col = h[i];
                        else col = make_double2(col.x + h[i].x, col.y + h[i].y);
                    }
                }
                // w -= sum_i h_i s_i V_i
                for (int t = r0 + threadIdx.x; t < r1; t += blockDim.x) {
                    cpx<R> q = w[t];
                    for (int i = 0; i <= j; ++i) {
                        const cpx<R> hi((R)(h[i].x * scale[i]), (R)(h[i].y * scale[i]));
                        q = q - hi * a.V[(size_t)i * a.n + t];
                    }
                    w[t] = q;
                }
                __syncthreads();
            }
            // norm of w
            double acc = 0;
            for (int t = r0 + threadIdx.x; t < r1; t += blockDim.x) {
                cpx<R> q = w[t];
                acc += (double)q.re * q.re + (double)q.im * q.im;
            }
            block_partial(acc, 0.0, 0, wsum, nullptr);
            flush(2 * (CG_MAXM + 2), 1);
            if (!grid_sync(a.st, G, a.timeout)) return;
            gather(2 * (CG_MAXM + 2), 1);
            if (threadIdx.x == 0) {
                const double nrm = sqrt(h[0].x);
                double2 *col = Rm + j * (CG_MAXM + 1);
                col[j + 1] = make_double2(nrm, 0);
                // previous rotations
                for (int i = 0; i < j; ++i) {
                    double2 p = col[i], q = col[i + 1];
                    double2 sv = sn[i];
                    // p' = c p + s q ; q' = c q - conj(s) p
                    double2 pn = make_double2(cs[i] * p.x + (sv.x * q.x - sv.y * q.y), cs[i] * p.y + (sv.x * q.y + sv.y * q.x));
                    double2 qn = make_double2(cs[i] * q.x - (sv.x * p.x + sv.y * p.y), cs[i] * q.y - (sv.x * p.y - sv.y * p.x));
                    col[i] = pn;
                    col[i + 1] = qn;
                }
                double2 p = col[j], q = col[j + 1];
                double ap = hypot(p.x, p.y), aq = hypot(q.x, q.y);
                double c, sr, si;
                if (aq == 0) { c = 1; sr = 0; si = 0; }
                else if (ap == 0) { c = 0; sr = 1; si = 0; }
                else {
                    double tt = hypot(ap, aq);
                    c = ap / tt;
                    // s = (p/|p|) conj(q) / t
                    double ur = p.x / ap, ui = p.y / ap;
                    sr = (ur * q.x + ui * q.y) / tt;
                    si = (ui * q.x - ur * q.y) / tt;
                }
                cs[j] = c;
                sn[j] = make_double2(sr, si);
                col[j] = make_double2(c * p.x + (sr * q.x - si * q.y), c * p.y + (sr * q.y + si * q.x));
                col[j + 1] = make_double2(0, 0);
                double2 gj = g[j];
                // g[j+1] = -conj(s) g[j] ; g[j] = c g[j]
                g[j + 1] = make_double2(-(sr * gj.x + si * gj.y), -(sr * gj.y - si * gj.x));
                g[j] = make_double2(c * gj.x, c * gj.y);
                const double est = hypot(g[j + 1].x, g[j + 1].y);
                if (!isfinite(nrm) || !isfinite(est)) atomicExch(&a.st->status, 2);
                scale[j + 1] = nrm > 0 ? 1.0 / nrm : 0.0;
                stop = (est <= tol_abs) || nrm == 0 || !isfinite(est);
                kcols = j + 1;
            }
            __syncthreads();
            k = j + 1;
            if (stop) { conv = true; break; }
        }
        // y = R^-1 g (thread 0), x += sum_i y_i s_i V_i
        if (threadIdx.x == 0) {
            for (int i = k - 1; i >= 0; --i) {
                double2 sacc = g[i];
                for (int l = i + 1; l < k; ++l) {
                    double2 r = Rm[l * (CG_MAXM + 1) + i], yl = y[l];
                    sacc.x -= r.x * yl.x - r.y * yl.y;
                    sacc.y -= r.x * yl.y + r.y * yl.x;
                }
                double2 d = Rm[i * (CG_MAXM + 1) + i];
                double dd = d.x * d.x + d.y * d.y;
                y[i] = dd > 0 ? make_double2((sacc.x * d.x + sacc.y * d.y) / dd, (sacc.y * d.x - sacc.x * d.y) / dd)
                              : make_double2(0, 0);
            }
        }
        __syncthreads();
        for (int t = r0 + threadIdx.x; t < r1; t += blockDim.x) {
            cpx<R> q = a.x[t];
            for (int i = 0; i < k; ++i) {
                const cpx<R> yi((R)(y[i].x * scale[i]), (R)(y[i].y * scale[i]));
                q = q + yi * a.V[(size_t)i * a.n + t];
            }
            a.x[t] = q;
        }
        have_x = true;
        its += k;
        // x must be complete before the next residual's matvec
        if (!grid_sync(a.st, G, a.timeout)) return;
        if (conv) break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&a.st->iters, its);
}

// Launch the persistent coarse GMRES for (Q_c - sigma) e_c = r_c (e_c from 0).
// `state` points at a zero-initialised CGState (one reduction slot).
template <typename R>
void coarse_gmres_persistent(Ctx &c, double sigma, const void *rc, void *ec, DevBuf &Vbuf, DevBuf &pbuf, void *state) {
    const int ntv = c.prm.n_tv;
    const int n = c.nagg * 2 * ntv;
    const int m = std::min(c.prm.coarse_restart, CG_MAXM);
    int dev_sms = 0;
    MG_CUDA(cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, c.device));
    int per_sm = 0;
    MG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, coarse_gmres_kernel<R>, CG_THREADS, 0));
    MG_REQUIRE(per_sm >= 1, MGEIG_ECUDA);
    int G = (n + CG_THREADS - 1) / CG_THREADS;
    G = std::max(1, std::min(G, dev_sms * per_sm));
    Vbuf.alloc((size_t)(m + 1) * n * sizeof(cpx<R>));
    pbuf.alloc((size_t)G * CG_SLOTS * sizeof(double2));
    CGArgs<R> a;
    a.nagg = c.nagg; a.ntv = ntv; a.n = n;
    for (int mu = 0; mu < 4; ++mu) a.cd[mu] = c.cdims[mu];
    a.Dc = static_cast<const cpx<R> *>(c.Dc.p);
    a.sigma = (R)sigma;
    a.b = static_cast<const cpx<R> *>(rc);
    a.x = static_cast<cpx<R> *>(ec);
    a.V = Vbuf.as<cpx<R>>();
    a.partial = pbuf.as<double2>();
    a.st = static_cast<CGState *>(state);
    a.m = m;
    a.maxiter = c.prm.coarse_maxiter;
    a.tol = c.prm.coarse_tol;
    a.timeout = 4000000000LL;   // about 2 s of SM clock per barrier wait
    void *args[] = {&a};
    TimeScope ts(c.timer, K_COARSE_SOLVE, 0);
    MG_CUDA(cudaLaunchCooperativeKernel((void *)coarse_gmres_kernel<R>, dim3(G), dim3(CG_THREADS), args, 0, c.stream));
}

template void coarse_gmres_persistent<float>(Ctx &, double, const void *, void *, DevBuf &, DevBuf &, void *);
template void coarse_gmres_persistent<double>(Ctx &, double, const void *, void *, DevBuf &, DevBuf &, void *);

}  // namespace mgeig
