// Host orchestration of the solvers (native C++ driving the kernels):
//   GMRES(m) on either level, the two-grid cycle B (Eq. 2.3, mu = 0 pre- and
//   nu post-smoothing steps), the FP64 flexible GMRES of every shifted solve
//   (Sec. 2.2: double precision FGMRES preconditioned by single precision
//   multigrid), the multigrid setup and the Rayleigh quotient iteration of
//   Algorithm 1.
//
// Scalars of the Krylov methods (Hessenberg columns, norms) are reduced on the
// device and read back once per Arnoldi step; the Givens rotations and the
// small triangular solves run on the host.
#include <chrono>
#include <cmath>
#include <algorithm>
#include <numeric>

#include <cstdlib>
#include <cstring>

#include <mutex>

#include "internal.h"

namespace mgeig {

// Progress log on stderr when the environment variable MGEIG_LOG is set.
static bool log_on() {
    static const bool on = std::getenv("MGEIG_LOG") != nullptr;
    return on;
}
static double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// ---------------------------------------------------------------------------
// device buffers, timer

void DevBuf::alloc(size_t n) {
    if (bytes >= n && p) return;
    free();
    if (n == 0) return;
    MG_CUDA(cudaMalloc(&p, n));
    bytes = n;
}

void DevBuf::free() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
}

cudaEvent_t Timer::begin(int) {
    if (next + 2 > pool.size()) {
        flush();
        while (pool.size() < next + 2) {
            cudaEvent_t e;
            MG_CUDA(cudaEventCreate(&e));
            pool.push_back(e);
        }
    }
    cudaEvent_t a = pool[next++];
    MG_CUDA(cudaEventRecord(a, stream));
    return a;
}

void Timer::end(int cls, cudaEvent_t a, double b) {
    cudaEvent_t e = pool[next++];
    MG_CUDA(cudaEventRecord(e, stream));
    pending.push_back({cls, a, e});
    bytes[cls] = b;
    if (pending.size() >= 1024) flush();
}

void Timer::flush() {
    if (!pending.empty()) {
        MG_CUDA(cudaEventSynchronize(pending.back().b));
        for (auto &p : pending) {
            float t = 0;
            MG_CUDA(cudaEventElapsedTime(&t, p.a, p.b));
            ms[p.cls] += t;
        }
        pending.clear();
    }
    next = 0;
}

void Timer::reset() {
    flush();
    for (int k = 0; k < K_NCLASS; ++k) { launches[k] = 0; ms[k] = 0; total_bytes[k] = 0; }
}

Timer::~Timer() {
    for (auto e : pool) cudaEventDestroy(e);
}

// ---------------------------------------------------------------------------
// reductions

constexpr int RED_SLOTS = 512;       // cpx<double> results on the device
// slots: Hessenberg passes H1, H2, norm HN, the persistent coarse solver's
// state CGS (status word and iteration counter), uploads from UP on
constexpr int H1 = 0, H2 = 128, HN = 256, CGS = 257, NFETCH = 258, UP = 300;

void ensure_reduction(Ctx &c, int max_vectors) {
    (void)max_vectors;
    if (!c.red_partial.p) {
        c.red_partial.alloc((size_t)(MAX_ITERATED + 8) * 1024 * sizeof(double2));   // >= (vectors + 1) x 1024 blocks
        c.red_out.alloc(RED_SLOTS * sizeof(double2));
        MG_CUDA(cudaMemset(c.red_out.p, 0, RED_SLOTS * sizeof(double2)));
        MG_CUDA(cudaMallocHost(&c.pinned, 2 * RED_SLOTS * sizeof(double2)));
    }
}

void sync(Ctx &c) { MG_CUDA(cudaStreamSynchronize(c.stream)); }

static cpx<double> *dslot(Ctx &c, int i) { return c.red_out.as<cpx<double>>() + i; }
static cpx<double> *hslot(Ctx &c, int i) { return reinterpret_cast<cpx<double> *>(c.pinned) + i; }
static cpx<double> *upslot(Ctx &c, int i) { return reinterpret_cast<cpx<double> *>(c.pinned) + RED_SLOTS + i; }

struct CoarseState { unsigned int count, gen; int status, iters; };

// copy device slots [0, n) to the host mirror and wait; every fetch also
// brings back the persistent coarse solver's state and raises its errors
static void fetch(Ctx &c, int n) {
    n = std::max(n, NFETCH);
    MG_CUDA(cudaMemcpyAsync(c.pinned, c.red_out.p, n * sizeof(double2), cudaMemcpyDeviceToHost, c.stream));
    sync(c);
    const CoarseState *cs = reinterpret_cast<const CoarseState *>(c.pinned + 2 * CGS);
    if (cs->status != 0) {
        const int code = cs->status == 1 ? MGEIG_ETIMEOUT : MGEIG_EBREAKDOWN;
        MG_CUDA(cudaMemsetAsync(dslot(c, CGS), 0, sizeof(CoarseState), c.stream));
        sync(c);
        throw Error{code};
    }
}

// upload host coefficients to device slots starting at UP
static cpx<double> *upload(Ctx &c, const std::vector<cpx<double>> &v) {
    MG_REQUIRE((int)v.size() <= RED_SLOTS - UP, MGEIG_EINVAL);
    // the previous upload may still be read by an in-flight kernel
    sync(c);
    for (size_t i = 0; i < v.size(); ++i) *upslot(c, (int)i) = v[i];
    MG_CUDA(cudaMemcpyAsync(dslot(c, UP), upslot(c, 0), v.size() * sizeof(double2), cudaMemcpyHostToDevice, c.stream));
    return dslot(c, UP);
}

static bool finite(cpx<double> z) { return std::isfinite(z.re) && std::isfinite(z.im); }

// the Gram-Schmidt building blocks on caller-owned FP64 device vectors
void blas_dot_host(Ctx &c, bool f32, int k, const void *const *X, const void *y, size_t n, double *out) {
    ensure_reduction(c, k);
    if (f32) blas_multidot<float>(c, X, k, y, n, dslot(c, H1));
    else blas_multidot<double>(c, X, k, y, n, dslot(c, H1));
    fetch(c, H1 + k);
    for (int j = 0; j < k; ++j) {
        out[2 * j] = hslot(c, H1 + j)->re;
        out[2 * j + 1] = hslot(c, H1 + j)->im;
    }
}

void blas_axpy_host(Ctx &c, bool f32, int k, const void *const *X, const double *coef, void *y, size_t n) {
    ensure_reduction(c, k);
    std::vector<cpx<double>> cv(k);
    for (int j = 0; j < k; ++j) cv[j] = cpx<double>(coef[2 * j], coef[2 * j + 1]);
    if (f32) blas_multi_axpy<float>(c, y, X, k, upload(c, cv), 1.0, n);
    else blas_multi_axpy<double>(c, y, X, k, upload(c, cv), 1.0, n);
    sync(c);
}

// ---------------------------------------------------------------------------
// workspace

struct Ctx::Work {
    int outer_m = 0, coarse_m = 0, smooth_k = 0, ntv = 0;
    bool mixed = false;
    DevBuf Wall;                 // ntv FP64 test vectors, contiguous
    DevBuf P64all;               // ntv FP64 interpolation vectors
    DevBuf PRall;                // ntv level-precision vectors (mixed only)
    std::vector<DevBuf> V64;     // FGMRES Arnoldi basis (FP64)
    std::vector<DevBuf> Z;       // FGMRES preconditioned vectors (level precision)
    DevBuf x64, t64, q64;        // FP64 temporaries
    DevBuf rR, zR, tR, eR;       // level-precision fine temporaries
    std::vector<DevBuf> S;       // GMRES smoother basis
    DevBuf rc, ec, ct;           // coarse vectors
    DevBuf cgS;                  // persistent coarse solver's global scratch
    DevBuf Wc, AWc, Edev, Einv;  // deflation: P^dag w_j, (Q_c - sigma) P^dag w_j, E, E^-1
    DevBuf Mextra, Xall;         // Algorithm 1 vectors beyond the N_tv test vectors; rotation scratch
    DevBuf Wfrozen;              // the setup's test vectors that stay in P (p_modes < N_tv)
    std::vector<void *> modes;   // iterated vectors: W[0..N_tv) then the extra ones
    std::vector<void *> Psrc;    // the N_tv vectors P is built from (W, or the first iterated vectors)
    bool defl_valid = false;
    double defl_sigma = 0;
    std::vector<void *> W, P64, P;
    // fine-grid deflation of the eigensolver's shifted solves by the iterated vectors
    DevBuf QZ64all;              // Q z_j (FP64)
    DevBuf ZRall, QZRall;        // level-precision copies of z_j and Q z_j (mixed only)
    DevBuf AZRall;               // (Q - sigma) z_j of the active subset, level precision
    DevBuf fdEinv, fdCoef;       // (Z_S^dag (Q - sigma) Z_S)^-1; coefficients c, d = E^-1 c
    std::vector<void *> QZ64, fdZ, fdQZ;   // FP64 Q z_j; level-precision z_j and Q z_j
    std::vector<void *> fdZs, fdAZs;       // the active subset: z_j and (Q - sigma) z_j
    std::vector<cpx<double>> Gz, Hz;       // Z^dag Z and Z^dag Q Z (row-major, fd_n x fd_n)
    int fd_n = 0;                          // maintained vectors (0: deflation off)
    int fd_k = 0;                          // vectors of the active deflation (0: off)
    int fg_mode = MODE_QSIGMA;             // operator of the FGMRES: Q - sigma, or D - sigma gamma5
};

static size_t f64_bytes(const Ctx &c) { return c.fine_ncpx() * sizeof(double2); }
static size_t fR_bytes(const Ctx &c) { return c.fine_ncpx() * 2 * c.level_bytes(); }
static size_t cR_bytes(const Ctx &c) { return c.coarse_ncpx() * 2 * c.level_bytes(); }

void mg_alloc(Ctx &c) {
    ensure_reduction(c, 64);
    if (!c.work) c.work = new Ctx::Work();
    Ctx::Work &w = *c.work;
    const int ntv = c.prm.n_tv;
    w.outer_m = c.prm.outer_restart;
    w.coarse_m = c.prm.coarse_restart;
    w.smooth_k = c.prm.gmres_smooth_k;
    w.ntv = ntv;
    w.mixed = c.mixed();
    w.Wall.alloc(f64_bytes(c) * ntv);
    w.P64all.alloc(f64_bytes(c) * ntv);
    if (c.mixed()) w.PRall.alloc(fR_bytes(c) * ntv);
    w.W.resize(ntv); w.P64.resize(ntv); w.P.resize(ntv);
    for (int j = 0; j < ntv; ++j) {
        w.W[j] = static_cast<char *>(w.Wall.p) + f64_bytes(c) * j;
        w.P64[j] = static_cast<char *>(w.P64all.p) + f64_bytes(c) * j;
        w.P[j] = c.mixed() ? static_cast<char *>(w.PRall.p) + fR_bytes(c) * j : w.P64[j];
    }
    w.V64.resize(w.outer_m + 1);
    for (auto &b : w.V64) b.alloc(f64_bytes(c));
    w.Z.resize(w.outer_m);
    for (auto &b : w.Z) b.alloc(fR_bytes(c));
    w.x64.alloc(f64_bytes(c)); w.t64.alloc(f64_bytes(c)); w.q64.alloc(f64_bytes(c));
    w.rR.alloc(fR_bytes(c)); w.zR.alloc(fR_bytes(c)); w.tR.alloc(fR_bytes(c)); w.eR.alloc(fR_bytes(c));
    if (c.prm.smoother == MGEIG_GMRES) {
        w.S.resize(w.smooth_k + 1);
        for (auto &b : w.S) b.alloc(fR_bytes(c));
    }
    w.rc.alloc(cR_bytes(c)); w.ec.alloc(cR_bytes(c)); w.ct.alloc(cR_bytes(c));
    w.Wc.alloc(cR_bytes(c) * ntv); w.AWc.alloc(cR_bytes(c) * ntv);
    w.Edev.alloc((size_t)ntv * ntv * sizeof(double2)); w.Einv.alloc((size_t)ntv * ntv * sizeof(double2));
    w.defl_valid = false;
    w.Psrc = w.W;
    c.Dc.alloc((size_t)9 * c.nagg * 4 * ntv * ntv * 2 * c.level_bytes());
    // periodic neighbours of every aggregate in the nine directions of the coarse stencil
    std::vector<int> nbr((size_t)9 * c.nagg);
    for (int s = 0; s < c.nagg; ++s) {
        int x[4], rem = s;
        for (int mu = 0; mu < 4; ++mu) { x[mu] = rem % c.cdims[mu]; rem /= c.cdims[mu]; }
        nbr[s] = s;
        for (int d = 1; d < 9; ++d) {
            const int mu = (d - 1) / 2, step = (d & 1) ? 1 : -1;
            int y[4] = {x[0], x[1], x[2], x[3]};
            y[mu] = (y[mu] + step + c.cdims[mu]) % c.cdims[mu];
            nbr[(size_t)d * c.nagg + s] = ((y[3] * c.cdims[2] + y[2]) * c.cdims[1] + y[1]) * c.cdims[0] + y[0];
        }
    }
    c.cnbr.alloc(nbr.size() * sizeof(int));
    MG_CUDA(cudaMemcpy(c.cnbr.p, nbr.data(), nbr.size() * sizeof(int), cudaMemcpyHostToDevice));
}

void mg_free(Ctx &c) {
    if (!c.work) return;
    Ctx::Work &w = *c.work;
    w.Wall.free(); w.P64all.free(); w.PRall.free();
    for (auto &b : w.V64) b.free();
    for (auto &b : w.Z) b.free();
    for (auto &b : w.S) b.free();
    w.x64.free(); w.t64.free(); w.q64.free();
    w.rR.free(); w.zR.free(); w.tR.free(); w.eR.free();
    w.rc.free(); w.ec.free(); w.ct.free();
    w.cgS.free();
    w.Wc.free(); w.AWc.free(); w.Edev.free(); w.Einv.free();
    w.Mextra.free(); w.Xall.free(); w.Wfrozen.free();
    w.QZ64all.free(); w.ZRall.free(); w.QZRall.free(); w.AZRall.free(); w.fdEinv.free(); w.fdCoef.free();
    delete c.work;
    c.work = nullptr;
    c.Dc.free(); c.Dc16.free(); c.Dcs.free();
    c.cnbr.free();
}

void *mg_test_vector(Ctx &c, int j) { return c.work->W[j]; }
void mg_use_test_vectors(Ctx &c) { c.work->Psrc = c.work->W; }

// ---------------------------------------------------------------------------
// Givens-based least squares of GMRES (host)

struct Hess {
    int m;
    std::vector<cpx<double>> H;   // (m+1) x m, column-major
    std::vector<double> cs;
    std::vector<cpx<double>> sn, g;
    explicit Hess(int m_) : m(m_), H((size_t)(m_ + 1) * m_), cs(m_), sn(m_), g(m_ + 1) {}
    cpx<double> &h(int i, int j) { return H[(size_t)j * (m + 1) + i]; }
    void start(double beta) { std::fill(g.begin(), g.end(), cpx<double>()); g[0] = cpx<double>(beta); }
    // column j holds the new Hessenberg column (rows 0..j+1); returns |g_{j+1}|
    double add_column(int j) {
        for (int i = 0; i < j; ++i) {
            cpx<double> a = h(i, j), b = h(i + 1, j);
            h(i, j) = cs[i] * a + sn[i] * b;
            h(i + 1, j) = cs[i] * b - conj(sn[i]) * a;
        }
        cpx<double> a = h(j, j), b = h(j + 1, j);
        double aa = std::hypot(a.re, a.im), bb = std::hypot(b.re, b.im);
        if (bb == 0) { cs[j] = 1; sn[j] = cpx<double>(); }
        else if (aa == 0) { cs[j] = 0; sn[j] = cpx<double>(1); }
        else {
            double t = std::hypot(aa, bb);
            cs[j] = aa / t;
            sn[j] = (1.0 / t) * (cpx<double>(a.re / aa, a.im / aa) * conj(b));
        }
        h(j, j) = cs[j] * a + sn[j] * b;
        h(j + 1, j) = cpx<double>();
        g[j + 1] = -(conj(sn[j]) * g[j]);
        g[j] = cs[j] * g[j];
        return std::hypot(g[j + 1].re, g[j + 1].im);
    }
    std::vector<cpx<double>> solve(int k) {
        std::vector<cpx<double>> y(k);
        for (int i = k - 1; i >= 0; --i) {
            cpx<double> s = g[i];
            for (int l = i + 1; l < k; ++l) s = s - h(i, l) * y[l];
            cpx<double> d = h(i, i);
            double dd = d.re * d.re + d.im * d.im;
            y[i] = dd > 0 ? (1.0 / dd) * (s * conj(d)) : cpx<double>();
        }
        return y;
    }
};

// w <- w - X X^dag w for the orthonormal X[0..k) (classical Gram-Schmidt).  The
// first pass also returns ||w||^2; a second pass runs only when the first one
// removed more than half of ||w||^2 (the Daniel-Gragg-Kaufman-Stewart
// criterion ||w'|| < ||w|| / sqrt 2), otherwise ||w'||^2 = ||w||^2 - sum |h_i|^2.
// h[0..k) receives the summed coefficients; returns ||w'||^2.
template <typename R>
static double gs_dgks(Ctx &c, const void *const *X, int k, void *w, size_t n, cpx<double> *h) {
    std::vector<const void *> Xw(X, X + k);
    Xw.push_back(w);
    blas_multidot<R>(c, Xw.data(), k + 1, w, n, dslot(c, H1));
    if (k > 0) blas_multi_axpy<R>(c, w, X, k, dslot(c, H1), -1.0, n);
    fetch(c, H1 + k + 1);
    const double ww = hslot(c, H1 + k)->re;
    double s = 0;
    for (int i = 0; i < k; ++i) {
        h[i] = *hslot(c, H1 + i);
        MG_REQUIRE(finite(h[i]), MGEIG_EBREAKDOWN);
        s += h[i].re * h[i].re + h[i].im * h[i].im;
    }
    MG_REQUIRE(std::isfinite(ww), MGEIG_EBREAKDOWN);
    if (k == 0) return ww;
    if (ww - s > 0.5 * ww) return ww - s;
    blas_multidot<R>(c, X, k, w, n, dslot(c, H2));
    blas_multi_axpy<R>(c, w, X, k, dslot(c, H2), -1.0, n);
    blas_norm2<R>(c, w, n, dslot(c, HN));
    fetch(c, HN + 1);
    for (int i = 0; i < k; ++i) {
        h[i] = h[i] + *hslot(c, H2 + i);
        MG_REQUIRE(finite(h[i]), MGEIG_EBREAKDOWN);
    }
    return hslot(c, HN)->re;
}

// Arnoldi step: w is orthogonalised against basis[0..j] (gs_dgks),
// Hessenberg column j filled (rows 0..j+1).  Returns the norm of w.
template <typename R>
static double arnoldi_step(Ctx &c, std::vector<void *> &basis, int j, void *w, size_t n, Hess &H) {
    std::vector<const void *> X(basis.begin(), basis.begin() + j + 1);
    std::vector<cpx<double>> h(j + 1);
    const double w2 = gs_dgks<R>(c, X.data(), j + 1, w, n, h.data());
    for (int i = 0; i <= j; ++i) H.h(i, j) = h[i];
    double nrm = std::sqrt(std::max(0.0, w2));
    MG_REQUIRE(std::isfinite(nrm), MGEIG_EBREAKDOWN);
    H.h(j + 1, j) = cpx<double>(nrm);
    return nrm;
}

// Restarted GMRES on flat arrays of precision R.  x is the initial guess when
// x_nonzero, else it is set to the solution from zero.  tol = 0 runs exactly
// maxiter steps.  Returns the iteration count.
template <typename R, typename Op>
static int gmres(Ctx &c, Op op, const void *b, void *x, bool x_nonzero, size_t n, double tol, int restart,
                 int maxiter, std::vector<DevBuf> &basis_buf) {
    std::vector<void *> basis;
    for (auto &d : basis_buf) basis.push_back(d.p);
    const int m = std::min<int>(restart, (int)basis.size() - 1);
    blas_norm2<R>(c, b, n, dslot(c, HN));
    fetch(c, HN + 1);
    const double bnorm = std::sqrt(hslot(c, HN)->re);
    MG_REQUIRE(std::isfinite(bnorm), MGEIG_EBREAKDOWN);
    if (!x_nonzero) blas_zero<R>(c, x, n);
    if (bnorm == 0) return 0;
    int its = 0;
    bool have_x = x_nonzero;
    Hess H(m);
    while (its < maxiter) {
        if (have_x) {
            op(x, basis[0]);
            // basis0 = b - A x
            blas_scale<R>(c, cpx<double>(-1), basis[0], n);
            blas_axpy<R>(c, cpx<double>(1), b, basis[0], n);
        } else {
            blas_copy<R>(c, b, basis[0], n);
        }
        blas_norm2<R>(c, basis[0], n, dslot(c, HN));
        fetch(c, HN + 1);
        const double beta = std::sqrt(hslot(c, HN)->re);
        MG_REQUIRE(std::isfinite(beta), MGEIG_EBREAKDOWN);
        if (beta <= tol * bnorm || beta == 0) break;
        blas_scale<R>(c, cpx<double>(1.0 / beta), basis[0], n);
        H.start(beta);
        const int mm = std::min(m, maxiter - its);
        int k = 0;
        double est = beta;
        for (int j = 0; j < mm; ++j) {
            op(basis[j], basis[j + 1]);
            const double nrm = arnoldi_step<R>(c, basis, j, basis[j + 1], n, H);
            est = H.add_column(j);
            k = j + 1;
            if (est <= tol * bnorm || nrm == 0) break;
            blas_scale<R>(c, cpx<double>(1.0 / nrm), basis[j + 1], n);
        }
        std::vector<cpx<double>> y = H.solve(k);
        std::vector<const void *> X(basis.begin(), basis.begin() + k);
        blas_multi_axpy<R>(c, x, X.data(), k, upload(c, y), 1.0, n);
        have_x = true;
        its += k;
        if (est <= tol * bnorm) break;
    }
    return its;
}

// ---------------------------------------------------------------------------
// the two-grid cycle

// complex Gauss-Jordan inverse with partial pivoting (row-major n x n)
static bool invert(int n, std::vector<cpx<double>> A, std::vector<cpx<double>> &inv) {
    inv.assign((size_t)n * n, cpx<double>());
    for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = cpx<double>(1);
    for (int col = 0; col < n; ++col) {
        int piv = col;
        double best = -1;
        for (int r = col; r < n; ++r) {
            cpx<double> z = A[(size_t)r * n + col];
            double m = std::hypot(z.re, z.im);
            if (m > best) { best = m; piv = r; }
        }
        if (!(best > 0) || !std::isfinite(best)) return false;
        if (piv != col)
            for (int k = 0; k < n; ++k) {
                std::swap(A[(size_t)piv * n + k], A[(size_t)col * n + k]);
                std::swap(inv[(size_t)piv * n + k], inv[(size_t)col * n + k]);
            }
        cpx<double> d = A[(size_t)col * n + col];
        double dd = d.re * d.re + d.im * d.im;
        cpx<double> di(d.re / dd, -d.im / dd);
        for (int k = 0; k < n; ++k) {
            A[(size_t)col * n + k] = A[(size_t)col * n + k] * di;
            inv[(size_t)col * n + k] = inv[(size_t)col * n + k] * di;
        }
        for (int r = 0; r < n; ++r) {
            if (r == col) continue;
            cpx<double> f = A[(size_t)r * n + col];
            if (f.re == 0 && f.im == 0) continue;
            for (int k = 0; k < n; ++k) {
                A[(size_t)r * n + k] = A[(size_t)r * n + k] - f * A[(size_t)col * n + k];
                inv[(size_t)r * n + k] = inv[(size_t)r * n + k] - f * inv[(size_t)col * n + k];
            }
        }
    }
    return true;
}

// (Q_c - sigma) W_c and E^-1 = (W_c^dag (Q_c - sigma) W_c)^-1 for the current
// test vectors and shift (cached until the shift or P changes)
template <typename R>
static void deflation_prepare(Ctx &c, double sigma) {
    Ctx::Work &w = *c.work;
    if (!c.prm.coarse_deflate || c.in_setup || (w.defl_valid && w.defl_sigma == sigma)) return;
    const int k = c.prm.n_tv;
    const size_t n = c.coarse_ncpx(), vb = cR_bytes(c);
    std::vector<const void *> Wp(k);
    for (int i = 0; i < k; ++i) Wp[i] = static_cast<const char *>(w.Wc.p) + vb * i;
    for (int j = 0; j < k; ++j) {
        void *awj = static_cast<char *>(w.AWc.p) + vb * j;
        coarse_apply<R>(c, c.Dc.p, sigma, Wp[j], awj, false);
        blas_multidot<R>(c, Wp.data(), k, awj, n, w.Edev.as<cpx<double>>() + (size_t)j * k);
    }
    std::vector<cpx<double>> Ecol((size_t)k * k), E((size_t)k * k), Ei;
    MG_CUDA(cudaMemcpyAsync(Ecol.data(), w.Edev.p, Ecol.size() * sizeof(double2), cudaMemcpyDeviceToHost, c.stream));
    sync(c);
    for (int j = 0; j < k; ++j)
        for (int i = 0; i < k; ++i) E[(size_t)i * k + j] = Ecol[(size_t)j * k + i];   // E_ij = <W_i, A W_j>
    MG_REQUIRE(invert(k, E, Ei), MGEIG_EBREAKDOWN);
    MG_CUDA(cudaMemcpyAsync(w.Einv.p, Ei.data(), Ei.size() * sizeof(double2), cudaMemcpyHostToDevice, c.stream));
    sync(c);
    w.defl_valid = true;
    w.defl_sigma = sigma;
}

// Coarse solve (Q_c - sigma) e = r_c: one persistent cooperative launch (GMRES
// on the deflated D_c form, see coarse_gmres.cu)
template <typename R>
static void coarse_solve(Ctx &c, double sigma, const void *rc, void *ec) {
    Ctx::Work &w = *c.work;
    deflation_prepare<R>(c, sigma);
    CoarseSolveBufs B;
    B.scratch = &w.cgS;
    B.state = dslot(c, CGS);
    B.k = (c.prm.coarse_deflate && !c.in_setup) ? c.prm.n_tv : 0;
    B.W = w.Wc.p;
    B.AW = w.AWc.p;
    B.Einv = w.Einv.p;
    coarse_gmres_persistent<R>(c, B, sigma, rc, ec);
}

// Adds the persistent coarse solver's iterations since the last call to the
// stats (and their coarse-operator bytes to the timer); raises its errors.
void coarse_iters_take(Ctx &c) {
    if (!c.red_out.p) return;
    CoarseState s;
    MG_CUDA(cudaMemcpyAsync(&s, dslot(c, CGS), sizeof(s), cudaMemcpyDeviceToHost, c.stream));
    sync(c);
    MG_CUDA(cudaMemsetAsync(reinterpret_cast<char *>(dslot(c, CGS)) + offsetof(CoarseState, iters), 0, sizeof(int),
                            c.stream));
    if (s.status != 0) MG_CUDA(cudaMemsetAsync(dslot(c, CGS), 0, sizeof(CoarseState), c.stream));
    sync(c);
    c.st.coarse_iters += s.iters;
    const double ntv = c.prm.n_tv;
    c.timer.total_bytes[K_COARSE_SOLVE] += (double)s.iters * 9.0 * c.nagg * 4 * ntv * ntv * 2 * c.level_bytes();
    if (s.status == 1) throw Error{MGEIG_ETIMEOUT};
    if (s.status != 0) throw Error{MGEIG_EBREAKDOWN};
}

// z = B r for fine vectors r, z of precision R (r is not modified)
template <typename R>
static void mg_cycle(Ctx &c, double sigma, const void *r, void *z) {
    Ctx::Work &w = *c.work;
    c.st.mg_cycles += 1;
    restrict_vec<R>(c, (const void *const *)w.P.data(), r, w.rc.p);
    coarse_solve<R>(c, sigma, w.rc.p, w.ec.p);
    prolong_vec<R>(c, (const void *const *)w.P.data(), w.ec.p, z);
    if constexpr (sizeof(R) == 4) {
        if (c.prm.smoother == MGEIG_LEARNED && !c.in_setup) {
            // z += M(r - (Q - sigma) z): the learned smoother on the residual of the coarse correction
            const size_t n = c.fine_ncpx();
            apply_fine<R>(c, MODE_QSIGMA, sigma, z, w.tR.p);
            blas_scale<R>(c, cpx<double>(-1), w.tR.p, n);
            blas_axpy<R>(c, cpx<double>(1), r, w.tR.p, n);
            net_smooth(c, w.tR.p, z);
            return;
        }
    }
    if (c.prm.smoother == MGEIG_SAP || c.prm.smoother == MGEIG_LEARNED) {
        for (int k = 0; k < c.prm.sap_cycles; ++k) {
            sap_sweep<R>(c, 0, sigma, r, true, z);
            sap_sweep<R>(c, 1, sigma, r, true, z);
        }
    } else {
        const size_t n = c.fine_ncpx();
        auto op = [&](const void *x, void *y) { apply_fine<R>(c, MODE_QSIGMA, sigma, x, y); };
        for (int k = 0; k < c.prm.smooth_steps; ++k) {
            // tR = r - A z ; eR = GMRES_k(A, tR) ; z += eR
            apply_fine<R>(c, MODE_QSIGMA, sigma, z, w.tR.p);
            blas_scale<R>(c, cpx<double>(-1), w.tR.p, n);
            blas_axpy<R>(c, cpx<double>(1), r, w.tR.p, n);
            gmres<R>(c, op, w.tR.p, w.eR.p, false, n, 0.0, c.prm.gmres_smooth_k, c.prm.gmres_smooth_k, w.S);
            blas_axpy<R>(c, cpx<double>(1), w.eR.p, z, n);
        }
    }
}

// ---------------------------------------------------------------------------
// P and the coarse operator from the test vectors

void mg_rebuild(Ctx &c) {
    Ctx::Work &w = *c.work;
    const int ntv = c.prm.n_tv;
    const size_t vb = cR_bytes(c);
    if (c.mixed()) {
        build_interp<float>(c, (const void *const *)w.Psrc.data(), ntv, w.P.data());
        build_coarse<float>(c, (const void *const *)w.P.data(), c.Dc.p);
        if (c.prm.coarse_links != MGEIG_LINKS_LEVEL) compress_coarse(c);
        // coarse images P^dag w_j of the test vectors (the deflation space)
        for (int j = 0; j < ntv; ++j) {
            convert_f64_to_f32(c, w.Psrc[j], w.rR.p, c.fine_ncpx());
            restrict_vec<float>(c, (const void *const *)w.P.data(), w.rR.p, static_cast<char *>(w.Wc.p) + vb * j);
        }
    } else {
        build_interp<double>(c, (const void *const *)w.Psrc.data(), ntv, w.P64.data());
        build_coarse<double>(c, (const void *const *)w.P.data(), c.Dc.p);
        for (int j = 0; j < ntv; ++j)
            restrict_vec<double>(c, (const void *const *)w.P.data(), w.Psrc[j], static_cast<char *>(w.Wc.p) + vb * j);
    }
    w.defl_valid = false;
}

// Gram-Schmidt (each step twice) of FP64 vectors v[0..n) in place
static void orthonormalise(Ctx &c, std::vector<void *> &v, int n) {
    const size_t N = c.fine_ncpx();
    for (int j = 0; j < n; ++j) {
        std::vector<const void *> X(v.begin(), v.begin() + j);
        std::vector<cpx<double>> h(j);
        const double nrm = std::sqrt(std::max(0.0, gs_dgks<double>(c, X.data(), j, v[j], N, h.data())));
        MG_REQUIRE(std::isfinite(nrm) && nrm > 0, MGEIG_EBREAKDOWN);
        blas_scale<double>(c, cpx<double>(1.0 / nrm), v[j], N);
    }
}

// Gram-Schmidt (each step twice) of v[from..n) against all earlier vectors
static void orthonormalise_from(Ctx &c, std::vector<void *> &v, int from) {
    const size_t N = c.fine_ncpx();
    const int n = (int)v.size();
    for (int j = from; j < n; ++j) {
        std::vector<const void *> X(v.begin(), v.begin() + j);
        std::vector<cpx<double>> h(j);
        const double nrm = std::sqrt(std::max(0.0, gs_dgks<double>(c, X.data(), j, v[j], N, h.data())));
        MG_REQUIRE(std::isfinite(nrm) && nrm > 0, MGEIG_EBREAKDOWN);
        blas_scale<double>(c, cpx<double>(1.0 / nrm), v[j], N);
    }
}

// one preconditioner application on an FP64 fine vector, FP64 result
template <typename R>
static void mg_cycle_f64(Ctx &c, double sigma, const void *r64, void *z64) {
    Ctx::Work &w = *c.work;
    if (sizeof(R) == 4) {
        convert_f64_to_f32(c, r64, w.rR.p, c.fine_ncpx());
        mg_cycle<R>(c, sigma, w.rR.p, w.zR.p);
        convert_f32_to_f64(c, w.zR.p, z64, c.fine_ncpx());
    } else {
        mg_cycle<R>(c, sigma, r64, z64);
    }
}

template <typename R>
static void smooth_random(Ctx &c, void *w64) {
    Ctx::Work &w = *c.work;
    const size_t n = c.fine_ncpx();
    void *rhs = w.rR.p, *z = w.zR.p;
    if (sizeof(R) == 4) convert_f64_to_f32(c, w64, rhs, n);
    else blas_copy<double>(c, w64, rhs, n);
    if (c.prm.smoother != MGEIG_GMRES) {
        blas_zero<R>(c, z, n);
        for (int k = 0; k < c.prm.setup_smooth; ++k) {
            sap_sweep<R>(c, 0, 0.0, rhs, true, z);
            sap_sweep<R>(c, 1, 0.0, rhs, true, z);
        }
    } else {
        auto op = [&](const void *x, void *y) { apply_fine<R>(c, MODE_QSIGMA, 0.0, x, y); };
        gmres<R>(c, op, rhs, z, false, n, 0.0, c.prm.gmres_smooth_k, c.prm.gmres_smooth_k * c.prm.setup_smooth, w.S);
    }
    if (sizeof(R) == 4) convert_f32_to_f64(c, z, w64, n);
    else blas_copy<double>(c, z, w64, n);
}

template <typename R>
static void setup_impl(Ctx &c, uint64_t seed) {
    Ctx::Work &w = *c.work;
    const int ntv = c.prm.n_tv;
    w.Psrc = w.W;
    random_spinors(c, seed, w.Wall.p, ntv, 0x5EED0001u);
    c.setup_seed = seed;
    for (int j = 0; j < ntv; ++j) smooth_random<R>(c, w.W[j]);
    orthonormalise(c, w.W, ntv);
    mg_rebuild(c);
    for (int it = 0; it < c.prm.setup_iters; ++it) {
        const double t0 = now_s();
        for (int j = 0; j < ntv; ++j) {
            mg_cycle_f64<R>(c, 0.0, w.W[j], w.t64.p);
            blas_copy<double>(c, w.t64.p, w.W[j], c.fine_ncpx());
        }
        orthonormalise(c, w.W, ntv);
        mg_rebuild(c);
        if (log_on()) {
            const long long ci = c.st.coarse_iters;
            coarse_iters_take(c);
            fprintf(stderr, "mgeig setup iter %d coarse %lld %.3fs\n", it, c.st.coarse_iters - ci, now_s() - t0);
        }
    }
    sync(c);
}

void setup(Ctx &c, uint64_t seed) {
    c.in_setup = true;
    try {
        if (c.mixed()) setup_impl<float>(c, seed);
        else setup_impl<double>(c, seed);
    } catch (...) {
        c.in_setup = false;
        throw;
    }
    c.in_setup = false;
    c.have_setup = true;
}

// ---------------------------------------------------------------------------
// Fine-grid deflation of the shifted solves of Algorithm 1 by the iterated
// vectors Z = [z_1 .. z_k] (the current eigenvector approximations and guards).
// Near an eigenvalue, Q - sigma is nearly singular on the eigenvector being
// refined and, inside a cluster, on its neighbours; only N_tv of them are in P.
// With E = Z^dag (Q - sigma) Z (FP64, from the FP64 products Z^dag Z and
// Z^dag Q Z) the preconditioner of the outer FGMRES becomes
//     z = Z E^-1 Z^dag r + B (r - (Q - sigma) Z E^-1 Z^dag r),
// so span(Z) is solved exactly (Galerkin) and the two-grid method B only sees
// the deflated residual.  The iteration still solves (Q - sigma) x = v.

// Q z_i, its level-precision copies and row/column i of Z^dag Z, Z^dag Q Z: the
// entries j < upto (all of them after z_i changed; j <= i when every row is
// rebuilt in order, the Hermitian matrices giving the rest)
static void fdefl_update(Ctx &c, const std::vector<void *> &M, int i, int upto = -1) {
    Ctx::Work &w = *c.work;
    const size_t N = c.fine_ncpx();
    const int k = upto < 0 ? w.fd_n : upto;
    apply_fine<double>(c, MODE_QSIGMA, 0.0, M[i], w.QZ64[i]);
    std::vector<const void *> X(M.begin(), M.begin() + k);
    blas_multidot<double>(c, X.data(), k, M[i], N, dslot(c, H1));
    blas_multidot<double>(c, X.data(), k, w.QZ64[i], N, dslot(c, H2));
    fetch(c, H2 + k);
    const int kk = w.fd_n;   // the matrices' leading dimension
    for (int j = 0; j < k; ++j) {
        const cpx<double> g = *hslot(c, H1 + j), h = *hslot(c, H2 + j);   // <z_j, z_i>, <z_j, Q z_i>
        w.Gz[(size_t)j * kk + i] = g;
        w.Gz[(size_t)i * kk + j] = conj(g);
        w.Hz[(size_t)j * kk + i] = h;
        w.Hz[(size_t)i * kk + j] = conj(h);   // Q is Hermitian
    }
    w.Gz[(size_t)i * kk + i] = cpx<double>(w.Gz[(size_t)i * kk + i].re);
    w.Hz[(size_t)i * kk + i] = cpx<double>(w.Hz[(size_t)i * kk + i].re);
    if (c.mixed()) {
        convert_f64_to_f32(c, M[i], w.fdZ[i], N);
        convert_f64_to_f32(c, w.QZ64[i], w.fdQZ[i], N);
    } else {
        w.fdZ[i] = M[i];
        w.fdQZ[i] = w.QZ64[i];
    }
}

static void fdefl_all(Ctx &c, const std::vector<void *> &M) {
    for (int i = 0; i < c.work->fd_n; ++i) fdefl_update(c, M, i, i + 1);
}

static void fdefl_begin(Ctx &c, const std::vector<void *> &M, int k) {
    Ctx::Work &w = *c.work;
    w.fd_n = w.fd_k = 0;
    if (!c.prm.fine_deflate) return;
    MG_REQUIRE(k >= 1 && k <= MAX_ITERATED, MGEIG_EINVAL);
    w.QZ64all.alloc(f64_bytes(c) * k);
    w.AZRall.alloc(fR_bytes(c) * k);
    w.QZ64.resize(k);
    w.fdZ.resize(k);
    w.fdQZ.resize(k);
    for (int j = 0; j < k; ++j) w.QZ64[j] = static_cast<char *>(w.QZ64all.p) + f64_bytes(c) * j;
    if (c.mixed()) {
        w.ZRall.alloc(fR_bytes(c) * k);
        w.QZRall.alloc(fR_bytes(c) * k);
        for (int j = 0; j < k; ++j) {
            w.fdZ[j] = static_cast<char *>(w.ZRall.p) + fR_bytes(c) * j;
            w.fdQZ[j] = static_cast<char *>(w.QZRall.p) + fR_bytes(c) * j;
        }
    }
    w.fdEinv.alloc((size_t)MAX_ITERATED * MAX_ITERATED * sizeof(double2));
    w.fdCoef.alloc((size_t)3 * MAX_ITERATED * sizeof(double2));
    w.Gz.assign((size_t)k * k, cpx<double>());
    w.Hz.assign((size_t)k * k, cpx<double>());
    w.fd_n = k;
    fdefl_all(c, M);
}

static void fdefl_end(Ctx &c) {
    Ctx::Work &w = *c.work;
    w.fd_n = w.fd_k = 0;
    w.QZ64all.free(); w.ZRall.free(); w.QZRall.free(); w.AZRall.free(); w.fdEinv.free(); w.fdCoef.free();
    w.QZ64.clear(); w.fdZ.clear(); w.fdQZ.clear(); w.fdZs.clear(); w.fdAZs.clear();
}

// The deflation space of the solve for vector i at shift sigma: z_i and every
// z_j whose Rayleigh quotient theta_j = <z_j, Q z_j> / <z_j, z_j> lies within
// fine_deflate_radius of sigma (all iterated vectors when the radius is < 0);
// E^-1 = (Z^dag Q Z - sigma Z^dag Z)^-1 and (Q - sigma) Z in the level precision.
template <typename R>
static void fdefl_prepare(Ctx &c, double sigma, int i) {
    Ctx::Work &w = *c.work;
    const int nz = w.fd_n;
    w.fd_k = 0;
    if (!nz) return;
    const size_t N = c.fine_ncpx();
    const double rad = c.prm.fine_deflate_radius;
    std::vector<int> S{i};
    for (int j = 0; j < nz; ++j) {
        if (j == i) continue;
        const double theta = w.Hz[(size_t)j * nz + j].re / w.Gz[(size_t)j * nz + j].re;
        if (rad < 0 || std::fabs(theta - sigma) <= rad) S.push_back(j);
    }
    const int k = (int)S.size();
    std::vector<cpx<double>> E((size_t)k * k), Ei;
    for (int a = 0; a < k; ++a)
        for (int b = 0; b < k; ++b) {
            const size_t q = (size_t)S[a] * nz + S[b];
            E[(size_t)a * k + b] = w.Hz[q] - cpx<double>(sigma) * w.Gz[q];
        }
    MG_REQUIRE(invert(k, E, Ei), MGEIG_EBREAKDOWN);
    MG_CUDA(cudaMemcpyAsync(w.fdEinv.p, Ei.data(), Ei.size() * sizeof(double2), cudaMemcpyHostToDevice, c.stream));
    w.fdZs.resize(k);
    w.fdAZs.resize(k);
    for (int a = 0; a < k; ++a) {
        w.fdZs[a] = w.fdZ[S[a]];
        w.fdAZs[a] = static_cast<char *>(w.AZRall.p) + fR_bytes(c) * a;
        blas_copy<R>(c, w.fdQZ[S[a]], w.fdAZs[a], N);
        blas_axpy<R>(c, cpx<double>(-sigma), w.fdZs[a], w.fdAZs[a], N);
    }
    sync(c);
    w.fd_k = k;
}

// z = M r for the FP64 Arnoldi vector v (z in the level precision R): the
// two-grid cycle, deflated by Z when the eigensolver has set it up
template <typename R>
static void precondition(Ctx &c, double sigma, const void *v64, void *z) {
    Ctx::Work &w = *c.work;
    const size_t n = c.fine_ncpx();
    const int k = w.fd_k;
    const bool dsys = w.fg_mode == MODE_DSIGMA;
    if (sizeof(R) == 4) convert_f64_to_f32(c, v64, w.rR.p, n);
    else if (k || dsys) blas_copy<double>(c, v64, w.rR.p, n);
    // for D - sigma gamma5 = gamma5 (Q - sigma) the preconditioner is B gamma5
    // (the lower spins are the second half of either layout: FP64 [12][V], FP32 float4 [6][V])
    if (dsys) blas_scale<R>(c, cpx<double>(-1), static_cast<char *>(w.rR.p) + n / 2 * sizeof(cpx<R>), n / 2);
    const void *r = (sizeof(R) == 4 || k || dsys) ? w.rR.p : v64;
    cpx<double> *cf = w.fdCoef.as<cpx<double>>();
    cpx<double> *d = cf + MAX_ITERATED, *unused = cf + 2 * MAX_ITERATED;
    if (k) {
        blas_multidot<R>(c, (const void *const *)w.fdZs.data(), k, w.rR.p, n, cf);           // Z^dag r
        small_gemv(c, w.fdEinv.as<cpx<double>>(), k, cf, 0.0, d, unused);                   // d = E^-1 Z^dag r
        blas_multi_axpy<R>(c, w.rR.p, (const void *const *)w.fdAZs.data(), k, d, -1.0, n);  // r -= (Q - sigma) Z d
    }
    mg_cycle<R>(c, sigma, r, z);
    if (k) blas_multi_axpy<R>(c, z, (const void *const *)w.fdZs.data(), k, d, 1.0, n);      // z += Z d
}

// ---------------------------------------------------------------------------
// FGMRES (FP64) with the two-grid preconditioner

template <typename R>
static int fgmres_impl(Ctx &c, double sigma, const void *b, void *x, double tol, int maxiter) {
    Ctx::Work &w = *c.work;
    const size_t n = c.fine_ncpx();
    const int m = w.outer_m;
    std::vector<void *> V;
    for (auto &d : w.V64) V.push_back(d.p);
    blas_norm2<double>(c, b, n, dslot(c, HN));
    fetch(c, HN + 1);
    const double bnorm = std::sqrt(hslot(c, HN)->re);
    MG_REQUIRE(std::isfinite(bnorm), MGEIG_EBREAKDOWN);
    blas_zero<double>(c, x, n);
    if (bnorm == 0) return MGEIG_OK;
    int its = 0;
    bool have_x = false;
    Hess H(m);
    while (its < maxiter) {
        if (have_x) {
            apply_fine<double>(c, w.fg_mode, sigma, x, V[0]);
            blas_scale<double>(c, cpx<double>(-1), V[0], n);
            blas_axpy<double>(c, cpx<double>(1), b, V[0], n);
        } else {
            blas_copy<double>(c, b, V[0], n);
        }
        blas_norm2<double>(c, V[0], n, dslot(c, HN));
        fetch(c, HN + 1);
        const double beta = std::sqrt(hslot(c, HN)->re);
        MG_REQUIRE(std::isfinite(beta), MGEIG_EBREAKDOWN);
        if (beta <= tol * bnorm) return MGEIG_OK;
        blas_scale<double>(c, cpx<double>(1.0 / beta), V[0], n);
        H.start(beta);
        const int mm = std::min(m, maxiter - its);
        int k = 0;
        double est = beta;
        for (int j = 0; j < mm; ++j) {
            void *zj = w.Z[j].p;
            precondition<R>(c, sigma, V[j], zj);
            if (sizeof(R) == 4) apply_fine_f64_from_f32(c, w.fg_mode, sigma, zj, V[j + 1]);
            else apply_fine<double>(c, w.fg_mode, sigma, zj, V[j + 1]);
            const double nrm = arnoldi_step<double>(c, V, j, V[j + 1], n, H);
            est = H.add_column(j);
            k = j + 1;
            c.st.outer_iters += 1;
            if (est <= tol * bnorm || nrm == 0) break;
            blas_scale<double>(c, cpx<double>(1.0 / nrm), V[j + 1], n);
        }
        std::vector<cpx<double>> y = H.solve(k);
        for (int i = 0; i < k; ++i) blas_axpy_to_f64<R>(c, y[i], w.Z[i].p, x, n);
        have_x = true;
        its += k;
        if (est <= tol * bnorm) return MGEIG_OK;
    }
    return MGEIG_ENOCONV;
}

// (D - sigma gamma5) x = b, the non-Hermitian system of DD-alpha-AMG (Sec. 2),
// by the same FGMRES with the preconditioner B gamma5 (D_sigma^-1 = (Q - sigma)^-1 gamma5)
int fgmres_solve_d(Ctx &c, double sigma, const void *b64, void *x64, double tol) {
    Ctx::Work &w = *c.work;
    w.fg_mode = MODE_DSIGMA;
    struct Reset { Ctx::Work &w; ~Reset() { w.fg_mode = MODE_QSIGMA; } } reset{w};
    return fgmres_solve(c, sigma, b64, x64, tol);
}

int fgmres_solve(Ctx &c, double sigma, const void *b64, void *x64, double tol, int maxiter) {
    c.st.solves += 1;
    if (maxiter <= 0) maxiter = c.prm.outer_maxiter;
    return c.mixed() ? fgmres_impl<float>(c, sigma, b64, x64, tol, maxiter)
                     : fgmres_impl<double>(c, sigma, b64, x64, tol, maxiter);
}

// ---------------------------------------------------------------------------
// small dense Hermitian eigenproblem (cyclic Jacobi), for the Ritz rotation

static void herm_eig(int n, std::vector<cpx<double>> A, std::vector<double> &w, std::vector<cpx<double>> &Vm) {
    auto a = [&](int i, int j) -> cpx<double> & { return A[(size_t)i * n + j]; };
    Vm.assign((size_t)n * n, cpx<double>());
    for (int i = 0; i < n; ++i) Vm[(size_t)i * n + i] = cpx<double>(1);
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0, tot = 0;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) {
                double m2 = a(i, j).re * a(i, j).re + a(i, j).im * a(i, j).im;
                tot += m2;
                if (i != j) off += m2;
            }
        if (off <= 1e-32 * tot || off == 0) break;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) {
                cpx<double> apq = a(p, q);
                double mag = std::hypot(apq.re, apq.im);
                if (mag == 0) continue;
                cpx<double> e(apq.re / mag, apq.im / mag);   // e^{i phi}
                double app = a(p, p).re, aqq = a(q, q).re;
                double theta = (aqq - app) / (2 * mag);
                double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1));
                double cth = 1 / std::sqrt(t * t + 1), sth = t * cth;
                // G = [[c, s], [-s e^{-i phi}, c e^{-i phi}]] on (p, q); A <- G^dag A G, V <- V G
                cpx<double> em = conj(e);
                for (int k = 0; k < n; ++k) {
                    cpx<double> akp = a(k, p), akq = a(k, q);
                    a(k, p) = cth * akp - sth * (em * akq);
                    a(k, q) = sth * akp + cth * (em * akq);
                    cpx<double> vkp = Vm[(size_t)k * n + p], vkq = Vm[(size_t)k * n + q];
                    Vm[(size_t)k * n + p] = cth * vkp - sth * (em * vkq);
                    Vm[(size_t)k * n + q] = sth * vkp + cth * (em * vkq);
                }
                for (int k = 0; k < n; ++k) {
                    cpx<double> apk = a(p, k), aqk = a(q, k);
                    a(p, k) = cth * apk - sth * (e * aqk);
                    a(q, k) = sth * apk + cth * (e * aqk);
                }
            }
    }
    w.resize(n);
    for (int i = 0; i < n; ++i) w[i] = a(i, i).re;
}

// Ritz vectors of Q in span(X[0..n)), ordered by |theta| then theta, written
// back into X[0..n).  Scratch: the Xall vector set.
static void ritz_rotate(Ctx &c, std::vector<void *> &Xv, int n) {
    Ctx::Work &w = *c.work;
    const size_t N = c.fine_ncpx();
    w.Xall.alloc(f64_bytes(c) * n);
    std::vector<cpx<double>> H((size_t)n * n);
    std::vector<const void *> X(Xv.begin(), Xv.begin() + n);
    for (int j = 0; j < n; ++j) {
        apply_fine<double>(c, MODE_QSIGMA, 0.0, Xv[j], w.q64.p);
        blas_multidot<double>(c, X.data(), n, w.q64.p, N, dslot(c, H1));
        fetch(c, n);
        for (int i = 0; i < n; ++i) H[(size_t)i * n + j] = *hslot(c, H1 + i);
    }
    for (int i = 0; i < n; ++i)
        for (int j = i; j < n; ++j) {
            cpx<double> s = 0.5 * (H[(size_t)i * n + j] + conj(H[(size_t)j * n + i]));
            H[(size_t)i * n + j] = s;
            H[(size_t)j * n + i] = conj(s);
        }
    std::vector<double> th;
    std::vector<cpx<double>> Y;
    herm_eig(n, H, th, Y);
    std::vector<int> ord(n);
    std::iota(ord.begin(), ord.end(), 0);
    std::sort(ord.begin(), ord.end(), [&](int a, int b) {
        double fa = std::fabs(th[a]), fb = std::fabs(th[b]);
        return fa != fb ? fa < fb : th[a] < th[b];
    });
    for (int k = 0; k < n; ++k) {
        std::vector<cpx<double>> coef(n);
        for (int i = 0; i < n; ++i) coef[i] = Y[(size_t)i * n + ord[k]];
        void *dst = static_cast<char *>(w.Xall.p) + f64_bytes(c) * k;
        blas_zero<double>(c, dst, N);
        blas_multi_axpy<double>(c, dst, X.data(), n, upload(c, coef), 1.0, N);
    }
    for (int k = 0; k < n; ++k) blas_copy<double>(c, static_cast<char *>(w.Xall.p) + f64_bytes(c) * k, Xv[k], N);
}

// lambda = <v|Q v>, eps^2 = ||Q v - lambda v||^2 ; returns (lambda, eps)
static std::pair<double, double> rayleigh(Ctx &c, const void *v) {
    Ctx::Work &w = *c.work;
    const size_t N = c.fine_ncpx();
    apply_fine<double>(c, MODE_QSIGMA, 0.0, v, w.q64.p);
    const void *X[1] = {v};
    blas_multidot<double>(c, X, 1, w.q64.p, N, dslot(c, H1));
    blas_resid_norm2(c, w.q64.p, v, dslot(c, H1), N, dslot(c, HN));
    fetch(c, HN + 1);
    const double lam = hslot(c, H1)->re;
    const double eps = std::sqrt(std::max(0.0, hslot(c, HN)->re));
    MG_REQUIRE(std::isfinite(lam) && std::isfinite(eps), MGEIG_EBREAKDOWN);
    return {lam, eps};
}

// Start vectors of Algorithm 1 beyond the N_tv test vectors: Philox uniforms
// (stream 0x5EED0003), setup_smooth two-grid iterations at sigma = 0 with the
// setup's P, then Gram-Schmidt against all earlier vectors.
template <typename R>
static void extra_start_vectors(Ctx &c, int n_tv, int n_run) {
    Ctx::Work &w = *c.work;
    const int n_extra = n_run - n_tv;
    random_spinors(c, c.setup_seed, w.Mextra.p, n_extra, 0x5EED0003u);
    c.in_setup = true;
    for (int k = 0; k < c.prm.setup_smooth; ++k)
        for (int j = n_tv; j < n_run; ++j) {
            mg_cycle_f64<R>(c, 0.0, w.modes[j], w.t64.p);
            blas_copy<double>(c, w.t64.p, w.modes[j], c.fine_ncpx());
        }
    c.in_setup = false;
    orthonormalise(c, w.modes, n_run);
}

int eigensolve(Ctx &c, int n_want, double tol, double *evals, double *evecs_host, double *resid) {
    Ctx::Work &w = *c.work;
    const size_t N = c.fine_ncpx();
    const int ntv = c.prm.n_tv;
    const int guard = c.prm.n_guard < 0 ? std::min(std::max(n_want, ntv), MAX_ITERATED - n_want) : c.prm.n_guard;
    const int n_eig = n_want + guard;
    MG_REQUIRE(n_eig <= MAX_ITERATED, MGEIG_EINVAL);
    w.modes.assign(w.W.begin(), w.W.end());
    if (n_eig > ntv) {
        w.Mextra.alloc(f64_bytes(c) * (n_eig - ntv));
        for (int j = ntv; j < n_eig; ++j) w.modes.push_back(static_cast<char *>(w.Mextra.p) + f64_bytes(c) * (j - ntv));
        if (c.mixed()) extra_start_vectors<float>(c, ntv, n_eig);
        else extra_start_vectors<double>(c, ntv, n_eig);
    }
    std::vector<void *> &M = w.modes;
    if (c.prm.ritz_start) ritz_rotate(c, M, std::max(ntv, n_eig));
    // P from the first p iterated vectors and, when p < N_tv, the setup's test
    // vectors p .. N_tv - 1 (a frozen copy): a P built from a subset of the modes
    const int p_modes = c.prm.p_modes < 0 ? ntv : std::min(c.prm.p_modes, ntv);
    std::vector<void *> Wfix;
    if (p_modes < ntv) {
        w.Wfrozen.alloc(f64_bytes(c) * (ntv - p_modes));
        for (int j = p_modes; j < ntv; ++j) {
            Wfix.push_back(w.Wfrozen.as<char>() + f64_bytes(c) * (j - p_modes));
            blas_copy<double>(c, M[j], Wfix.back(), N);
        }
    }
    auto set_psrc = [&]() {
        w.Psrc.assign(M.begin(), M.begin() + p_modes);
        w.Psrc.insert(w.Psrc.end(), Wfix.begin(), Wfix.end());
    };
    set_psrc();
    mg_rebuild(c);
    std::vector<double> lam(n_eig, 0.0), eps(n_eig, 1.0);
    fdefl_begin(c, M, n_eig);
    struct FdEnd { Ctx &c; ~FdEnd() { fdefl_end(c); } } fd_end{c};
    int sweeps = 0;
    const bool rr = c.prm.ritz_each_sweep != 0;
    // with the per-sweep Rayleigh-Ritz step converged pairs are locked, the
    // vectors stay in |lambda| order and only the n_want lowest must converge
    auto unconverged = [&]() {
        const int n = rr ? n_want : n_eig;
        for (int i = 0; i < n; ++i)
            if (eps[i] > tol) return true;
        return false;
    };
    int status = MGEIG_OK;
    while (unconverged() && sweeps < c.prm.max_sweeps) {
        ++sweeps;
        std::vector<char> locked(n_eig);
        for (int i = 0; i < n_eig; ++i) locked[i] = eps[i] <= tol;
        for (int i = 0; i < n_eig; ++i) {
            if (eps[i] <= tol) continue;
            // damped shift of Algorithm 1, with a floor on the damping
            const double sigma = lam[i] * std::max(1.0 - std::max(eps[i], c.prm.shift_floor), 0.0);
            const double t0 = now_s();
            const int outer0 = c.st.outer_iters;
            // guard vectors only widen the span: a few FGMRES steps suffice
            const bool is_guard = rr && i >= n_want;
            // inexact solve: the new vector's eigen-residual is about tau |lambda - sigma|,
            // so tau shrinks to 0.1 tol / |lambda - sigma| near convergence
            const double dls = std::fabs(lam[i] - sigma);
            const double tau = (is_guard || dls == 0 || !c.prm.adaptive_tol)
                                   ? c.prm.solve_tol
                                   : std::min(c.prm.solve_tol, std::max(0.1 * tol / dls, 1e-12));
            if (c.mixed()) fdefl_prepare<float>(c, sigma, i);
            else fdefl_prepare<double>(c, sigma, i);
            // a guard vector's solve may take a cheaper coarse solve
            struct CoarseCap {
                Ctx &c;
                int saved;
                CoarseCap(Ctx &cc, bool guard) : c(cc), saved(cc.prm.coarse_maxiter) {
                    if (guard && c.prm.guard_coarse_maxiter > 0) c.prm.coarse_maxiter = c.prm.guard_coarse_maxiter;
                }
                ~CoarseCap() { c.prm.coarse_maxiter = saved; }
            } cap{c, is_guard};
            int rc = fgmres_solve(c, sigma, M[i], w.x64.p, tau,
                                  is_guard ? std::min(c.prm.guard_maxiter, c.prm.outer_maxiter) : c.prm.outer_maxiter);
            if (rc != MGEIG_OK && rc != MGEIG_ENOCONV) return rc;
            // Gram-Schmidt against v_j, j < i (Algorithm 1), and every locked pair
            std::vector<const void *> X;
            for (int j = 0; j < n_eig; ++j)
                if (j < i || (rr && locked[j] && j != i)) X.push_back(M[j]);
            std::vector<cpx<double>> hx(X.size());
            const double nrm = std::sqrt(std::max(0.0, gs_dgks<double>(c, X.data(), (int)X.size(), w.x64.p, N,
                                                                          hx.data())));
            MG_REQUIRE(std::isfinite(nrm) && nrm > 0, MGEIG_EBREAKDOWN);
            blas_scale<double>(c, cpx<double>(1.0 / nrm), w.x64.p, N);
            blas_copy<double>(c, w.x64.p, M[i], N);
            if (i < p_modes) mg_rebuild(c);   // P holds the first p_modes iterated vectors
            w.fd_k = 0;   // the solve is over
            if (w.fd_n) fdefl_update(c, M, i);
            auto le = rayleigh(c, M[i]);
            lam[i] = le.first;
            eps[i] = le.second;
            if (log_on()) {
                const long long ci = c.st.coarse_iters;
                coarse_iters_take(c);
                fprintf(stderr, "mgeig rqi sweep %d i %d sigma %.6e lambda %.12e eps %.3e outer %d coarse %lld %s %.3fs\n",
                        sweeps, i, sigma, lam[i], eps[i], c.st.outer_iters - outer0, c.st.coarse_iters - ci,
                        rc == MGEIG_OK ? "ok" : "cap", now_s() - t0);
            }
        }
        if (rr) {
            // lock the converged pairs; the nearly converged ones (eps <= ritz_keep)
            // are only orthonormalised, Rayleigh-Ritz on the others, orthogonal to both
            std::vector<void *> order;
            std::vector<int> K, U;
            for (int i = 0; i < n_eig; ++i)
                if (eps[i] <= tol) order.push_back(M[i]);
                else if (eps[i] <= c.prm.ritz_keep) K.push_back(i);
                else U.push_back(i);
            const int nl = (int)order.size(), nk = (int)K.size();
            if (!K.empty() || !U.empty()) {
                for (int i : K) order.push_back(M[i]);
                for (int i : U) order.push_back(M[i]);
                orthonormalise_from(c, order, nl);
                if (!U.empty()) {
                    std::vector<void *> Mu(order.begin() + nl + nk, order.end());
                    ritz_rotate(c, Mu, (int)Mu.size());
                }
                for (int i : K) U.push_back(i);
                for (int i : U) {
                    auto le = rayleigh(c, M[i]);
                    lam[i] = le.first;
                    eps[i] = le.second;
                }
            }
            // keep every vector in |lambda| order (a permutation of the pointers)
            std::vector<int> perm(n_eig);
            std::iota(perm.begin(), perm.end(), 0);
            std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) {
                double fa = std::fabs(lam[a]), fb = std::fabs(lam[b]);
                return fa != fb ? fa < fb : lam[a] < lam[b];
            });
            std::vector<void *> M2(n_eig);
            std::vector<double> l2(n_eig), e2(n_eig);
            for (int k = 0; k < n_eig; ++k) { M2[k] = M[perm[k]]; l2[k] = lam[perm[k]]; e2[k] = eps[perm[k]]; }
            for (int k = 0; k < n_eig; ++k) { M[k] = M2[k]; lam[k] = l2[k]; eps[k] = e2[k]; }
            set_psrc();
            mg_rebuild(c);
            fdefl_all(c, M);
            if (log_on()) {
                double mx = 0;
                for (int i = 0; i < n_want; ++i) mx = std::max(mx, eps[i]);
                fprintf(stderr, "mgeig rqi sweep %d locked %d max eps (wanted) %.3e\n", sweeps, nl, mx);
            }
        }
    }
    c.st.sweeps = sweeps;
    if (c.ds_blas() || c.ds_stencil()) {
        // the reported pairs are certified in FP64: their Rayleigh quotients and
        // residuals again with the FP64 stencil and FP64 inner products
        struct Fp64 {
            Ctx &c;
            explicit Fp64(Ctx &cc) : c(cc) { c.force_fp64 = true; }
            ~Fp64() { c.force_fp64 = false; }
        } fp64{c};
        for (int i = 0; i < (rr ? n_want : n_eig); ++i) {
            auto le = rayleigh(c, M[i]);
            lam[i] = le.first;
            eps[i] = le.second;
        }
    }
    if (unconverged()) status = MGEIG_ENOCONV;
    // order by |lambda|, then lambda
    std::vector<int> ord(n_eig);
    std::iota(ord.begin(), ord.end(), 0);
    std::sort(ord.begin(), ord.end(), [&](int a, int b) {
        double fa = std::fabs(lam[a]), fb = std::fabs(lam[b]);
        return fa != fb ? fa < fb : lam[a] < lam[b];
    });
    for (int k = 0; k < n_want; ++k) {
        if (evals) evals[k] = lam[ord[k]];
        if (resid) resid[k] = eps[ord[k]];
    }
    if (evecs_host) {
        // host layout, unit norm, largest-modulus component real positive
        for (int k = 0; k < n_want; ++k) {
            unpack_spinor_f64(c, M[ord[k]], static_cast<double *>(c.staging.p), 1);
            MG_CUDA(cudaMemcpyAsync(evecs_host + (size_t)k * N * 2, c.staging.p, N * 16, cudaMemcpyDeviceToHost, c.stream));
            sync(c);
            double *v = evecs_host + (size_t)k * N * 2;
            size_t best = 0;
            double bm = -1;
            for (size_t i = 0; i < N; ++i) {
                double m2 = v[2 * i] * v[2 * i] + v[2 * i + 1] * v[2 * i + 1];
                if (m2 > bm * (1 + 1e-12)) { bm = m2; best = i; }
            }
            const double mag = std::sqrt(bm);
            const double pr = v[2 * best] / mag, pi = -v[2 * best + 1] / mag;   // conj phase
            for (size_t i = 0; i < N; ++i) {
                double re = v[2 * i], im = v[2 * i + 1];
                v[2 * i] = re * pr - im * pi;
                v[2 * i + 1] = re * pi + im * pr;
            }
        }
    }
    return status;
}

// ---------------------------------------------------------------------------
// Approximate low-mode averaging (Sec. 3.1, 3.2): from N orthonormal approximate
// eigenvectors v_i, the pairs that pass the cutoff eps_i / |lambda_i| <= c,
// A_ij = <v_i | Q | v_j>, Q~^-1_low = sum (A^-1)_ij |v_i><v_j|, the oblique
// projector R~ = 1 - sum Q |v_i> (A^-1)_ij <v_j|, and the two parts of the loop
// L(t) = sum_{x in t} tr Q^-1_{x,x}: the low-mode part from the vectors, the
// high-mode part Q^-1 R~ stochastically with Z2 noise (Q s = R~ eta).

struct Lma {
    DevBuf Vall, QVall;                 // N vectors and Q v_i (FP64)
    int n = 0;
    std::vector<void *> V, QV;          // the kept vectors and their products
    std::vector<cpx<double>> Ainv;      // row-major, kept x kept
};

void *lma_vectors(Ctx &c, int n) {
    if (!c.lma) c.lma = new Lma();
    c.lma->Vall.alloc(f64_bytes(c) * n);
    c.lma->QVall.alloc(f64_bytes(c) * n);
    return c.lma->Vall.p;
}

void lma_free(Ctx &c) {
    if (!c.lma) return;
    c.lma->Vall.free();
    c.lma->QVall.free();
    delete c.lma;
    c.lma = nullptr;
}

void lma_prepare(Ctx &c, int n, void *Vdev, bool ritz, double cutoff, double *lam, double *eps, int *kept,
                 int *n_kept, double *A_out, double *Ainv_out, double *Llow) {
    Lma &L = *c.lma;
    MG_REQUIRE(Vdev == L.Vall.p && n >= 1 && n <= MAX_ITERATED, MGEIG_EINVAL);
    const size_t N = c.fine_ncpx();
    std::vector<void *> V(n), QV(n);
    for (int i = 0; i < n; ++i) {
        V[i] = L.Vall.as<char>() + f64_bytes(c) * i;
        QV[i] = L.QVall.as<char>() + f64_bytes(c) * i;
    }
    orthonormalise(c, V, n);
    if (ritz) ritz_rotate(c, V, n);   // Ritz vectors of Q in span(V), by |theta|
    L.V.clear();
    L.QV.clear();
    for (int i = 0; i < n; ++i) {
        auto le = rayleigh(c, V[i]);
        apply_fine<double>(c, MODE_QSIGMA, 0.0, V[i], QV[i]);
        if (lam) lam[i] = le.first;
        if (eps) eps[i] = le.second;
        const bool keep = le.second <= cutoff * std::fabs(le.first);
        if (kept) kept[i] = keep ? 1 : 0;
        if (keep) { L.V.push_back(V[i]); L.QV.push_back(QV[i]); }
    }
    const int nk = (int)L.V.size();
    L.n = nk;
    if (n_kept) *n_kept = nk;
    L.Ainv.clear();
    if (!nk) return;
    std::vector<cpx<double>> A((size_t)nk * nk);
    std::vector<const void *> X(L.V.begin(), L.V.end());
    for (int j = 0; j < nk; ++j) {
        blas_multidot<double>(c, X.data(), nk, L.QV[j], N, dslot(c, H1));
        fetch(c, H1 + nk);
        for (int i = 0; i < nk; ++i) A[(size_t)i * nk + j] = *hslot(c, H1 + i);   // <v_i | Q v_j>
    }
    MG_REQUIRE(invert(nk, A, L.Ainv), MGEIG_EBREAKDOWN);
    if (A_out) std::memcpy(A_out, A.data(), A.size() * sizeof(cpx<double>));
    if (Ainv_out) std::memcpy(Ainv_out, L.Ainv.data(), L.Ainv.size() * sizeof(cpx<double>));
    if (Llow) {
        const int T = c.dims[3];
        TmpBuf M;
        M.alloc((size_t)T * nk * nk * sizeof(double2));
        timeslice_dots(c, X.data(), nk, X.data(), nk, M.p);
        std::vector<cpx<double>> Mh((size_t)T * nk * nk);
        MG_CUDA(cudaMemcpyAsync(Mh.data(), M.p, Mh.size() * sizeof(double2), cudaMemcpyDeviceToHost, c.stream));
        sync(c);
        for (int t = 0; t < T; ++t) {
            cpx<double> acc;
            for (int j = 0; j < nk; ++j)
                for (int i = 0; i < nk; ++i)
                    acc = acc + L.Ainv[(size_t)i * nk + j] * Mh[((size_t)t * nk + j) * nk + i];
            Llow[2 * t] = acc.re;
            Llow[2 * t + 1] = acc.im;
        }
    }
}

// mode 0: y = Q~^-1_low x ; mode 1: y = R~ x  (FP64 internal spinors, y != x)
void lma_apply(Ctx &c, int mode, const void *x64, void *y64) {
    MG_REQUIRE(c.lma && (mode == 0 || mode == 1), MGEIG_ENOTSETUP);
    Lma &L = *c.lma;
    const size_t N = c.fine_ncpx();
    const int nk = L.n;
    if (mode == 0) blas_zero<double>(c, y64, N);
    else blas_copy<double>(c, x64, y64, N);
    if (!nk) return;
    std::vector<const void *> X(L.V.begin(), L.V.end());
    blas_multidot<double>(c, X.data(), nk, x64, N, dslot(c, H1));
    fetch(c, H1 + nk);
    std::vector<cpx<double>> coef(nk);
    for (int i = 0; i < nk; ++i) {
        cpx<double> acc;
        for (int j = 0; j < nk; ++j) acc = acc + L.Ainv[(size_t)i * nk + j] * *hslot(c, H1 + j);
        coef[i] = acc;
    }
    std::vector<const void *> B(mode == 0 ? L.V.begin() : L.QV.begin(), mode == 0 ? L.V.end() : L.QV.end());
    blas_multi_axpy<double>(c, y64, B.data(), nk, upload(c, coef), mode == 0 ? 1.0 : -1.0, N);
}

// L_high(t) = 1/nstoch sum_n sum_{x in t} <eta_n(x) | s_n(x)>, Q s_n = R~ eta_n
void lma_loop_high(Ctx &c, int nstoch, uint64_t seed, double tol, double *Lhigh, int *outer_iters) {
    MG_REQUIRE(c.lma, MGEIG_ENOTSETUP);
    const int T = c.dims[3];
    TmpBuf eta, b, sv, M;
    eta.alloc(f64_bytes(c) * nstoch);
    b.alloc(f64_bytes(c));
    sv.alloc(f64_bytes(c));
    M.alloc((size_t)T * sizeof(double2));
    z2_spinors(c, seed, eta.p, nstoch, 0x5EED0002u);
    std::vector<double> acc(2 * T, 0.0);
    std::vector<double2> Mh(T);
    const int outer0 = c.st.outer_iters;
    for (int k = 0; k < nstoch; ++k) {
        const void *ek = eta.as<char>() + f64_bytes(c) * k;
        lma_apply(c, 1, ek, b.p);
        const int rc = fgmres_solve(c, 0.0, b.p, sv.p, tol);
        MG_REQUIRE(rc == MGEIG_OK, rc);
        const void *X[1] = {ek};
        const void *Y[1] = {sv.p};
        timeslice_dots(c, X, 1, Y, 1, M.p);
        MG_CUDA(cudaMemcpyAsync(Mh.data(), M.p, T * sizeof(double2), cudaMemcpyDeviceToHost, c.stream));
        sync(c);
        for (int t = 0; t < T; ++t) { acc[2 * t] += Mh[t].x; acc[2 * t + 1] += Mh[t].y; }
    }
    for (int t = 0; t < 2 * T; ++t) Lhigh[t] = acc[t] / nstoch;
    if (outer_iters) *outer_iters = c.st.outer_iters - outer0;
}

// ---------------------------------------------------------------------------
// training of the learned smoother on pairs the two-grid method produces

void net_train(Ctx &c, int steps, int batch, double lr, uint64_t seed, double *losses) {
    Ctx::Work &w = *c.work;
    const size_t n = c.fine_ncpx();
    TmpBuf v64, R, E;
    v64.alloc(f64_bytes(c) * batch);
    R.alloc(fR_bytes(c) * batch);
    E.alloc(fR_bytes(c) * batch);
    for (int step = 0; step < steps; ++step) {
        random_spinors(c, seed + (uint64_t)step, v64.p, batch, 0x5EED0004u);
        for (int f = 0; f < batch; ++f) {
            void *rf = R.as<char>() + fR_bytes(c) * f;
            void *ef = E.as<char>() + fR_bytes(c) * f;
            convert_f64_to_f32(c, v64.as<char>() + f64_bytes(c) * f, w.rR.p, n);
            // coarse correction x_c = P Q_c^-1 P^dag v and the residual r = v - Q x_c
            restrict_vec<float>(c, (const void *const *)w.P.data(), w.rR.p, w.rc.p);
            coarse_solve<float>(c, 0.0, w.rc.p, w.ec.p);
            prolong_vec<float>(c, (const void *const *)w.P.data(), w.ec.p, w.zR.p);
            apply_fine<float>(c, MODE_QSIGMA, 0.0, w.zR.p, rf);
            blas_scale<float>(c, cpx<double>(-1), rf, n);
            blas_axpy<float>(c, cpx<double>(1), w.rR.p, rf, n);
            // the target: the SAP correction of r (D e = gamma5 r from e = 0)
            blas_zero<float>(c, ef, n);
            for (int k = 0; k < c.prm.sap_cycles; ++k) {
                sap_sweep<float>(c, 0, 0.0, rf, true, ef);
                sap_sweep<float>(c, 1, 0.0, rf, true, ef);
            }
        }
        const double L = net_train_step(c, R.p, E.p, batch, lr);
        if (losses) losses[step] = L;
        if (log_on() && (step % 50 == 0 || step == steps - 1)) fprintf(stderr, "mgeig net step %d loss %.4e\n", step, L);
    }
    coarse_iters_take(c);
}

// ---------------------------------------------------------------------------
// single-step entry points used for parity checks (FP64 in / out)

template <typename R>
static void to_level(Ctx &c, const void *in64, void *outR) {
    if (sizeof(R) == 4) convert_f64_to_f32(c, in64, outR, c.fine_ncpx());
    else blas_copy<double>(c, in64, outR, c.fine_ncpx());
}
template <typename R>
static void from_level(Ctx &c, const void *inR, void *out64) {
    if (sizeof(R) == 4) convert_f32_to_f64(c, inR, out64, c.fine_ncpx());
    else blas_copy<double>(c, inR, out64, c.fine_ncpx());
}

void sap_smooth_f64(Ctx &c, double sigma, const void *b64, void *z64, int cycles) {
    Ctx::Work &w = *c.work;
    if (c.mixed()) {
        to_level<float>(c, b64, w.rR.p);
        to_level<float>(c, z64, w.zR.p);
        for (int k = 0; k < cycles; ++k) {
            sap_sweep<float>(c, 0, sigma, w.rR.p, false, w.zR.p);
            sap_sweep<float>(c, 1, sigma, w.rR.p, false, w.zR.p);
        }
        from_level<float>(c, w.zR.p, z64);
    } else {
        for (int k = 0; k < cycles; ++k) {
            sap_sweep<double>(c, 0, sigma, b64, false, z64);
            sap_sweep<double>(c, 1, sigma, b64, false, z64);
        }
    }
}

void mg_cycle_host(Ctx &c, double sigma, const double *r64, double *z64) {
    if (c.mixed()) mg_cycle_f64<float>(c, sigma, r64, z64);
    else mg_cycle_f64<double>(c, sigma, r64, z64);
}

// coarse vectors: FP64 flat <-> level precision flat
__global__ void flat_f64_to_f32(size_t n, const double2 *in, float2 *out) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = make_float2((float)in[i].x, (float)in[i].y);
}
__global__ void flat_f32_to_f64(size_t n, const float2 *in, double2 *out) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = make_double2(in[i].x, in[i].y);
}

// n complex values: FP64 -> FP32 (to32) or FP32 -> FP64
void coarse_flat_convert(Ctx &c, const void *in, void *out, size_t n, bool to32) {
    if (to32) flat_f64_to_f32<<<grid_for(n, 256), 256, 0, c.stream>>>(n, (const double2 *)in, (float2 *)out);
    else flat_f32_to_f64<<<grid_for(n, 256), 256, 0, c.stream>>>(n, (const float2 *)in, (double2 *)out);
    MG_CHECK_LAUNCH();
}

static void coarse_in(Ctx &c, const void *x64, void *xR) {
    const size_t n = c.coarse_ncpx();
    if (c.mixed()) flat_f64_to_f32<<<grid_for(n, 256), 256, 0, c.stream>>>(n, (const double2 *)x64, (float2 *)xR);
    else MG_CUDA(cudaMemcpyAsync(xR, x64, n * 16, cudaMemcpyDeviceToDevice, c.stream));
    MG_CHECK_LAUNCH();
}
static void coarse_out(Ctx &c, const void *xR, void *x64) {
    const size_t n = c.coarse_ncpx();
    if (c.mixed()) flat_f32_to_f64<<<grid_for(n, 256), 256, 0, c.stream>>>(n, (const float2 *)xR, (double2 *)x64);
    else MG_CUDA(cudaMemcpyAsync(x64, xR, n * 16, cudaMemcpyDeviceToDevice, c.stream));
    MG_CHECK_LAUNCH();
}

void coarse_apply_f64(Ctx &c, double sigma, const void *x64, void *y64) {
    Ctx::Work &w = *c.work;
    coarse_in(c, x64, w.rc.p);
    if (c.mixed()) coarse_apply<float>(c, c.Dc.p, sigma, w.rc.p, w.ec.p);
    else coarse_apply<double>(c, c.Dc.p, sigma, w.rc.p, w.ec.p);
    coarse_out(c, w.ec.p, y64);
}

void restrict_f64(Ctx &c, const void *r64, void *rc64) {
    Ctx::Work &w = *c.work;
    if (c.mixed()) {
        to_level<float>(c, r64, w.rR.p);
        restrict_vec<float>(c, (const void *const *)w.P.data(), w.rR.p, w.rc.p);
    } else {
        restrict_vec<double>(c, (const void *const *)w.P.data(), r64, w.rc.p);
    }
    coarse_out(c, w.rc.p, rc64);
}

void prolong_f64(Ctx &c, const void *ec64, void *e64) {
    Ctx::Work &w = *c.work;
    coarse_in(c, ec64, w.ec.p);
    if (c.mixed()) {
        prolong_vec<float>(c, (const void *const *)w.P.data(), w.ec.p, w.zR.p);
        from_level<float>(c, w.zR.p, e64);
    } else {
        prolong_vec<double>(c, (const void *const *)w.P.data(), w.ec.p, e64);
    }
}

__global__ void dc_to_f64(size_t n, const float2 *in, double2 *out) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = make_double2(in[i].x, in[i].y);
}
// column-major blocks -> row-major [9][nagg][row][col]
__global__ void dc_transpose(size_t nblk, int n2, const double2 *in, double2 *out) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t per = (size_t)n2 * n2;
    if (i >= nblk * per) return;
    size_t b = i / per, o = i % per;
    int row = (int)(o / n2), col = (int)(o % n2);
    out[i] = in[b * per + (size_t)col * n2 + row];
}

void coarse_op_f64(Ctx &c, void *out64) {
    const int n2 = 2 * c.prm.n_tv;
    const size_t nblk = (size_t)9 * c.nagg, tot = nblk * n2 * n2;
    TmpBuf tmp;
    tmp.alloc(tot * 16);
    if (c.mixed()) dc_to_f64<<<grid_for(tot, 256), 256, 0, c.stream>>>(tot, c.Dc.as<float2>(), tmp.as<double2>());
    else MG_CUDA(cudaMemcpyAsync(tmp.p, c.Dc.p, tot * 16, cudaMemcpyDeviceToDevice, c.stream));
    dc_transpose<<<grid_for(tot, 256), 256, 0, c.stream>>>(nblk, n2, tmp.as<double2>(), static_cast<double2 *>(out64));
    MG_CHECK_LAUNCH();
    sync(c);
    tmp.free();
}

void interp_f64(Ctx &c, void *const *out64) {
    Ctx::Work &w = *c.work;
    for (int j = 0; j < c.prm.n_tv; ++j) {
        if (c.mixed()) convert_f32_to_f64(c, w.P[j], out64[j], c.fine_ncpx());
        else MG_CUDA(cudaMemcpyAsync(out64[j], w.P64[j], f64_bytes(c), cudaMemcpyDeviceToDevice, c.stream));
    }
}

// ---------------------------------------------------------------------------
// The two-grid cycle without device allocation (mgeig_mg_cycle_dev_noalloc).
//
// Some callers cannot allocate device memory when they need a preconditioner
// application: a solver embedded in a framework whose pool allocator owns all
// free GPU memory, a latency-critical loop that must not take the driver's
// allocation lock or let cudaFree synchronise the device, or a host thread
// that runs while another library holds the GPU to a fixed memory budget.
// For them the cycle's coarse vectors and the persistent coarse solver's
// scratch (Krylov basis, projected right-hand side, per-block partial sums,
// barrier and status words) live in one file-scope device array of
// NOALLOC_SCRATCH_BYTES; every GPU that loads this library holds it until
// the process exits.  All calls share it, so calls that overlap on the GPU
// (other streams, other contexts on the same device, other host threads) race.

constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(16) << 20;   // 16 MiB
static __device__ __align__(256) unsigned char noalloc_scratch[NOALLOC_SCRATCH_BYTES];

size_t mg_cycle_noalloc_limit() { return NOALLOC_SCRATCH_BYTES; }

// Device address of noalloc_scratch on `device` (which must be current): in host
// code the array's name only stands in for the symbol, so the address is looked
// up with cudaGetSymbolAddress once per device and cached.
static void *noalloc_scratch_address(int device) {
    constexpr int MAX_DEVICES = 64;
    static std::mutex mu;
    static void *addr[MAX_DEVICES] = {};
    MG_REQUIRE(device >= 0 && device < MAX_DEVICES, MGEIG_EINVAL);
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[device]) {
        void *p = nullptr;
        MG_CUDA(cudaGetSymbolAddress(&p, noalloc_scratch));
        addr[device] = p;
    }
    return addr[device];
}

// Looks the array's address up at context creation (mgeig_create), so that the
// module holding it is loaded and the array is reserved before any
// mgeig_mg_cycle_dev_noalloc call: with CUDA's lazy module loading that would
// otherwise happen inside the first call.
void noalloc_prepare(Ctx &c) { (void)noalloc_scratch_address(c.device); }

// Gauss-Jordan inverse of the row-major n x n matrix A (destroyed), n <= 24,
// with the operations of invert() in the same order (identical results) but
// on the caller's arrays.
static bool invert_fixed(int n, cpx<double> *A, cpx<double> *inv) {
    for (int i = 0; i < n * n; ++i) inv[i] = cpx<double>();
    for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = cpx<double>(1);
    for (int col = 0; col < n; ++col) {
        int piv = col;
        double best = -1;
        for (int r = col; r < n; ++r) {
            cpx<double> z = A[(size_t)r * n + col];
            double m = std::hypot(z.re, z.im);
            if (m > best) { best = m; piv = r; }
        }
        if (!(best > 0) || !std::isfinite(best)) return false;
        if (piv != col)
            for (int k = 0; k < n; ++k) {
                std::swap(A[(size_t)piv * n + k], A[(size_t)col * n + k]);
                std::swap(inv[(size_t)piv * n + k], inv[(size_t)col * n + k]);
            }
        cpx<double> d = A[(size_t)col * n + col];
        double dd = d.re * d.re + d.im * d.im;
        cpx<double> di(d.re / dd, -d.im / dd);
        for (int k = 0; k < n; ++k) {
            A[(size_t)col * n + k] = A[(size_t)col * n + k] * di;
            inv[(size_t)col * n + k] = inv[(size_t)col * n + k] * di;
        }
        for (int r = 0; r < n; ++r) {
            if (r == col) continue;
            cpx<double> f = A[(size_t)r * n + col];
            if (f.re == 0 && f.im == 0) continue;
            for (int k = 0; k < n; ++k) {
                A[(size_t)r * n + k] = A[(size_t)r * n + k] - f * A[(size_t)col * n + k];
                inv[(size_t)r * n + k] = inv[(size_t)r * n + k] - f * inv[(size_t)col * n + k];
            }
        }
    }
    return true;
}

// deflation_prepare with host arrays on the stack instead of the heap
template <typename R>
static void deflation_prepare_fixed(Ctx &c, double sigma) {
    Ctx::Work &w = *c.work;
    if (w.defl_valid && w.defl_sigma == sigma) return;
    constexpr int KMAX = 24;
    const int k = c.prm.n_tv;
    MG_REQUIRE(k <= KMAX, MGEIG_EINVAL);
    const size_t n = c.coarse_ncpx(), vb = cR_bytes(c);
    const void *Wp[KMAX];
    for (int i = 0; i < k; ++i) Wp[i] = static_cast<const char *>(w.Wc.p) + vb * i;
    for (int j = 0; j < k; ++j) {
        void *awj = static_cast<char *>(w.AWc.p) + vb * j;
        coarse_apply<R>(c, c.Dc.p, sigma, Wp[j], awj, false);
        blas_multidot<R>(c, Wp, k, awj, n, w.Edev.as<cpx<double>>() + (size_t)j * k);
    }
    cpx<double> Ecol[KMAX * KMAX], E[KMAX * KMAX], Ei[KMAX * KMAX];
    MG_CUDA(cudaMemcpyAsync(Ecol, w.Edev.p, (size_t)k * k * sizeof(double2), cudaMemcpyDeviceToHost, c.stream));
    sync(c);
    for (int j = 0; j < k; ++j)
        for (int i = 0; i < k; ++i) E[(size_t)i * k + j] = Ecol[(size_t)j * k + i];   // E_ij = <W_i, A W_j>
    MG_REQUIRE(invert_fixed(k, E, Ei), MGEIG_EBREAKDOWN);
    MG_CUDA(cudaMemcpyAsync(w.Einv.p, Ei, (size_t)k * k * sizeof(double2), cudaMemcpyHostToDevice, c.stream));
    sync(c);
    w.defl_valid = true;
    w.defl_sigma = sigma;
}

template <typename R>
static int mg_cycle_noalloc_impl(Ctx &c, double sigma, const void *r, void *z) {
    Ctx::Work &w = *c.work;
    const size_t cb = c.coarse_ncpx() * sizeof(cpx<R>);
    const int k = c.prm.coarse_deflate ? c.prm.n_tv : 0;
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    // layout: solver state words | r_c | e_c | the coarse solver's scratch
    const size_t off_rc = 256, off_ec = off_rc + up(cb), off_S = off_ec + up(cb);
    const size_t need = off_S + up(coarse_gmres_scratch_bytes(c, k));
    if (need > NOALLOC_SCRATCH_BYTES) {
        fprintf(stderr, "libmgeig: mgeig_mg_cycle_dev_noalloc needs %zu bytes of scratch for this coarse grid, "
                        "its static array holds %zu\n", need, NOALLOC_SCRATCH_BYTES);
        return MGEIG_ESCRATCH;
    }
    char *s = static_cast<char *>(noalloc_scratch_address(c.device));
    // the barrier counters, status and iteration words must start at zero
    MG_CUDA(cudaMemsetAsync(s, 0, 256, c.stream));
    if (k) deflation_prepare_fixed<R>(c, sigma);
    c.st.mg_cycles += 1;
    restrict_vec<R>(c, (const void *const *)w.P.data(), r, s + off_rc);
    coarse_gmres_at<R>(c, sigma, s + off_rc, s + off_ec, s + off_S, s, k, w.Wc.p, w.AWc.p, w.Einv.p);
    prolong_vec<R>(c, (const void *const *)w.P.data(), s + off_ec, z);
    for (int q = 0; q < c.prm.sap_cycles; ++q) {
        sap_sweep<R>(c, 0, sigma, r, true, z);
        sap_sweep<R>(c, 1, sigma, r, true, z);
    }
    int state[4];   // barrier count, generation, status (0 ok, 1 timeout, 2 breakdown), iterations
    MG_CUDA(cudaMemcpyAsync(state, s, sizeof(state), cudaMemcpyDeviceToHost, c.stream));
    sync(c);
    c.st.coarse_iters += state[3];
    if (state[2] == 1) return MGEIG_ETIMEOUT;
    if (state[2] != 0) return MGEIG_EBREAKDOWN;
    return MGEIG_OK;
}

int mg_cycle_noalloc(Ctx &c, double sigma, const void *r, void *z) {
    return c.mixed() ? mg_cycle_noalloc_impl<float>(c, sigma, r, z) : mg_cycle_noalloc_impl<double>(c, sigma, r, z);
}

}  // namespace mgeig
