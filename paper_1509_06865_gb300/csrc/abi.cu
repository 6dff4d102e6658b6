// The C ABI of libmgeig (declared in include/mgeig.h).  Every entry point
// catches the library's internal errors and returns a status code.
#include <chrono>
#include <cstring>

#include "internal.h"

using namespace mgeig;

struct mgeig_ctx {
    Ctx c;
};

namespace {

template <typename F>
int guarded(mgeig_ctx *ctx, F f) {
    if (!ctx) return MGEIG_EINVAL;
    try {
        MG_CUDA(cudaSetDevice(ctx->c.device));
        return f(ctx->c);
    } catch (const Error &e) {
        return e.code;
    } catch (const std::bad_alloc &) {
        return MGEIG_ENOMEM;
    }
}

bool divides_all(const int *blk, const int *dims) {
    for (int mu = 0; mu < 4; ++mu)
        if (blk[mu] < 1 || dims[mu] % blk[mu]) return false;
    return true;
}

// the lattice checks of mgeig_create: every extent >= 2, 12 V below 2^31
int check_dims(const int dims[4], long long *V_out = nullptr) {
    long long V = 1;
    for (int mu = 0; mu < 4; ++mu) {
        if (dims[mu] < 2) return MGEIG_EINVAL;
        V *= dims[mu];
    }
    if (V >= (1LL << 31) / 12) return MGEIG_EINVAL;
    if (V_out) *V_out = V;
    return MGEIG_OK;
}

// the parameter checks of mgeig_set_params for a lattice of extents dims
int validate(const int dims[4], const mgeig_params &p) {
    for (int mu = 0; mu < 4; ++mu)
        if (p.bc[mu] != 1 && p.bc[mu] != -1) return MGEIG_EINVAL;
    if (!divides_all(p.agg, dims) || !divides_all(p.sap_block, dims)) return MGEIG_EINVAL;
    int avol = 1, bvol = 1;
    for (int mu = 0; mu < 4; ++mu) {
        const int nb = dims[mu] / p.sap_block[mu];
        if (nb < 2 || nb % 2) return MGEIG_EINVAL;
        avol *= p.agg[mu];
        bvol *= p.sap_block[mu];
    }
    if (avol > 1024 || bvol > 1024) return MGEIG_EINVAL;
    if (p.n_tv < 2 || p.n_tv > 24 || 6 * avol < p.n_tv) return MGEIG_EINVAL;
    if (p.sap_cycles < 0 || p.sap_mr_iters < 1 || p.smooth_steps < 0 || p.gmres_smooth_k < 1) return MGEIG_EINVAL;
    if (p.setup_smooth < 0 || p.setup_iters < 0) return MGEIG_EINVAL;
    if (p.outer_restart < 1 || p.outer_restart > 100 || p.outer_maxiter < 1) return MGEIG_EINVAL;
    if (p.coarse_restart < 1 || p.coarse_restart > COARSE_PERSISTENT_MAXM || p.coarse_maxiter < 1) return MGEIG_EINVAL;
    if (p.coarse_deflate != 0 && p.coarse_deflate != 1) return MGEIG_EINVAL;
    if (p.ritz_each_sweep != 0 && p.ritz_each_sweep != 1) return MGEIG_EINVAL;
    if (!(p.shift_floor >= 0 && p.shift_floor < 1) || p.guard_maxiter < 1) return MGEIG_EINVAL;
    if (!(p.ritz_keep >= 0) || !std::isfinite(p.ritz_keep)) return MGEIG_EINVAL;
    if (p.fine_deflate != 0 && p.fine_deflate != 1) return MGEIG_EINVAL;
    if (!std::isfinite(p.fine_deflate_radius)) return MGEIG_EINVAL;
    if ((p.adaptive_tol != 0 && p.adaptive_tol != 1) || (p.ritz_start != 0 && p.ritz_start != 1)) return MGEIG_EINVAL;
    if (p.coarse_links < MGEIG_LINKS_LEVEL || p.coarse_links > MGEIG_LINKS_F16) return MGEIG_EINVAL;
    if (p.coarse_links != MGEIG_LINKS_LEVEL && p.precision != MGEIG_MIXED) return MGEIG_EINVAL;
    if (!(p.barrier_timeout > 0) || !(p.barrier_timeout <= 60)) return MGEIG_EINVAL;
    if (p.p_modes < -1 || p.p_modes == 0) return MGEIG_EINVAL;
    if (p.coarse_blocks < 0) return MGEIG_EINVAL;
    if (p.blas_ds != 0 && p.blas_ds != 1) return MGEIG_EINVAL;
    if (p.stencil_ds != 0 && p.stencil_ds != 1) return MGEIG_EINVAL;
    if (p.blas_blocks < 0 || p.blas_blocks > 64) return MGEIG_EINVAL;
    if (p.guard_coarse_maxiter < 0) return MGEIG_EINVAL;
    if (!(p.coarse_tol >= 0) || !(p.solve_tol > 0)) return MGEIG_EINVAL;
    if (p.precision != MGEIG_FP64 && p.precision != MGEIG_MIXED) return MGEIG_EINVAL;
    if (p.smoother != MGEIG_SAP && p.smoother != MGEIG_GMRES && p.smoother != MGEIG_LEARNED) return MGEIG_EINVAL;
    if (p.smoother == MGEIG_LEARNED && (p.precision != MGEIG_MIXED || !net_supported_dims(dims))) return MGEIG_EINVAL;
    if (p.max_sweeps < 1 || p.n_guard < -1) return MGEIG_EINVAL;
    return MGEIG_OK;
}

size_t spinor_bytes(const Ctx &c) { return c.fine_ncpx() * 16; }

// host (caller) spinors -> internal FP64 device layout at dst
void host_to_internal(Ctx &c, const double *host, void *dst) {
    MG_CUDA(cudaMemcpyAsync(c.staging.p, host, spinor_bytes(c), cudaMemcpyHostToDevice, c.stream));
    pack_spinor_f64(c, c.staging.as<double>(), dst, 1);
}

void internal_to_host(Ctx &c, const void *src, double *host) {
    unpack_spinor_f64(c, src, c.staging.as<double>(), 1);
    MG_CUDA(cudaMemcpyAsync(host, c.staging.p, spinor_bytes(c), cudaMemcpyDeviceToHost, c.stream));
    sync(c);
}

}  // namespace

namespace mgeig {
void refresh_clover(Ctx &c) {
    if (c.clover_loaded) pack_clover(c, c.clov_user.as<double>());
    else build_clover(c);
}
}  // namespace mgeig

extern "C" {

void mgeig_default_params(mgeig_params *p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->m0 = 0.0;
    p->csw = 1.0;
    for (int mu = 0; mu < 4; ++mu) { p->bc[mu] = 1; p->agg[mu] = 4; p->sap_block[mu] = 4; }
    p->n_tv = 20;
    p->sap_cycles = 3;
    p->sap_mr_iters = 4;
    p->smooth_steps = 2;
    p->gmres_smooth_k = 8;
    p->setup_smooth = 3;
    p->setup_iters = 10;
    p->outer_restart = 20;
    p->outer_maxiter = 50;
    p->coarse_restart = 30;
    p->coarse_maxiter = 24;
    p->coarse_tol = 5e-2;
    p->solve_tol = 1e-2;
    p->precision = MGEIG_MIXED;
    p->smoother = MGEIG_SAP;
    p->max_sweeps = 50;
    p->n_guard = -1;
    p->coarse_deflate = 1;
    p->ritz_each_sweep = 1;
    p->shift_floor = 1e-6;
    p->guard_maxiter = 4;
    p->ritz_keep = 1e-6;
    p->fine_deflate = 1;
    p->fine_deflate_radius = -1.0;
    p->adaptive_tol = 1;
    p->ritz_start = 1;
    p->coarse_links = MGEIG_LINKS_LEVEL;
    p->barrier_timeout = 2.0;
    p->p_modes = -1;
    p->coarse_blocks = 0;
    p->blas_ds = 1;
    p->stencil_ds = 0;
    p->blas_blocks = 0;
    p->guard_coarse_maxiter = 0;
}

int mgeig_create(mgeig_ctx **out, const int dims[4], int device) {
    if (!out || !dims) return MGEIG_EINVAL;
    *out = nullptr;
    long long V = 1;
    if (check_dims(dims, &V) != MGEIG_OK) return MGEIG_EINVAL;
    mgeig_ctx *ctx = new (std::nothrow) mgeig_ctx();
    if (!ctx) return MGEIG_ENOMEM;
    Ctx &c = ctx->c;
    c.device = device;
    int stride = 1;
    for (int mu = 0; mu < 4; ++mu) {
        c.dims[mu] = dims[mu];
        c.g.L[mu] = dims[mu];
        c.g.stride[mu] = stride;
        stride *= dims[mu];
        c.g.bc[mu] = 1;
    }
    c.g.V = (int)V;
    mgeig_default_params(&c.prm);
    int rc = guarded(ctx, [&](Ctx &c) {
        MG_CUDA(cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking));
        MG_CUDA(cudaDeviceGetAttribute(&c.sms, cudaDevAttrMultiProcessorCount, c.device));
        c.timer.stream = c.stream;
        c.U64.alloc((size_t)V * 4 * 9 * 16);
        c.U32.alloc((size_t)V * 4 * 3 * 16);
        c.clov64.alloc((size_t)V * 36 * 16);
        c.clov32.alloc((size_t)V * 18 * 16);
        c.staging.alloc((size_t)V * 4 * 9 * 16);   // largest host-layout transfer: the gauge field
        ensure_reduction(c, 64);
        noalloc_prepare(c);
        return MGEIG_OK;
    });
    if (rc != MGEIG_OK) {
        mgeig_destroy(ctx);
        return rc;
    }
    *out = ctx;
    return MGEIG_OK;
}

void mgeig_destroy(mgeig_ctx *ctx) {
    if (!ctx) return;
    Ctx &c = ctx->c;
    cudaSetDevice(c.device);
    if (c.stream) cudaStreamSynchronize(c.stream);
    try { c.timer.reset(); } catch (...) {}
    mg_free(c);
    net_free(c);
    lma_free(c);
    c.U64.free(); c.U32.free(); c.clov64.free(); c.clov32.free(); c.Uds.free(); c.clovds.free(); c.clov_user.free(); c.staging.free();
    c.red_partial.free(); c.red_out.free(); c.Dc.free(); c.Dc16.free(); c.Dcs.free();
    for (auto &b : c.user_bufs) b.free();
    if (c.pinned) cudaFreeHost(c.pinned);
    if (c.stream) cudaStreamDestroy(c.stream);
    delete ctx;
}

int mgeig_check_params(const int dims[4], const mgeig_params *p) {
    if (!dims || !p) return MGEIG_EINVAL;
    const int rc = check_dims(dims);
    return rc != MGEIG_OK ? rc : validate(dims, *p);
}

int mgeig_set_params(mgeig_ctx *ctx, const mgeig_params *p) {
    if (!ctx || !p) return MGEIG_EINVAL;
    return guarded(ctx, [&](Ctx &c) {
        int rc = validate(c.dims, *p);
        if (rc != MGEIG_OK) return rc;
        sync(c);
        mg_free(c);
        c.prm = *p;
        for (int mu = 0; mu < 4; ++mu) {
            c.g.bc[mu] = p->bc[mu];
            c.cdims[mu] = c.dims[mu] / p->agg[mu];
        }
        c.nagg = c.cdims[0] * c.cdims[1] * c.cdims[2] * c.cdims[3];
        c.agg_vol = p->agg[0] * p->agg[1] * p->agg[2] * p->agg[3];
        c.sap_vol = p->sap_block[0] * p->sap_block[1] * p->sap_block[2] * p->sap_block[3];
        c.sap_nblk = (int)(c.g.V / c.sap_vol);
        c.have_setup = false;
        if (c.have_gauge) refresh_clover(c);
        mg_alloc(c);
        sync(c);
        return MGEIG_OK;
    });
}

int mgeig_load_gauge(mgeig_ctx *ctx, const double *U) {
    if (!ctx || !U) return MGEIG_EINVAL;
    return guarded(ctx, [&](Ctx &c) {
        MG_CUDA(cudaMemcpyAsync(c.staging.p, U, (size_t)c.g.V * 4 * 9 * 16, cudaMemcpyHostToDevice, c.stream));
        pack_gauge(c, c.staging.as<double>());
        c.clover_loaded = false;
        c.clov_user.free();
        build_clover(c);
        c.have_gauge = true;
        c.have_setup = false;
        sync(c);
        return MGEIG_OK;
    });
}

int mgeig_load_gauge_dev(mgeig_ctx *ctx, const void *U_dev) {
    if (!ctx || !U_dev) return MGEIG_EINVAL;
    return guarded(ctx, [&](Ctx &c) {
        pack_gauge(c, static_cast<const double *>(U_dev));
        c.clover_loaded = false;
        c.clov_user.free();
        build_clover(c);
        c.have_gauge = true;
        c.have_setup = false;
        sync(c);
        return MGEIG_OK;
    });
}

int mgeig_load_clover(mgeig_ctx *ctx, const double *A) {
    if (!ctx) return MGEIG_EINVAL;
    return guarded(ctx, [&](Ctx &c) {
        if (!c.have_gauge) return MGEIG_ENOTSETUP;
        sync(c);
        if (A) {
            const size_t bytes = (size_t)c.g.V * 72 * 16;
            c.clov_user.alloc(bytes);
            MG_CUDA(cudaMemcpyAsync(c.clov_user.p, A, bytes, cudaMemcpyHostToDevice, c.stream));
            c.clover_loaded = true;
        } else {
            c.clover_loaded = false;
            c.clov_user.free();
        }
        refresh_clover(c);
        c.have_setup = false;
        sync(c);
        return MGEIG_OK;
    });
}

int mgeig_get_clover(mgeig_ctx *ctx, double *A) {
    if (!ctx || !A) return MGEIG_EINVAL;
    return guarded(ctx, [&](Ctx &c) {
        if (!c.have_gauge) return MGEIG_ENOTSETUP;
        TmpBuf tmp;
        tmp.alloc((size_t)c.g.V * 72 * 16);
        unpack_clover(c, tmp.as<double>());
        MG_CUDA(cudaMemcpyAsync(A, tmp.p, (size_t)c.g.V * 72 * 16, cudaMemcpyDeviceToHost, c.stream));
        sync(c);
        tmp.free();
        return MGEIG_OK;
    });
}

int mgeig_alloc_dev(mgeig_ctx *ctx, size_t bytes, void **ptr) {
    if (!ctx || !ptr) return MGEIG_EINVAL;
    *ptr = nullptr;
    return guarded(ctx, [&](Ctx &c) {
        DevBuf b;
        b.alloc(bytes);
        c.user_bufs.push_back(b);
        *ptr = b.p;
        return MGEIG_OK;
    });
}

int mgeig_pack_spinors(mgeig_ctx *ctx, int prec, const double *host, void *dev, int n_fields) {
    if (!ctx || !host || !dev || n_fields < 1) return MGEIG_EINVAL;
    if (prec != MGEIG_PREC_F64 && prec != MGEIG_PREC_F32) return MGEIG_EINVAL;
    return guarded(ctx, [&](Ctx &c) {
        TmpBuf t;
        if (prec == MGEIG_PREC_F32) t.alloc(spinor_bytes(c));
        for (int f = 0; f < n_fields; ++f) {
            const double *h = host + (size_t)f * c.fine_ncpx() * 2;
            if (prec == MGEIG_PREC_F64) {
                host_to_internal(c, h, static_cast<char *>(dev) + (size_t)f * spinor_bytes(c));
            } else {
                host_to_internal(c, h, t.p);
                convert_f64_to_f32(c, t.p, static_cast<char *>(dev) + (size_t)f * spinor_bytes(c) / 2, c.fine_ncpx());
            }
        }
        sync(c);
        t.free();
        return MGEIG_OK;
    });
}

int mgeig_unpack_spinors(mgeig_ctx *ctx, int prec, const void *dev, double *host, int n_fields) {
    if (!ctx || !host || !dev || n_fields < 1) return MGEIG_EINVAL;
    if (prec != MGEIG_PREC_F64 && prec != MGEIG_PREC_F32) return MGEIG_EINVAL;
    return guarded(ctx, [&](Ctx &c) {
        TmpBuf t;
        if (prec == MGEIG_PREC_F32) t.alloc(spinor_bytes(c));
        for (int f = 0; f < n_fields; ++f) {
            double *h = host + (size_t)f * c.fine_ncpx() * 2;
            if (prec == MGEIG_PREC_F64) {
                internal_to_host(c, static_cast<const char *>(dev) + (size_t)f * spinor_bytes(c), h);
            } else {
                convert_f32_to_f64(c, static_cast<const char *>(dev) + (size_t)f * spinor_bytes(c) / 2, t.p, c.fine_ncpx());
                internal_to_host(c, t.p, h);
            }
        }
        return MGEIG_OK;
    });
}

static int check_op(int op, int prec) {
    if (op != MGEIG_OP_Q && op != MGEIG_OP_D) return MGEIG_EINVAL;
    if (prec != MGEIG_PREC_F64 && prec != MGEIG_PREC_F32) return MGEIG_EINVAL;
    return MGEIG_OK;
}

int mgeig_apply(mgeig_ctx *ctx, double sigma, int op, int prec, const double *x, double *y, int nrhs) {
    if (!ctx || !x || !y || nrhs < 1) return MGEIG_EINVAL;
    if (check_op(op, prec) != MGEIG_OK) return MGEIG_EINVAL;
    return guarded(ctx, [&](Ctx &c) {
        if (!c.have_gauge) return MGEIG_ENOTSETUP;
        const int mode = op == MGEIG_OP_Q ? MODE_QSIGMA : MODE_DSIGMA;
        const size_t sb = spinor_bytes(c);
        TmpBuf a, b, a32, b32;
        a.alloc(sb * nrhs);
        b.alloc(sb * nrhs);
        if (prec == MGEIG_PREC_F32) { a32.alloc(sb / 2 * nrhs); b32.alloc(sb / 2 * nrhs); }
        for (int r = 0; r < nrhs; ++r) {
            host_to_internal(c, x + (size_t)r * c.fine_ncpx() * 2, a.as<char>() + sb * r);
            if (prec == MGEIG_PREC_F32) convert_f64_to_f32(c, a.as<char>() + sb * r, a32.as<char>() + sb / 2 * r, c.fine_ncpx());
        }
        // all right-hand sides in one launch (links and clover read once for all)
        if (prec == MGEIG_PREC_F64) apply_fine_nrhs<double>(c, mode, sigma, a.p, b.p, nrhs);
        else apply_fine_nrhs<float>(c, mode, sigma, a32.p, b32.p, nrhs);
        for (int r = 0; r < nrhs; ++r) {
            if (prec == MGEIG_PREC_F32) convert_f32_to_f64(c, b32.as<char>() + sb / 2 * r, b.as<char>() + sb * r, c.fine_ncpx());
            internal_to_host(c, b.as<char>() + sb * r, y + (size_t)r * c.fine_ncpx() * 2);
        }
        a.free(); b.free(); a32.free(); b32.free();
        return MGEIG_OK;
    });
}

int mgeig_apply_dev(mgeig_ctx *ctx, double sigma, int op, int prec, const void *x, void *y) {
    if (!ctx || !x || !y) return MGEIG_EINVAL;
    const bool ds = prec == MGEIG_PREC_F64_DS || prec == MGEIG_PREC_F32_F64_DS;
    if (check_op(op, ds ? MGEIG_PREC_F64 : prec) != MGEIG_OK) return MGEIG_EINVAL;
    return guarded(ctx, [&](Ctx &c) {
        if (!c.have_gauge) return MGEIG_ENOTSETUP;
        const int mode = op == MGEIG_OP_Q ? MODE_QSIGMA : MODE_DSIGMA;
        if (ds) apply_fine_ds(c, mode, sigma, x, y, prec == MGEIG_PREC_F32_F64_DS);
        else if (prec == MGEIG_PREC_F64) apply_fine_fp64(c, mode, sigma, x, y);
        else apply_fine<float>(c, mode, sigma, x, y);
        return MGEIG_OK;
    });
}

int mgeig_apply_dev_nrhs(mgeig_ctx *ctx, double sigma, int op, int prec, const void *x, void *y, int nrhs) {
    if (!ctx || !x || !y || nrhs < 1) return MGEIG_EINVAL;
    if (check_op(op, prec) != MGEIG_OK) return MGEIG_EINVAL;
    return guarded(ctx, [&](Ctx &c) {
        if (!c.have_gauge) return MGEIG_ENOTSETUP;
        const size_t fb = c.fine_ncpx() * (prec == MGEIG_PREC_F64 ? 16 : 8) * (size_t)nrhs;
        const char *xb = static_cast<const char *>(x), *yb = static_cast<const char *>(y);
        if (xb < yb + fb && yb < xb + fb) return MGEIG_EINVAL;   // the fields must not overlap
        const int mode = op == MGEIG_OP_Q ? MODE_QSIGMA : MODE_DSIGMA;
        if (prec == MGEIG_PREC_F64) apply_fine_nrhs<double>(c, mode, sigma, x, y, nrhs);
        else apply_fine_nrhs<float>(c, mode, sigma, x, y, nrhs);
        return MGEIG_OK;
    });
}

static int need_setup(Ctx &c) {
    if (!c.have_gauge) return MGEIG_ENOTSETUP;
    if (!c.work) return MGEIG_ENOTSETUP;
    return MGEIG_OK;
}

static void begin_stats(Ctx &c) {
    std::memset(&c.st, 0, sizeof(c.st));
    c.st.kernel_launches = -c.launches;
}
static void end_stats(Ctx &c, mgeig_stats *out, std::chrono::steady_clock::time_point t0) {
    coarse_iters_take(c);
    c.st.kernel_launches += c.launches;
    c.st.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (out) *out = c.st;
}

int mgeig_setup(mgeig_ctx *ctx, uint64_t seed, mgeig_stats *stats) {
    return guarded(ctx, [&](Ctx &c) {
        int rc = need_setup(c);
        if (rc) return rc;
        auto t0 = std::chrono::steady_clock::now();
        begin_stats(c);
        setup(c, seed);
        end_stats(c, stats, t0);
        return MGEIG_OK;
    });
}

int mgeig_set_test_vectors(mgeig_ctx *ctx, const double *W) {
    if (!W) return MGEIG_EINVAL;
    return guarded(ctx, [&](Ctx &c) {
        int rc = need_setup(c);
        if (rc) return rc;
        for (int j = 0; j < c.prm.n_tv; ++j) host_to_internal(c, W + (size_t)j * c.fine_ncpx() * 2, mg_test_vector(c, j));
        mg_use_test_vectors(c);
        mg_rebuild(c);
        sync(c);
        c.have_setup = true;
        return MGEIG_OK;
    });
}

int mgeig_get_test_vectors(mgeig_ctx *ctx, double *W) {
    if (!W) return MGEIG_EINVAL;
    return guarded(ctx, [&](Ctx &c) {
        if (!c.have_setup) return MGEIG_ENOTSETUP;
        for (int j = 0; j < c.prm.n_tv; ++j) internal_to_host(c, mg_test_vector(c, j), W + (size_t)j * c.fine_ncpx() * 2);
        return MGEIG_OK;
    });
}

int mgeig_get_interp(mgeig_ctx *ctx, double *P) {
    if (!P) return MGEIG_EINVAL;
    return guarded(ctx, [&](Ctx &c) {
        if (!c.have_setup) return MGEIG_ENOTSETUP;
        const int ntv = c.prm.n_tv;
        std::vector<TmpBuf> tmp(ntv);
        std::vector<void *> ptr(ntv);
        for (int j = 0; j < ntv; ++j) { tmp[j].alloc(spinor_bytes(c)); ptr[j] = tmp[j].p; }
        interp_f64(c, ptr.data());
        for (int j = 0; j < ntv; ++j) internal_to_host(c, ptr[j], P + (size_t)j * c.fine_ncpx() * 2);
        for (auto &t : tmp) t.free();
        return MGEIG_OK;
    });
}

int mgeig_get_coarse_op(mgeig_ctx *ctx, double *Dc) {
    if (!Dc) return MGEIG_EINVAL;
    return guarded(ctx, [&](Ctx &c) {
        if (!c.have_setup) return MGEIG_ENOTSETUP;
        const int n2 = 2 * c.prm.n_tv;
        const size_t bytes = (size_t)9 * c.nagg * n2 * n2 * 16;
        TmpBuf t;
        t.alloc(bytes);
        coarse_op_f64(c, t.p);
        MG_CUDA(cudaMemcpyAsync(Dc, t.p, bytes, cudaMemcpyDeviceToHost, c.stream));
        sync(c);
        t.free();
        return MGEIG_OK;
    });
}

int mgeig_restrict(mgeig_ctx *ctx, const double *r, double *rc) {
    if (!r || !rc) return MGEIG_EINVAL;
    return guarded(ctx, [&](Ctx &c) {
        if (!c.have_setup) return MGEIG_ENOTSETUP;
        TmpBuf a, b;
        a.alloc(spinor_bytes(c));
        b.alloc(c.coarse_ncpx() * 16);
        host_to_internal(c, r, a.p);
        restrict_f64(c, a.p, b.p);
        MG_CUDA(cudaMemcpyAsync(rc, b.p, c.coarse_ncpx() * 16, cudaMemcpyDeviceToHost, c.stream));
        sync(c);
        return MGEIG_OK;
    });
}

int mgeig_prolong(mgeig_ctx *ctx, const double *ec, double *e) {
    if (!ec || !e) return MGEIG_EINVAL;
    return guarded(ctx, [&](Ctx &c) {
        if (!c.have_setup) return MGEIG_ENOTSETUP;
        TmpBuf a, b;
        a.alloc(c.coarse_ncpx() * 16);
        b.alloc(spinor_bytes(c));
        MG_CUDA(cudaMemcpyAsync(a.p, ec, c.coarse_ncpx() * 16, cudaMemcpyHostToDevice, c.stream));
        prolong_f64(c, a.p, b.p);
        internal_to_host(c, b.p, e);
        return MGEIG_OK;
    });
}

int mgeig_coarse_apply(mgeig_ctx *ctx, double sigma, const double *xc, double *yc) {
    if (!xc || !yc) return MGEIG_EINVAL;
    return guarded(ctx, [&](Ctx &c) {
        if (!c.have_setup) return MGEIG_ENOTSETUP;
        TmpBuf a, b;
        a.alloc(c.coarse_ncpx() * 16);
        b.alloc(c.coarse_ncpx() * 16);
        MG_CUDA(cudaMemcpyAsync(a.p, xc, c.coarse_ncpx() * 16, cudaMemcpyHostToDevice, c.stream));
        coarse_apply_f64(c, sigma, a.p, b.p);
        MG_CUDA(cudaMemcpyAsync(yc, b.p, c.coarse_ncpx() * 16, cudaMemcpyDeviceToHost, c.stream));
        sync(c);
        return MGEIG_OK;
    });
}

int mgeig_coarse_apply_nrhs(mgeig_ctx *ctx, double sigma, const double *xc, double *yc, int nrhs) {
    if (!xc || !yc || nrhs < 1 || nrhs > 16) return MGEIG_EINVAL;
    return guarded(ctx, [&](Ctx &c) {
        if (!c.have_setup) return MGEIG_ENOTSETUP;
        const size_t n = c.coarse_ncpx(), b64 = n * 16 * nrhs;
        TmpBuf a, b, a32, b32;
        a.alloc(b64);
        b.alloc(b64);
        MG_CUDA(cudaMemcpyAsync(a.p, xc, b64, cudaMemcpyHostToDevice, c.stream));
        if (c.mixed()) {
            a32.alloc(b64 / 2);
            b32.alloc(b64 / 2);
            coarse_flat_convert(c, a.p, a32.p, n * nrhs, true);
            coarse_apply_nrhs(c, sigma, a32.p, b32.p, nrhs);
            coarse_flat_convert(c, b32.p, b.p, n * nrhs, false);
        } else {
            for (int r = 0; r < nrhs; ++r)
                coarse_apply<double>(c, c.Dc.p, sigma, a.as<char>() + n * 16 * r, b.as<char>() + n * 16 * r, false);
        }
        MG_CUDA(cudaMemcpyAsync(yc, b.p, b64, cudaMemcpyDeviceToHost, c.stream));
        sync(c);
        return MGEIG_OK;
    });
}

int mgeig_coarse_apply_dev_nrhs(mgeig_ctx *ctx, double sigma, const void *X, void *Y, int nrhs) {
    if (!X || !Y || nrhs < 1 || nrhs > 16) return MGEIG_EINVAL;
    return guarded(ctx, [&](Ctx &c) {
        if (!c.have_setup) return MGEIG_ENOTSETUP;
        if (!c.mixed()) return MGEIG_EINVAL;
        const size_t fb = c.coarse_ncpx() * 8 * (size_t)nrhs;
        const char *xb = static_cast<const char *>(X), *yb = static_cast<const char *>(Y);
        if (xb < yb + fb && yb < xb + fb) return MGEIG_EINVAL;
        coarse_apply_nrhs(c, sigma, X, Y, nrhs);
        return MGEIG_OK;
    });
}

int mgeig_sap(mgeig_ctx *ctx, double sigma, const double *b, double *z, int cycles) {
    if (!b || !z || cycles < 0) return MGEIG_EINVAL;
    return guarded(ctx, [&](Ctx &c) {
        if (!c.have_gauge || !c.work) return MGEIG_ENOTSETUP;
        TmpBuf a, bb;
        a.alloc(spinor_bytes(c));
        bb.alloc(spinor_bytes(c));
        host_to_internal(c, b, a.p);
        host_to_internal(c, z, bb.p);
        sap_smooth_f64(c, sigma, a.p, bb.p, cycles);
        internal_to_host(c, bb.p, z);
        return MGEIG_OK;
    });
}

int mgeig_mg_cycle(mgeig_ctx *ctx, double sigma, const double *r, double *z) {
    if (!r || !z) return MGEIG_EINVAL;
    return guarded(ctx, [&](Ctx &c) {
        if (!c.have_setup) return MGEIG_ENOTSETUP;
        TmpBuf a, b;
        a.alloc(spinor_bytes(c));
        b.alloc(spinor_bytes(c));
        host_to_internal(c, r, a.p);
        mg_cycle_host(c, sigma, a.as<double>(), b.as<double>());
        internal_to_host(c, b.p, z);
        coarse_iters_take(c);   // raises the coarse solver's timeout or breakdown
        return MGEIG_OK;
    });
}

int mgeig_mg_cycle_dev_noalloc(mgeig_ctx *ctx, double sigma, const void *r, void *z) {
    if (!r || !z || !std::isfinite(sigma)) return MGEIG_EINVAL;
    return guarded(ctx, [&](Ctx &c) {
        if (!c.have_setup) return MGEIG_ENOTSETUP;
        if (c.prm.smoother != MGEIG_SAP || c.timer.on) return MGEIG_EINVAL;
        // the prolongation writes z before the smoother reads r: they must not overlap
        const size_t nb = c.fine_ncpx() * 2 * c.level_bytes();
        const char *rb = static_cast<const char *>(r), *zb = static_cast<const char *>(z);
        if (rb < zb + nb && zb < rb + nb) return MGEIG_EINVAL;
        return mg_cycle_noalloc(c, sigma, r, z);
    });
}

int mgeig_solve(mgeig_ctx *ctx, double sigma, const double *b, double *x, double tol, mgeig_stats *stats) {
    if (!b || !x || !(tol > 0)) return MGEIG_EINVAL;
    return guarded(ctx, [&](Ctx &c) {
        if (!c.have_setup) return MGEIG_ENOTSETUP;
        auto t0 = std::chrono::steady_clock::now();
        begin_stats(c);
        TmpBuf a, bb;
        a.alloc(spinor_bytes(c));
        bb.alloc(spinor_bytes(c));
        host_to_internal(c, b, a.p);
        int rc = fgmres_solve(c, sigma, a.p, bb.p, tol);
        internal_to_host(c, bb.p, x);
        end_stats(c, stats, t0);
        return rc;
    });
}

int mgeig_solve_batch(mgeig_ctx *const *ctxs, int nctx, const double *sigmas, int nsig, const double *const *b,
                      double *const *x, int nrhs, double tol, mgeig_stats *stats) {
    if (!ctxs || nctx < 1 || !sigmas || nsig < 1 || !b || !x || nrhs < 1 || !(tol > 0)) return MGEIG_EINVAL;
    for (int k = 0; k < nctx; ++k)
        if (!ctxs[k] || !b[k] || !x[k]) return MGEIG_EINVAL;
    for (int s = 0; s < nsig; ++s)
        if (!std::isfinite(sigmas[s])) return MGEIG_EINVAL;
    mgeig_stats total{};
    int status = MGEIG_OK;
    const auto t0 = std::chrono::steady_clock::now();
    for (int k = 0; k < nctx; ++k) {
        int rc = guarded(ctxs[k], [&](Ctx &c) {
            if (!c.have_setup) return MGEIG_ENOTSETUP;
            begin_stats(c);
            const size_t nd = c.fine_ncpx() * 2;   // doubles per host spinor
            TmpBuf a, bb;
            a.alloc(spinor_bytes(c));
            bb.alloc(spinor_bytes(c));
            int worst = MGEIG_OK;
            // shift-major order: the coarse deflation data of a shift serves all right-hand sides
            for (int s = 0; s < nsig; ++s)
                for (int r = 0; r < nrhs; ++r) {
                    host_to_internal(c, b[k] + nd * r, a.p);
                    const int rc1 = fgmres_solve(c, sigmas[s], a.p, bb.p, tol);
                    if (rc1 != MGEIG_OK && rc1 != MGEIG_ENOCONV) return rc1;
                    if (rc1 == MGEIG_ENOCONV) worst = MGEIG_ENOCONV;
                    internal_to_host(c, bb.p, x[k] + nd * ((size_t)s * nrhs + r));
                }
            coarse_iters_take(c);
            c.st.kernel_launches += c.launches;
            total.solves += c.st.solves;
            total.outer_iters += c.st.outer_iters;
            total.mg_cycles += c.st.mg_cycles;
            total.coarse_iters += c.st.coarse_iters;
            total.fine_applies += c.st.fine_applies;
            total.kernel_launches += c.st.kernel_launches;
            return worst;
        });
        if (rc != MGEIG_OK && rc != MGEIG_ENOCONV) return rc;
        if (rc == MGEIG_ENOCONV) status = MGEIG_ENOCONV;
    }
    total.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (stats) *stats = total;
    return status;
}

int mgeig_solve_d(mgeig_ctx *ctx, double sigma, const double *b, double *x, double tol, mgeig_stats *stats) {
    if (!b || !x || !(tol > 0)) return MGEIG_EINVAL;
    return guarded(ctx, [&](Ctx &c) {
        if (!c.have_setup) return MGEIG_ENOTSETUP;
        auto t0 = std::chrono::steady_clock::now();
        begin_stats(c);
        TmpBuf a, bb;
        a.alloc(spinor_bytes(c));
        bb.alloc(spinor_bytes(c));
        host_to_internal(c, b, a.p);
        int rc = fgmres_solve_d(c, sigma, a.p, bb.p, tol);
        internal_to_host(c, bb.p, x);
        end_stats(c, stats, t0);
        return rc;
    });
}

int mgeig_eigensolve(mgeig_ctx *ctx, int n_eig, double tol, double *evals, double *evecs, double *resid,
                     mgeig_stats *stats) {
    return guarded(ctx, [&](Ctx &c) {
        if (!c.have_setup) return MGEIG_ENOTSETUP;
        if (n_eig < 1 || n_eig > MAX_ITERATED || !(tol > 0)) return MGEIG_EINVAL;
        auto t0 = std::chrono::steady_clock::now();
        begin_stats(c);
        int rc = eigensolve(c, n_eig, tol, evals, evecs, resid);
        sync(c);
        end_stats(c, stats, t0);
        return rc;
    });
}

int mgeig_set_timing(mgeig_ctx *ctx, int on) {
    return guarded(ctx, [&](Ctx &c) {
        c.timer.reset();
        c.timer.on = on != 0;
        c.timer.mask = ~0u;
        return MGEIG_OK;
    });
}

int mgeig_set_timing_classes(mgeig_ctx *ctx, unsigned int mask) {
    return guarded(ctx, [&](Ctx &c) {
        c.timer.reset();
        c.timer.on = mask != 0;
        c.timer.mask = mask;
        return MGEIG_OK;
    });
}

int mgeig_kernel_times(mgeig_ctx *ctx, int n, long long *launches, double *ms, double *bytes, const char **names) {
    static const char *kNames[K_NCLASS] = {"stencil_f64", "stencil_f32", "sap_f64",      "sap_f32",
                                           "restrict",    "prolong",     "coarse_apply", "coarse_build",
                                           "interp_build", "blas_f64",   "blas_low",     "other",
                                           "coarse_gmres", "net"};
    return guarded(ctx, [&](Ctx &c) {
        c.timer.flush();
        for (int k = 0; k < n && k < K_NCLASS; ++k) {
            if (launches) launches[k] = c.timer.launches[k];
            if (ms) ms[k] = c.timer.ms[k];
            if (bytes) bytes[k] = c.timer.total_bytes[k];
            if (names) names[k] = kNames[k];
        }
        return (int)K_NCLASS;
    });
}

int mgeig_lma_prepare(mgeig_ctx *ctx, int n, const double *V, double cutoff, double *lam, double *eps, int *kept,
                      int *n_kept, double *A, double *Ainv, double *Llow) {
    if (n < 1 || n > MAX_ITERATED || !(cutoff > 0)) return MGEIG_EINVAL;
    return guarded(ctx, [&](Ctx &c) {
        if (!c.have_gauge) return MGEIG_ENOTSETUP;
        if (!V && !c.have_setup) return MGEIG_ENOTSETUP;
        if (!V && n > c.prm.n_tv) return MGEIG_EINVAL;
        void *dev = lma_vectors(c, n);
        const size_t sb = spinor_bytes(c);
        for (int i = 0; i < n; ++i) {
            void *dst = static_cast<char *>(dev) + sb * i;
            if (V) host_to_internal(c, V + (size_t)i * c.fine_ncpx() * 2, dst);
            else MG_CUDA(cudaMemcpyAsync(dst, mg_test_vector(c, i), sb, cudaMemcpyDeviceToDevice, c.stream));
        }
        lma_prepare(c, n, dev, V == nullptr, cutoff, lam, eps, kept, n_kept, A, Ainv, Llow);
        sync(c);
        return MGEIG_OK;
    });
}

int mgeig_lma_apply(mgeig_ctx *ctx, int mode, const double *x, double *y) {
    if (!x || !y || (mode != 0 && mode != 1)) return MGEIG_EINVAL;
    return guarded(ctx, [&](Ctx &c) {
        if (!c.lma) return MGEIG_ENOTSETUP;
        TmpBuf a, b;
        a.alloc(spinor_bytes(c));
        b.alloc(spinor_bytes(c));
        host_to_internal(c, x, a.p);
        lma_apply(c, mode, a.p, b.p);
        internal_to_host(c, b.p, y);
        return MGEIG_OK;
    });
}

int mgeig_lma_loop_high(mgeig_ctx *ctx, int nstoch, uint64_t seed, double tol, double *Lhigh, mgeig_stats *stats) {
    if (nstoch < 1 || !(tol > 0) || !Lhigh) return MGEIG_EINVAL;
    return guarded(ctx, [&](Ctx &c) {
        if (!c.lma || !c.have_setup) return MGEIG_ENOTSETUP;
        auto t0 = std::chrono::steady_clock::now();
        begin_stats(c);
        lma_loop_high(c, nstoch, seed, tol, Lhigh, nullptr);
        end_stats(c, stats, t0);
        return MGEIG_OK;
    });
}

int mgeig_net_init(mgeig_ctx *ctx, uint64_t seed) {
    return guarded(ctx, [&](Ctx &c) {
        net_init(c, seed);
        return MGEIG_OK;
    });
}

int mgeig_net_set_weights(mgeig_ctx *ctx, const float *W) {
    if (!W) return MGEIG_EINVAL;
    return guarded(ctx, [&](Ctx &c) {
        net_set_weights(c, W);
        return MGEIG_OK;
    });
}

int mgeig_net_get_weights(mgeig_ctx *ctx, float *W) {
    if (!W) return MGEIG_EINVAL;
    return guarded(ctx, [&](Ctx &c) {
        net_get_weights(c, W);
        return MGEIG_OK;
    });
}

int mgeig_net_train(mgeig_ctx *ctx, int steps, int batch, double lr, uint64_t seed, double *losses) {
    if (steps < 1 || batch < 1 || batch > 64 || !(lr > 0)) return MGEIG_EINVAL;
    return guarded(ctx, [&](Ctx &c) {
        if (!c.have_setup) return MGEIG_ENOTSETUP;
        if (!c.mixed() || !net_supported(c)) return MGEIG_EINVAL;
        net_train(c, steps, batch, lr, seed, losses);
        return MGEIG_OK;
    });
}

int mgeig_net_loss_grads(mgeig_ctx *ctx, const double *x, const double *t, int batch, double *loss, float *G) {
    if (!x || !t || !loss || !G || batch < 1 || batch > 64) return MGEIG_EINVAL;
    return guarded(ctx, [&](Ctx &c) {
        *loss = net_loss_grads(c, x, t, batch, G);
        return MGEIG_OK;
    });
}

int mgeig_net_apply(mgeig_ctx *ctx, const double *r, double *e) {
    if (!r || !e) return MGEIG_EINVAL;
    return guarded(ctx, [&](Ctx &c) {
        const size_t sb = spinor_bytes(c);
        TmpBuf a, a32, z32;
        a.alloc(sb);
        a32.alloc(sb / 2);
        z32.alloc(sb / 2);
        host_to_internal(c, r, a.p);
        convert_f64_to_f32(c, a.p, a32.p, c.fine_ncpx());
        MG_CUDA(cudaMemsetAsync(z32.p, 0, sb / 2, c.stream));
        net_smooth(c, a32.p, z32.p);
        convert_f32_to_f64(c, z32.p, a.p, c.fine_ncpx());
        internal_to_host(c, a.p, e);
        return MGEIG_OK;
    });
}

int mgeig_multidot_dev(mgeig_ctx *ctx, int prec, int k, const void *const *X, const void *y, long long n,
                       double *d) {
    if (!ctx || !X || !y || !d || k < 1 || k > 32 || n < 1) return MGEIG_EINVAL;
    if (prec != MGEIG_PREC_F64 && prec != MGEIG_PREC_F32) return MGEIG_EINVAL;
    for (int j = 0; j < k; ++j)
        if (!X[j]) return MGEIG_EINVAL;
    return guarded(ctx, [&](Ctx &c) {
        blas_dot_host(c, prec == MGEIG_PREC_F32, k, X, y, (size_t)n, d);
        return MGEIG_OK;
    });
}

int mgeig_multi_axpy_dev(mgeig_ctx *ctx, int prec, int k, const void *const *X, const double *cf, void *y,
                         long long n) {
    if (!ctx || !X || !y || !cf || k < 1 || k > 32 || n < 1) return MGEIG_EINVAL;
    if (prec != MGEIG_PREC_F64 && prec != MGEIG_PREC_F32) return MGEIG_EINVAL;
    for (int j = 0; j < k; ++j)
        if (!X[j] || X[j] == y) return MGEIG_EINVAL;
    return guarded(ctx, [&](Ctx &c) {
        blas_axpy_host(c, prec == MGEIG_PREC_F32, k, X, cf, y, (size_t)n);
        return MGEIG_OK;
    });
}

int mgeig_fma_peak(mgeig_ctx *ctx, int prec, int reps, double *flops) {
    if (!ctx || !flops || reps < 1 || (prec != MGEIG_PREC_F64 && prec != MGEIG_PREC_F32)) return MGEIG_EINVAL;
    return guarded(ctx, [&](Ctx &c) {
        *flops = fma_peak_flops(c, prec, reps);
        return MGEIG_OK;
    });
}

int mgeig_get_stream(mgeig_ctx *ctx, void **stream) {
    if (!ctx || !stream) return MGEIG_EINVAL;
    *stream = (void *)ctx->c.stream;
    return MGEIG_OK;
}

int mgeig_get_launch_count(mgeig_ctx *ctx, long long *count) {
    if (!ctx || !count) return MGEIG_EINVAL;
    *count = ctx->c.launches;
    return MGEIG_OK;
}

const char *mgeig_strerror(int status) {
    switch (status) {
        case MGEIG_OK: return "ok";
        case MGEIG_EINVAL: return "invalid argument";
        case MGEIG_ENOTSETUP: return "gauge field or multigrid setup missing";
        case MGEIG_ECUDA: return "CUDA runtime error";
        case MGEIG_ENOCONV: return "iteration cap reached before convergence";
        case MGEIG_EBREAKDOWN: return "numerical breakdown (NaN/Inf or zero vector)";
        case MGEIG_ENOMEM: return "device memory allocation failed";
        case MGEIG_ETIMEOUT: return "a bounded device-side wait expired";
        case MGEIG_ESCRATCH: return "coarse grid too large for the static scratch of mgeig_mg_cycle_dev_noalloc";
        default: return "unknown status";
    }
}

}  // extern "C"
