// Host-side internals of libmgeig: the context, device buffers, launch wrappers.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/mgeig.h"
#include "common.cuh"

namespace mgeig {

// Status propagation: every CUDA runtime error becomes MGEIG_ECUDA, with the
// message kept in the context for mgeig_strerror-style diagnostics on stderr.
struct Error {
    int code;
};

#define MG_CUDA(call)                                                                      \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            fprintf(stderr, "libmgeig: %s failed: %s (%s:%d)\n", #call, cudaGetErrorString(e_), \
                    __FILE__, __LINE__);                                                   \
            (void)cudaGetLastError(); /* a launch error must not be reported again later */ \
            throw ::mgeig::Error{e_ == cudaErrorMemoryAllocation ? MGEIG_ENOMEM : MGEIG_ECUDA}; \
        }                                                                                  \
    } while (0)

// every kernel launch of the library is followed by this check, which also
// counts it on the context `c` in scope
#define MG_CHECK_LAUNCH()                \
    do {                                 \
        MG_CUDA(cudaGetLastError());     \
        ++c.launches;                    \
    } while (0)

#define MG_REQUIRE(cond, code)           \
    do {                                 \
        if (!(cond)) throw ::mgeig::Error{code}; \
    } while (0)

// A device allocation owned by the context.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    void alloc(size_t n);
    void free();
    template <typename T> T *as() const { return static_cast<T *>(p); }
};

// A scoped device allocation, released when it goes out of scope.
struct TmpBuf : DevBuf {
    TmpBuf() = default;
    TmpBuf(const TmpBuf &) = delete;
    TmpBuf &operator=(const TmpBuf &) = delete;
    ~TmpBuf() { free(); }
};

// Kernel classes with per-class CUDA event timing (off unless enabled).
enum KernelClass {
    K_STENCIL_F64 = 0, K_STENCIL_F32, K_SAP_F64, K_SAP_F32, K_RESTRICT, K_PROLONG,
    K_COARSE_APPLY, K_COARSE_BUILD, K_PBUILD, K_BLAS_F64, K_BLAS_LOW, K_OTHER, K_COARSE_SOLVE, K_NET, K_NCLASS
};

struct Timer {
    bool on = false;
    unsigned int mask = ~0u;            // kernel classes that record events while on
    cudaStream_t stream = nullptr;
    long long launches[K_NCLASS] = {};
    double ms[K_NCLASS] = {};
    double bytes[K_NCLASS] = {};        // algorithmic bytes of the last launch
    double total_bytes[K_NCLASS] = {};  // algorithmic bytes summed over launches
    std::vector<cudaEvent_t> pool;
    struct Pending { int cls; cudaEvent_t a, b; };
    std::vector<Pending> pending;
    size_t next = 0;
    cudaEvent_t begin(int cls);
    void end(int cls, cudaEvent_t a, double bytes);
    void flush();
    void reset();
    ~Timer();
};

// RAII bracket around one launch of a kernel class.
struct TimeScope {
    Timer &t; int cls; double bytes; cudaEvent_t a = nullptr;
    TimeScope(Timer &t_, int cls_, double bytes_) : t(t_), cls(cls_), bytes(bytes_) {
        if (t.on && (t.mask >> cls & 1u)) a = t.begin(cls);
        t.launches[cls] += 1;
        t.total_bytes[cls] += bytes_;
    }
    ~TimeScope() { if (a) t.end(cls, a, bytes); else t.bytes[cls] = bytes; }
};

struct Ctx;
struct Net;   // the learned smoother's weights and activations (learned.cu)
struct Lma;   // approximate low-mode averaging state (solver.cu)

// ----- fine operator (fine_op.cu) -----
void pack_gauge(Ctx &c, const double *dev_host_layout);
void build_clover(Ctx &c);
// packs a caller's clover term (device, [site][2][6][6] complex128, no mass term)
void pack_clover(Ctx &c, const double *dev_in);
// the clover term of the operator: the loaded one, else built from the gauge field
void refresh_clover(Ctx &c);
void unpack_clover(Ctx &c, double *dev_out);
template <typename R> void apply_fine(Ctx &c, int mode, double sigma, const void *x, void *y);
// nrhs fields stored back to back, one launch
template <typename R> void apply_fine_nrhs(Ctx &c, int mode, double sigma, const void *x, void *y, int nrhs);
// x in FP32 internal layout, y FP64: y = op(x) in FP64 arithmetic
void apply_fine_f64_from_f32(Ctx &c, int mode, double sigma, const void *x32, void *y64);
void apply_fine_fp64(Ctx &c, int mode, double sigma, const void *x, void *y);
void apply_fine_ds(Ctx &c, int mode, double sigma, const void *x, void *y, bool x_fp32);
void pack_spinor_f64(Ctx &c, const double *host_layout_dev, void *out, int n);
void unpack_spinor_f64(Ctx &c, const void *in, double *host_layout_dev, int n);
void convert_f64_to_f32(Ctx &c, const void *in64, void *out32, size_t ncomplex);
void convert_f32_to_f64(Ctx &c, const void *in32, void *out64, size_t ncomplex);
void random_spinors(Ctx &c, uint64_t seed, void *out64, int n, uint32_t tag);
constexpr int MAX_ITERATED = 64;   // vectors iterated by Algorithm 1

// ----- BLAS-1 on flat complex arrays (blas.cu) -----
// Results of reductions land in device memory (cpx<double>); *_host variants sync.
template <typename R> void blas_multidot(Ctx &c, const void *const *X, int k, const void *y, size_t n, cpx<double> *d_out);
template <typename R> void blas_multi_axpy(Ctx &c, void *y, const void *const *X, int k, const cpx<double> *d_coef, double sign, size_t n);
void small_gemv(Ctx &c, const cpx<double> *A, int k, const cpx<double> *x, double s, cpx<double> *y, cpx<double> *ys);
template <typename R> void blas_norm2(Ctx &c, const void *x, size_t n, cpx<double> *d_out);
template <typename R> void blas_axpy(Ctx &c, cpx<double> a, const void *x, void *y, size_t n);
template <typename R> void blas_scale(Ctx &c, cpx<double> a, void *x, size_t n);
template <typename R> void blas_copy(Ctx &c, const void *x, void *y, size_t n);
template <typename R> void blas_zero(Ctx &c, void *x, size_t n);
// y (FP64) += a * x (R)
template <typename R> void blas_axpy_to_f64(Ctx &c, cpx<double> a, const void *x, void *y64, size_t n);
// y = x - lambda_dev[0] * v ; out = ||y||^2  (FP64; lambda on the device)
void blas_resid_norm2(Ctx &c, const void *qv, const void *v, const cpx<double> *d_lambda, size_t n, cpx<double> *d_out);

// ----- multigrid (mg.cu) -----
template <typename R> void build_interp(Ctx &c, const void *const *W64, int ntv, void *const *P);
template <typename R> void restrict_vec(Ctx &c, const void *const *P, const void *r, void *rc);
template <typename R> void prolong_vec(Ctx &c, const void *const *P, const void *ec, void *e);
template <typename R> void build_coarse(Ctx &c, const void *const *P, void *Dc);
template <typename R> void coarse_apply(Ctx &c, const void *Dc, double sigma, const void *x, void *y, bool dform = false);
template <typename R> void coarse_gamma5(Ctx &c, const void *x, void *y);
template <typename R> void sap_sweep(Ctx &c, int colour, double sigma, const void *rhs, bool rhs_gamma5, void *z);

// ----- 16-bit coarse links (links16.cu) -----
void compress_coarse(Ctx &c);   // Dc (FP32) -> Dc16, Dcs in the format of prm.coarse_links
void coarse_apply_links16(Ctx &c, double sigma, const void *x, void *y, bool dform);
// Y = (Q_c - sigma) X for nrhs <= 16 FP32 coarse vectors back to back (tensor cores with BF16 links)
void coarse_apply_nrhs(Ctx &c, double sigma, const void *X, void *Y, int nrhs);
// n flat complex values FP64 -> FP32 (to32) or back (solver.cu)
void coarse_flat_convert(Ctx &c, const void *in, void *out, size_t n, bool to32);

// ----- persistent coarse GMRES (coarse_gmres.cu) -----
constexpr int COARSE_PERSISTENT_MAXM = 32;
struct CoarseSolveBufs {
    DevBuf *scratch;             // global scratch of the solver (coarse_gmres_scratch_bytes)
    void *state;                 // CGState (barrier, status, iteration counter)
    int k;                       // deflation vectors (0: none)
    const void *W, *AW, *Einv;   // k coarse vectors each; E^-1 (k x k complex double)
};
template <typename R>
void coarse_gmres_persistent(Ctx &c, const CoarseSolveBufs &B, double sigma, const void *rc, void *ec);
// the same solve with caller-placed scratch (coarse_gmres.cu): `scratch` holds
// coarse_gmres_scratch_bytes(c, k) bytes, `state` 16 bytes that are zero on entry
size_t coarse_gmres_scratch_bytes(Ctx &c, int k);
template <typename R>
void coarse_gmres_at(Ctx &c, double sigma, const void *rc, void *ec, void *scratch, void *state, int k,
                     const void *W, const void *AW, const void *Einv);

// ----- the context -----
struct Ctx {
    int dims[4];
    Geom g;
    int device = 0;
    int sms = 152;               // streaming multiprocessors of the device
    cudaStream_t stream = nullptr;
    mgeig_params prm;
    bool have_gauge = false;
    bool have_setup = false;
    bool in_setup = false;    // the setup's coarse solves run without deflation
    uint64_t setup_seed = 0;
    Timer timer;

    // fine fields
    DevBuf U64, U32, clov64, clov32;
    DevBuf Uds, clovds;          // double-float copies of U64, clov64 (float2 per double)
    bool ds_fields_valid = false;
    DevBuf clov_user;         // a clover term loaded by mgeig_load_clover (host layout)
    bool clover_loaded = false;
    DevBuf staging;           // host-layout transfer buffer
    std::vector<DevBuf> user_bufs;

    // reduction scratch
    DevBuf red_partial;       // per-block partial sums
    DevBuf red_out;           // reduction results (cpx<double>)
    size_t red_blocks = 0;
    double *pinned = nullptr; // host mirror of red_out

    // multigrid geometry
    int cdims[4] = {0, 0, 0, 0};
    int nagg = 0, agg_vol = 0;
    int sap_nblk = 0, sap_vol = 0;

    // test vectors (FP64) and interpolation / coarse operator in the level precision
    std::vector<DevBuf> W;    // ntv FP64 fine vectors
    std::vector<DevBuf> P;    // ntv vectors, R precision
    DevBuf Dc;                // [9][nagg][2N][2N] (column-major blocks), R precision
    DevBuf Dc16, Dcs;         // 16-bit links [9][nagg][re|im][2N][2N] and their scales [9][nagg]
    DevBuf cnbr;              // coarse neighbour table int32 [9][nagg]: self, then +mu, -mu for mu = 0..3

    size_t fine_ncpx() const { return (size_t)g.V * 12; }
    size_t coarse_ncpx() const { return (size_t)nagg * 2 * prm.n_tv; }
    bool mixed() const { return prm.precision == MGEIG_MIXED; }
    // FP64-storage BLAS and FP64-output stencil in double-float arithmetic
    // (mixed precision only)
    bool ds_blas() const { return prm.blas_ds != 0 && mixed() && !force_fp64; }
    bool ds_stencil() const { return prm.stencil_ds != 0 && mixed() && !force_fp64; }
    bool force_fp64 = false;     // set while a result is certified in FP64
    size_t level_bytes() const { return mixed() ? sizeof(float) : sizeof(double); }

    // host workspace counters
    mgeig_stats st{};
    long long launches = 0;   // kernel launches since the context was created

    // solver workspace (allocated lazily, see solver.cu)
    struct Work;
    Work *work = nullptr;
    Net *net = nullptr;       // the learned smoother (allocated on first use)
    Lma *lma = nullptr;       // approximate low-mode averaging (mgeig_lma_prepare)
};

// ----- solvers (solver.cu) -----
void ensure_reduction(Ctx &c, int max_vectors);
void sync(Ctx &c);
void read_reduction(Ctx &c, int n);   // copies n cpx<double> from red_out into pinned
cpx<double> host_red(Ctx &c, int i);

void mg_alloc(Ctx &c);
void coarse_iters_take(Ctx &c);
void mg_free(Ctx &c);
void *mg_test_vector(Ctx &c, int j);
void mg_use_test_vectors(Ctx &c);   // P is rebuilt from the test vectors (not the eigensolver's modes)
void mg_rebuild(Ctx &c);   // P and coarse operator from c.W
void setup(Ctx &c, uint64_t seed);
void mg_cycle_host(Ctx &c, double sigma, const double *r_dev64_internal, double *z_dev64_internal);
// the two-grid cycle on level-precision device spinors, scratch in a static device array
int mg_cycle_noalloc(Ctx &c, double sigma, const void *r, void *z);
size_t mg_cycle_noalloc_limit();
void noalloc_prepare(Ctx &c);   // the static array's address, looked up once per device
int fgmres_solve(Ctx &c, double sigma, const void *b64, void *x64, double tol, int maxiter = 0);
int fgmres_solve_d(Ctx &c, double sigma, const void *b64, void *x64, double tol);
int eigensolve(Ctx &c, int n_eig, double tol, double *evals, double *evecs_host, double *resid);
void sap_smooth_f64(Ctx &c, double sigma, const void *b64, void *z64, int cycles);
void coarse_apply_f64(Ctx &c, double sigma, const void *x64, void *y64);
void restrict_f64(Ctx &c, const void *r64, void *rc64);
void prolong_f64(Ctx &c, const void *ec64, void *e64);
void coarse_op_f64(Ctx &c, void *out64);
void interp_f64(Ctx &c, void *const *out64);

int grid_for(size_t n, int threads);

// ----- the learned smoother (learned.cu) -----
bool net_supported_dims(const int dims[4]);   // extents divisible by the 4 x 4 x 4 x 2 box
bool net_supported(const Ctx &c);             // the same for the context's lattice
void net_init(Ctx &c, uint64_t seed);
void net_set_weights(Ctx &c, const float *host);   // [3][81][32][32] FP32
void net_get_weights(Ctx &c, float *host);
void net_free(Ctx &c);
// z += ||r|| f(r / ||r||) for one FP32 spinor r (z FP32)
void net_smooth(Ctx &c, const void *r, void *z);
// one Adam step on batch pairs (FP32 spinors r_f, SAP corrections e_f back to back); returns the loss
double net_train_step(Ctx &c, const void *r, const void *e, int batch, double lr);
// loss and weight gradients for host channel data x, t [batch][V][24] FP64
double net_loss_grads(Ctx &c, const double *x, const double *t, int batch, float *G_host);
// ----- approximate low-mode averaging (lma.cu kernels, solver.cu host code) -----
// M[t][j][i] = sum_{x in timeslice t} <X_j(x) | Y_i(x)> for FP64 internal spinors (device output)
void timeslice_dots(Ctx &c, const void *const *X, int nj, const void *const *Y, int ni, void *M_dev);
void z2_spinors(Ctx &c, uint64_t seed, void *out64, int n, uint32_t tag);
// n FP64 internal vectors at V (device, overwritten by their orthonormalisation);
// outputs as in mgeig_lma_prepare (any may be NULL)
void lma_prepare(Ctx &c, int n, void *V, bool ritz, double cutoff, double *lam, double *eps, int *kept, int *n_kept,
                 double *A, double *Ainv, double *Llow);
void *lma_vectors(Ctx &c, int n);   // device room for n FP64 spinors owned by the LMA state
void lma_apply(Ctx &c, int mode, const void *x64, void *y64);
void lma_loop_high(Ctx &c, int nstoch, uint64_t seed, double tol, double *Lhigh, int *outer_iters);
void lma_free(Ctx &c);
// training pairs from the method and the training loop (solver.cu)
void net_train(Ctx &c, int steps, int batch, double lr, uint64_t seed, double *losses);
// FMA throughput (FLOP/s) of the library's own peak kernel, FP64 or FP32 (peak.cu)
double fma_peak_flops(Ctx &c, int prec, int reps);
void blas_dot_host(Ctx &c, bool f32, int k, const void *const *X, const void *y, size_t n, double *out);
void blas_axpy_host(Ctx &c, bool f32, int k, const void *const *X, const double *coef, void *y, size_t n);

}  // namespace mgeig
