/*
 * mgeig.h -- C ABI of libmgeig, a single-GPU (GB300, sm_103a) multigrid Rayleigh
 * quotient eigensolver for the Hermitian clover-improved Wilson operator.
 *
 * Method: Bali, Collins, Frommer, Kahl, Kanamori, Mueller, Rottmann, Simeth,
 * "(Approximate) Low-Mode Averaging with a new Multigrid Eigensolver",
 * arXiv:1509.06865 (Lattice 2015).  Section and equation numbers below refer
 * to that paper.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Lattice dims[4] = {Lx, Ly, Lz, Lt}; V = Lx*Ly*Lz*Lt sites.  Site index
 *    s = ((t*Lz + z)*Ly + y)*Lx + x.
 *  - Host gauge field: complex128 U[t][z][y][x][mu][a][b] (mu = 0..3 for
 *    x, y, z, t), stored as interleaved (re, im) doubles: V*4*9 complex numbers.
 *  - Host spinor field: complex128 psi[t][z][y][x][spin][colour], V*12 complex.
 *    Chiral gamma basis with gamma5 = -g1 g2 g3 g4 = diag(1, 1, -1, -1) (Sec. 2).
 *  - The operator (Sec. 2; the paper does not print D, this is the standard
 *    form, mass normalisation, Wilson r = 1):
 *      D psi(x) = (4 + m0) psi(x)
 *               - 1/2 sum_mu [(1 - g_mu) U_mu(x) psi(x+mu) + (1 + g_mu) U_mu(x-mu)^dag psi(x-mu)]
 *               + c_sw (i/4) sum_{mu,nu} sigma_{mu nu} F_{mu nu}(x) psi(x),
 *    with the four-leaf clover F = (Q_{mu nu} - Q_{mu nu}^dag)/8, sigma = (i/2)[g_mu, g_nu],
 *    g_k = [[0, i s_k], [-i s_k, 0]], g_4 = [[0, 1], [1, 0]].
 *    Q = gamma5 D (Hermitian), D_sigma = D - sigma gamma5 = gamma5 (Q - sigma).
 *    bc[mu] = +1 (periodic) or -1 (antiperiodic) multiplies every hop across
 *    the lattice edge in direction mu.
 *  - Every call returns MGEIG_OK (0) or a negative status; mgeig_strerror()
 *    names it.  Host buffers stay owned by the caller; the library copies in
 *    and out and never keeps a caller pointer.  The context owns all device
 *    memory (allocated in mgeig_create / mgeig_set_params / mgeig_setup) and
 *    frees it in mgeig_destroy.  A context is bound to one device and one
 *    CUDA stream; calls on one context must not overlap.
 */
#ifndef MGEIG_H
#define MGEIG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define MGEIG_OK 0
#define MGEIG_EINVAL (-1)      /* bad argument, size or parameter                       */
#define MGEIG_ENOTSETUP (-2)   /* gauge field or multigrid setup missing                */
#define MGEIG_ECUDA (-3)       /* a CUDA runtime call failed                            */
#define MGEIG_ENOCONV (-4)     /* iteration cap hit; outputs hold the best iterate      */
#define MGEIG_EBREAKDOWN (-5)  /* NaN/Inf or a zero Krylov vector where none may appear */
#define MGEIG_ENOMEM (-6)      /* device allocation failed                              */
#define MGEIG_ETIMEOUT (-7)    /* a bounded device-side wait expired (grid barrier)     */
#define MGEIG_ESCRATCH (-8)    /* coarse grid too large for the static scratch of
                                  mgeig_mg_cycle_dev_noalloc                            */

/* precision of the multigrid preconditioner (Sec. 2.2: double precision FGMRES
 * around a single precision multigrid method) */
#define MGEIG_FP64 0   /* every level in FP64                                    */
#define MGEIG_MIXED 1  /* FP32 smoother / P / coarse solve, FP64 outer and RQI    */

/* smoother of the two-grid cycle (Sec. 2) */
#define MGEIG_SAP 0    /* SAP on D_sigma with right-hand side gamma5 r            */
#define MGEIG_GMRES 1  /* restarted GMRES(k) on Q - sigma                         */
#define MGEIG_LEARNED 2 /* the learned smoother (mgeig_net_*) on the residual after
                           the coarse correction; MGEIG_MIXED only; the setup and
                           the start vectors of Algorithm 1 still smooth with SAP */

/* operator selector of mgeig_apply */
#define MGEIG_OP_Q 0   /* y = (Q - sigma) x                                       */
#define MGEIG_OP_D 1   /* y = (D - sigma gamma5) x                                */

/* arithmetic of mgeig_apply */
#define MGEIG_PREC_F64 0
#define MGEIG_PREC_F32 1
/* mgeig_apply_dev only: the mixed solver's FP64-output stencil in double-float
 * arithmetic (two floats per value, about 2^-46 relative; links and clover
 * from double-float copies of the FP64 arrays) */
#define MGEIG_PREC_F64_DS 2       /* x and y FP64                                  */
#define MGEIG_PREC_F32_F64_DS 3   /* x FP32, y FP64 (the outer FGMRES matvec)      */

/* storage of the coarse operator's links in the mixed-precision preconditioner
 * (an extension of the Sec. 2.2 precision split beyond the paper: the coarse operator in
 * 16 bits with one FP32 scale per 2N_tv x 2N_tv link block, FP32 arithmetic) */
#define MGEIG_LINKS_LEVEL 0   /* the level precision (FP32 in MGEIG_MIXED)            */
#define MGEIG_LINKS_BF16 1    /* bfloat16 entries / per-link FP32 scale               */
#define MGEIG_LINKS_F16 2     /* IEEE half entries / per-link FP32 scale              */

typedef struct mgeig_ctx mgeig_ctx;

/* Solver parameters.  The paper fixes none of the smoother, coarse-grid and
 * setup parameters (it cites the DD-alpha-AMG papers); mgeig_default_params
 * fills in the values this library uses. */
typedef struct mgeig_params {
    double m0;            /* bare mass                                          */
    double csw;           /* clover coefficient c_sw                            */
    int bc[4];            /* fermion boundary phase per direction, +1 or -1     */
    int agg[4];           /* aggregate extent per direction (divides dims)      */
    int n_tv;             /* test vectors N_tv (2..24); coarse blocks 2N_tv^2   */
    int sap_block[4];     /* SAP block extent; an even number >= 2 of blocks    */
    int sap_cycles;       /* post-smoothing SAP cycles nu                       */
    int sap_mr_iters;     /* minimal-residual steps per block solve             */
    int smooth_steps;     /* GMRES smoother: restarts nu                        */
    int gmres_smooth_k;   /* GMRES smoother: Krylov steps per restart           */
    int setup_smooth;     /* setup: smoother iterations on the random vectors   */
    int setup_iters;      /* setup: multigrid iterations per test vector        */
    int outer_restart;    /* FGMRES restart length                              */
    int outer_maxiter;    /* FGMRES iteration cap per solve                     */
    int coarse_restart;   /* coarse GMRES restart length (1..32)                */
    int coarse_maxiter;   /* coarse GMRES iteration cap per solve               */
    double coarse_tol;    /* coarse GMRES relative residual                     */
    double solve_tol;     /* FGMRES relative residual of each shifted solve     */
    int precision;        /* MGEIG_FP64 or MGEIG_MIXED                          */
    int smoother;         /* MGEIG_SAP or MGEIG_GMRES                           */
    int max_sweeps;       /* Rayleigh quotient iteration: sweep cap             */
    int n_guard;          /* extra iterated vectors beyond n_eig (n_eig + n_guard
                             <= 64); -1 = max(n_eig, n_tv)                      */
    int coarse_deflate;   /* 1: outside the setup the coarse solve treats
                             span{P^dag w_j} of the test vectors exactly (Galerkin
                             deflation), 0: plain                               */
    int ritz_each_sweep;  /* 1: after every sweep of Algorithm 1 the iterated
                             vectors become the Ritz vectors of Q in their span */
    double shift_floor;   /* damping floor: sigma = lambda max(1 - max(eps,
                             shift_floor), 0); keeps the shifted system solvable
                             by the single-precision preconditioner              */
    int guard_maxiter;    /* FGMRES step cap for the guard vectors' solves     */
    double ritz_keep;     /* unconverged pairs with eps <= ritz_keep stay out of
                             the per-sweep Rayleigh-Ritz step (their own RQI step
                             converges them; a rotation with rough neighbours of a
                             nearly equal Ritz value would spoil them again)     */
    int fine_deflate;     /* 1: inside the eigensolver every shifted solve is
                             deflated on the fine grid by the iterated vectors Z:
                             the preconditioner becomes
                             z = Z E^-1 Z^dag r + B (r - (Q - sigma) Z E^-1 Z^dag r),
                             E = Z^dag (Q - sigma) Z formed in FP64; 0: plain B */
    double fine_deflate_radius;  /* Z of the solve for v_i: v_i and the iterated
                             vectors whose Rayleigh quotient lies within this
                             distance of sigma (< 0: all iterated vectors)      */
    int adaptive_tol;     /* 1: the shifted solve of v_i runs to relative
                             residual min(solve_tol, 0.1 tol / |lambda_i - sigma|)
                             (the new eigen-residual is about that times
                             |lambda_i - sigma|); 0: solve_tol for every solve   */
    int ritz_start;       /* 1: Algorithm 1 starts from the Ritz vectors of Q in
                             the span of the setup's test vectors (same span,
                             same P), ordered by |theta|; 0: from the test
                             vectors in the order the setup leaves them          */
    int coarse_links;     /* MGEIG_LINKS_*: how the coarse operator is stored and
                             read by the coarse solver and coarse applies (16-bit
                             links only with MGEIG_MIXED)                        */
    int p_modes;          /* P is built from the first p_modes iterated vectors of
                             Algorithm 1 and the setup's test vectors p_modes ..
                             n_tv - 1 (kept as the setup left them); -1 = n_tv:
                             every test vector is replaced by a mode            */
    double barrier_timeout;   /* seconds (of SM clock) a block of the persistent
                             coarse solver waits at a grid barrier before it gives
                             up, raises MGEIG_ETIMEOUT and returns              */
    int coarse_blocks;    /* thread blocks of the persistent coarse solver (one
                             per SM at most, each owning a contiguous slice of
                             the coarse rows); 0 = one per SM, capped by the
                             rows.  Fewer blocks make the two grid barriers of an
                             Arnoldi step cheaper and each block's matvec longer */
    int blas_ds;          /* 1 (MGEIG_MIXED only): the inner products and vector
                             updates of the FP64 vectors (Gram-Schmidt and the
                             Rayleigh quotients of Algorithm 1, the Arnoldi steps
                             of the outer FGMRES) in double-float arithmetic on
                             the FP32 pipe, about 2^-46 relative (the compensated
                             dot product of Ogita, Rump and Oishi); 0: in FP64   */
    int stencil_ds;       /* 1 (MGEIG_MIXED only): the solver's FP64-output
                             stencil (the outer FGMRES matvec, residuals,
                             Rayleigh quotients inside Algorithm 1) in
                             double-float arithmetic from double-float copies of
                             the links and clover; 0 (default): in FP64.  The
                             residuals Algorithm 1 reports are always recomputed
                             in FP64, and mgeig_apply* with MGEIG_PREC_F64 is
                             always FP64.  (On GB300 the double-float stencil is
                             slower than the FP64 one: its long dependent
                             TwoSum chains at 12 warps per SM are latency bound.) */
    int blas_blocks;      /* thread blocks per SM of the BLAS-1 kernels (inner
                             products, vector updates), at most 64; 0 = the
                             measured defaults: 4 per SM for inner products and
                             FP32 multi-vector updates, 16 for the others        */
    int guard_coarse_maxiter; /* coarse GMRES iteration cap inside the solves of
                             Algorithm 1's guard vectors (capped at guard_maxiter
                             outer steps, they only widen the Rayleigh-Ritz
                             space); 0 = coarse_maxiter                          */
} mgeig_params;

/* Work counters and timings of the last setup / eigensolve / solve call. */
typedef struct mgeig_stats {
    int sweeps;           /* Algorithm 1 while-loop passes                      */
    int solves;           /* shifted solves (Algorithm 1, v <- (Q - sigma)^-1 v)*/
    int outer_iters;      /* FGMRES iterations                                  */
    int mg_cycles;        /* two-grid preconditioner applications               */
    long long coarse_iters;   /* coarse GMRES iterations                        */
    long long fine_applies;   /* fine stencil applications (both precisions)    */
    double seconds;       /* wall time of the call                              */
    long long kernel_launches;   /* CUDA kernels the call launched             */
} mgeig_stats;

/* Fill p with the library defaults (m0 = 0, c_sw = 1, periodic, 4^4 aggregates,
 * N_tv = 20, SAP 4^4 blocks, 3 cycles x 4 MR steps, mixed precision). */
void mgeig_default_params(mgeig_params *p);

/* Create a context for an Lx x Ly x Lz x Lt lattice on CUDA device `device`.
 * Requires every extent >= 2.  *out receives the context (NULL on error). */
int mgeig_create(mgeig_ctx **out, const int dims[4], int device);

/* Free every device buffer and the context.  NULL is accepted. */
void mgeig_destroy(mgeig_ctx *ctx);

/* Validate and store parameters; (re)builds the clover term when a gauge field
 * is loaded and drops an existing multigrid setup.  EINVAL names no field: the
 * checks are agg/sap_block dividing dims, an even number >= 2 of SAP blocks per
 * direction, 2 <= n_tv <= 24, bc = +-1, positive iteration counts. */
int mgeig_set_params(mgeig_ctx *ctx, const mgeig_params *p);

/* The checks of mgeig_create (lattice) and mgeig_set_params (parameters) for
 * the lattice dims without a context: MGEIG_OK if a context of that lattice
 * would accept p, else MGEIG_EINVAL.  Host only: no device call, no allocation,
 * usable without a GPU.  Besides the checks listed above: aggregate and SAP
 * block volumes <= 1024, n_tv <= 6 x aggregate volume, 16-bit coarse links and
 * the learned smoother only with MGEIG_MIXED, the learned smoother only on
 * extents divisible by 4 x 4 x 4 x 2, 0 < barrier_timeout <= 60. */
int mgeig_check_params(const int dims[4], const mgeig_params *p);

/* Copy a host gauge field (layout above) to the device and build the clover
 * term from it (four-leaf clover, FP64, Sec. 2 / the operator above). */
int mgeig_load_gauge(mgeig_ctx *ctx, const double *U);

/* Same as mgeig_load_gauge for a gauge field already in device memory (same
 * host layout, complex128), e.g. a buffer allocated with mgeig_alloc_dev. */
int mgeig_load_gauge_dev(mgeig_ctx *ctx, const void *U_dev);

/* Replace the clover term of the operator (Sec. 2: D is the clover-improved
 * Wilson operator) by a caller's A(x) = c_sw (i/4) sum_{mu nu} sigma_{mu nu} F_{mu nu}(x),
 * e.g. one computed with another clover definition or improvement coefficient.
 *   A   host complex128 [site][chirality 2][6][6], the layout of mgeig_get_clover
 *       (c_sw included, the mass term 4 + m0 not), or NULL to go back to the
 *       term the library builds from the gauge field.  Each 6x6 block must be
 *       Hermitian: only the real diagonal and the upper triangle are read.
 *       Copied; the caller keeps ownership.
 * Needs a loaded gauge field (MGEIG_ENOTSETUP otherwise); the loaded term stays
 * in use across mgeig_set_params (which re-adds the new mass) until the next
 * mgeig_load_clover(ctx, NULL) or gauge load.  Drops an existing multigrid
 * setup (the operator changed). */
int mgeig_load_clover(mgeig_ctx *ctx, const double *A);

/* Copy the clover term A(x) = c_sw (i/4) sum sigma F (without the mass term) to
 * host memory as complex128 [site][chirality 2][6][6]; row/col = 3*spin' + colour
 * with spin' = spin mod 2 inside the chirality block. */
int mgeig_get_clover(mgeig_ctx *ctx, double *A);

/* y = (Q - sigma) x (op = MGEIG_OP_Q) or (D - sigma gamma5) x (MGEIG_OP_D) for
 * nrhs host spinors stored one after another, computed in FP64 or in FP32
 * (inputs rounded to FP32, result widened back), all right-hand sides in one
 * launch (mgeig_apply_dev_nrhs).  Fine stencil, Sec. 2. */
int mgeig_apply(mgeig_ctx *ctx, double sigma, int op, int prec,
                const double *x, double *y, int nrhs);

/* Same on device memory: x, y are device spinors in the library's internal
 * layout (FP64: double2 [12][V]; FP32: float4 [6][V], component k = 3*spin +
 * colour, float4 q holds components 2q, 2q+1), one field each.  Launched on the
 * context's stream, asynchronous.  For timing the stencil without copies.
 * prec may also be MGEIG_PREC_F64_DS or MGEIG_PREC_F32_F64_DS (any context
 * precision). */
int mgeig_apply_dev(mgeig_ctx *ctx, double sigma, int op, int prec,
                    const void *x, void *y);

/* The stencil of mgeig_apply_dev on nrhs device fields at once: x and y each
 * hold nrhs fields of the internal layout of precision prec stored back to back
 * (field k at byte offset k * V * 12 * (16 for FP64, 8 for FP32)); x and y must
 * not overlap (MGEIG_EINVAL).  One launch for all fields, so the links and the
 * clover term are read from HBM once for all of them (the multi right-hand-side
 * form of the fine stencil, Sec. 2, as used for many right-hand sides of Z2
 * noise, Sec. 3, Eqs. 3.4-3.6).  Asynchronous on the context's stream. */
int mgeig_apply_dev_nrhs(mgeig_ctx *ctx, double sigma, int op, int prec, const void *x, void *y, int nrhs);

/* Device buffer of `bytes` bytes owned by the context (freed by destroy), e.g.
 * for mgeig_apply_dev operands.  *ptr = NULL on error. */
int mgeig_alloc_dev(mgeig_ctx *ctx, size_t bytes, void **ptr);

/* Convert n_fields host-layout complex128 spinors (host memory) into the
 * internal device layout of precision prec at dev (mgeig_apply_dev layout). */
int mgeig_pack_spinors(mgeig_ctx *ctx, int prec, const double *host, void *dev, int n_fields);

/* Inverse of mgeig_pack_spinors: n_fields internal-layout device spinors of
 * precision prec -> host-layout complex128 spinors in host memory. */
int mgeig_unpack_spinors(mgeig_ctx *ctx, int prec, const void *dev, double *host, int n_fields);

/* Multigrid setup (Sec. 2.1, paragraph after Algorithm 1): N_tv random test
 * vectors (Philox4x32-10 uniforms, key = seed, counters (site, pair, vector,
 * 0x5EED0001)), setup_smooth smoother iterations each, then setup_iters times
 * {one two-grid iteration per test vector at sigma = 0; Gram-Schmidt in FP64;
 * rebuild P and the coarse operator}. */
int mgeig_setup(mgeig_ctx *ctx, uint64_t seed, mgeig_stats *stats);

/* Replace the test vectors with n_tv host spinors and rebuild P and the coarse
 * operator from them (no orthonormalisation across vectors). */
int mgeig_set_test_vectors(mgeig_ctx *ctx, const double *W);

/* Copy the current test vectors (n_tv host spinors, FP64) out. */
int mgeig_get_test_vectors(mgeig_ctx *ctx, double *W);

/* Interpolation P (Eq. 2.4): the n_tv fine spinors whose restriction to each
 * aggregate and chirality are the orthonormal columns of P. */
int mgeig_get_interp(mgeig_ctx *ctx, double *P);

/* Coarse operator D_c = P^dag D P (Eq. 2.5) as complex128
 * [direction 9][coarse site][2 n_tv][2 n_tv]; direction 0 = self, 1 + 2 mu =
 * +mu, 2 + 2 mu = -mu; row/col = c*n_tv + j (chirality c, test vector j). */
int mgeig_get_coarse_op(mgeig_ctx *ctx, double *Dc);

/* r_c = P^dag r (host fine spinor -> host coarse vector [coarse site][2][n_tv]). */
int mgeig_restrict(mgeig_ctx *ctx, const double *r, double *rc);

/* e = P e_c (host coarse vector -> host fine spinor). */
int mgeig_prolong(mgeig_ctx *ctx, const double *ec, double *e);

/* y_c = (gamma5^c D_c - sigma) x_c = (Q_c - sigma) x_c (Eq. 2.6). */
int mgeig_coarse_apply(mgeig_ctx *ctx, double sigma, const double *xc, double *yc);

/* y_c = (Q_c - sigma) x_c for nrhs <= 16 host coarse vectors stored one after
 * another (Eq. 2.6).  With MGEIG_MIXED and MGEIG_LINKS_BF16 one launch on the
 * tensor cores (BF16 links with their per-link FP32 scale, right-hand sides
 * rounded to BF16 after the scale is applied, FP32 accumulation); with the
 * other link formats the CUDA-core coarse apply per right-hand side. */
int mgeig_coarse_apply_nrhs(mgeig_ctx *ctx, double sigma, const double *xc, double *yc, int nrhs);

/* The same on device memory, MGEIG_MIXED only: X and Y hold nrhs FP32 coarse
 * vectors (complex64 [coarse site][2][n_tv] each) back to back, must not
 * overlap (MGEIG_EINVAL).  Asynchronous on the context's stream. */
int mgeig_coarse_apply_dev_nrhs(mgeig_ctx *ctx, double sigma, const void *X, void *Y, int nrhs);

/* cycles SAP cycles (red then black blocks, sap_mr_iters MR steps per block)
 * for D_sigma z = b from z (both host spinors; z updated in place). */
int mgeig_sap(mgeig_ctx *ctx, double sigma, const double *b, double *z, int cycles);

/* One two-grid preconditioner application z = B r at shift sigma (Eq. 2.3
 * with no pre- and nu post-smoothing steps): coarse GMRES on Q_c - sigma (tol,
 * coarse_maxiter), prolongation, then the smoother.  Host spinors. */
int mgeig_mg_cycle(mgeig_ctx *ctx, double sigma, const double *r, double *z);

/* The same two-grid application z = B r, for callers that cannot allocate
 * device memory while they run (a framework whose pool allocator holds all free
 * GPU memory, a latency-bound loop that must not take the driver's allocation
 * lock or let cudaFree synchronise the device).  The paper has no counterpart.
 *   r, z   device spinors in the context's level precision and internal layout
 *          (MGEIG_PREC_F32 for MGEIG_MIXED, MGEIG_PREC_F64 for MGEIG_FP64, as
 *          mgeig_pack_spinors writes them); r is read, z is overwritten.  The
 *          caller owns both; they must not overlap (MGEIG_EINVAL otherwise:
 *          the prolongation writes z before the smoother reads r).
 * The result equals mgeig_mg_cycle's.  On success the call allocates nothing:
 * the coarse vectors and the coarse solver's scratch live in one static device
 * array of 16 MiB that every GPU loading this library holds until the process
 * exits.  Coarse grids needing more return MGEIG_ESCRATCH: it holds three coarse
 * vectors (n_agg x 2 n_tv complex values in the level precision each) plus the
 * coarse solver's per-block partial sums, and, on coarse grids too large for the
 * solver to keep its per-block vectors in shared memory, another
 * (2 coarse_restart + 5) coarse vectors; the 16^3 x 32 lattice with 4^4
 * aggregates and 20 test vectors fits in both precisions.  mgeig_create looks
 * up the array's device address (cudaGetSymbolAddress, once per device), which
 * also loads the code module that holds the array, so calls on a context made
 * after mgeig_create allocate no device memory of the library's own.  (With
 * CUDA's lazy loading the driver may still load a kernel's code the first time
 * it runs; a caller that must exclude that makes one call ahead of time or sets
 * CUDA_MODULE_LOADING=EAGER.)  All calls share the array, so calls that overlap
 * on the GPU race.  Needs the SAP smoother and kernel timing off (MGEIG_EINVAL
 * otherwise); the coarse-grid deflation data for sigma is computed on the first
 * call at a new sigma, as in mgeig_mg_cycle.  The call synchronises the
 * context's stream before it returns (it reads the coarse solver's status words
 * back), so the cycle has finished when it returns. */
int mgeig_mg_cycle_dev_noalloc(mgeig_ctx *ctx, double sigma, const void *r, void *z);

/* Solve (Q - sigma) x = b with FP64 flexible GMRES preconditioned by the two-grid
 * method (Sec. 2.2) to relative residual tol.  ENOCONV if outer_maxiter is hit. */
int mgeig_solve(mgeig_ctx *ctx, double sigma, const double *b, double *x, double tol,
                mgeig_stats *stats);

/* Many shifted systems of many fields (Algorithm 1's shifted systems, and the
 * Z2 noise right-hand sides of Sec. 3, Eqs. 3.4-3.6): for every context k
 * (set up, any lattice, any device) solve (Q - sigmas[s]) x = b_j for the nsig
 * shifts and the nrhs host right-hand sides b[k] (nrhs spinors of that lattice
 * one after another) to relative residual tol with the FGMRES of mgeig_solve;
 * x[k] receives nsig * nrhs solutions ordered [shift][rhs].  The systems of a
 * context run one after another, shift-major (the coarse deflation data of a
 * shift is computed once for all its right-hand sides).  Returns ENOCONV when
 * any system hits outer_maxiter (all outputs filled), the first other error of a
 * context otherwise.  stats (may be NULL) sums the counters of all contexts. */
int mgeig_solve_batch(mgeig_ctx *const *ctxs, int nctx, const double *sigmas, int nsig, const double *const *b,
                      double *const *x, int nrhs, double tol, mgeig_stats *stats);

/* Solve the non-Hermitian (D - sigma gamma5) x = b (sigma = 0: the Wilson-clover
 * system D x = b that DD-alpha-AMG solves, Sec. 2) with the same FP64 flexible
 * GMRES, now on D_sigma, right-preconditioned by B gamma5 (D_sigma^-1 =
 * (Q - sigma)^-1 gamma5; with the SAP smoother this is the two-grid method on
 * D_sigma itself, SAP acting on D_sigma z = r).  ENOCONV if outer_maxiter is hit. */
int mgeig_solve_d(mgeig_ctx *ctx, double sigma, const double *b, double *x, double tol, mgeig_stats *stats);

/* Algorithm 1: the n_eig eigenpairs of Q of smallest |lambda| to eigen-residual
 * ||Q v - lambda v|| <= tol, starting from the setup's test vectors (rotated to
 * Ritz vectors of Q in their span, ordered by |theta|).  The iteration runs on
 * n_eig + n_guard vectors and returns the n_eig of smallest |lambda|: the guard
 * vectors lower the chance that a wanted mode is missed (the failure noted in
 * Sec. 2.1 after Algorithm 1).  Needs mgeig_setup.
 * Outputs (any may be NULL): evals[n_eig], evecs[n_eig host spinors, unit norm,
 * phase such that the largest-modulus component is real positive],
 * resid[n_eig]; sorted by |lambda| ascending, then lambda.  Iterated vectors
 * beyond the n_tv test vectors start from Philox uniforms (stream 0x5EED0003,
 * the setup's seed) smoothed by setup_smooth two-grid iterations; P always holds
 * the first n_tv of them.  n_eig + n_guard <= 64.
 * ENOCONV when max_sweeps is hit (outputs hold the current iterates). */
int mgeig_eigensolve(mgeig_ctx *ctx, int n_eig, double tol, double *evals, double *evecs,
                     double *resid, mgeig_stats *stats);

/* Per-kernel timing with CUDA events on the context stream (off by default;
 * switching it on or off resets the counters).  mgeig_kernel_times returns,
 * for kernel class k < n, the number of launches[k], their total device time
 * ms[k] (0 while timing is off) and the total algorithmic bytes[k] they move
 * (the bytes a perfect kernel would read and write once); names[k] is a static
 * string.  Returns the number of classes, or a negative status. */
int mgeig_set_timing(mgeig_ctx *ctx, int on);
/* As mgeig_set_timing(ctx, 1), but only the kernel classes whose bit is set in
 * mask (bit k = class k of mgeig_kernel_times) record CUDA events, so that one
 * class can be timed with little overhead on the rest; mask 0 switches timing
 * off.  The paper has no counterpart. */
int mgeig_set_timing_classes(mgeig_ctx *ctx, unsigned int mask);
int mgeig_kernel_times(mgeig_ctx *ctx, int n, long long *launches, double *ms,
                       double *bytes, const char **names);

/* The cudaStream_t (as void *) on which every call of this context launches
 * its kernels, for callers that record CUDA events around device-pointer calls
 * such as mgeig_apply_dev.  Owned by the context. */
int mgeig_get_stream(mgeig_ctx *ctx, void **stream);

/* Number of CUDA kernels this context has launched since it was created (all
 * calls, including mgeig_load_gauge*); *count is written on success.  The
 * paper has no counterpart: it lets a caller count the device work of a step. */
int mgeig_get_launch_count(mgeig_ctx *ctx, long long *count);

/* ---------------------------------------------------------------------------
 * Approximate low-mode averaging (Sec. 3.1, 3.2): eigenpairs of low accuracy,
 * e.g. the setup's test vectors (Sec. 3.3: no Rayleigh quotient iteration),
 * used through the corrected low-mode inverse and an oblique projector.
 * -------------------------------------------------------------------------- */

/* Take n approximate eigenvectors (host spinors V, or NULL for the Ritz vectors of
 * Q in the span of the setup's first n test vectors, by |theta|), orthonormalise
 * them (Gram-Schmidt in FP64) and keep the
 * pairs whose relative accuracy passes the cutoff eps_i / |lambda_i| <= cutoff
 * (Sec. 3.3 uses 0.75), lambda_i = <v_i|Q|v_i>, eps_i = ||Q v_i - lambda_i v_i||.
 * Outputs (any may be NULL): lam[n], eps[n], kept[n] (1 kept, 0 cut), *n_kept;
 * A[k][k] and Ainv[k][k] (complex128, row-major, k = *n_kept) with
 * A_ij = <v_i|Q|v_j> over the kept pairs in their original order; Llow[Lt]
 * (complex128) the low-mode part of the loop per timeslice,
 * L_low(t) = sum_{x in t} tr (Q~^-1_low)_{x,x},  Q~^-1_low = sum_ij (A^-1)_ij |v_i><v_j|.
 * The state stays in the context for mgeig_lma_apply / mgeig_lma_loop_high. */
int mgeig_lma_prepare(mgeig_ctx *ctx, int n, const double *V, double cutoff, double *lam, double *eps, int *kept,
                      int *n_kept, double *A, double *Ainv, double *Llow);

/* y = Q~^-1_low x (mode 0) or y = R~ x with the oblique projector
 * R~ = 1 - sum_ij Q |v_i> (A^-1)_ij <v_j| (mode 1), host spinors, FP64. */
int mgeig_lma_apply(mgeig_ctx *ctx, int mode, const double *x, double *y);

/* The high-mode part of the loop per timeslice, estimated with nstoch Z2 + iZ2
 * noise vectors eta_n (Philox key seed, stream 0x5EED0002: the entries
 * (+-1 +- i)/sqrt 2 from the sign bits of the words of counter (site, component
 * pair, n, stream)):  Lhigh[t] = 1/nstoch sum_n sum_{x in t} <eta_n(x)|s_n(x)>, where
 * Q s_n = R~ eta_n is solved by the FGMRES of mgeig_solve (sigma = 0) to relative
 * residual tol, so that Q^-1 R~ = Q^-1 - Q~^-1_low (Sec. 3.1 with the oblique
 * projector of Sec. 3.2).  Needs mgeig_lma_prepare and mgeig_setup. */
int mgeig_lma_loop_high(mgeig_ctx *ctx, int nstoch, uint64_t seed, double tol, double *Lhigh, mgeig_stats *stats);

/* ---------------------------------------------------------------------------
 * The learned smoother (the paper has none; an extension of the
 * smoother M of Eq. 2.3): a 3-layer 4D convolutional network (3^4 taps,
 * 24 -> 32 -> 32 -> 24 real channels, no bias, GELU in its tanh form between
 * the layers), applied as M(r) = ||r|| f(r / ||r||), trained on the GPU with the
 * library's own tensor-core kernels on (residual, SAP correction) pairs that the
 * two-grid method produces.  Weights: FP32 [layer 3][tap 81][out 32][in 32],
 * tap = ((dt+1)*3 + (dz+1))*9 + (dy+1)*3 + (dx+1); unused channels zero.
 * The lattice extents must be multiples of 4, 4, 4, 2 (MGEIG_EINVAL).
 * -------------------------------------------------------------------------- */

/* He-normal initialisation of the weights from `seed` (64-bit Mersenne twister,
 * Box-Muller), standard deviation 0.5 sqrt(2 / (81 c_in)); resets Adam. */
int mgeig_net_init(mgeig_ctx *ctx, uint64_t seed);

/* Copy the FP32 master weights in (resets Adam) or out (layout above). */
int mgeig_net_set_weights(mgeig_ctx *ctx, const float *W);
int mgeig_net_get_weights(mgeig_ctx *ctx, float *W);

/* `steps` Adam steps (learning rate lr) on `batch` fresh pairs each: random
 * Philox vectors v (stream 0x5EED0004, key seed + step), the coarse correction
 * x_c = P (Q_c)^-1 P^dag v, the residual r = v - Q x_c, the target e = the SAP
 * correction of r (sap_cycles cycles on D e = gamma5 r from e = 0); loss
 * 1/(2 batch) sum ||f(r/||r||) - e/||r||||^2.  losses[steps] (may be NULL)
 * receives the loss of every step.  Needs mgeig_setup; MGEIG_MIXED only. */
int mgeig_net_train(mgeig_ctx *ctx, int steps, int batch, double lr, uint64_t seed, double *losses);

/* Loss and weight gradients (FP32, layout of the weights) for caller data: x and
 * t are FP64 channel fields [batch][site][24] (channel 2k = Re, 2k+1 = Im of
 * spin-colour component k), loss = 1/(2 batch) sum ||f(x) - t||^2.  For checking
 * the GPU forward and backward kernels; weights as set. */
int mgeig_net_loss_grads(mgeig_ctx *ctx, const double *x, const double *t, int batch, double *loss, float *G);

/* e = M(r) = ||r|| f(r / ||r||) for one host spinor (computed from its FP32
 * rounding, result widened to FP64). */
int mgeig_net_apply(mgeig_ctx *ctx, const double *r, double *e);

/* Inner products d_j = <X_j, y> = sum_i conj(X_j[i]) y[i], j < k, of device
   vectors of n complex values (interleaved re, im; FP64 for prec =
   MGEIG_PREC_F64, FP32 for MGEIG_PREC_F32; 16-byte aligned): the projection
   coefficients of the Gram-Schmidt step of Algorithm 1 (Sec. 2.1), of the
   Arnoldi process of the outer FGMRES (FP64) and of the fine-grid deflation
   (FP32).  X: host array of k device pointers (1 <= k <= 32); y: device
   pointer; d: host, 2k doubles (re, im).  FP64 vectors: double-float arithmetic
   when the context's blas_ds = 1 and precision MGEIG_MIXED, else FP64; FP32
   vectors: FP32 products, per-thread FP32 sums, FP64 across threads.  Blocks
   until d is written.  Returns MGEIG_EINVAL for prec or k out of range, n < 1
   or a NULL pointer. */
int mgeig_multidot_dev(mgeig_ctx *ctx, int prec, int k, const void *const *X, const void *y, long long n,
                       double *d);

/* y += sum_j c_j X_j, j < k (the update of the same Gram-Schmidt, Arnoldi and
   deflation steps), for the device vectors of mgeig_multidot_dev; c: host, 2k
   doubles (re, im).  y must not be one of the X_j.  Same arithmetic rule and
   errors; returns when y is written. */
int mgeig_multi_axpy_dev(mgeig_ctx *ctx, int prec, int k, const void *const *X, const double *c, void *y,
                         long long n);

/* FMA throughput of the device in FP64 (prec = MGEIG_PREC_F64) or FP32
 * (MGEIG_PREC_F32), in FLOP/s (2 per FMA), measured with the library's own
 * kernel (independent FMA chains on every SM, best of `reps` launches timed with
 * CUDA events on the context's stream).  The paper has no counterpart: it is the
 * arithmetic roof of the kernels whose FP64 work, not memory, bounds them. */
int mgeig_fma_peak(mgeig_ctx *ctx, int prec, int reps, double *flops);

/* Name of a status code. */
const char *mgeig_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* MGEIG_H */
