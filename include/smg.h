/*
 * smg.h -- C ABI of libsmg, a GB300 (sm_103a) staggered multigrid solver.
 *
 * The library solves M x = b for the staggered operator M = m + D
 * (arXiv:2212.12559, Sec. 2.2; naive or HISQ-shaped with Naik links) with
 * flexible GCR preconditioned by the Kahler-Dirac multigrid K-cycle of
 * Sec. 2.1 and 2.3 (Table 1), to a relative residual of the full (non-Schur)
 * operator (Sec. 3.2).
 *
 * Conventions shared by every call:
 *  - A lattice has extents dims = {Lx, Ly, Lz, Lt}, each even and >= 4
 *    (Kahler-Dirac hypercubes, Sec. 2.2), periodic boundaries.  Site index
 *    x + Lx*(y + Ly*(z + Lz*t)).
 *  - A colour field is V x 3 complex numbers, FP64, real/imaginary
 *    interleaved ([V][3][2] doubles).  A link field is [4][V][3][3] complex
 *    FP64 (row-major 3x3; entry [mu][x][a][b] links x to x+mu).
 *  - `where` says where a caller buffer lives: SMG_HOST (pageable or pinned
 *    host memory) or SMG_DEVICE (device memory on the context's GPU).
 *  - The caller owns every buffer it passes; the library copies what it
 *    keeps and never retains a caller pointer after a call returns.
 *  - Every call returns an smg_status.  On failure smg_last_error() gives a
 *    one-line reason.  No call aborts the process or traps the GPU.
 *  - All device work is ordered on the context's stream (smg_set_stream);
 *    calls return after that work has completed unless stated otherwise.
 */
#ifndef SMG_H
#define SMG_H

#include <stdint.h>

#if defined(__GNUC__)
#define SMG_API __attribute__((visibility("default")))
#else
#define SMG_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct smg_ctx smg_ctx;

typedef enum {
  SMG_OK = 0,
  SMG_ERR_ARG = -1,            /* invalid argument or size */
  SMG_ERR_CUDA = -2,           /* a CUDA runtime call failed */
  SMG_ERR_OOM = -3,            /* device allocation failed */
  SMG_ERR_STATE = -4,          /* call out of order (e.g. solve before mg_setup) */
  SMG_ERR_NOT_CONVERGED = -5,  /* iteration cap reached; x holds the best iterate */
  SMG_ERR_BREAKDOWN = -6,      /* NaN/Inf or zero norm met inside a solver */
  SMG_ERR_TIMEOUT = -7         /* a bounded device wait gave up */
} smg_status;

enum { SMG_HOST = 0, SMG_DEVICE = 1 };

/* Precision of the preconditioner (the outer GCR and its residuals are always FP64). */
enum {
  SMG_PREC_DOUBLE = 0,   /* FP64 vectors, FP64 links / blocks / stencils */
  SMG_PREC_SINGLE = 1,   /* FP32 vectors and storage */
  SMG_PREC_HALF = 2      /* FP32 vectors and arithmetic, FP16 storage with FP32 scales */
};

#define SMG_MAX_COARSE 3

/* Multigrid parameters; Table 1 of the paper gives the defaults in the comments. */
typedef struct smg_mg_params {
  int n_coarse;                    /* coarsenings: 1 = fine+KD+1 coarse level, 2 = one more */
  int agg[SMG_MAX_COARSE][4];      /* aggregate extents of each coarsening (4^4, then 2^4) */
  int nvec[SMG_MAX_COARSE];        /* near-null vectors per coarsening; coarse dof = 2*nvec */
  double setup_tol;                /* CGNE relative residual for near-null vectors: 1e-6 */
  int setup_maxiter;               /* CGNE iteration cap: 2000 (0 = use phi0 as given) */
  double inner_tol;                /* inner GCR tolerance on levels >= 1: 0.25 (levels >= 2: see
                                      coarse_inner_tol) */
  int inner_maxiter;               /* inner GCR iteration cap: 8 (at most 16) */
  int smoother_s;                  /* CA-GCR(s) post-smoother length: 8 */
  int dense_max;                   /* coarsest level solved exactly when its dof <= dense_max */
  int nkrylov;                     /* outer GCR restart length: 16 */
  int max_outer;                   /* outer GCR iteration cap */
  int precision;                   /* SMG_PREC_* of the preconditioner */
  int use_graph;                   /* 1: replay the K-cycle from a captured CUDA graph */
  int persistent;                  /* 1: run the last coarse GCR level as one cooperative launch
                                      (FP32 preconditioner, at most 16 systems) */
  int truncate_naik;               /* Table 1 level-1 operator: 0 = KD-preconditioned HISQ
                                      A = (B+m)^{-1} M; 1 = truncated A' = (B+m)^{-1}(m + D_fat),
                                      the Naik hops dropped from the pseudo-fine operator only
                                      (Sec. 3.1); the outer GCR keeps the full M.  Default 0. */
  int block_coarse;                /* Sec. 2.3: 1 = every coarse level uses the block-preconditioned
                                      operator X^{-1} A_hat (X its self blocks) in its GCR, smoother
                                      and the next Galerkin product, with the right-hand side
                                      X^{-1} R r; the near-null CGNE runs on A_hat.  A dense
                                      coarsest level is inverted from A_hat, which gives the same
                                      solution.  Default 0 (un-preconditioned A_hat). */
  int coarsest_deflate;            /* Table 1 coarsest solver: k > 0 = SVD-deflated Chebyshev-basis
                                      CA-GCR when the coarsest level is not solved densely.  Setup:
                                      the k lowest singular triplets of the coarsest operator by a
                                      Chebyshev-filtered subspace iteration on A^dag A from the start
                                      block phi0[n_coarse] (k + max(4, k/4) <= 64 fields).  Solve:
                                      x0 = V diag(1/sigma) U^dag b, then CA-GCR(coarsest_cheb_s)
                                      cycles with a Chebyshev basis on [sigma_k, sigma_max] until
                                      0.25 ||b|| or inner_maxiter cycles.  Default 0 (GCR). */
  int coarsest_cheb_s;             /* Chebyshev basis length of that CA-GCR, 1..16.  Default 8:
                                      Table 1 uses 16, but on coarse operators whose eigenvalues
                                      lie well off the real interval a 16-long basis leaves the
                                      Gram matrix numerically singular (in FP32 vectors the
                                      correction is lost) */
  int coarsest_schur;              /* Table 1 level-3 operator: 1 = the deflated coarsest solve runs
                                      on the even/odd Schur complement S = 1 - K_eo K_oe of the
                                      block-preconditioned operator 1 + K (needs block_coarse,
                                      coarsest_deflate > 0 and even coarse extents): right-hand side
                                      c_e - K_eo c_o, singular triplets and CA-GCR of S, then
                                      x_o = c_o - K_oe x_e.  Default 0. */
  int schur_coarse;                /* Table 1 level-2 operator: 1 = every coarse level that is not
                                      the coarsest runs its GCR and post-smoother on the Schur
                                      complement S of its block-preconditioned operator (needs
                                      block_coarse and even coarse extents), right-hand side
                                      c_e - K_eo c_o, preconditioned by the K-cycle on the embedded
                                      residual (r_e, 0) (for x_o = c_o - K_oe x_e the full residual
                                      is exactly that), x_o reconstructed.  Default 0. */
  int coarsest_basis;              /* basis of the coarsest CA-GCR: 0 = Chebyshev polynomials of
                                      [sigma_k, sigma_max] (Table 1, default); 1 = the shifted power
                                      basis ((A - c)/h)^k r of the disk around that interval's
                                      centre, well conditioned when the spectrum fills a disk
                                      rather than lying near the real interval (both span the same
                                      Krylov space) */
  double coarse_inner_tol;         /* inner GCR tolerance of levels >= 2 (the Galerkin levels and
                                      the coarsest level's iterative solve); 0 = inner_tol.  Table 1
                                      gives every level 0.25; a tighter level-1 rule with Table 1's
                                      rule below it cuts the coarse work at light masses */
  int coarse_inner_maxiter;        /* iteration cap of those levels, 1..16; 0 = inner_maxiter */
  int galerkin_tc;                 /* Galerkin product A_hat = R A P (Sec. 2.1) with SMG_PREC_HALF:
                                      1 (default) = from the FP16 prolongator the K-cycle uses, the
                                      operator parts applied in FP32 with the level's stored links /
                                      stencil, and the restriction P^dag (A P) on the tensor cores
                                      (FP16 operands, FP32 sums) wherever that kernel serves the
                                      transfer (32 or 64 near-null vectors); entries then carry FP16
                                      rounding, as the stored stencil does.  0 = always the FP64
                                      product from the FP64 prolongator */
} smg_mg_params;

/* Fills *p with the defaults above (two-level, 4^4 aggregates, 24 vectors, FP64). */
SMG_API void smg_default_params(smg_mg_params* p);

typedef struct smg_solve_info {
  int converged;          /* 1 when the recomputed residual meets tol */
  int iterations;         /* outer GCR iterations */
  int restarts;           /* outer GCR restarts (true-residual recomputations) */
  double true_residual;   /* ||b - M x|| / ||b|| recomputed in FP64 at exit */
  double seconds;         /* wall time of the call */
} smg_solve_info;

/* ---------------------------------------------------------------- lifetime */
/* Creates a context for one lattice on the current CUDA device. */
SMG_API int smg_create(const int dims[4], smg_ctx** out);
SMG_API int smg_destroy(smg_ctx* ctx);
SMG_API const char* smg_last_error(const smg_ctx* ctx);
/* Orders all further work on `stream` (a cudaStream_t; NULL = the context's own stream). */
SMG_API int smg_set_stream(smg_ctx* ctx, void* stream);

/* ------------------------------------------------------------------ problem */
/* Sec. 2.2 / 3.1: fat links (distance 1) and optional Naik links (distance 3,
 * NULL for the naive operator) with coefficient c_naik.  Copies the links;
 * invalidates the KD blocks and the multigrid setup.  The time boundary set
 * by smg_set_boundary applies to these links. */
SMG_API int smg_set_gauge(smg_ctx* ctx, const void* fat, const void* naik, double c_naik, int where);
/* Boundary conditions of the fermion field: flags 0 = periodic in all four
 * directions (default), SMG_BC_T_ANTIPERIODIC = psi(x + L_t t) = -psi(x),
 * the hops that wrap around the time extent carry -1.  The paper does not
 * state its boundary conditions; the antiperiodic time boundary is the usual
 * one for propagators.  Implemented on the stored links: smg_set_gauge
 * negates the time links whose hop wraps (fat links on the last time slice,
 * Naik links on the last three), which leaves the KD blocks (no block holds a
 * wrapping hop) and every kernel unchanged; smg_force returns the gradient
 * with respect to the links the caller passed.  Takes effect at the next
 * smg_set_gauge (the current gauge field, KD blocks and setup are dropped:
 * smg_set_gauge and smg_mg_setup must follow).  SMG_ERR_ARG on unknown
 * flags. */
enum { SMG_BC_T_ANTIPERIODIC = 1 };
SMG_API int smg_set_boundary(smg_ctx* ctx, int flags);
/* M = m + D with the given real mass.  Rebuilds the KD blocks (B+m)^{-1}
 * (Sec. 3.1); keeps the near-null vectors and the coarse operators, which
 * stay those of the mass they were built with (Sec. 3.2: operators from the
 * lightest mass are reused for the others). */
SMG_API int smg_set_mass(smg_ctx* ctx, double mass);

/* Sec. 2.1 / 2.3 / Table 1: builds the hierarchy for the current gauge field
 * and mass.  phi0[l] is the random start of the near-null CGNE of
 * coarsening l: nvec[l] fields of the level's size (V*3 complex on the fine
 * level, V_l*2*nvec[l-1] complex on coarse level l), FP64 interleaved,
 * [nvec][sites][dof], in `where` memory.  With setup_maxiter = 0 the starts
 * are used as the near-null vectors unchanged. */
SMG_API int smg_mg_setup(smg_ctx* ctx, const smg_mg_params* params, const void* const* phi0, int where);

/* Sec. 3.2 generates the near-null vectors and the coarsest level's singular
 * vectors once, at the lightest mass, saves them and reuses them for every
 * later solve.  smg_save_setup writes the current setup to the file `path`:
 * the parameters, the near-null vectors of every coarsening as the setup
 * produced them (before chiral doubling and block orthonormalisation), the
 * CGNE iteration counts and, with a deflated coarsest level, its singular
 * values and vectors; a hash of the contents closes the file.  Nothing about
 * the gauge field is stored.  SMG_ERR_STATE before mg_setup; SMG_ERR_ARG when
 * the file cannot be written. */
SMG_API int smg_save_setup(smg_ctx* ctx, const char* path);
/* Rebuilds the hierarchy from a file written by smg_save_setup, for the
 * context's current gauge field and mass (set_gauge and set_mass first): the
 * saved vectors are block-orthonormalised and coarsened exactly as
 * smg_mg_setup does (no CGNE, no singular-vector iteration), so with the
 * gauge field, mass and parameters of the save every coarse operator is bit
 * for bit the one saved with.  params: NULL for the saved parameters, or
 * parameters with the same level structure (n_coarse, agg, nvec,
 * block_coarse, coarsest_schur, coarsest_deflate) whose other settings
 * (precision, inner rules, smoother, graph, persistence, ...) replace the
 * saved ones, e.g. to run the same vectors in FP64.  Replaces any previous
 * setup.  SMG_ERR_ARG when the file is missing, truncated, fails its hash,
 * was saved for other lattice extents or does not match params' level
 * structure; SMG_ERR_STATE without a gauge field or mass. */
SMG_API int smg_load_setup(smg_ctx* ctx, const char* path, const smg_mg_params* params);

/* Sec. 3.2: solves M x = b to ||b - M x|| <= tol ||b|| (recomputed in FP64).
 * b, x: V*3 complex FP64.  x is output only (zero initial guess).
 * Returns SMG_ERR_NOT_CONVERGED (with x the last iterate) at max_outer. */
SMG_API int smg_solve(smg_ctx* ctx, const void* b, void* x, double tol, int where, smg_solve_info* info);

/* Sec. 3.3: nrhs sources times nshift masses solved together as one batch.
 * b: [nrhs][V][3]; x: [nshift][nrhs][V][3]; info: nshift*nrhs entries (may be
 * NULL).  The near-null vectors and coarse operators of the current setup
 * serve every mass; M and (B+m)^{-1} use each system's own mass. */
SMG_API int smg_multi_solve(smg_ctx* ctx, int nrhs, const void* b, int nshift, const double* masses, void* x,
                    double tol, int where, smg_solve_info* info);

/* Sec. 4 (propagator workflow): M(m_i) x_i = b for nshift masses by
 * conjugate gradients on M^dag M = m^2 + D^dag D with every shift in one
 * Krylov space (one product by D^dag D per iteration for all of them), then
 * x_i = M(m_i)^dag y_i.  FP64 on the full operator (Naik included); needs
 * set_gauge only (no mass, no setup).  b: V*3 complex FP64; x: [nshift][V][3];
 * masses > 0, any order; info: nshift entries with the recomputed
 * ||b - M(m_i) x_i|| / ||b|| and the shared iteration count (may be NULL).
 * Returns SMG_ERR_NOT_CONVERGED when a residual misses tol after maxiter. */
SMG_API int smg_multishift_cg(smg_ctx* ctx, const void* b, int nshift, const double* masses, void* x, double tol,
                              int maxiter, int where, smg_solve_info* info);

/* Sec. 4: the propagator workflow's split: the n_mg lightest masses by the MG
 * solver of the current setup (as smg_multi_solve: near-null vectors and
 * coarse operators of the setup mass serve every mass), the others by
 * smg_multishift_cg (at most cg_maxiter iterations).  b: V*3; x: [nmass][V][3]
 * in the order of `masses`; info: nmass entries in that order (may be NULL). */
SMG_API int smg_propagators(smg_ctx* ctx, const void* b, int nmass, const double* masses, int n_mg, void* x,
                            double tol, int cg_maxiter, int where, smg_solve_info* info);

/* ------------------------------------------------------ test / bench hooks */
/* Operators applied to nsys FP64 fields (in/out [nsys][V][3]) in precision
 * `prec` (SMG_PREC_*; inputs are rounded to it, outputs widened to FP64). */
enum {
  SMG_OP_M = 0,      /* m + D                     (Sec. 2.2)          */
  SMG_OP_MDAG = 1,   /* m - D = M^dag                                  */
  SMG_OP_KD = 2,     /* (B+m)^{-1}                (Eq. 2, Sec. 3.1)   */
  SMG_OP_KDDAG = 3,  /* (B+m)^{-dag}                                   */
  SMG_OP_A = 4,      /* (B+m)^{-1} M              (Eq. 2)             */
  SMG_OP_ADAG = 5    /* M^dag (B+m)^{-dag}                             */
};
SMG_API int smg_apply_fine(smg_ctx* ctx, int op, int prec, int nsys, const void* in, void* out, int where);
/* Maps (Sec. 2.2): parity, hypercube index, position in hypercube, aggregate
 * index and position in aggregate for aggregates agg[4]; five int32 arrays of V. */
SMG_API int smg_get_maps(smg_ctx* ctx, const int agg[4], int* parity, int* kd_block, int* kd_pos, int* agg_idx,
                 int* agg_pos, int where);
/* (B+m)^{-1} for the current mass: [V/16][48][48] complex FP64 row-major. */
SMG_API int smg_get_kd_inverse(smg_ctx* ctx, void* out, int where);
/* Block-orthonormal near-null vectors of coarsening l: [nvec][sites][dof] FP64. */
SMG_API int smg_get_null_vectors(smg_ctx* ctx, int l, void* out, int where);
/* Coarse operator produced by coarsening l, as the level uses it: A_hat, or
 * X^{-1} A_hat with block_coarse; [Vc][N][9][N] FP64 (Sec. 2.1, 2.3). */
SMG_API int smg_get_coarse_op(smg_ctx* ctx, int l, void* out, int where);
/* X^{-1} of the self blocks of coarsening l's A_hat, [Vc][N][N] FP64 row-major
 * (Sec. 2.3).  SMG_ERR_STATE unless the setup used block_coarse. */
SMG_API int smg_get_coarse_xinv(smg_ctx* ctx, int l, void* out, int where);
/* Deflation of the coarsest level (coarsest_deflate = k): sigma[k] the k
 * lowest singular values (ascending); info[4] = {Chebyshev interval lower
 * end sigma_k, upper end (sigma_max estimate), subspace iterations, largest
 * relative residual |A^dag A v - sigma^2 v| / b of the k pairs}.
 * SMG_ERR_STATE without a deflated coarsest level. */
SMG_API int smg_get_deflation(smg_ctx* ctx, double* sigma, double* info);
/* One solve of coarse level l + 2 (the level coarsening l produces) as the
 * K-cycle runs it (dense inverse, deflated Chebyshev CA-GCR, or GCR with the
 * K-cycle below), in the setup's precision, on nsys right-hand sides
 * [nsys][Vc][N] complex FP64; out likewise. */
SMG_API int smg_coarse_solve(smg_ctx* ctx, int l, int nsys, const void* in, void* out, int where);
/* Restriction / prolongation of coarsening l and the coarse operator of
 * level l in precision `prec`, on nsys FP64 fields. */
SMG_API int smg_restrict(smg_ctx* ctx, int l, int prec, int nsys, const void* in, void* out, int where);
SMG_API int smg_prolong(smg_ctx* ctx, int l, int prec, int nsys, const void* in, void* out, int where);
SMG_API int smg_coarse_apply(smg_ctx* ctx, int l, int prec, int nsys, const void* in, void* out, int where);
/* Fermion-force outer product: F_mu(x) = -c eta_mu(x) [Y(x) X(x+k mu)^dag - X(x) Y(x+k mu)^dag]
 * with k = 1, c = 1 (which = 0, fat links) or k = 3, c = c_naik (which = 1, Naik links).
 * X, Y: V*3 complex FP64; F: [4][V][3][3] complex FP64. */
SMG_API int smg_force(smg_ctx* ctx, const void* X, const void* Y, int which, void* F, int where);
/* Fermion action S = phi^dag (M^dag M)^{-1} phi for the current gauge field
 * and mass, by two multigrid solves to `tol`: Z = M^{-1} (eps phi),
 * Y = eps Z = M^{-dag} phi (eps M eps = M^dag), X = M^{-1} Y, S = |Y|^2, and
 * dS/dm = -2 m |X|^2.  X, Y (V*3 complex FP64, may be NULL) receive the
 * vectors that smg_force turns into the link derivative (HMC fermion force;
 * Sec. 4 names gauge generation as a use of the solver).  info: 2 entries
 * (may be NULL).  Returns SMG_ERR_NOT_CONVERGED if a solve missed tol. */
SMG_API int smg_fermion_action(smg_ctx* ctx, const void* phi, void* X, void* Y, double tol, int where, double* S,
                               double* dSdm, smg_solve_info* info);
/* Iterations used by the near-null CGNE of coarsening l (max over vectors). */
SMG_API int smg_setup_iterations(smg_ctx* ctx, int l, int* iters);
/* Wall-clock seconds that the last smg_mg_setup spent on coarsening l, by
 * phase (Sec. 3.2 and Table 2 count setup apart from the solves):
 * secs[0] near-null CGNE, secs[1] chiral doubling, block orthonormalisation
 * and prolongator packing, secs[2] the Galerkin stencil R A P, secs[3] the
 * rest (stencil dagger, block preconditioning, packing to storage precision,
 * dense inverse or deflation of the coarsest level).  The stream is
 * synchronised at each phase boundary.  After smg_load_setup, secs[0] is 0. */
SMG_API int smg_setup_times(smg_ctx* ctx, int l, double secs[4]);

/* Kernels that smg_time_kernel can time. */
enum {
  SMG_KERNEL_DSLASH = 0,    /* m + D on the fine lattice                    */
  SMG_KERNEL_KD = 1,        /* (B+m)^{-1} per hypercube                     */
  SMG_KERNEL_RESTRICT = 2,  /* R of coarsening l                            */
  SMG_KERNEL_PROLONG = 3,   /* P of coarsening l                            */
  SMG_KERNEL_COARSE = 4,    /* 9-point coarse operator of coarsening l      */
  SMG_KERNEL_A = 5,         /* A = (B+m)^{-1} M on the fine lattice (Eq. 2):  */
                            /* the dslash and block launches of one apply   */
  SMG_KERNEL_COARSE_SOLVE = 6  /* one solve of the level coarsening l produces,
                                  as the K-cycle runs it (dense inverse,
                                  deflated Chebyshev CA-GCR, Schur form or GCR
                                  with the K-cycle below), synthetic rhs  */
};
/* Average device milliseconds of one launch of `kernel` on nsys systems, in
 * the setup's preconditioner precision (FP64 before mg_setup), timed with
 * CUDA events on the context's stream over nrep back-to-back launches after
 * one warm-up launch.  Inputs are library-owned zero fields. */
SMG_API int smg_time_kernel(smg_ctx* ctx, int kernel, int l, int nsys, int nrep, double* ms_per_launch);
/* The 9-point coarse apply (Sec. 3.1) on a synthetic stencil of coarse
 * extents cdims[4] with N components per site, nsys right-hand sides, storage
 * precision `prec` (FP32 vectors; FP64 for SMG_PREC_DOUBLE): average device
 * milliseconds per launch over nrep back-to-back launches (CUDA events on the
 * context's stream).  Allocates and frees its own stencil and fields. */
SMG_API int smg_bench_coarse_apply(smg_ctx* ctx, const int cdims[4], int N, int nsys, int prec, int nrep,
                                   double* ms_per_launch);
/* Kernels of the 9-point coarse apply (Sec. 3.1: the paper's coarse stencil
 * exposes extra parallelism beyond the volume; here the choice is a kernel
 * per shape).  CORES: one CTA per site and system, a warp per row, any
 * precision; MMA: mma.sync tensor-core GEMM over several systems (FP16
 * stencil, FP32 vectors, N % 16 == 0, N <= 128, nsys >= 2); TC_*: tcgen05 + TMA
 * GEMM over up to 16 systems per launch (FP16 stencil, FP32 vectors, N = 128,
 * nsys >= 2) with 1 or 2 persistent CTAs per SM and a 4- or 6-stage stencil
 * ring; ROWS: CUDA cores, any precision, the V*N output rows of each system
 * split evenly over a grid that fills every SM once, a half warp per row
 * (no partly filled last wave when V is not a multiple of the resident
 * CTAs); ROWS_MULTI: the same for up to 8 systems per CTA (FP32 vectors,
 * FP16 or FP32 stencil, N % 4 == 0, nsys >= 2), each stencil chunk loaded
 * once for the group, vectors kept in FP32 (the near-null CGNE's batched
 * applies).  AUTO: the autotuner's choice (below). */
enum {
  SMG_COARSE_AUTO = 0,
  SMG_COARSE_CORES = 1,
  SMG_COARSE_MMA = 2,
  SMG_COARSE_TC_1x4 = 3,
  SMG_COARSE_TC_2x4 = 4,
  SMG_COARSE_TC_1x6 = 5,
  SMG_COARSE_ROWS = 6,
  SMG_COARSE_ROWS_MULTI = 7
};
/* The coarse apply (Sec. 3.1) of a caller's stencil: stencil is FP64
 * [Vc][N][9][N] complex ([site][row][direction][column]; direction 0 self,
 * 1 + 2mu forward, 2 + 2mu backward) on the periodic coarse lattice cdims[4],
 * packed to the storage of `prec` as smg_mg_setup packs its own (FP16 with
 * one FP32 scale per row for SMG_PREC_HALF); in, out: [nsys][Vc][N] FP64,
 * rounded to the vector precision of `prec`; path: SMG_COARSE_*.
 * SMG_ERR_ARG when the path does not serve the shape; SMG_ERR_TIMEOUT when a
 * bounded wait of the tcgen05 kernel gave up. */
SMG_API int smg_coarse_apply_stencil(smg_ctx* ctx, const int cdims[4], int N, int prec, int path,
                                     const void* stencil, int nsys, const void* in, void* out, int where);
/* Host only: the SMG_COARSE_* kernels that serve N components, nsys systems
 * and precision `prec`, the untuned default first; writes up to cap of them
 * and returns how many there are (SMG_ERR_ARG on bad arguments). */
SMG_API int smg_coarse_paths(int N, int nsys, int prec, int* paths, int cap);

/* Autotuner of launch shapes (an implementation service; the paper has no
 * counterpart).  The first time a kernel family meets a shape with more than
 * one candidate (today: the coarse apply's kernels), every candidate runs on
 * that shape's real operator data into scratch output, timed with CUDA
 * events on the calling stream, and the fastest serves the shape for the rest
 * of the process; nothing is tuned while a stream is being captured into a
 * graph (the untuned default serves instead).  mode: 1 = tune (default),
 * 0 = always the untuned default.  The table is process-wide. */
SMG_API int smg_tune_mode(int mode);
/* The table as text, one shape per line: key, chosen path id, its name, then
 * name=ms for each timed candidate, tab separated.  Writes at most cap bytes
 * (NUL-terminated) and returns the size the whole text needs. */
SMG_API long long smg_tune_table(char* buf, long long cap);
/* Writes the table to a file / merges a file's entries (key and path id of
 * each line) into the table, so that a later process skips the timing.
 * SMG_ERR_ARG on an unreadable or malformed file. */
SMG_API int smg_tune_save(const char* path);
SMG_API int smg_tune_load(const char* path);
SMG_API int smg_tune_clear(void);

/* Launch plan of the persistent coarse-level solver (host only, no device
 * needed): a level of V sites with N components, nsys systems, nvec_next
 * near-null vectors of the next level (0: coarsest, no restriction), storage
 * SMG_PREC_SINGLE or SMG_PREC_HALF, on a device with `sms` SMs and `smem_cap`
 * bytes of shared memory per block.  out: grid, rows per CTA, site slots per
 * CTA, resident (1/0), systems per staging round, dynamic shared bytes, and
 * the shared-memory offsets of the stencil rows, row scales, prolongator rows
 * and staging area.  Returns SMG_ERR_ARG on a bad shape. */
SMG_API int smg_persist_plan(int V, int N, int nsys, int nvec_next, int prec, int sms, long long smem_cap,
                             long long out[10]);

/* Test hook for the bounded waits (no counterpart in the paper): the grid
 * barriers of the persistent coarse-level solver give up after limit_ns
 * nanoseconds (default 2 s; 1000 <= limit_ns <= 2e9) and, with
 * extra_arrivals = 1, expect one arrival that never comes, so that every
 * barrier wait runs out.  The kernel then records an error, lets its bulk
 * copies land and returns; the solve returns SMG_ERR_TIMEOUT and clears the
 * barrier words.  (limit 2e9, extra 0) restores normal operation. */
SMG_API int smg_debug_persist_barrier(smg_ctx* ctx, long long limit_ns, int extra_arrivals);

/* Total kernels launched by the library in this process (a CUDA-graph replay
 * counts every kernel node it runs). */
SMG_API long long smg_kernel_launches(void);

/* Batched inner products that allocate nothing: out[s] = <x_s, y_s> =
 * sum_i conj(x[s][i]) y[s][i] for s < nsys, FP64 complex, all three buffers in
 * device memory ([nsys][n] interleaved complex; out: nsys complex).  The paper
 * has no counterpart: this is a service for callers that cannot allocate on
 * the call path (a framework whose caching allocator owns the device heap, or
 * a latency-critical loop that cannot take cudaMalloc's implicit device
 * synchronisation).  It reduces in a fixed file-scope device array of
 * 8192 partial sums (128 KiB per device, held until the process exits), so
 * nsys must not exceed 8192 (SMG_ERR_ARG otherwise); x, y and out must be
 * 16-byte aligned (SMG_ERR_ARG otherwise); no cudaMalloc/cudaFree or
 * allocating library routine is called.  The first call on a device looks up
 * that array's device address (cudaGetSymbolAddress) and should come before
 * any stream capture.  Work is enqueued on the context's stream and the call
 * returns without waiting.  Every call shares the array (its counter is
 * cleared at the start of each call): calls that overlap on the GPU race. */
SMG_API int smg_dot_noalloc(smg_ctx* ctx, const void* x, const void* y, long long n, int nsys, void* out);

#ifdef __cplusplus
}
#endif

#endif /* SMG_H */
