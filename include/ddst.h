/*
 * ddst.h -- C ABI of the GB300 overlapping solution-transfer domain decomposition.
 *
 * Method: arXiv 2510.25991, "An overlapping domain decomposition method based on
 * solution-transfer operators".  The library solves the variable-coefficient elliptic
 * boundary value problem of Sec. 1, Eq. (basic),
 *
 *     -div(a grad u) + b . grad u + c u = f   in the unit square / cube,   u = g on the boundary,
 *
 * discretized by the five-point (2D) / seven-point (3D) finite-difference stencil of Sec. 2.1 /
 * Sec. 5.2 on a uniform grid with n cells per side (h = 1/n).  The domain is cut into slabs of
 * w cells normal to x; the N_ds = n/w - 1 interior interfaces Gamma_j are coupled by the local
 * Dirichlet solution-transfer operators S_{j,j-1}, S_{j,j+1} of the overlapping double slabs
 * Psi_j (Sec. 2.2, Eq. (defS); Alg. 1, Alg. 2).  The equilibrium system (I - K) u_Gamma = fhat
 * (Sec. 1, Eq. (modelS)) is solved by unrestarted GMRES (Sec. 5), after which the volume is
 * reconstructed by local solves.  Mixed precision (FP32 local operators, FP64 Krylov and FP64
 * global residual refinement) is this library's addition; the paper computes in FP64.
 *
 * Conventions shared by every entry point
 *  - Arrays are FP64 and C-contiguous with x the slowest axis.  Nodal arrays (a, c, g and the
 *    gradient dL/da, dL/dg) have (n+1)^dim entries; interior arrays (f, u, dL/du, dL/df) have
 *    (n-1)^dim entries.  Interface vectors are N_ds blocks of n_Gamma = (n-1)^(dim-1) values,
 *    block j holding Gamma_j ordered like the remaining axes (y, then z).
 *  - An array argument may point to host or to device memory; the library detects which with
 *    cudaPointerGetAttributes and stages host arrays through its own device buffers.  Arrays
 *    are owned by the caller and only read/written during the call.
 *  - Every call is ordered on the CUDA stream given to ddst_setup (NULL = the legacy default
 *    stream) and returns after the stream has finished the call's work.
 *  - No entry point aborts, traps or waits without bound.  Errors return a status, record a
 *    message (ddst_last_error) and leave the context usable.  A call out of order returns
 *    DDST_ERR_STATE.
 *  - Device memory of a context is allocated by the library (cudaMalloc) and released by
 *    ddst_destroy.
 *  - Threads: calls on one context must not overlap; different contexts may be used from
 *    different threads at the same time (kernel shared-memory limits are raised under a lock,
 *    the context-free error message is per thread).  ddst_residual_noalloc calls share one
 *    scratch array and must be serialized by the caller.
 *  - Devices: a context belongs to the device that is current at ddst_setup, and that device
 *    must be current for every later call on it.  Several GPUs are driven with one process
 *    per GPU.
 */
#ifndef DDST_H
#define DDST_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DDST_OK = 0,
  DDST_ERR_INVALID_ARG = 1,   /* bad size, pointer or option                               */
  DDST_ERR_OOM = 2,           /* cudaMalloc failed                                         */
  DDST_ERR_CUDA = 3,          /* any other CUDA runtime error                              */
  DDST_ERR_SINGULAR = 4,      /* a local pivot block was singular (info.fail_slab/_block)  */
  DDST_ERR_NOT_CONVERGED = 5, /* GMRES or refinement missed its tolerance                  */
  DDST_ERR_TIMEOUT = 6,       /* a bounded device wait ran out                             */
  DDST_ERR_STATE = 7,         /* call out of order (e.g. solve before build_transfer)      */
  DDST_ERR_NOT_IMPLEMENTED = 8
} ddst_status;

/* Arithmetic of the local operators, transfer operators and their application. */
enum {
  DDST_FP64 = 0,   /* everything FP64                                                      */
  DDST_MIXED = 1,  /* FP32 factors, FP32 transfer operators (FP32 accumulation; the
                      tensor-core products as 3xTF32, accurate to FP32), FP64 GMRES
                      vectors, FP64 global residual refinement                             */
  DDST_MIXED_TF32 = 3, /* DDST_MIXED with one TF32 product (not 3xTF32) per tensor-core step
                      of the transfer build and the large-block factorization: about a third
                      of their tensor work, TF32-accurate operators (relative error ~1e-3),
                      more FP64 refinement steps for the same final accuracy            */
  DDST_AUTO = 2    /* DDST_MIXED, or DDST_FP64 when an FP32 pivot falls below its floor
                      (1e3 eps |diag|).  The block elimination does not pivot, so this
                      happens only for indefinite local operators (Helmholtz slabs wider
                      than about half a wavelength) whose leading block minors pass near
                      zero; ddst_get_precision reports which one was used.                */
};

typedef struct ddst_ctx ddst_ctx;

/* Uniform grid on the unit square (dim = 2) or cube (dim = 3) with n cells per side. */
typedef struct {
  int dim;
  int64_t n;
} ddst_grid;

/* PDE coefficients of Sec. 1, Eq. (basic). */
typedef struct {
  const double* a;  /* nodal diffusion coefficient, (n+1)^dim values, all > 0 (required)       */
  double b[3];      /* constant convection vector (unused components ignored)                  */
  const double* c;  /* nodal reaction coefficient, (n+1)^dim values, or NULL for c = 0         */
} ddst_coeffs;

typedef struct {
  int precision;        /* DDST_FP64, DDST_MIXED, DDST_MIXED_TF32 or DDST_AUTO                */
  double gmres_tol;     /* relative residual target of each interface GMRES solve; <= 0 picks
                           1e-10 for DDST_FP64 and, for DDST_MIXED (inner solve of the
                           refinement), 1e-3 with explicit transfer operators or 1e-2 when some
                           are applied matrix-free                                            */
  int gmres_max_iter;   /* Krylov dimension cap (unrestarted GMRES; used clamped to 1..1000)  */
  double refine_tol;    /* FP64 refinement stops when its error estimate, rho / (1 - rho) times
                           the last correction (rho: observed contraction, the larger of the
                           last two ratios; taken as >= 1/2 while only one ratio is known; no
                           estimate while rho >= 1), is <= refine_tol * ||u||               */
  int refine_max;       /* maximum number of refinement steps (0 = plain DD solve)            */
  int k_max;            /* HODLR rank cap per block (used clamped to 1..128)                  */
  int oversample;       /* extra random samples beyond k_max; the sketch width k_max +
                           oversample is capped at 128                                        */
  int leaf_size;        /* HODLR leaf size (used clamped to 8..256)                          */
  uint64_t seed;        /* seed of the counter-based Gaussian sketch generator                */
  int check_every;      /* GMRES iterations between host convergence checks; 0 = automatic:
                           every iteration for matrix-free operators, every 8 otherwise       */
  int factor_chunks;    /* pivot sweeps split along y into warm-started chunks per slab and
                           direction: 0 automatic, 1 exact sequential sweeps, k > 1 forced     */
  int factor_warmup;    /* warm-up rows of a chunk (0: 4 w in FP32, 10 w in FP64)              */
  int tensor_cores;     /* 1: DDST_MIXED transfer build (block sizes <= 64) and large-block
                           factorization on the tcgen05 tensor cores (3xTF32); 0: FP32 FMA
                           kernels (kept for validation); -1 automatic: 1 unless a tuned
                           cache entry (autotune_cache) says otherwise                        */
  int explicit_S;       /* transfer operators: 1 formed explicitly (Alg. 1 with the identity as
                           test matrix; required by ddst_compress), 0 applied matrix-free through
                           two sweeps of local solves per GMRES iteration (no S stored), -1
                           automatic: matrix-free when some block is larger than 128 (or 64 in
                           FP64), explicit otherwise                                          */
  int recompute_factors; /* 1: release the local factors once the transfer operators exist and
                           recompute them at the start of every solve, adjoint or matrix-free
                           application (the HBM they take is free in between, at the cost of
                           one factorization per call); 0: keep them                          */
  const char* autotune_cache; /* path of the autotuner's cache file (text, one line per
                           device and set of problem shapes), or NULL.  At setup, an entry for
                           this device and these shapes replaces the knobs left automatic:
                           precision (only DDST_AUTO), tensor_cores (-1), explicit_S (-1),
                           gmres_tol (<= 0), check_every (0), factor_chunks (0) and
                           interface_solver (-1).
                           ddst_autotune writes the entry.  The string is read during the
                           call only.                                                         */
  int interface_solver; /* 0: GMRES on (I - K) u_Gamma = fhat (the paper's solver); -1
                           automatic: GMRES unless a tuned cache entry says 1; 1: direct,
                           by block cyclic reduction of the block-tridiagonal system (the
                           direct solvers of Sec. 4), factored from the explicit S at the first
                           solve after ddst_build_transfer (dense blocks, also after
                           ddst_compress) and reused by every later solve and adjoint.  Needs
                           explicit transfer operators and n_Gamma <= 8192 (else
                           NOT_IMPLEMENTED at the solve).  Cost: per level, the inversion of
                           half the remaining diagonal blocks and about three products of
                           n_Gamma^3 per block; memory about 5 N_ds n_Gamma^2 elements plus
                           packed scratch during the factorization                            */
} ddst_options;

/* Per-call report.  Times are milliseconds measured with CUDA events on the context stream. */
typedef struct {
  int gmres_iters;        /* GMRES iterations summed over refinement steps                    */
  int gmres_iters_first;  /* iterations of the first interface solve                          */
  int refine_iters;       /* DD solves performed (1 = no refinement correction needed)        */
  double rel_residual;    /* final ||b - A u||_2 / ||b||_2 in FP64                            */
  double est_rel_error;   /* refinement error bound rho/(1-rho) ||last correction|| / ||u||,   */
                          /* per problem; a batch reports its largest problem's bound          */
  double t_factor, t_transfer, t_compress, t_solve;
  int64_t bytes_factors;  /* device bytes of the local factors (held only during setup and each
                             call when recompute_factors is set)                              */
  int64_t bytes_transfer; /* device bytes of the transfer operators (dense or HODLR)          */
  int max_rank;           /* largest HODLR rank (0 when dense)                                */
  int fail_slab;          /* first slab with a singular pivot, else -1                        */
  int fail_block;         /* its block (y index, 1-based), else -1                            */
  int factor_chunks;      /* chunks per slab sweep actually used (1 = sequential; a failed
                             warm-up check falls back to 1)                                   */
  double factor_check;    /* largest relative warm-up check difference (0 when sequential)    */
  double t_direct;        /* milliseconds of the direct interface factorization (0 if none)  */
  double refine_rho;      /* slowest refinement contraction observed: the largest ratio
                             ||correction_k|| / ||correction_{k-1}|| over the problems (corrections
                             at the FP64 rounding level excluded); 0 with one DD solve          */
} ddst_info;

/* Fills *opt with defaults: MIXED, gmres_tol automatic (see above), refine_tol 1e-9,
 * refine_max 8, gmres_max_iter 1000, k_max 64, oversample 10, leaf_size 128, seed 1234,
 * check_every 0 (automatic), tensor_cores -1 (automatic), explicit_S -1, recompute_factors 0,
 * autotune_cache NULL.
 * Testing hooks (environment variables, read at each use; they exercise the error paths without
 * a device fault):
 *  - DDST_FAIL_ALLOC=k: the k-th device allocation of the library after the variable was set
 *    fails as out of memory (DDST_ERR_OOM) without calling cudaMalloc.
 *  - DDST_WAIT_CYCLES=c: the pipeline waits of the tensor-core transfer build give up after c
 *    clock cycles instead of about 4e9 (2 s); a short budget makes a wait expire on purpose and
 *    ddst_build_transfer returns DDST_ERR_TIMEOUT.  Waits for copies or MMAs already issued keep
 *    the full budget, so nothing is in flight when the kernel exits. */
void ddst_options_default(ddst_options* opt);

/* Builds the local operators A_j(I_j, I_j) of every double slab and factors them
 * (Sec. 2.5 and Alg. 2: "compute local discretization", "factorize").
 * grid/coeffs: one problem; slab_width: w cells (n % w == 0, n/w >= 2, block size
 * m = (2w-1)(n-1)^(dim-2) <= 8192).  Blocks up to 128 (64 in FP64) are factored by one CTA per
 * slab and sweep direction (two-sided block LU, explicit inverses F, B and diagonal blocks G of
 * A_j^{-1}); larger blocks, padded to a multiple of 128, by a one-sided block LU whose dense
 * inverses are formed by 128-wide Gauss-Jordan panels on the tensor cores (FP32) or FMA (FP64),
 * all slabs of a block size advancing together.  opt may be NULL (defaults).  stream:
 * cudaStream_t or NULL.  On success *out receives a new context.  Errors: INVALID_ARG, OOM,
 * CUDA, SINGULAR. */
ddst_status ddst_setup(const ddst_grid* grid, const ddst_coeffs* coeffs, int slab_width,
                       const ddst_options* opt, void* stream, ddst_ctx** out);

/* Same for nprob independent problems sharing one context (batched kernels over all slabs of
 * all problems).  grids, coeffs and slab_widths are arrays of nprob entries. */
ddst_status ddst_setup_batch(int nprob, const ddst_grid* grids, const ddst_coeffs* coeffs,
                             const int* slab_widths, const ddst_options* opt, void* stream,
                             ddst_ctx** out);

/* Forms every S_{j,j-1} and S_{j,j+1} explicitly (Sec. 2.2, Eq. (defS)) from one transposed
 * multi-right-hand-side solve per double slab with the central interface points as sources.
 * In a matrix-free context (options.explicit_S) nothing is formed: S is applied through the
 * local factors (two sweeps of local solves per application; Sec. 2.5, the LU column of the
 * comparison in Sec. 5.1), and this call only marks the operators ready.
 * Requires ddst_setup.  Errors: STATE, OOM, CUDA. */
ddst_status ddst_build_transfer(ddst_ctx* ctx);

/* Compresses every S_{j,j'} into HODLR form (Sec. 2.4: weak admissibility, cluster tree
 * shared by source and target interface) by randomized sampling with Gaussian sketches; each
 * off-diagonal block is truncated at sigma_{r+1} <= tol * ||S_{j,j'}||_2 (rank <= k_max).
 * tol <= 0 keeps the dense operators.  In DDST_MIXED the sketch and range finder run in FP32 and
 * reject samples below 1e3 eps_32 of their own norm, which floors the compression error near 1e-5
 * of ||S_{j,j'}||_2: requests below about 1e-5 are met only in DDST_FP64 (the FP64 refinement of
 * ddst_solve still reaches its refine_tol).  Requires ddst_build_transfer.  Errors: STATE, OOM, CUDA,
 * INVALID_ARG (cluster tree deeper than 12 levels: raise leaf_size), NOT_IMPLEMENTED (tol > 0 on a
 * matrix-free context: compression samples the explicit operators). */
ddst_status ddst_compress(ddst_ctx* ctx, double tol);

/* Compresses every S_{j,j'} into nested-basis HBS form (Sec. 2.4: weak admissibility, cluster
 * tree shared by source and target interface, O(k N) storage and apply) from s = 3 rank +
 * oversample Gaussian samples Y = S Omega and Z = S^T Psi per operator (Alg. 1), drawn on the
 * device from options.seed.  Fixed rank `rank` per tree node, leaves of at most 2 rank indices.
 * Per node: U = the leading `rank` columns of the column-pivoted QR of Y_t P (P an orthonormal
 * basis of the null space of the node's rows of Omega), V likewise from Z and Psi, the diagonal
 * remainder D = (I - U U^T) Y_t Omega_t^+ + U U^T ((I - V V^T) Z_t Psi_t^+)^T, and the reduced
 * samples passed to the parent; the root keeps the reduced 2 rank x 2 rank matrix.  Exact (to
 * rounding) when every off-diagonal block row and column of the tree has rank <= `rank`.  The
 * node algebra runs in the working precision (FP32 in DDST_MIXED).  Solves then apply the HBS
 * operators; ddst_compress (either tol) or ddst_build_transfer drops them.  Requires
 * ddst_build_transfer.  Errors: STATE, OOM, CUDA, INVALID_ARG (rank outside 1..32, oversample
 * < 0 or 3 rank + oversample > 96), NOT_IMPLEMENTED (a context that applies any operator
 * matrix-free). */
ddst_status ddst_compress_hbs(ddst_ctx* ctx, int rank, int oversample);

/* A dense operator compressed on its own into HBS form (the algorithm of ddst_compress_hbs). */
typedef struct ddst_hbs ddst_hbs;

/* Compresses the dense ng x ng row-major FP64 host matrix S into HBS form with fixed rank
 * `rank`, `nsamples` samples (>= 3 rank, <= 96) and leaves of at most `leaf` (<= 64) indices of
 * the balanced bisection tree (node t of level l covers [t ng / 2^l, (t+1) ng / 2^l)).  omega
 * and psi: the ng x nsamples row-major FP64 host test matrices, or both NULL to draw them on the
 * device.  precision: DDST_FP64 or DDST_MIXED (FP32 storage and node algebra).  The caller
 * keeps its arrays; *out is released with ddst_hbs_destroy.  The paper compresses the transfer
 * operators only (this entry point exposes the same compression for any dense operator).
 * Errors: INVALID_ARG (NULL or device pointers, bad sizes, a leaf's size plus rank above
 * nsamples), OOM, CUDA. */
ddst_status ddst_hbs_create(const double* S, int64_t ng, int rank, int nsamples, int leaf,
                            const double* omega, const double* psi, int precision,
                            ddst_hbs** out);

/* y = S_H x (transpose = 0) or S_H^T x (transpose = 1): the upward pass (V^T x per leaf, then
 * the inner levels), the root, and the downward pass (D x + U y_parent).  x, y: ng values, host
 * or device arrays; returns after y is written.  Errors: INVALID_ARG, CUDA. */
ddst_status ddst_hbs_apply(ddst_hbs* h, const double* x, double* y, int transpose);

/* The dense expansion of S_H, row-major ng x ng into a host array.  Errors: INVALID_ARG, CUDA. */
ddst_status ddst_hbs_expand(ddst_hbs* h, double* out);

/* Tree depth L (levels below the root) and stored numbers of the representation (leaves
 * n^2 + 2 n k, inner nodes 8 k^2, root 4 k^2).  Either output may be NULL.  Errors: INVALID_ARG. */
ddst_status ddst_hbs_stats(const ddst_hbs* h, int* levels, int64_t* entries);

/* Releases a handle from ddst_hbs_create (NULL is ignored). */
void ddst_hbs_destroy(ddst_hbs* h);

/* Solves for one problem (contexts made by ddst_setup): equivalent loads (Sec. 2.2, Eq.
 * (equilib1)), GMRES on (I - K) u_Gamma = fhat, volume reconstruction, then FP64 residual
 * refinement u += DD(b - A u) until the error bound rho/(1-rho) ||correction|| (rho: observed
 * contraction ratio of the corrections, no bound while it is >= 1) is <= refine_tol ||u||; the
 * bound is info->est_rel_error.  In a batch the test holds for every problem on its own (its own
 * corrections and its own ||u||), not for the concatenated vector.
 * f: interior load; g: nodal Dirichlet data (only boundary nodes are read); u: interior
 * output.  info may be NULL.  Errors: STATE, INVALID_ARG, NOT_CONVERGED (u still written). */
ddst_status ddst_solve(ddst_ctx* ctx, const double* f, const double* g, double* u,
                       ddst_info* info);

/* IMEX backward-Euler time marching (Sec. 6, Example 1, Eq. (convdiff)) on a context set up
 * for the screened operator -div(a grad u) + c u with reaction c = 1/dt (and no convection b):
 * each of nsteps steps solves it for f = U_n / dt - v . grad_h U_n (central differences at the
 * interior nodes, U_n = 0 on the boundary) with zero Dirichlet data, so the factors, transfer
 * operators and (interface_solver = 1) factored equilibrium system are reused by every step.
 * The refinement of step n + 1 starts from U_n.  Arrays per problem (nprob pointers each):
 * vel[q] holds dim nodal velocity components, component d at offset d (n+1)^dim; u0[q] the
 * interior initial state; u[q] receives U_nsteps.  info sums GMRES iterations and refinement
 * steps over the steps (est_rel_error, rel_residual and refine_rho: the worst step); t_solve is
 * the whole march.  The paper's example has Neumann and periodic sides; this driver keeps the
 * library's Dirichlet boundary.  Errors: INVALID_ARG (nsteps < 0, dt <= 0, NULL), STATE,
 * NOT_CONVERGED (the march stops at the step that missed refine_tol; u holds that step). */
ddst_status ddst_march(ddst_ctx* ctx, int nsteps, double dt, const double* const* vel,
                       const double* const* u0, double* const* u, ddst_info* info);

/* Batched form: f, g, u are arrays of nprob pointers (one per problem). */
ddst_status ddst_solve_batch(ddst_ctx* ctx, const double* const* f, const double* const* g,
                             double* const* u, ddst_info* info);

/* Discrete adjoint of the last ddst_solve: lambda = A^{-T} dL_du through the transposed DD
 * (transposed local solves through the same factors, transposed transfer operators, GMRES
 * on (I - K)^T), refined against the FP64 residual of A^T.  Writes dL_df = lambda (interior),
 * dL_dg (nodal; boundary nodes only, interior entries set to 0) and dL_da (nodal; may be
 * NULL to skip).  Any output pointer may be NULL.  Errors: STATE, NOT_CONVERGED. */
ddst_status ddst_solve_adjoint(ddst_ctx* ctx, const double* dL_du, double* dL_df,
                               double* dL_dg, double* dL_da, ddst_info* info);

/* Batched adjoint: arrays of nprob pointers. */
ddst_status ddst_solve_adjoint_batch(ddst_ctx* ctx, const double* const* dL_du,
                                     double* const* dL_df, double* const* dL_dg,
                                     double* const* dL_da, ddst_info* info);

/* Interface traces u_Gamma of problem prob from the last solve (N_ds * n_Gamma values, host or
 * device array): the refined solution u on the interfaces Gamma_j (Sec. 2.2), which solves the
 * equilibrium system (I - K) u_Gamma = fhat of Sec. 1, Eq. (modelS) to the refinement's
 * accuracy.  Errors: INVALID_ARG (bad prob or NULL), STATE (no solve yet), CUDA. */
ddst_status ddst_interface_trace(ddst_ctx* ctx, int prob, double* uG);

/* Copies S_{j,j-1} (side = -1) or S_{j,j+1} (side = +1) of problem prob, slab j (1-based),
 * as a dense row-major n_Gamma x n_Gamma FP64 matrix (expanded from HODLR or HBS if compressed) into
 * a host or device array.  Errors: INVALID_ARG (bad prob, j or side; no such block at the
 * ends), STATE (transfer operators not built), NOT_IMPLEMENTED (matrix-free context), CUDA. */
ddst_status ddst_get_transfer(ddst_ctx* ctx, int prob, int j, int side, double* out);

/* y = (I - K) x (transpose = 0) or y = (I - K)^T x (transpose = 1) for problem prob with the
 * current (dense, HODLR or HBS) operators (Sec. 2.2, Eq. (modelS)); x and y hold N_ds * n_Gamma
 * values, host or device arrays; returns after y is written (synchronizes the context stream).
 * Errors: INVALID_ARG, STATE (transfer operators not built), CUDA. */
ddst_status ddst_apply_interface(ddst_ctx* ctx, int prob, const double* x, double* y,
                                 int transpose);

/* Diagnostic timing of the interface operator, the matrix-vector product of every GMRES
 * iteration (Eq. (modelS)): runs `reps` applications of (I - K) (or its transpose) to the
 * context's own interface work vectors, back to back on the context stream, and returns the
 * mean device time per application in *ms (CUDA events on that stream).  The work vectors'
 * contents are overwritten.  Errors: INVALID_ARG (NULL or reps < 1), STATE (operators not
 * built), CUDA. */
ddst_status ddst_time_apply(ddst_ctx* ctx, int transpose, int reps, float* ms);

/* Sizes of problem prob: number of double slabs n_ds, interface length n_gamma, and the
 * largest HODLR rank of the context (the HBS rank after ddst_compress_hbs; 0 while dense).  Any output may be NULL.
 * Errors: INVALID_ARG (NULL ctx or bad prob; message via ddst_last_error(NULL), since ctx is
 * const). */
ddst_status ddst_query(const ddst_ctx* ctx, int prob, int* n_ds, int64_t* n_gamma,
                       int* max_rank);

/* Arithmetic the context was set up with: DDST_FP64, DDST_MIXED or DDST_MIXED_TF32 (what
 * DDST_AUTO chose).
 * Errors: INVALID_ARG for a NULL argument (message via ddst_last_error(NULL)). */
ddst_status ddst_get_precision(const ddst_ctx* ctx, int* precision);

/* Allocation-free FP64 residual of the finite-difference system.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate device memory while
 * they run (a locked memory budget, an allocator that forbids new device allocations, or host
 * threads that must not take the driver's allocation locks); every other entry point here
 * allocates its context and work buffers with cudaMalloc.
 * Computes r = b(f, g) - A u for the problem (grid, coeffs), where b carries the load f and
 * the Dirichlet data g exactly as ddst_solve builds it, and writes norms[0] = ||r||_2,
 * norms[1] = ||b||_2 (so norms[0] / norms[1] is the relative residual ddst_solve reports).
 * All arrays must be DEVICE memory of the current device, or managed memory (this call
 * stages nothing; another GPU's memory is refused): f, u, r interior
 * ((n-1)^dim), g and coeffs->a / coeffs->c nodal ((n+1)^dim), norms two doubles.
 * At most 16,777,216 interior unknowns (e.g. a 4097^2 grid); larger grids return
 * DDST_ERR_INVALID_ARG.  The scratch is a 1 MiB file-scope device array (one FP64 partial sum
 * per 256 unknowns and per norm) that every GPU which loads the library holds until the
 * process exits; every call overwrites the partial sums it reads, so nothing has to start at
 * zero.  All calls share that array: calls that overlap on the GPU (on different streams)
 * race and must be serialized by the caller.  The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) with that device current; make that first call before
 * any stream capture.  Stream-ordered on `stream`; returns once the work is enqueued (it does
 * not wait for it).  Errors: INVALID_ARG (message via ddst_last_error(NULL)), CUDA. */
ddst_status ddst_residual_noalloc(const ddst_grid* grid, const ddst_coeffs* coeffs,
                                  const double* f, const double* g, const double* u, double* r,
                                  double* norms, void* stream);

/* Number of CUDA kernels this library has launched in the calling process so far (a
 * diagnostic for benchmarks: the difference across a timed region counts its launches). */
int64_t ddst_kernel_launches(void);

/* The direct interface solve alone (interface_solver = 1 machinery, whatever the option):
 * x = (I - K)^{-1} rhs (transpose 0) or (I - K)^{-T} rhs (transpose 1) for problem prob, rhs and
 * x of N_ds n_Gamma values in the interface order above, by block cyclic reduction of the
 * explicit transfer operators (factored at the first call, kept until ddst_build_transfer runs
 * again).  Sec. 1, Eq. (modelS); Sec. 4, direct solvers.  Errors: INVALID_ARG, STATE (no
 * transfer operators), NOT_IMPLEMENTED (matrix-free operators, n_Gamma > 8192), SINGULAR (a
 * diagonal block of the reduction fell below 1e3 eps; fail_slab names the interface block),
 * OOM. */
ddst_status ddst_solve_interface(ddst_ctx* ctx, int prob, const double* rhs, double* x,
                                 int transpose);

/* Sharding of independent problems over ranks (one process per GPU, no data-path collective):
 * item i (cost[i] >= 0, e.g. its unknowns) goes to rank owner[i] in [0, world), by longest
 * processing time first (items by decreasing cost, each to the least-loaded rank; ties by
 * index and rank), so every rank computes the same assignment without communication.  load
 * (optional, world values) receives each rank's summed cost.  Host only; no GPU needed.
 * Errors: INVALID_ARG. */
ddst_status ddst_partition(int nitems, const double* cost, int world, int* owner, double* load);

/* ---- Autotuner --------------------------------------------------------------------------
 * The method leaves its schedule to the implementation: how the pivot sweeps are split, the
 * tensor-core precision, whether S is formed or applied through local solves, and how the
 * inner GMRES tolerance is balanced against refinement steps.  ddst_autotune times these knobs
 * on the caller's own problems (one coordinate at a time, starting from the automatic
 * choices): each candidate is a full setup, transfer build, compression (compress_tol > 0) and
 * two solves, and its cost is factor + transfer + compression time plus the faster solve, all
 * CUDA-event times.  A candidate is rejected unless it solves to refine_tol with a refinement
 * contraction (ddst_info.refine_rho) of at most 0.1, so a cheaper but less accurate operator
 * wins only if the FP64 refinement still converges fast on it.  Only knobs left automatic in
 * *base are tuned.  The chosen options go to rep->chosen and, when base->autotune_cache is set,
 * into that file under the key of this device and these problem shapes (ddst_autotune_key),
 * replacing an older entry.  f, g: nprob right-hand sides as for ddst_solve_batch.
 * solves_per_setup (>= 1) weighs the solve against the one-time work in the cost: setup
 * phases + direct interface factorization + solves_per_setup x one solve (the second of the two,
 * without one-time work); the interface solver is tuned too (GMRES or block cyclic reduction).
 * The cache key does not include solves_per_setup: the last tuning of a shape is the one kept.
 * Errors: INVALID_ARG; the status of the untuned configuration when even that fails. */
typedef struct {
  ddst_options chosen;  /* base with the tuned knobs set (autotune_cache copied from base)     */
  int candidates;       /* configurations run, the untuned one included                       */
  int rejected;         /* candidates that failed or contracted slower than 0.1              */
  double default_ms;    /* cost of the untuned configuration                                  */
  double best_ms;       /* cost of the chosen configuration                                   */
  double best_rho;      /* refinement contraction observed with the chosen configuration     */
  int cache_written;    /* 1 when the entry was stored in base->autotune_cache                */
} ddst_tune_report;

ddst_status ddst_autotune(int nprob, const ddst_grid* grids, const ddst_coeffs* coeffs,
                          const int* slab_widths, const double* const* f,
                          const double* const* g, double compress_tol, int solves_per_setup,
                          const ddst_options* base, void* stream, ddst_tune_report* rep);

/* The cache key of a set of problems on the current device: the device name, compute
 * capability and SM count ("nodevice" without a GPU), the requested precision, and per problem
 * its dimension, n, slab width and whether it has a reaction term.  Writes a NUL-terminated
 * string of at most len bytes.  Errors: INVALID_ARG (NULL argument, or len too small). */
ddst_status ddst_autotune_key(int nprob, const ddst_grid* grids, const ddst_coeffs* coeffs,
                              const int* slab_widths, int precision, char* buf, size_t len);

/* Cache file access (host only; no GPU needed).  ddst_autotune_lookup sets *found and, when the
 * key is present, replaces the automatic knobs of *opt as ddst_setup does; lines that do not
 * parse are ignored.  ddst_autotune_store writes opt's knobs under key, replacing an existing
 * entry (the file is rewritten through a temporary file and renamed).  Errors: INVALID_ARG
 * (NULL argument, or a file that cannot be written). */
ddst_status ddst_autotune_lookup(const char* path, const char* key, ddst_options* opt, int* found);
ddst_status ddst_autotune_store(const char* path, const char* key, const ddst_options* opt);

/* The options a context runs with, automatic choices resolved (gmres_tol, check_every,
 * tensor_cores, precision after a DDST_AUTO fallback) and tuned knobs applied.
 * Errors: INVALID_ARG for a NULL argument. */
ddst_status ddst_get_options(const ddst_ctx* ctx, ddst_options* opt);

/* Message of the last error on ctx.  With ctx NULL: the last error the calling thread got
 * without a context (a failed ddst_setup, a NULL context, ddst_query, ddst_get_precision,
 * ddst_residual_noalloc); the message is kept per thread.  The string stays valid until the
 * next error on the same context (or thread) or ddst_destroy. */
const char* ddst_last_error(const ddst_ctx* ctx);

/* Releases the context and all its device memory.  NULL is ignored. */
void ddst_destroy(ddst_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* DDST_H */
