/*
 * tlr.h -- C ABI of the GB300 tile-low-rank (TLR) Cholesky / LDL^T library.
 *
 * Method: Boukaram, Zampini, Turkiyyah, Keyes, "H2OPUS-TLR: High Performance
 * Tile Low Rank Symmetric Factorizations using Adaptive Randomized
 * Approximation" (arXiv 2108.11932).  Section and algorithm numbers below
 * refer to that paper.
 *
 * Conventions (all entry points):
 *   - Every call returns a tlr_status; no C++ exception crosses the ABI.
 *   - Work is enqueued on the context's CUDA stream.  Calls that return host
 *     values (logdet, info, ranks, tile export) synchronize that stream.
 *   - Inputs are owned by the caller and only read during the call.  Objects
 *     returned through `tlr_mat**` are owned by the library until tlr_free.
 *   - Matrices are column-major FP64 unless stated.  "device" pointers must be
 *     device memory of the context's GPU; "host" pointers are plain host memory.
 *   - Point order: callers pass points, right-hand sides and vectors in their
 *     ORIGINAL order; the library keeps the KD-tree permutation internally.
 *   - A failed factorization leaves the matrix in state FAILED; every later
 *     call on it except tlr_get_info/tlr_free returns TLR_ERR_STATE.
 */
#ifndef TLR_GB300_H
#define TLR_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tlr_ctx tlr_ctx; /* device, stream, allocator, workspaces */
typedef struct tlr_mat tlr_mat; /* a TLR matrix or its factor, device-resident */

typedef enum {
  TLR_OK = 0,
  TLR_ERR_ARG = -1,      /* invalid argument (null pointer, bad size, bad option) */
  TLR_ERR_NOMEM = -2,    /* device or host allocation failed */
  TLR_ERR_NOT_SPD = -3,  /* a diagonal tile lost definiteness (Section 5.1); see tlr_info.k_fail */
  TLR_ERR_CUDA = -4,     /* a CUDA runtime call failed */
  TLR_ERR_TIMEOUT = -5,  /* a bounded device wait expired */
  TLR_ERR_STATE = -6,    /* object in the wrong state (e.g. solve on an unfactored matrix) */
  TLR_ERR_LIMIT = -7     /* a size exceeds a compiled-in limit */
} tlr_status;

/* Kernel of the generated covariance matrix (Section 6):
 *   A_ij = exp(-||x_i - x_j||_2 / ell) + nugget * delta_ij.                   */
enum { TLR_KERNEL_EXP = 0 };
typedef struct {
  int type;      /* TLR_KERNEL_EXP */
  double ell;    /* length scale > 0 */
  double nugget; /* added to the diagonal, > -1 (a negative nugget shifts the covariance down, which
                    makes it indefinite: the case of the safeguards of Section 5.1) */
} tlr_kernel;

/* Arithmetic of the ARA sampling / projection products (the chains of
 * Equation 2 / Equation 3).  Orthogonalization, convergence norms, the dense
 * diagonal-tile factorization and the triangular solves are FP64 always.     */
enum {
  TLR_PREC_FP64 = 0, /* everything FP64 */
  TLR_PREC_FP32 = 1, /* sampling/projection chains in FP32 with FP32 accumulation for every
                        tile whose estimated FP32 rounding error u32 sqrt(K) (|A_ik|_F +
                        sum_j |L_ij|_F |L_kj|_F) is below 1/8 of the ARA threshold, FP64 for
                        the others; eps < 1e-4 uses FP64 throughout */
  TLR_PREC_MIXED = 2 /* the products that form ARA samples and projections (construction:
                        T Omega, T^T Q; factorization: Urow_i W_i of Equation 2's chain and
                        Urow_k Z of its transpose) on the 16-bit tensor cores (FP16 inputs, FP32
                        accumulation, power-of-two block scaling), truncated to the fewest 7-bit
                        planes s
                        (2 <= s <= 8) whose worst-case error K (s+1) 2^(eA+eB-7s) per entry keeps
                        the sample's column norm (the projection's Frobenius norm) within 1/8 of
                        the ARA threshold; chosen per 128 x 16 output block on the device from
                        the blocks' exponents.  eps < 1e-4 keeps all 8 planes (FP64-exact) */
};

/* Definiteness safeguards (Section 5.1). */
enum {
  TLR_COMP_NONE = 0,
  TLR_COMP_SHIFT = 1, /* factor A + shift*I (Section 5.1, "diagonal shifting") */
  TLR_COMP_SCHUR = 2, /* A(k,k) - D_k + diag(rowsum|D_k - Dbar_k|) (Section 5.1.1) */
  TLR_COMP_MODCHOL = 3 /* Cholesky only: a diagonal tile that is not positive definite is factored by
                          the modified Cholesky of Algorithm 8 (Section 5.1.2, tlr_dense_modchol) */
};

/* Tile pivoting (Algorithm 9, Section 5.2). */
enum {
  TLR_PIVOT_NONE = 0,
  TLR_PIVOT_FROBENIUS = 1 /* Cholesky only, FP64 precision, compensation NONE or SHIFT, N a multiple of b:
                             at step k every remaining diagonal tile holds A(i,i) - D_i (the terms of the
                             finished columns are added as each column ends); the one with the largest
                             Frobenius norm (the first on ties) is exchanged with tile k, rows and columns,
                             before the step proceeds as in Algorithm 6.  The factor is that of P A P^T;
                             tlr_get_perm returns the point order with the exchanges, and the solve,
                             logdet and products take and return vectors in the original order.  With
                             SHIFT the shift is added to every diagonal tile before the first step. */
};

typedef struct {
  int bs;           /* ARA sampling block width (Algorithm 1), 1..64; 0 = 16 */
  int max_slots;    /* dynamic-batch width: tiles sampled concurrently (Algorithm 5
                       subset ri); 0 = every tile of the column */
  int precision;    /* TLR_PREC_* */
  int compensation; /* TLR_COMP_* */
  double shift;     /* diagonal shift for TLR_COMP_SHIFT (Section 5.1: s <= eps) */
  uint64_t seed;    /* Philox key of the Gaussian blocks */
  int ldl;          /* internal: set by tlr_ldlt */
  int pivot;        /* TLR_PIVOT_* */
  int reserved[6];
} tlr_opts;

/* Fill `o` with defaults: bs 16, all tiles in the batch, FP64, no compensation, seed 0. */
void tlr_opts_default(tlr_opts* o);

/* Optional device allocator.  If both are NULL the library uses
 * cudaMallocAsync/cudaFreeAsync on the context stream.  `alloc` returns NULL on
 * failure (the call then returns TLR_ERR_NOMEM). */
typedef void* (*tlr_alloc_fn)(size_t bytes, void* user);
typedef void (*tlr_free_fn)(void* ptr, void* user);

/* Create a context on `device`, enqueuing work on `cuda_stream` (a cudaStream_t, or NULL for the
 * legacy default stream).  hbm_budget: device bytes the serving queue (tlr_submit) may let the
 * context hold while it admits requests (0 = no limit); every device allocation of the library
 * goes through the context and is counted. */
tlr_status tlr_create(tlr_ctx** ctx, int device, size_t hbm_budget, void* cuda_stream, tlr_alloc_fn alloc,
                      tlr_free_fn free_fn, void* user);
tlr_status tlr_destroy(tlr_ctx* ctx);

/* TLR construction (Section 1, Figure 1; Section 6 clustering paragraph):
 * KD-order the N points (host, row-major N x d, d in 1..3), generate the kernel
 * matrix tile by tile on the device and compress every lower off-diagonal b x b
 * tile with batched ARA (Algorithm 1) to the absolute 2-norm threshold eps.
 * Diagonal tiles stay dense.  If b does not divide N the last tile is padded
 * with identity rows/columns.  *A receives a new matrix in state "A".
 * Entries are evaluated in 64-bit fixed point from the points on a per-matrix
 * grid (no FP64 arithmetic), within 4 x 2^-52 (1 + |log a_ij|) relative of the
 * FP64 formula; entries below 2^-1020 are 0.  Errors: TLR_ERR_ARG (null
 * pointers, N <= 0, d outside 1..3, b < 1, eps <= 0, ell <= 0, nugget <= -1,
 * opts.bs > min(64, b)), TLR_ERR_NOMEM. */
tlr_status tlr_compress(tlr_ctx* ctx, const double* points_host, int64_t N, int d,
                        const tlr_kernel* kernel, int b, double eps, const tlr_opts* opts,
                        tlr_mat** A);

/* Same construction from points that are already on the device in KD order
 * (pts: device, N x d row-major, ordered as tlr_kd_order returns).  perm_host
 * (host, N entries, may be NULL for the identity) gives the original index of
 * each ordered point, so that later calls keep using the original order. */
tlr_status tlr_compress_ordered(tlr_ctx* ctx, const double* pts, const int64_t* perm_host, int64_t N,
                                int d, const tlr_kernel* kernel, int b, double eps,
                                const tlr_opts* opts, tlr_mat** A);

/* Rank trimming of every off-diagonal tile U_ij V_ij^T of A, a compressed matrix (state A) or a factor,
 * as tlr_trim_tiles does for one tile: ranks never grow and each tile's error is its first dropped
 * singular value (<= eps); U_ij keeps orthonormal columns.  In place (new panels).  Errors: TLR_ERR_ARG,
 * TLR_ERR_STATE (a failed factorization), TLR_ERR_LIMIT (as tlr_trim_tiles). */
tlr_status tlr_trim(tlr_ctx* ctx, tlr_mat* A, double eps);

/* Deep copy (device-to-device) of a TLR matrix or factor. */
tlr_status tlr_copy(tlr_ctx* ctx, const tlr_mat* src, tlr_mat** dst);

/* Left-looking TLR Cholesky, Algorithm 6 (updateDense, chol, cholARAUpdate
 * with dynamic batching per Algorithm 5, batchTrsm, updateTiles).  In place:
 * A := L with A ~= L L^T.  Every updated tile is recompressed to eps.  With
 * opts.pivot = TLR_PIVOT_FROBENIUS, Algorithm 9 (tile pivoting): A := L with
 * P A P^T ~= L L^T, P recorded in the factor's point order.
 * TLR_ERR_NOT_SPD if a diagonal tile is not positive definite (k_fail in tlr_info).
 * TLR_ERR_ARG for options outside their rules (bs > min(64, b); MODCHOL with
 * b > 2048; pivoting with precision other than FP64, compensation other than
 * NONE or SHIFT, or N not a multiple of b). */
tlr_status tlr_potrf(tlr_ctx* ctx, tlr_mat* A, double eps, const tlr_opts* opts);

/* Pivot-free left-looking TLR LDL^T, Algorithm 10 (five-product sampling
 * chain of Equation 3, dense unpivoted LDL^T of the diagonal tiles, batchTrsm
 * followed by batchIDMult).  In place: A := (L, D), L unit lower on the diagonal
 * tiles.  TLR_ERR_NOT_SPD if a pivot of D is exactly zero or not finite.
 * TLR_ERR_ARG also for TLR_COMP_MODCHOL and for tile pivoting (Cholesky only). */
tlr_status tlr_ldlt(tlr_ctx* ctx, tlr_mat* A, double eps, const tlr_opts* opts);

/* Batched factorization of `count` independent matrices (Cholesky if ldl == 0,
 * else LDL^T), each in place as with tlr_potrf / tlr_ldlt.  The matrices advance
 * column by column together and every step of every matrix shares the same
 * launches (one dynamic ARA batch per column step for all matrices; sizes,
 * thresholds and options may differ per matrix, except the ARA block width
 * opts.bs, which all matrices of one call share: a call mixing block widths
 * returns TLR_ERR_ARG without factoring any).  Each matrix draws its own
 * Gaussian blocks (its opts.seed), so its result does not depend on the batch.
 * eps[m] and opts[m] (opts may be NULL for defaults) per matrix; status[m]
 * (host) receives each matrix's outcome (TLR_ERR_NOT_SPD leaves it FAILED).
 * Returns TLR_OK unless the call itself failed. */
tlr_status tlr_factor_batch(tlr_ctx* ctx, int count, tlr_mat** A, const double* eps, const tlr_opts* opts,
                            int ldl, tlr_status* status);

/* Continuous batching of factorizations (no counterpart in the paper: the
 * serving loop of a many-request deployment).  A session holds factorizations in
 * flight; tlr_session_step advances every unfinished one by one column, all of
 * them in the same launches (each matrix at its own column index), and matrices
 * may be added between steps.  A matrix added to a session is factored in place
 * (Cholesky if ldl == 0, else LDL^T) exactly as tlr_potrf / tlr_ldlt would: same
 * result bit for bit.  All matrices of a session use one ARA block width. */
typedef struct tlr_session tlr_session;
tlr_status tlr_session_create(tlr_ctx* ctx, tlr_session** s);
tlr_status tlr_session_destroy(tlr_session* s);
/* Queue A (state "A") for factorization; *ticket identifies it in this session. */
tlr_status tlr_session_add(tlr_session* s, tlr_mat* A, double eps, const tlr_opts* opts, int ldl, int* ticket);
/* One column step of every unfinished factorization; *unfinished (may be NULL)
 * receives how many remain. */
tlr_status tlr_session_step(tlr_session* s, int* unfinished);
/* *finished = 1 once the ticket's factorization ended; *result its status. */
tlr_status tlr_session_poll(tlr_session* s, int ticket, int* finished, tlr_status* result);

/* Serving queue (no counterpart in the paper: the request loop of a deployment that evaluates
 * many Gaussian-process likelihoods, the use Section 1 gives for the factorization).  A request
 * is one covariance matrix to build, factor, solve with nrhs right-hand sides and take the log
 * determinant of.  tlr_submit copies the request into the context's queue; tlr_progress does one
 * scheduling step:
 *   1. admission, in submission order: the next queued request is built (tlr_compress) and joins
 *      the factorizations in flight when the context's device bytes plus the request's estimated
 *      footprint fit in tlr_create's hbm_budget (always when nothing is in flight);
 *   2. one column step of every factorization in flight, all of them in the same launches
 *      (tlr_session: a request that joins mid-flight gets the result it would get alone);
 *   3. each finished factorization: on TLR_ERR_NOT_SPD it is rebuilt and refactored once as
 *      A + eps I (Section 5.1, diagonal shift); otherwise it is solved (its right-hand sides copied
 *      in, the solution copied back to the queue's host memory), its logdet taken, and its device
 *      memory released.
 * tlr_poll reports a request; once it is done, the first tlr_poll that sees it copies the solution
 * into x (if x is not NULL) and releases the request (its ticket is then unknown: TLR_ERR_ARG).
 * All requests of a context share one ARA block width (the first request's opts.bs).
 * tlr_progress and tlr_poll synchronize the context stream; they are not thread-safe. */
typedef struct {
  const double* points; /* host, N x d row-major, original point order; copied by tlr_submit */
  int64_t N;
  int d;
  tlr_kernel kernel;
  int b;                /* tile size */
  double eps;           /* absolute tile threshold */
  int ldl;              /* 0: L L^T (Algorithm 6), 1: L D L^T (Algorithm 10) */
  int nrhs;             /* right-hand sides, 0..1024 */
  const double* rhs;    /* host, N x nrhs column-major (leading dimension N), original point order;
                           copied by tlr_submit (may be NULL when nrhs == 0) */
  tlr_opts opts;        /* bs, precision, compensation, seed, max_slots of this request */
} tlr_request;
typedef struct {
  int done;             /* 0: queued or in flight (the fields below are not set yet) */
  tlr_status status;    /* TLR_OK, or the error that ended the request */
  int retried;          /* 1: refactored as A + eps I after a loss of definiteness */
  int sign;             /* sign of det (LDL^T of an indefinite matrix: -1 possible) */
  double logdet;        /* log |det| of the factored matrix */
  double wait_s;        /* host seconds from tlr_submit to admission */
  double run_s;         /* host seconds from admission to the result */
  int64_t bytes;        /* device bytes of the factor while it was resident */
  double mean_rank;     /* mean rank of the factor's off-diagonal tiles */
} tlr_result;
tlr_status tlr_submit(tlr_ctx* ctx, const tlr_request* req, uint64_t* ticket);
/* One scheduling step.  *queued / *in_flight (either may be NULL) receive the requests waiting for
 * admission and those being factored after the step; both 0 means every request is done. */
tlr_status tlr_progress(tlr_ctx* ctx, int* queued, int* in_flight);
/* res->done = 0 while the request runs; x: host N x nrhs, leading dimension ldx >= N, or NULL. */
tlr_status tlr_poll(tlr_ctx* ctx, uint64_t ticket, tlr_result* res, double* x, int64_t ldx);

/* Solve (L L^T) X = B or (L D L^T) X = B with the TLR triangular solve of
 * Algorithm 7 (forward) and its transpose (backward).  B: device, N x nrhs,
 * leading dimension ldb >= N, original point order; overwritten with X.
 * The factor keeps a solve plan per group width (right-hand sides are taken in
 * groups of at most 32; up to 4 widths are kept): two N x width work arrays and
 * the job tables, allocated on the first solve of that width and freed with the
 * factor.  The first solve of a width runs the plan's launches directly; the
 * next captures them once as a CUDA graph, which later solves replay (same
 * kernels, bitwise the same results).  Solves with one factor must not run
 * concurrently (they share the plan's work arrays). */
tlr_status tlr_solve(tlr_ctx* ctx, const tlr_mat* F, int nrhs, double* B, int64_t ldb);

/* Preconditioned conjugate gradients (Section 6: a low-accuracy TLR factor of
 * A + eps I as the CG preconditioner, run until ||A x - b|| / ||b|| <= tol).
 * A: a compressed matrix (state "A", the operator, applied with tlr_matvec);
 * F: a factor of the same N (the preconditioner, applied with tlr_solve, so its
 * solves replay a captured graph after the first).  B: device, N x nrhs,
 * leading dimension ldb >= N, original point order (read only); X: device,
 * N x nrhs, ldx >= N, receives the solutions (started from 0).  Each column
 * runs its own iteration (textbook PCG, Saad Algorithm 9.1) and stops when its
 * updated residual is at most tol ||b|| or after maxit iterations; iters[c]
 * (host) receives its iteration count and relres[c] (host) its true relative
 * residual ||b - A x|| / ||b||.  A zero column gives x = 0 after 0 iterations.
 * Errors: TLR_ERR_ARG (null pointers, nrhs < 0, tol <= 0, maxit < 0, N
 * mismatch or above 2^31 - 1), TLR_ERR_STATE (A not in state "A" or F not
 * factored). */
tlr_status tlr_pcg(tlr_ctx* ctx, const tlr_mat* A, const tlr_mat* F, int nrhs, const double* B, int64_t ldb,
                   double* X, int64_t ldx, double tol, int maxit, int* iters, double* relres);

/* log|det| of the factored matrix: 2 sum log diag(L_kk) (Cholesky) or
 * sum log|D_ii| (LDL^T); *sign = sign of the determinant.  Host outputs. */
tlr_status tlr_logdet(tlr_ctx* ctx, const tlr_mat* F, double* logdet, int* sign);

/* Matrix products with the TLR data (Section 4.4), original point order:
 *   op TLR_OP_A   : Y = A X     (F in state "A": symmetric TLR product)
 *   op TLR_OP_L   : Y = L X     (factor)
 *   op TLR_OP_LT  : Y = L^T X   (factor)
 *   op TLR_OP_LLT : Y = L L^T X or L D L^T X (factor)
 * X, Y: device, N x nrhs, leading dimensions ldx, ldy >= N; X and Y must not overlap. */
enum { TLR_OP_A = 0, TLR_OP_L = 1, TLR_OP_LT = 2, TLR_OP_LLT = 3 };
tlr_status tlr_matvec(tlr_ctx* ctx, const tlr_mat* F, int op, int nrhs, const double* X,
                      int64_t ldx, double* Y, int64_t ldy);

/* Exact kernel-matrix product Y = A X, A generated on the fly from the points
 * (used to measure backward errors and residuals, the way Section 6 checks its
 * factorizations).  Points host row-major N x d in ORIGINAL order; X, Y device
 * N x nrhs (ldx, ldy >= N).  TLR_ERR_ARG for a NULL pointer, N <= 0, d outside
 * 1..3, nrhs < 0, ldx or ldy < N, a kernel type other than TLR_KERNEL_EXP,
 * ell <= 0 or nugget <= -1 (the same rule as tlr_kernel_matvec_noalloc). */
tlr_status tlr_kernel_matvec(tlr_ctx* ctx, const double* points_host, int64_t N, int d,
                             const tlr_kernel* kernel, int nrhs, const double* X, int64_t ldx,
                             double* Y, int64_t ldy);

/* Allocation-free variant of tlr_kernel_matvec.  The paper has no counterpart:
 * this is a library service for callers that cannot allocate device memory
 * (a memory manager owns the whole device heap, cudaMalloc's implicit
 * synchronization is not acceptable, or no tlr_ctx exists).  It computes the
 * same Y = A X; instead of library-allocated device memory it stages the
 * points in a fixed device array compiled into the library (3 MiB, held by
 * every GPU that loads the library until the process exits), so it needs no
 * context and calls no allocator.
 *   cuda_stream: cudaStream_t of the CURRENT device (NULL: legacy default
 *     stream); the call is enqueued on it and returns without synchronizing.
 *   points_host: host, row-major N x d, original order; copied during the call
 *     (if it is page-locked, leave it unchanged until the stream has run the call).
 *     The copy is an asynchronous host-to-device copy on cuda_stream: if that stream is being
 *     captured, the copy becomes a node of the graph and reads points_host again at every
 *     replay, so points_host must then stay valid and unchanged for every replay.
 *   X, Y: device, N x nrhs, column-major, ldx, ldy >= N (caller-owned).
 * Limits and errors: N * d <= 393216 (131072 points in 3D), else TLR_ERR_LIMIT;
 * bad arguments TLR_ERR_ARG; a failing CUDA call TLR_ERR_CUDA.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current): make that first call before any stream
 * capture.  All calls share the array and it keeps the last call's points;
 * calls whose work overlaps on the GPU (other streams, other host threads)
 * race on it and must be serialized by the caller. */
tlr_status tlr_kernel_matvec_noalloc(void* cuda_stream, const double* points_host, int64_t N, int d,
                                     const tlr_kernel* kernel, int nrhs, const double* X,
                                     int64_t ldx, double* Y, int64_t ldy);

typedef struct {
  int64_t N;
  int b, nb, d;
  int state;           /* 0 = A, 1 = Cholesky factor, 2 = LDL^T factor, 3 = FAILED */
  int k_fail;          /* failing tile column for TLR_ERR_NOT_SPD, else -1 */
  int max_rank;        /* over lower off-diagonal tiles */
  double mean_rank;
  int64_t bytes;       /* device bytes of the representation */
  double flops_exec;   /* FP64 flops executed by the last factorization (all phases) */
  double flops_model;  /* paper-model flops: per-tile chains of Equation 2 */
  double ara_rounds;   /* total ARA rounds of the last factorization (all columns) */
  double seconds;      /* host wall time of the last factorization call */
  double flops_fp32;   /* FP32 flops of the sampling/projection chains (TLR_PREC_FP32) */
  double tile_rounds_fp32, tile_rounds_fp64; /* ARA tile-rounds sampled in FP32 / FP64 (TLR_PREC_FP32) */
} tlr_info;
tlr_status tlr_get_info(const tlr_mat* M, tlr_info* info);

/* Ranks of the lower off-diagonal tiles: host int array nb x nb, row-major,
 * entry (i, j) for i > j, zero elsewhere. */
tlr_status tlr_get_ranks(tlr_ctx* ctx, const tlr_mat* M, int* ranks);

/* KD permutation: host int64 array, perm[p] = original index of ordered point p. */
tlr_status tlr_get_perm(const tlr_mat* M, int64_t* perm);

/* Export tiles to host for inspection (KD order, padded, b rows each):
 *   diagonal tile k (i == j): b x b into U (V unused); LDL^T D_k (b) into V if V != NULL;
 *   off-diagonal (i > j): U_ij (b x r) into U and V_ij (b x r) into V, r = rank. */
tlr_status tlr_get_tile(tlr_ctx* ctx, const tlr_mat* M, int i, int j, double* U, double* V);

tlr_status tlr_free(tlr_ctx* ctx, tlr_mat* M);
const char* tlr_strerror(tlr_status s);

/* ---------------- building blocks (each one step of the method) ---------------- */

/* KD-tree ordering of Section 6 (host only): recursive split along the axis of
 * largest bounding-box extent (ties: lowest axis), points sorted by (coordinate,
 * index), left part b * 2^(ceil(log2(n/b)) - 1) points.  perm[p] = original
 * index of ordered point p.  points: host row-major N x d. */
tlr_status tlr_kd_order(const double* points, int64_t N, int d, int b, int64_t* perm);

/* Gaussian block Omega (b x bs, column-major, device) for (seed, stream,
 * column k, round t): Philox4x32-10 (Salmon et al., SC'11) counters
 * (pair index, t, k, stream), key (seed lo, seed hi), Box-Muller pairs. */
tlr_status tlr_omega(tlr_ctx* ctx, uint64_t seed, uint32_t stream, uint32_t k, uint32_t t,
                     int b, int bs, double* out);

/* Batched ARA (Algorithm 1) on explicit dense n x n operands: T[s] at
 * T + s*n*n (device, column-major).  Gaussian blocks (seed, stream, k, t) are
 * shared by all operands of a round.  Outputs per operand s: Q[s] and B[s]
 * (device, n x n capacity each, column-major, first rank[s] columns used,
 * T[s] ~= Q B^T) and rank[s] (device int).  eps: absolute 2-norm threshold. */
tlr_status tlr_ara_dense(tlr_ctx* ctx, int nops, int n, const double* T, int bs, double eps,
                         uint64_t seed, uint32_t stream, uint32_t k, double* Q, double* B,
                         int* rank);

/* ARA -> SVD rank trimming (Section 6: the post-processing step that applies the SVD to each low-rank
 * tile to bring its rank down to the minimum) of `ntiles` tiles Q_t B_t^T of one shape: Q and B device,
 * ntiles blocks of b x r column-major (leading dimension b, block t at t * b * r), Q_t with orthonormal
 * columns.  B_t = W S Z^T (Householder QR of B_t, then one-sided Jacobi SVD of its triangular factor);
 * the r'_t singular values above eps are kept, in descending order: Qout_t = Q_t Z_r, Bout_t = B_t Z_r
 * (= W_r S_r), columns r'_t .. r - 1 zero; rank (host, ntiles) receives r'_t.  The tile's error is its
 * first dropped singular value (<= eps).  Errors: TLR_ERR_ARG (null pointers, b < 1, r outside 0..b,
 * eps <= 0), TLR_ERR_LIMIT (b above ~11000: the CTA's shared memory). */
tlr_status tlr_trim_tiles(tlr_ctx* ctx, int ntiles, int b, int r, const double* Q, const double* B, double eps,
                          double* Qout, double* Bout, int* rank);

/* Dense FP64 Cholesky (lower, in place) of an n x n device matrix (lda >= n);
 * *info (host) = -1 on success, else the first failing column. */
tlr_status tlr_dense_potrf(tlr_ctx* ctx, int n, double* A, int lda, int* info);
/* Modified Cholesky (Algorithm 8, Section 5.1.2) of a symmetric n x n device matrix (lower triangle
 * read, lda >= n, n <= 2048): if A is positive definite, its Cholesky factor (*modified = 0);
 * otherwise (*modified = 1) the Cholesky factor of A + E = P L (D + F) L^T P^T, where P^T A P = L D L^T
 * is the symmetric factorization with the 1x1 / 2x2 pivoting of Bunch and Kaufman (1977) and F raises
 * each pivot block's eigenvalues to at least sqrt(u / 2) ||A||_inf (Cheng and Higham, 1998).  In
 * place: L in the lower triangle; after a modification the strict upper triangle holds A + E.
 * *info (host) = -1, or the failing column should A + E itself not factor. */
tlr_status tlr_dense_modchol(tlr_ctx* ctx, int n, double* A, int lda, int* modified, int* info);
/* Dense unpivoted LDL^T (in place: unit L below the diagonal, D on it). */
tlr_status tlr_dense_ldlt(tlr_ctx* ctx, int n, double* A, int lda, int* info);
/* X = L^{-1} B in place (L lower n x n, unit diagonal if unit != 0), B n x nrhs. */
tlr_status tlr_dense_trsm(tlr_ctx* ctx, int n, const double* L, int lda, int unit, int nrhs,
                          double* B, int ldb);

/* C = T X (trans = 0; trans = 2: the same product through the kernel that reads T by columns,
 * as the factorization reads its panels) or C = T^T X (trans = 1) for one dense n x n FP64 tile T (column-major,
 * leading dimension n) and X n x ncols (leading dimension ldx), C n x ncols (ldc): the
 * construction's ARA products (Algorithm 1 samples and projections of Section 6's tiles),
 * computed on the 16-bit tensor cores (tcgen05) by exact splitting into 7-bit chunks (Ozaki et
 * al., 2012) with an error of the order of an FP64 product.  n must be a positive multiple of 16
 * (TLR_ERR_LIMIT otherwise); all pointers are device memory owned by the caller; the call
 * returns after the product is complete. */
tlr_status tlr_split_product(tlr_ctx* ctx, int trans, int n, int ncols, const double* T, const double* X,
                             int ldx, double* C, int ldc);

/* Measurement utility (not part of the method): what the split products used since the last
 * reset.  counts[s] (s = 1..8; counts[0] unused) = output blocks (128 x 16 x one K slice)
 * computed with s 7-bit planes (8: FP64-exact; fewer: TLR_PREC_MIXED truncation); *bytes = int8
 * chunk bytes of the operands read, each operand block counted once.  Synchronizes the context
 * stream; reset != 0 zeroes the counters.  counts (9 entries) or bytes may be NULL. */
tlr_status tlr_split_planes(tlr_ctx* ctx, int64_t* counts, double* bytes, int reset);

/* Measurement utility (not part of the method): FP64 DFMA throughput of this
 * GPU in TFLOP/s, from a register-resident FMA loop timed with CUDA events. */
tlr_status tlr_fp64_peak(tlr_ctx* ctx, double* tflops);

/* Number of kernels this library launched on the context since creation. */
int64_t tlr_launch_count(const tlr_ctx* ctx);

/* Measurement utility (not part of the method): per-launch CUDA-event accounting of the
 * batched products, by family: 0-2 FP64 k_gemm NN / TN / NT, 3-5 FP32 k_gemm NN / TN / NT,
 * 6 the tensor-core split products (FP64-equivalent flops), 7 the fused orthogonalization rounds
 * (k_orth_round: 8 n q bs + 6 n bs^2 flops per slot).  Copies the accumulated
 * milliseconds, algorithmic flops (2 M N K per job, half for a triangular operand), algorithmic
 * bytes (split products only: slices read once, C written) and launch counts since the last call
 * (any pointer may be NULL; arrays of TLR_GEMM_FAMILIES), resets them, and turns the
 * accounting on (enable != 0) or off. */
#define TLR_GEMM_FAMILIES 8
tlr_status tlr_gemm_stats(tlr_ctx* ctx, int enable, double* ms, double* flops, double* bytes, int64_t* launches);

/* Measurement utility (not part of the method): phase profiler in the spirit
 * of the paper's phase breakdown (Section 6.1, Figure 8a).  Stream time between
 * consecutive phase boundaries (CUDA events) is charged to the earlier phase.
 * Copies the accumulated milliseconds and kernel launches of the n first phases
 * (order: gram, diag-update, potrf, sample, orthog, host-sync, project, trsm,
 * update-tiles, compress, solve, other; with n >= 13, ms[12] = host time blocked
 * in stream synchronizations) into ms / launches (either may be NULL),
 * resets them, and turns profiling on (enable != 0) or off. */
tlr_status tlr_profile(tlr_ctx* ctx, int enable, double* ms, int64_t* launches, int n);

#ifdef __cplusplus
}
#endif
#endif /* TLR_GB300_H */
