/*
 * snmf.h -- C ABI of the GB300 library for symmetric nonnegative matrix
 * factorization by the nonmonotone projected Barzilai-Borwein method (SNMPBB)
 * of Swart and Brust, "A Nonmonotone Gradient-Based Algorithm for Symmetric
 * Nonnegative Matrix Factorization and Graph Clustering".
 *
 * Problem (Sec. 1.2, Eq. (2)):    min_{W >= 0} || A - W W^T ||_F^2,  A symmetric n x n.
 * Penalty form (Sec. 2.1, Eq. (3)): f(W,H) = 1/2 ||A - W H||^2 + lambda/2 ||W - H^T||^2,
 *   solved by alternating Algorithm 1 (NMPBB) over W and H; Graph-SNMPBB (Sec. 2.2,
 *   Eq. (5)) adds gamma/2 tr(H L H^T); LAI-SNMPBB (Sec. 2.3, Eq. (8)) replaces A by a
 *   randomized eigen-sketch U E U^T.
 *
 * Conventions shared by every entry point
 *   - Matrices are row-major.  The factors W and Ht (= H^T) are n x (r * batch):
 *     restart j occupies columns [j r, (j+1) r).
 *   - Element type of W and Ht: double in SNMF_F64 precision, float otherwise.
 *   - Pointers marked "device" must be CUDA device (or managed) memory of the
 *     current device; "host" pointers are ordinary host memory.
 *   - The library never takes ownership of caller memory.  A is borrowed (must
 *     outlive the handle) when it lives on the device and its dtype equals the
 *     working precision; otherwise snmf_create makes an owned device copy.
 *   - All device work is issued on the CUDA stream given to snmf_create (NULL =
 *     legacy default stream).  Calls are synchronous with respect to the host on
 *     return.  A handle is not thread-safe.
 *   - No exceptions cross the ABI.  Every call returns an snmf_status; on error a
 *     message is available from snmf_last_error(handle).  Invalid arguments are
 *     rejected with SNMF_ERR_ARG before any kernel is launched.
 *   - There is no CPU fallback: a call that needs the GPU fails with
 *     SNMF_ERR_CUDA when no usable device is present.
 */
#ifndef SNMF_H
#define SNMF_H

#include <stdint.h>

#if defined(__GNUC__)
#define SNMF_API __attribute__((visibility("default")))
#else
#define SNMF_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct snmf_ctx* snmf_handle;

typedef enum {
  SNMF_OK = 0,
  SNMF_NOT_CONVERGED = 1,   /* max_iter reached before the tolerance */
  SNMF_ERR_ARG = -1,        /* invalid argument, rejected before any launch */
  SNMF_ERR_CUDA = -2,       /* CUDA runtime error or no device */
  SNMF_ERR_OOM = -3,        /* device allocation failed */
  SNMF_ERR_NUMERIC = -4,    /* NaN/Inf met in the FP64 scalar state */
  SNMF_ERR_TIMEOUT = -5,    /* a bounded device wait ran out */
  SNMF_ERR_STATE = -6       /* call out of order (e.g. solve on a destroyed handle) */
} snmf_status;

/* matrix kinds */
enum { SNMF_DENSE = 0, SNMF_CSR = 1, SNMF_DENSE_BATCH = 2 };
/* element types (matrix dtype) and working precisions */
enum { SNMF_F64 = 0, SNMF_F32 = 1, SNMF_BF16 = 2, SNMF_FP8 = 3 };
/* where a matrix passed to snmf_create lives */
enum { SNMF_ON_DEVICE = 0, SNMF_ON_HOST = 1 };
/* formulations: the penalty form (Sec. 2.1, Eq. (3)), the single-variable objective (Eq. (2)),
   and the naive symmetric use of Algorithm 1 that Sec. 2.1 describes before the penalty form
   (the W block with H = W^T held fixed and lambda = 0, then H <- W^T; the paper reports that it
   performs poorly, which the rank-one case shows: the block solve w <- A w / ||w||^2 alternates
   between two norms) */
enum { SNMF_PENALTY = 0, SNMF_DIRECT = 1, SNMF_NAIVE = 2 };
/* BB step variants */
enum { SNMF_BB1 = 0, SNMF_BB2 = 1 };

/*
 * Symmetric input matrix A (Sec. 1.2: V in the paper).
 *   dense: values is n x n row-major with leading dimension ld >= n (elements).
 *   CSR:   rowptr[n+1], colidx[nnz] (int32, each row's columns in [0, n)),
 *          values[nnz]; both triangles stored.
 * dtype is SNMF_F64 or SNMF_F32.  location says whether the three arrays are
 * device or host memory.
 *   dense batch (SNMF_DENSE_BATCH): nprob independent problems solved together
 *          (uneven batch; no counterpart in the paper, which solves one problem at a
 *          time).  batch_desc (host) holds 3 int64 per problem p: n_p, r_p and the element
 *          offset of A_p in values; A_p is n_p x n_p row-major with leading dimension n_p.
 *          Requires 1 <= r_p <= min(n_p, 64), penalty form, batch == 1, precision F64
 *          (with F64 values), F32 or BF16.  The factors W, Ht of snmf_solve are the
 *          problems' n_p x r_p row-major blocks packed back to back in problem order
 *          (offset of problem p = sum over q < p of n_q r_q elements); the r argument of
 *          snmf_create is ignored; n, ld, nnz, rowptr, colidx are unused.
 */
typedef struct {
  int32_t kind;
  int32_t dtype;
  int32_t location;
  int32_t reserved;
  int64_t n;
  int64_t nnz;
  int64_t ld;
  const void* values;
  const int32_t* rowptr;
  const int32_t* colidx;
  int32_t nprob;               /* SNMF_DENSE_BATCH: number of problems                 */
  int32_t reserved2;
  const int64_t* batch_desc;   /* SNMF_DENSE_BATCH: host, 3 * nprob entries (see above) */
} snmf_matrix;

/*
 * Solver options.  snmf_default_options fills the documented defaults.
 */
typedef struct {
  int32_t formulation;     /* SNMF_PENALTY (Sec. 2.1, default) | SNMF_DIRECT (Eq. (2)) |
                              SNMF_NAIVE (Sec. 2.1: W block with H = W^T, then H <- W^T; no
                              lambda, no graph term, plain BB step; Ht in/out is W)         */
  int32_t precision;       /* SNMF_F64 | SNMF_F32 (default) | SNMF_BF16 | SNMF_FP8: storage of A
                              for the A*X products; accumulation is FP32 (FP64 in SNMF_F64) and
                              objective, line search and BB inner products are FP64 throughout.
                              SNMF_FP8 (dense only): E4M3 codes of A / s_t with a power-of-two
                              scale s_t per 128 x 128 tile (the smallest 2^k with
                              max|A_t| / 2^k <= 448), round to nearest even, saturating; the
                              iteration's products decode the codes to BF16 (exactly) and run
                              on the tensor cores like SNMF_BF16 (X as BF16 hi + lo parts),
                              the final evaluation on CUDA cores with FP32 X               */
  int32_t batch;           /* b random restarts sharing A (columns r*b), default 1            */
  int32_t nonmonotone_M;   /* 0: eta averaging of Alg. 1 line 4; M > 0: max of the last M
                              objective values (M <= 64).  Default 10                          */
  int32_t bb_variant;      /* SNMF_BB1 <S,S>/<S,Y> (Alg. 1 line 3, default) | SNMF_BB2        */
  int32_t max_ls;          /* line-search trials per step, default 20 (Sec. 4.1 (5))           */
  int32_t inner_iters;     /* Algorithm 1 steps per block (penalty), default 5                */
  int32_t max_iter;        /* outer iterations (penalty) or steps (direct), default 500        */
  int32_t power_iters;     /* power iterations for rho = ||G||_2 (Eq. (2.11)), default 50      */
  int32_t step_controller; /* 0: plain BB step (Alg. 1 line 3).  1: learned step multiplier m =
                              2^(2 tanh o) on the BB step from the MLP o = W2 relu(W1 phi + b1) + b2
                              (weights in mlp_weights, used in BF16); the proposal is kept only if
                              the nonmonotone Armijo test accepts it at beta = 1, otherwise the
                              step falls back to the plain BB direction with ordinary backtracking.
                              3: lean learned step: the proposal replaces the BB step and is
                              backtracked like it (one direction per step instead of two; the
                              convergence safeguards are the clamp to [alpha_min, alpha_max] and
                              the unchanged nonmonotone acceptance test).
                              2: record mode: the plain BB trajectory, and at every step the
                              features phi and the best of 9 multipliers 2^(-2..2 by 1/2) are
                              recorded (snmf_controller_data).
                              4: rollout branch (training data for labels scored by a short
                              rollout): batch must be a multiple of 9; restart j belongs to group
                              j / 9 and takes candidate c = j % 9.  Every restart follows the
                              plain BB step, except at the inner step whose index is branch_step
                              (counted over the whole solve: outer iteration t, block h (0 W,
                              1 H), step k of the block -> 2 t inner_iters + h inner_iters + k),
                              where its next step is 2^((c - 4) / 2) times the BB step.  At
                              that step the restart with c = 4 records its features phi, with
                              the group index as the target, for snmf_controller_data.  Give
                              the restarts of a group the same start: they then agree up to the
                              branch, and the factors at the end of the solve score the nine
                              multipliers.  1, 2, 3 and 4 need the penalty form and r <= 64.
                              Features phi: ln(BB1 rho), ln(BB2 rho), ratio of successive
                              projected-gradient norms, ratio of successive objective decreases,
                              fraction of zero entries.                                        */
  double lambda_sym;       /* penalty weight lambda (Eq. (3)); < 0 -> 0.01 ||A||_F (Sec. 4.1 (1)) */
  double theta;            /* Armijo parameter, default 1e-3 (Sec. 2.4)                        */
  double phi;              /* relaxation factor, default 1.7 (Sec. 2.4)                        */
  double eta;              /* averaging weight for nonmonotone_M == 0, default 0.85            */
  double alpha_min;        /* BB clamp, default 1e-10                                          */
  double alpha_max;        /* BB clamp, default 1e10                                           */
  double beta_shrink;      /* backtracking factor, default 0.5                                 */
  double tol;              /* relative projected-gradient tolerance, default 1e-4              */
  double direct_rho_factor;/* direct form: rho_k = factor ||W^T W||_2, default 3               */
  double init_scale;       /* W == NULL init: U[0,1] * init_scale * sqrt(mean(A)/r), default 2
                              (Sec. 4.1 (4))                                                   */
  uint64_t seed;           /* Philox seed of the default initialisation                         */
  const float* mlp_weights;/* host, SNMF_MLP_NPARAMS floats: W1[64][5], b1[64], W2[64], b2 (copied) */
  int64_t timeout_cycles;  /* bound on device-side waits (clock64 cycles), 0 = default (2e9);
                              see snmf_set_timeout                                             */
  int32_t autotune;        /* 1: at snmf_create, time the candidate launch configurations of
                              the dense A*X product (split-K count; tcgen05 ring depth and CTAs
                              per SM) on this device and shape and keep the fastest; 0 (default):
                              built-in heuristics.  No counterpart in the paper.               */
  int32_t x_parts;         /* SNMF_BF16 tensor-core product: X enters as 2 BF16 parts hi + lo
                              (0 or 2, default: the product sees X to about 2^-17) or as 1 part,
                              X rounded to BF16 (one MMA pass, half the tensor work); the stored A
                              is BF16 either way.  No counterpart in the paper.                */
  const char* tune_cache;  /* JSON file of tuned configurations keyed by device name and SM
                              count (read before timing, updated after); NULL: this process only */
  int32_t sym_half;        /* SNMF_BF16 dense A: 1 = keep only the 128 x 128 tiles of A on and
                              above the diagonal (A is symmetric, Sec. 1.2; the lower triangle
                              is not read): about half the bytes of A in HBM and per product.
                              The tensor-core product reads a tile below the diagonal as the
                              transpose of its stored mirror.  Default 0.  No counterpart in
                              the paper.                                                       */
  int32_t branch_step;     /* step_controller 4: index of the inner step that takes the nine
                              multipliers (see step_controller); < 0: none.  Default -1.       */
} snmf_options;

/* Per-solve statistics (best restart = lowest objective). */
typedef struct {
  int32_t iters;           /* outer iterations (penalty) / steps (direct) performed          */
  int32_t converged;       /* 1 when every restart met the tolerance                          */
  int32_t ls_fail;         /* line searches with no accepted trial (beta set to 0)           */
  int32_t clipped_steps;   /* direct: steps whose relaxed update had clipped entries          */
  int32_t best_restart;
  int32_t ax_products;     /* A*X products issued (dense GEMM / SpMM / LAI pair)             */
  double f;                /* objective of the best restart at the returned point            */
  double residual;         /* ||A - W Ht^T||_F / ||A||_F (direct: Ht = W), FP64               */
  double pg_rel;           /* relative projected gradient of the best restart                 */
  double seconds;          /* device time of the solve (CUDA events)                          */
  int64_t kernel_launches; /* library kernels executed by the solve                          */
  int32_t graph_replays;   /* replays of the captured iteration                              */
  int32_t ctl_proposals;   /* learned controller: proposals made                             */
  int32_t ctl_accepted;    /* learned controller: proposals accepted at beta = 1             */
  int32_t reserved;
} snmf_stats;

#define SNMF_MLP_IN 5
#define SNMF_MLP_HIDDEN 64
#define SNMF_MLP_NPARAMS (SNMF_MLP_IN * SNMF_MLP_HIDDEN + SNMF_MLP_HIDDEN + SNMF_MLP_HIDDEN + 1)

/* Fill *opt with the defaults listed above.  Never fails. */
SNMF_API void snmf_default_options(snmf_options* opt);

/*
 * Create a solver for the symmetric matrix *A and rank r (Sec. 1.2).
 *   h      out: new handle (NULL on failure)
 *   A      input matrix; dense (any precision) or CSR (SNMF_F32/SNMF_F64 precision)
 *   r      rank, 1 <= r <= min(n, 256)
 *   opt    options or NULL for the defaults; copied
 *   stream cudaStream_t (as void*) for all device work of this handle
 * Errors: SNMF_ERR_ARG for r out of range, batch < 1, r*batch > 4096, non-square or
 * negative sizes, ld < n, CSR with nnz mismatch, unknown enum values; SNMF_ERR_OOM,
 * SNMF_ERR_CUDA.  ||A||_F^2 of the stored (possibly quantized) A is computed here.
 */
SNMF_API snmf_status snmf_create(snmf_handle* h, const snmf_matrix* A, int r,
                        const snmf_options* opt, void* stream);

/*
 * Graph-SNMPBB (Sec. 2.2, Eq. (5)): add gamma/2 tr(H L H^T) to the objective.
 *   L      an explicit symmetric n x n CSR matrix (SNMF_F32 or SNMF_F64 values,
 *          device or host), copied into library memory.
 *   gamma  >= 0; 0 removes the term.
 * Penalty form: the term enters the H block only (Sec. 2.2); direct form:
 * gamma/2 tr(W^T L W).  ||L||_2 is estimated here (power_iters power iterations from
 * s_i = 1 + (i mod 2), Rayleigh quotient) and gamma ||L||_2 is added to rho of the
 * regularised block, the Lipschitz constant of its gradient (rho_0 of Sec. 2.4 extended by
 * the graph term).  L == NULL is not available in this build (SNMF_ERR_ARG).
 * Errors: SNMF_ERR_ARG (size mismatch, gamma < 0, dense L).
 */
SNMF_API snmf_status snmf_set_graph_reg(snmf_handle h, const snmf_matrix* L, double gamma);

/*
 * LAI-SNMPBB (Sec. 2.3, Eq. (8)): build the randomized eigen-sketch A ~ U E U^T and
 * use it for every later A*X product of this handle.
 *   k           kept eigenpairs (largest |eigenvalue|), 1 <= k
 *   oversample  extra sketch columns p; l = k + p <= min(n, 128)
 *   power_iters subspace iterations Q <- orth(A Q) before Q^T A Q is formed
 *   seed        Philox seed of the Gaussian sketch matrix
 * ||A||^2 in the objective becomes sum(E^2).  Errors: SNMF_ERR_ARG.
 */
SNMF_API snmf_status snmf_lai_sketch(snmf_handle h, int k, int oversample, int power_iters,
                            uint64_t seed);

/*
 * SVD start (Sec. 4.1 guideline (4), recommended there for graph problems): with A ~ U E P^T
 * from the r largest singular triplets, W_0 = |U E^1/2| and H_0 = |E^1/2 P^T|.  For symmetric A
 * the singular triplets are the eigenpairs of largest |lambda| (P = U sign(lambda)), so both
 * are |U| |lambda|^1/2.  The library takes them from the same randomized eigen-sketch as
 * snmf_lai_sketch (Gaussian test matrix from Philox `seed`, l = r + oversample columns,
 * power_iters subspace iterations, CholeskyQR, Jacobi eigensolver), of A itself.
 *   W   device, n x (r batch), out: the start in every restart's columns
 *   Ht  device, n x (r batch), out (may be NULL): the same values (H_0^T = W_0)
 * Pass W and Ht to snmf_solve as the start.  Errors: SNMF_ERR_ARG (r + oversample > min(n, 128),
 * negative counts), SNMF_ERR_STATE (dense batch handle), SNMF_ERR_OOM, SNMF_ERR_CUDA.
 */
SNMF_API snmf_status snmf_svd_init(snmf_handle h, void* W, void* Ht, int oversample, int power_iters,
                                   uint64_t seed);

/*
 * Run the solver (Algorithm 1 per block, Sec. 2) from the given start.
 *   W   device, n x (r*batch), in/out.  NULL: the default initialisation
 *       init_scale * sqrt(mean(A)/r) * U[0,1] (Philox, opt.seed) is used and the
 *       result is kept inside the handle (read it with snmf_get_factors).
 *   Ht  device, n x (r*batch), in/out, penalty form only; NULL: Ht_0 = W_0 (Sec. 4.1 (4)).
 *   out optional statistics.
 * Returns SNMF_OK when every restart met the tolerance, SNMF_NOT_CONVERGED when
 * max_iter was reached first, or an error.
 * Dense batch handles: W and Ht are the packed per-problem blocks (total sum n_p r_p
 * elements); W == NULL initialises problem p with Philox seed opt.seed + p.  In *out,
 * iters is the maximum over problems, f the sum, residual and pg_rel the maxima, and
 * converged says whether every problem met the tolerance.
 */
SNMF_API snmf_status snmf_solve(snmf_handle h, void* W, void* Ht, snmf_stats* out);

/*
 * As snmf_solve, with W and Ht in HOST memory (same shapes and element types):
 * the start is copied to the device and the result back, inside the call.
 * W must not be NULL; Ht may be NULL (Ht_0 = W_0, result not returned).
 */
SNMF_API snmf_status snmf_solve_host(snmf_handle h, void* W, void* Ht, snmf_stats* out);

/*
 * Per-restart results of the last solve (host arrays of length batch; any may be NULL):
 * objective, relative residual, relative projected gradient, iterations.  Dense batch
 * handles: one entry per problem (length nprob), in problem order.
 */
SNMF_API snmf_status snmf_restart_stats(snmf_handle h, double* f, double* residual,
                               double* pg_rel, int32_t* iters);

/* Copy the factors held inside the handle (after a solve with W == NULL) to device
 * buffers W / Ht (n x r*batch; either may be NULL). */
SNMF_API snmf_status snmf_get_factors(snmf_handle h, void* W, void* Ht);

/*
 * Single product through the library's A*X kernels: Y = A X (X, Y device,
 * n x cols of the handle's factor element type, cols <= r*batch).  Also returns
 * <X, A X> in *xax (host, may be NULL).  Uses the LAI sketch when one is set.
 */
SNMF_API snmf_status snmf_apply(snmf_handle h, const void* X, void* Y, int cols, double* xax);

/*
 * Checkpoint and exact restart (no counterpart in the paper).  snmf_get_state copies the
 * per-restart scalar state of the last solve (iteration count, projected gradient at the start
 * pg0, last H-block projected gradient, counters, and the rest of the FP64 control record) into
 * `blob` (host) with a version header; blob == NULL only reports the size in *size.
 * snmf_set_state imports such a blob (same n, r, batch and formulation, same library version)
 * for the next snmf_solve, which then continues from it: give that solve the factors the
 * earlier solve returned (W, Ht in/out as usual); its iteration count continues and max_iter
 * bounds the total.  In the penalty and naive forms every block restarts its BB memory and
 * nonmonotone reference, so a solve of k outer iterations, exported, and a resumed solve of m more
 * reproduce a solve of k + m iterations bit for bit.  Restarts that had met the tolerance stay
 * stopped.  set_state(h, NULL, 0) drops an imported state.
 * Errors: SNMF_ERR_ARG (buffer too small, foreign or mismatched blob), SNMF_ERR_STATE (no solve
 * yet, dense batch handle).
 */
SNMF_API snmf_status snmf_get_state(snmf_handle h, void* blob, int64_t capacity, int64_t* size);
SNMF_API snmf_status snmf_set_state(snmf_handle h, const void* blob, int64_t size);

/*
 * Per-iteration statistics of the last solve (no counterpart in the paper): the device keeps a
 * ring of the last 256 outer iterations per restart (penalty and naive forms; written by the
 * control step at the start of every W block).  Copies, per restart j, up to `capacity`
 * records out[j][t][8] = {outer iteration, ||P grad|| / ||P grad_0||, ||P grad||, last alpha,
 * last beta, line searches without an accepted trial (cumulative), learned-step proposals
 * accepted (cumulative), 1 while the restart goes on and 0 on the record where it stopped (the
 * tolerance or the iteration limit was met, or the gradient was not finite)}, oldest first;
 * unused records are -1.  *count: records
 * per restart written.  The ring is not cleared between solves.
 */
SNMF_API snmf_status snmf_stats_ring(snmf_handle h, double* out, int capacity, int32_t* count);
#define SNMF_RING_VALUES 8

/*
 * Measurement utility (no counterpart in the paper): time `iters` back-to-back
 * A*X products of the handle's factor shape (n x r*batch) on the handle's stream
 * with CUDA events.  *ms_product: mean time of the whole product (kernel and
 * epilogue); *ms_kernel: mean time of the product kernel alone (0 for LAI).
 * Either pointer may be NULL.  Overwrites internal work buffers only.  On a dense batch
 * handle both report one grouped product A_p X_p over every problem (X = the current W).
 */
SNMF_API snmf_status snmf_profile_ax(snmf_handle h, int iters, double* ms_product,
                                     double* ms_kernel);

/*
 * Measurement utility (no counterpart in the paper): mean time (ms, CUDA events on the
 * handle's stream) of one launch of the D-step kernel (Z step, gradient at Z, D direction,
 * fused line search; Alg. 1 lines 2-4) and of the update kernel (relaxed update, gradient,
 * BB inner products) of a W block, each launched `iters` times on the buffers of the last
 * solve with every restart marked live.  Penalty form without graph term, r <= 64.  It
 * overwrites the handle's work buffers and the factors held in it (snmf_restart_stats keeps
 * the solve's results); SNMF_ERR_STATE before a solve.
 */
SNMF_API snmf_status snmf_profile_steps(snmf_handle h, int iters, double* ms_dstep, double* ms_update);

/*
 * Measurement utility (no counterpart in the paper): which row-kernel body runs the D step and
 * the update of this handle's penalty blocks, and their algorithmic bytes per launch (every
 * n x (r batch) array a launch reads or writes, once).  *body: 0 the general row kernel
 * (Z and D stored; D step 6 arrays, 7 with the learned step's second direction, update 8),
 * 1 the shared-memory tile body (same traffic), 2 the recomputing kernels (Z and D not stored:
 * D step 4 arrays, update 6), 3 the recomputing kernels with their row products on the tensor
 * cores (tcgen05 TF32 with hi / lo operand parts; r = 64, chosen by the autotuner when faster),
 * 4 the same arithmetic as persistent kernels (one CTA per SM over 128-row tiles, inputs streamed
 * by TMA into shared slots while the previous tile computes; same traffic as 2 and 3).
 * *rows_per_cta: rows of one tile.  Any pointer may be NULL.
 */
SNMF_API snmf_status snmf_step_config(snmf_handle h, int32_t* body, int32_t* rows_per_cta, int64_t* dstep_bytes,
                                      int64_t* update_bytes);

/*
 * The product configuration chosen by the autotuner (no counterpart in the paper):
 * split-K slices, tcgen05 ring stages and CTAs per SM (0 where the kernel has none), the
 * measured mean time in ms, and *from_cache = 1 when it came from the cache file or an
 * earlier handle of this process.  SNMF_ERR_STATE when the handle was not tuned.
 */
SNMF_API snmf_status snmf_tuned_config(snmf_handle h, int32_t* splits, int32_t* stages, int32_t* per_sm,
                                       double* ms, int32_t* from_cache);

/*
 * The tile shapes chosen by the same autotuner: *bn = columns of X per tensor-core product
 * tile (0 where the product kernel has no such choice) and *row_bm = rows per CTA of the row
 * kernels of a step (FP32 penalty form: the recomputing kernels' 64 / 128 (r = 16: 128 / 256)
 * where snmf_step_config reports body 2, else the general kernel's 32 / 64; 0 where the
 * shared-memory tile body with its fixed height runs).  SNMF_ERR_STATE when the handle was not
 * tuned.
 */
SNMF_API snmf_status snmf_tuned_tiles(snmf_handle h, int32_t* bn, int32_t* row_bm);

/*
 * Allocation-free dense product (the paper has no counterpart; this is a service of
 * the library).  Y = A X and <X, A X> for a dense FP32 or FP64 A, computed with the
 * same kernels as snmf_apply, for callers that must not allocate device memory after
 * start-up: programs that size and reserve every buffer once (cudaMalloc and cudaFree
 * can synchronize the device and stall other streams), programs whose device memory
 * is owned by another allocator such as a framework's caching pool, and programs
 * running at the device-memory limit.  It makes no handle and calls no cudaMalloc,
 * cudaFree or other allocating routine, on the device or on the host.
 *   A      device, n x n row-major, leading dimension lda >= n, element type dtype
 *   dtype  SNMF_F32 or SNMF_F64 (A, X and Y share it)
 *   X, Y   device, n x cols row-major (leading dimension cols); Y is overwritten
 *   xax    host, receives <X, A X> (may be NULL)
 *   stream cudaStream_t as void*; the call returns after the stream has finished it
 * Scratch: the split-K slices and FP64 partial sums live in one file-scope device
 * array of SNMF_NOALLOC_SCRATCH_BYTES that every GPU loading the library keeps until
 * the process exits: the first SNMF_NOALLOC_PARTIAL_BYTES hold the partial sums (one
 * 256-byte record per 64-row slice of A, plus the reduced scalar), the rest the split-K
 * slices.  It is shared by all calls and keeps the last call's contents (every word a
 * call reads was written by that call, so nothing needs clearing); calls that overlap
 * on the GPU race on it, so issue them one at a time.
 * Set-up: the array's device address is resolved with cudaGetSymbolAddress on the
 * first call made in a CUDA context (the current device's context at the time of the
 * call) and cached per context; a new context (after cudaDeviceReset, or a driver-API
 * caller's own context) is resolved again on its first call.  Make that first call
 * before any stream capture.
 * Limits: n <= SNMF_NOALLOC_MAX_ROWS and 2 * n * cols * sizeof(element) <=
 * SNMF_NOALLOC_MAX_SLICE_PAIR_BYTES; larger sizes, NULL pointers, lda < n or another
 * dtype return SNMF_ERR_ARG before any CUDA call.  CUDA failures return SNMF_ERR_CUDA.
 */
#define SNMF_NOALLOC_SCRATCH_BYTES (64ull << 20)
#define SNMF_NOALLOC_PARTIAL_BYTES (4ull << 20)
#define SNMF_NOALLOC_MAX_SLICE_PAIR_BYTES (SNMF_NOALLOC_SCRATCH_BYTES - SNMF_NOALLOC_PARTIAL_BYTES)
/* 64 rows per partial record of 256 bytes; 256 bytes stay free for the reduced scalar */
#define SNMF_NOALLOC_MAX_ROWS (64ll * (int64_t)((SNMF_NOALLOC_PARTIAL_BYTES - 256) / 256))
SNMF_API snmf_status snmf_apply_dense_noalloc(const void* A, int dtype, int64_t n, int64_t lda,
                                              const void* X, void* Y, int cols, double* xax,
                                              void* stream);

/*
 * Record-mode data (step_controller == 2 or 4; not in the paper: training data of the learned
 * step controller).  Copies up to `capacity` recorded samples (features feat[i][5] and target
 * log2 multipliers targ[i] in mode 2, the restart group j / 9 in mode 4; host arrays) gathered
 * since the last call, then clears the record.
 * *count receives the number copied.  SNMF_ERR_STATE when the handle is not in record mode.
 */
SNMF_API snmf_status snmf_controller_data(snmf_handle h, float* feat, float* targ, int capacity,
                                          int32_t* count);

/*
 * Train the step controller's MLP on the GPU (not in the paper).  Loss: mean over samples
 * of (2 tanh(o) - t)^2, o = W2 relu(W1 phi + b1) + b2; full-batch Adam (beta1 0.9, beta2
 * 0.999) for `steps` steps with learning rate lr, FP32.
 *   feats[count][5], targets[count]: host arrays; weights: host, SNMF_MLP_NPARAMS floats, in
 *   (initial) / out (trained); loss_out: final loss (may be NULL); grad0: gradient of the loss
 *   at the initial weights (host, SNMF_MLP_NPARAMS floats, may be NULL).
 * Uses the current CUDA device and the legacy default stream; allocates device memory.
 */
SNMF_API snmf_status snmf_mlp_train(const float* feats, const float* targets, int count, float* weights,
                                    int steps, double lr, double* loss_out, float* grad0);

/*
 * Evaluate the step controller's network as the solver does (not in the paper): for each
 * of `count` feature vectors feats[i][5] (host) the multiplier m = 2^(2 tanh o),
 * o = W2 relu(W1 phi + b1) + b2, with the weights rounded to BF16 exactly as snmf_create
 * rounds opt.mlp_weights and FP32 accumulation on the device, into mult[i] (host).
 *   weights: host, SNMF_MLP_NPARAMS floats (W1[64][5], b1[64], W2[64], b2).
 * Uses the current CUDA device and the legacy default stream; allocates device memory.
 * Errors: SNMF_ERR_ARG (NULL pointer, count < 1), SNMF_ERR_OOM, SNMF_ERR_CUDA.
 */
SNMF_API snmf_status snmf_mlp_eval(const float* weights, const float* feats, int count, float* mult);

/*
 * Failure detection (not in the paper): set the bound, in clock64 cycles, of every device-side
 * wait of this handle's kernels (the mbarrier waits of the tensor-core products); 0 restores
 * the default (2e9 cycles, about one second).  A wait that runs out makes the kernel record
 * an error code, drain the asynchronous copies and tensor-core operations it issued (with a
 * separate budget of about two seconds) and return; the call that launched it then returns
 * SNMF_ERR_TIMEOUT and the handle stays usable.  The same bound is set at create by
 * opt.timeout_cycles.  Errors: SNMF_ERR_ARG (cycles < 0), SNMF_ERR_STATE (NULL handle).
 */
SNMF_API snmf_status snmf_set_timeout(snmf_handle h, int64_t cycles);

/*
 * Similarity graph of data points for Graph-SNMPBB (Sec. 2.2 builds it on a similarity graph;
 * the recipe is the clustering workload's; no counterpart entry point in the paper).
 *   X            device, n x d row-major FP32 points
 *   k            neighbours per point (1 <= k <= 32, k < n): the k nearest other points by
 *                squared Euclidean distance (FP32), ties to the lower index
 *   sigma_rank   1 <= sigma_rank <= k: s_i = distance to the sigma_rank-th neighbour;
 *                S_ij = exp(-d_ij^2 / (s_i s_j)) on the kNN pairs, symmetrised as max(S, S^T)
 *   rowptr       device, n + 1 int32, out; colidx, a_hat: device, capacity entries, out: the CSR
 *                matrix A^ = D^-1/2 S D^-1/2 (d_i = sum_j S_ij), columns ascending per row
 *   s_values     device, capacity entries, out (may be NULL): S on the same pattern
 *   degree       device, n FP32, out (may be NULL): d_i
 *   capacity     entries available; 2 n k always suffices.  *nnz (host) receives the count;
 *                a count above capacity returns SNMF_ERR_ARG with *nnz set.
 * Work runs on `stream`; the call returns when it is done.  Allocates device scratch.
 * Errors: SNMF_ERR_ARG, SNMF_ERR_OOM, SNMF_ERR_CUDA; SNMF_ERR_NUMERIC when a distance is not
 * finite or a scale s_i is zero (more than sigma_rank - 1 copies of a point), with no output.
 */
SNMF_API snmf_status snmf_knn_graph(const float* X, int64_t n, int d, int k, int sigma_rank, int32_t* rowptr,
                                    int32_t* colidx, float* a_hat, float* s_values, float* degree,
                                    int64_t capacity, int64_t* nnz, void* stream);

/*
 * Cluster labels of the last solve's restart `restart` (the reading of the clustering
 * experiments: point i belongs to argmax_c H[c][i], i.e. the largest entry of row i of Ht; W in
 * the direct and naive forms; ties to the lowest c).  labels: device, n int32, out.
 */
SNMF_API snmf_status snmf_cluster_assign(snmf_handle h, int restart, int32_t* labels);

/*
 * Clustering scores (Sec. 4 reports accuracy and ARI): the contingency table of two labelings
 * (device int32 arrays of n >= 2 labels in [0, k_true) and [0, k_pred); k_true, k_pred <= 512 and
 * k_true k_pred <= 4096) on the
 * device; from it the adjusted Rand index of Hubert and Arabie and the accuracy of the best
 * one-to-one matching of predicted to true labels (Hungarian method) on the host.  table
 * (host, k_true x k_pred), ari, accuracy: outputs, each may be NULL.
 * Errors: SNMF_ERR_ARG (label out of range, sizes), SNMF_ERR_OOM, SNMF_ERR_CUDA.
 */
SNMF_API snmf_status snmf_cluster_scores(const int32_t* truth, const int32_t* pred, int64_t n, int k_true,
                                         int k_pred, int64_t* table, double* ari, double* accuracy, void* stream);

/* Release every resource of the handle.  NULL is accepted. */
SNMF_API snmf_status snmf_destroy(snmf_handle h);

/* Message of the last error on this handle (or of the last failed create when
 * h is NULL).  Never NULL; valid until the next call on the handle. */
SNMF_API const char* snmf_last_error(snmf_handle h);

#ifdef __cplusplus
}
#endif

#endif /* SNMF_H */
