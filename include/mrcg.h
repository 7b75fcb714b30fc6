/* mrcg.h -- C ABI of the GB300 (sm_103a) MINRES-CG solver.
 *
 * Method: Manguoglu & Mehrmann, "A robust iterative scheme for symmetric
 * indefinite systems" (arXiv 1805.12417).  A x = b with A sparse, symmetric,
 * indefinite, full rank and k << n negative eigenvalues (Sec. 1, Eq. 1) is
 * solved by an outer preconditioned MINRES iteration whose preconditioner
 *     M_mr = A + 2 V_hat |Lambda_hat| V_hat^T                  (Sec. 2)
 * (V_hat: n x k basis of the negative invariant subspace, Lambda_hat: its k
 * negative eigenvalues) is applied approximately by an inner CG solve of
 * M_mr z = y (Eq. 2, Algorithm 1).  The solve stage is the third of the
 * paper's three stages (the summary closing Sec. 2): the caller supplies the
 * eigenpairs (stage two); the inner preconditioner M_cg is the identity,
 * Jacobi or the MINRES-CG* preconditioner of Sec. 2.1 (stage one, see
 * mrcg_inner_prec).
 *
 * Conventions for every entry point:
 *  - Status codes are returned; nothing is thrown across the ABI.
 *  - Vector pointers (b, x, u, y, z, ...) may be host or device memory; the
 *    library detects which with cudaPointerGetAttributes.  Device pointers must
 *    be on the handle's device.  Host pointers are staged through the handle's
 *    own device buffers (copies are inside the call).
 *  - Every call is ordered on the handle's CUDA stream and returns only when
 *    its results are complete (host-visible status and info).
 *  - A handle is used by one host thread at a time.
 *  - CSR inputs: full symmetric storage, int64 row pointers (rowptr[0] = 0),
 *    int32 column indices in [0, n), float64 values.
 *
 * Environment variables, read when a handle is created (none is needed; the
 * defaults are the tuned path):
 *  - MRCG_AUTOTUNE=0      skip the launch-shape autotuners and keep the default
 *                         shapes (mrcg_solver_create tunes for n_pad >= 4096,
 *                         mrcg_batch_create for 2^20 rows or more,
 *                         mrcg_shifted_create for n x columns >= 2^22);
 *                         MRCG_AUTOTUNE=2 tunes batches and shifted families of
 *                         any size.
 *  - MRCG_SHAPE_F32 / MRCG_SHAPE_F64 = "variant,stages,grid_a,grid_b"
 *                         replay a shape reported by mrcg_launch_config (for
 *                         profilers, whose slowed launches mislead the tuner);
 *                         ignored when the shape does not fit the matrix.
 *  - MRCG_VAR_A (0-15), MRCG_STAGES (2-8), MRCG_BPSM_A, MRCG_BPSM_B
 *                         fix the step-a variant, its pipeline depth and the
 *                         blocks per SM of the two inner kernels; any of them
 *                         turns the autotuner off.
 *  - MRCG_PDL=0..3        graph edges between the inner kernels of step-a
 *                         variants 14 and 15 (0: plain; 1: programmatic both ways;
 *                         2, the default: programmatic from step b to the next
 *                         step a, which streams its static operands while step b
 *                         finishes; 3: programmatic from step a to step b).
 *  - MRCG_ILU_STAGE=0/1   ILU(0) sweeps read the factors from global memory (0)
 *                         or from per-block images copied into shared memory
 *                         (1); default: images in mixed precision, global in FP64.
 *  - MRCG_EIG_FP32=0      mrcg_negative_eigenpairs filters in FP64 throughout
 *                         (default: FP32 filter steps until the lowest Ritz
 *                         pairs reach 1e-5 of the spectral radius bound).
 *  - MRCG_IDX16=0         keep 32-bit column indices in the inner kernels
 *                         (16-bit deltas are used whenever |col - row| <= 32767).
 *  - MRCG_UNROLL=U        inner iterations per convergence check (even, >= 2).
 *  - MRCG_INNER_LOOP=host drive the inner loop from the host instead of a
 *                         conditional CUDA graph, so that a profiler sees each
 *                         kernel; results are bitwise the same.  All three
 *                         handle kinds.
 *  - MRCG_DEBUG           print failed CUDA calls and the tuner's choice to
 *                         stderr.
 *  - MRCG_TEST_STALL=1    test hook: the producer warp of the staged step-a
 *                         kernels (variants 5-10, 12-15) stops after the first tile, the
 *                         consumers' bounded waits give up and the call returns
 *                         MRCG_ERR_CUDA; the context stays usable.
 */
#ifndef MRCG_H
#define MRCG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mrcg_solver* mrcg_handle; /* opaque */

typedef enum {
  MRCG_OK = 0,
  MRCG_ERR_INVALID = 1,    /* malformed arguments or inputs */
  MRCG_ERR_NOT_SPD = 2,    /* inner CG met p^T M_mr p <= 0: M_mr is not SPD */
  MRCG_ERR_BREAKDOWN = 3,  /* MINRES Lanczos/Givens breakdown, or r^T M_cg^{-1} r = 0 in the
                              inner CG (possible only with MRCG_MCG_SMW, whose M_cg may be indefinite) */
  MRCG_ERR_MAXITER = 4,    /* iteration budget exhausted; x = last iterate */
  MRCG_ERR_NONFINITE = 5,  /* NaN/Inf met in the data or the recurrences */
  MRCG_ERR_CUDA = 6,       /* a CUDA runtime call failed */
  MRCG_ERR_OOM = 7         /* device allocation failed */
} mrcg_status;

/* Arithmetic of the inner CG.  The outer MINRES (Lanczos vectors, Givens
 * rotations, residual norms, true-residual check) is always FP64. */
typedef enum {
  MRCG_FP64 = 0,        /* inner CG in FP64 */
  MRCG_MIXED_FP32 = 1,  /* inner CG with FP32 copies of A, V_hat and FP32 vectors */
  MRCG_MIXED_BF16M = 2  /* MRCG_MIXED_FP32 with V_hat's values rounded to BF16 (round to nearest even
                         * from their FP32 values): every inner kernel computes with the same rounded
                         * V_hat, so M_mr of Eq. 5 is built on it, and the one-gather step a on 16-slice
                         * tiles streams it as BF16 (half of V_hat's bytes).  A stays FP32: its shifted
                         * diagonal is not a BF16 number.  Single-system handles (and the inner
                         * level of complex handles); batch and shifted-family handles return
                         * MRCG_ERR_INVALID for it. */
} mrcg_precision;

/* Inner preconditioner M_cg of Algorithm 1 (the solves with M_cg inside each CG step). */
typedef enum {
  MRCG_MCG_IDENTITY = 0, /* M_cg = I */
  MRCG_MCG_JACOBI = 1,   /* M_cg = diag(M_mr) */
  MRCG_MCG_SMW = 2,      /* MINRES-CG* (Sec. 2.1): M_cg^{-1} = Atilde^{-1} - 2 V_hat Lambda_hat^{-1} V_hat^T,
                            the Sherman-Morrison-Woodbury form of M_mr^{-1} with A^{-1} approximated by
                            Atilde^{-1} = diag(A)^{-1}.  Needs a nonzero diagonal in every row of A
                            (else MRCG_ERR_INVALID at create); positive definite when diag(A) > 0.
                            Costs one more pass over V_hat per inner iteration.  Single systems only
                            (mrcg_batch_create and mrcg_shifted_create reject it). */
  MRCG_MCG_ILU0 = 3,     /* the incomplete LU factorisation ILU(0) of A (the experiments' inner preconditioner,
                            Sec. 4) in block-Jacobi form: A's diagonal blocks of ilu_block consecutive rows are
                            factored at create (couplings between blocks dropped; ilu_block >= n is plain
                            ILU(0)) and each inner CG step solves with the factors, one warp per block, level by
                            level.  Indefinite A gives an indefinite M_cg (Sec. 2 discusses CG with an indefinite
                            preconditioner); a zero pivot is MRCG_ERR_BREAKDOWN at create.  Single systems only. */
  MRCG_MCG_SMW_ILU0 = 4  /* MINRES-CG* (Sec. 2.1) with Atilde = those ILU(0) factors:
                            M_cg^{-1} = (L U)^{-1} - 2 V_hat Lambda_hat^{-1} V_hat^T.  Single systems only. */
} mrcg_inner_prec;

typedef struct {
  int64_t n;              /* rows of A (n >= 1) */
  int64_t nnz;            /* stored nonzeros (rowptr[n]) */
  const int64_t* rowptr;  /* [n+1], host or device */
  const int32_t* colind;  /* [nnz], sorted within each row */
  const double* val;      /* [nnz] */
  int32_t k;              /* columns of V_hat, 0 <= k <= 32 */
  const double* V;        /* [n*k] column-major (column j at V + j*n); NULL iff k == 0 */
  const double* lambda;   /* [k] eigenvalues of the columns of V_hat, all < 0 */
  int32_t precision;      /* mrcg_precision */
  int32_t inner_prec;     /* mrcg_inner_prec */
  int32_t validate;       /* nonzero: check V^T V ~ I and ||A V - V Lambda|| at create */
  int32_t max_outer;      /* cap on outer MINRES steps per solve; <= 0 selects 200 */
  double restart_factor;  /* restart a MINRES cycle when relres_j > f * relres_{j-3}
                             (j >= 4 within the cycle); 0 selects 0.5, < 0 disables */
  void* stream;           /* cudaStream_t to order all work on; NULL = a stream of its own */
  int32_t ilu_block;      /* MRCG_MCG_ILU0 / MRCG_MCG_SMW_ILU0: rows per diagonal block, a multiple of 32 up to
                             16384 (8192 with MRCG_FP64); 0 selects 1024 (capped at the padded n) */
  int32_t reserved;       /* set to 0 */
} mrcg_create_args;

typedef struct {
  int32_t outer_iters;        /* outer MINRES steps, all cycles */
  int32_t restarts;           /* cycles started after the first */
  int64_t inner_iters_total;  /* inner CG iterations (M_mr products) in total */
  int64_t prec_calls;         /* inner CG solves (applications of P) */
  int64_t kernel_launches;    /* kernels of this library executed by the call */
  double true_relres;        /* ||b - A x||_2 / ||b||_2 at exit, FP64 */
  double solve_ms;            /* wall time of the call */
  double* relres_history;     /* caller array or NULL: true relres after each outer step */
  int32_t history_cap;        /* its capacity */
  int32_t history_len;        /* entries written */
  int32_t status;             /* mrcg_status of the solve */
} mrcg_info;

/* Create a solver for A with preconditioner M_mr = A + 2 V |Lambda| V^T
 * (Sec. 2).  Every input array is deep-copied; the caller may free it when
 * the call returns.  A is stored on the device in SELL-32 form (slices of 32
 * rows, column-major within a slice) with FP64 values and, in mixed mode, an
 * FP32 copy of A and V_hat.
 * Errors: MRCG_ERR_INVALID (bad sizes, unsorted or out-of-range columns,
 * lambda >= 0, a V_hat that fails validation, a zero diagonal entry of A with
 * MRCG_MCG_SMW, a bad ilu_block), MRCG_ERR_BREAKDOWN (a zero pivot in the
 * ILU(0) factorisation), MRCG_ERR_OOM, MRCG_ERR_CUDA. */
mrcg_status mrcg_solver_create(const mrcg_create_args* args, mrcg_handle* out);

/* Solve A x = b by MINRES-CG (Algorithm 1).  On entry x holds x0, on exit the
 * last iterate.  Stops when the FP64 true relative residual
 * ||b - A x|| / ||b|| <= outer_tol (Sec. 4.2); each inner CG solve stops when
 * its recursive residual falls to inner_tol times its right-hand side's norm.
 * max_iters bounds the TOTAL inner CG iterations (the paper caps the sum of
 * all iterations, Sec. 4.1-4.2); <= 0 means no bound beyond
 * 2^31.  info may be NULL.  Returns the solve status (MRCG_ERR_MAXITER keeps
 * x and info valid). */
mrcg_status mrcg_solve(mrcg_handle h, const double* b, double* x, double outer_tol, double inner_tol,
                       int64_t max_iters, mrcg_info* info);

/* y = A x in FP64 (the products with A that Algorithm 1 takes). */
mrcg_status mrcg_apply_A(mrcg_handle h, const double* x, double* y);

/* out = M_mr u = A u + 2 V (|Lambda| (V^T u))  (Sec. 2, the product procedure
 * after the definition of M_mr), computed in the inner CG's precision: FP64,
 * or FP32 data and accumulation in mixed mode (inputs rounded to FP32,
 * output widened to FP64). */
mrcg_status mrcg_apply_mmr(mrcg_handle h, const double* u, double* out);

/* One application of the preconditioner: z ~ M_mr^{-1} y by the inner CG
 * from z = 0 (Eq. 2), in the handle's precision, until
 * ||y - M_mr z||_recursive <= inner_tol ||y|| or max_iters iterations.
 * iters (may be NULL) receives the iteration count.  Returns MRCG_OK,
 * MRCG_ERR_MAXITER, MRCG_ERR_NOT_SPD, MRCG_ERR_NONFINITE, MRCG_ERR_BREAKDOWN
 * (MRCG_MCG_SMW only) or MRCG_ERR_CUDA (a staged copy of the inner kernels did
 * not arrive within its wait limit of about a second; the handle stays usable). */
mrcg_status mrcg_inner_solve(mrcg_handle h, const double* y, double* z, double inner_tol, int64_t max_iters,
                             int64_t* iters);

/* Diagnostic timing of the two kernels of one inner CG iteration (Eq. 2):
 *   ms[0]: step a  -- p = s + beta p fused into q = A p + V (2|Lambda| V^T p)
 *          and the partials p^T q and V^T M_cg^{-1} A p (the M_mr product
 *          of Sec. 2; V^T s then follows by recurrence),
 *   ms[1]: step b  -- z += alpha p, r -= alpha q, s = M_cg^{-1} r and the
 *          partials r^T s, r^T r.
 * Each is launched `iters` times (1 <= iters <= 4096) on the handle's stream,
 * outside the solver's graph, on a fixed synthetic right-hand side, and
 * bracketed by CUDA events; ms receives the average duration in
 * milliseconds (ms[1] is near zero for step-a variant 8, which has no step b).  Overwrites the handle's work vectors (not its matrix). */
mrcg_status mrcg_time_inner_kernels(mrcg_handle h, int32_t iters, double* ms);

/* In-situ time of one inner CG iteration (Eq. 2) as it runs inside the
 * solver: the handle's own inner-CG graph (the device-side loop, or the
 * host-driven loop under MRCG_INNER_LOOP=host) is launched on a fixed
 * synthetic right-hand side with no tolerance, for 2U and for 2U + iters
 * iterations (U = iterations per loop body), each bracketed by CUDA events
 * on the handle's stream, and *ms_per_iter receives the difference divided by
 * the difference of the iterations run (the per-solve kernels cancel).  An
 * FP32 recursion can end by itself once it reaches its rounding floor
 * (p^T q <= 0); a first probe run finds where, and the long run then stops at
 * three quarters of that count.  8 <= iters <= 65536.  Overwrites the
 * handle's work vectors (not its matrix).  Errors: MRCG_ERR_INVALID,
 * MRCG_ERR_BREAKDOWN (fewer than 8 iterations to time), MRCG_ERR_CUDA. */
mrcg_status mrcg_time_inner_graph(mrcg_handle h, int32_t iters, double* ms_per_iter);

/* Measured FP64 fused-multiply-add throughput of the current device, in
 * TFLOP/s (2 flops per FMA): eight independent FMA chains per thread, eight
 * 256-thread blocks per SM, best of seven CUDA-event-timed launches after
 * three warm-ups.  The denominator of the FP64 kernels' arithmetic roofline.
 * ms (may be NULL) receives the best launch's duration.  Allocates and frees
 * a small scratch buffer.  Errors: MRCG_ERR_INVALID (tflops NULL),
 * MRCG_ERR_OOM, MRCG_ERR_CUDA. */
mrcg_status mrcg_fp64_fma_peak(double* tflops, double* ms);

/* Launch configuration chosen for the handle's inner-CG kernels (at create,
 * by timing candidate shapes on this matrix unless MRCG_AUTOTUNE=0):
 * cfg[0] step-a variant (0: V_hat rows loaded before the SpMV, 1: after it,
 * 2: two slices per warp, 3 / 4: as 1 with registers capped for 6 / 8
 * resident blocks per SM, 5 / 6: every streamed operand staged in shared
 * memory by bulk copies, a persistent grid over tiles of 8 slices, registers
 * capped for 2 / 4 blocks per SM, 7: as 5 with each warp's gathers issued
 * one tile ahead, 8: the whole CG iteration in one staged kernel, with the
 * residual norm by expansion and no step b; M_cg = I only; 9 / 10: staged as
 * 5 with registers capped for 2 / 3 blocks per SM, 11: plain loads,
 * 12 / 13: 9 / 10 with each warp's gathers issued one tile ahead, 14 / 15:
 * tiles of 16 slices with two adjacent slices per consumer warp, registers
 * capped for 2 / 1 blocks per SM; variants 9-15 gather only p (one load per
 * matrix entry) with beta formed by expansion in step a and p = s + beta p
 * done by their own step b; M_cg = I or Jacobi),
 * cfg[1] step-a grid (blocks), cfg[2] step-b grid,
 * cfg[3] CG iterations per body of the device loop, cfg[4] k bucket of the
 * kernels (0, 8, 12, 16, 24 or 32), cfg[5] bytes per column index read by the
 * inner kernels (2: 16-bit col - row deltas, used when every delta fits; 4),
 * cfg[6] shared-memory stages of variants 5-10 and 12-15 (0 for the others).
 * cfg must hold 7 values. */
mrcg_status mrcg_launch_config(mrcg_handle h, int32_t* cfg);

/* ---- Batches of independent systems (many uneven systems in one launch sequence) ----
 *
 * The paper's motivating use solves many systems with related coefficient
 * matrices after one setup (Sec. 2: the costly eigenpair stage pays off when
 * many systems share a coefficient matrix or have close ones; Sec. 3, shifted
 * systems of shift-and-invert Arnoldi).  A batch
 * holds nsys independent systems A_i x_i = b_i, each with its own M_mr
 * (V_hat_i, Lambda_hat_i), and runs Algorithm 1 for all of them at once: every
 * kernel covers all systems, with per-system scalars, per-system reductions
 * and per-system convergence masks; the inner CG loop of all systems is one
 * device-side graph loop. */
typedef struct mrcg_batch* mrcg_batch_handle; /* opaque */

/* Create a batch from nsys (1..4096) create-argument records, deep-copied
 * like mrcg_solver_create.  All records must share precision and inner_prec;
 * max_outer, restart_factor and stream are taken from sys[0].  The sum of the
 * systems' rows (each padded to a multiple of 32) must stay below 2^31.
 * Errors: MRCG_ERR_INVALID, MRCG_ERR_NONFINITE, MRCG_ERR_OOM, MRCG_ERR_CUDA. */
mrcg_status mrcg_batch_create(int32_t nsys, const mrcg_create_args* sys, mrcg_batch_handle* out);

/* Solve every system of the batch by MINRES-CG with the rules of mrcg_solve.
 * B and X hold the systems' vectors back to back in system order
 * (sum of n_i entries, host or device); X holds x0 on entry.  max_iters bounds
 * the total inner iterations of EACH system.  infos (may be NULL) receives one
 * record per system; kernel_launches there counts the launches of the whole
 * batched call.  Returns MRCG_OK when every system converged, else the
 * status of the first system (in order) that did not. */
mrcg_status mrcg_batched_solve(mrcg_batch_handle h, const double* B, double* X, double outer_tol, double inner_tol,
                               int64_t max_iters, mrcg_info* infos);

/* Number of systems in the batch (0 for NULL). */
int32_t mrcg_batch_size(mrcg_batch_handle h);

/* Launch shape of the batch engine, chosen at create by timing calibration
 * solves on the batch itself (unless MRCG_AUTOTUNE=0, or the batch holds
 * fewer than 2^20 rows): cfg[0] rows per chunk (the unit one block reduces
 * and a converged system skips: 1024, 2048, 4096 or 8192), cfg[1] step-a
 * grid, cfg[2] step-b grid, cfg[3] chunks.  cfg must hold 4 values. */
mrcg_status mrcg_batch_launch_config(mrcg_batch_handle h, int32_t* cfg);

/* Release a batch (NULL is a no-op). */
void mrcg_batch_destroy(mrcg_batch_handle h);

/* ---- Shifted families with blocks of right-hand sides ----
 *
 * Columns c = j * nrhs + r (0 <= c < nshift * nrhs <= 64) solve
 *     (L - sigma_j I) x_c = b_c,
 * the family of shifted systems of shift-and-invert Arnoldi (Sec. 3) with one
 * sparsity pattern.  Because the eigenvectors of L - sigma_j I are those of L,
 * every shift shares V_hat: for shift j, M_mr,j uses the first k_j columns of
 * V_hat and Lambda_hat_j = lambda_L[0..k_j) - sigma_j (Sec. 2, definition of
 * M_mr).  L, V_hat and all vectors are stored once; each iteration reads L and
 * V_hat once for all columns.  Identity inner preconditioner only. */
typedef struct mrcg_shifted* mrcg_shifted_handle; /* opaque */

/* L: CSR of the unshifted matrix (n, nnz, rowptr, colind, val as for
 * mrcg_solver_create); L->V: n x L->k column-major eigenvectors of L
 * (L->k <= 32, orthonormal), L->lambda: their eigenvalues of L (any sign);
 * L->precision, L->max_outer, L->restart_factor, L->stream as usual
 * (L->inner_prec must be MRCG_MCG_IDENTITY).  sigma[nshift], k_per_shift[nshift]
 * (0 <= k_j <= L->k, with lambda_L[l] - sigma_j < 0 for l < k_j).
 * Errors: MRCG_ERR_INVALID (also for nshift * nrhs_per_shift > 64),
 * MRCG_ERR_NONFINITE, MRCG_ERR_OOM, MRCG_ERR_CUDA. */
mrcg_status mrcg_shifted_create(const mrcg_create_args* L, int32_t nshift, const double* sigma,
                                const int32_t* k_per_shift, int32_t nrhs_per_shift, mrcg_shifted_handle* out);

/* Solve all columns by MINRES-CG (rules of mrcg_solve, per column).  B and X
 * are n x (nshift * nrhs) row-major blocks (element (i, c) at i * ncols + c),
 * host or device; X holds x0 on entry.  max_iters bounds each column's total
 * inner iterations.  infos (may be NULL): one record per column.  Returns
 * MRCG_OK when every column converged, else the first failing column's status. */
mrcg_status mrcg_shifted_solve(mrcg_shifted_handle h, const double* B, double* X, double outer_tol,
                               double inner_tol, int64_t max_iters, mrcg_info* infos);

/* Number of columns (nshift * nrhs_per_shift; 0 for NULL). */
int32_t mrcg_shifted_columns(mrcg_shifted_handle h);

/* Launch shape of the shifted-family engine, chosen at create by timing
 * calibration solves on the handle's own matrix (unless MRCG_AUTOTUNE=0, or
 * the blocks hold fewer than 2^22 values): cfg[0] row-kernel grid (blocks),
 * cfg[1] blocks per SM (0: the occupancy limit, untuned), cfg[2] 1 when the
 * SpMV takes four rows of at most 8 entries per warp (ELL-8), 0 for one row
 * per warp (CSR), cfg[3] V_hat width bucket (8, 16, 24, 32), cfg[4] padded
 * columns (32 or 64).  cfg must hold 5 values. */
mrcg_status mrcg_shifted_launch_config(mrcg_shifted_handle h, int32_t* cfg);

/* Release a shifted-family handle (NULL is a no-op). */
void mrcg_shifted_destroy(mrcg_shifted_handle h);

/* Allocation-free M_mr product: out = A u + 2 V (|Lambda| (V^T u)) in FP64.
 * The paper has no counterpart; this entry point exists for callers that
 * cannot call cudaMalloc at all (code running inside another framework's
 * fixed memory pool, plugins whose host forbids device allocations after
 * start-up, paths that must not take the allocator's locks).  It needs no
 * handle: the caller passes DEVICE arrays -- CSR A (rowptr[n+1], colind[nnz],
 * val[nnz], same rules as mrcg_create_args), V (n x k column-major, k <= 32),
 * lambda[k], u[n] and out[n] -- and the only scratch is a fixed 262,656-byte
 * static device array inside the library, which every GPU that loads the
 * library keeps until the process exits.  Nothing is allocated or freed.
 *  - The first call in each CUDA context (normally: on each device, in its
 *    primary context) looks up that array's device address with
 *    cudaGetSymbolAddress, with the device current, and caches it for that
 *    context.  Make that first call before any stream capture.  After a
 *    cudaDeviceReset the library's module is loaded afresh and the array may
 *    move: the next call sees a new context and looks the address up again
 *    (so it, too, should come before any capture).
 *  - Work is enqueued on `stream` (NULL = the default stream) and the call
 *    returns without waiting; out is complete when the stream reaches it.
 *  - All calls share the one scratch array and each call rewrites it (a
 *    counter is cleared at the start of each call): calls that can overlap on
 *    the GPU (different streams, several host threads) race and must be
 *    serialised by the caller.
 * Errors: MRCG_ERR_INVALID for n < 1, n > 2^31-1, k < 0, k > 32 or NULL
 * arrays; MRCG_ERR_CUDA if the address lookup or a launch fails. */
mrcg_status mrcg_mmr_apply_noalloc(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* val,
                                   int32_t k, const double* V, const double* lambda, const double* u, double* out,
                                   void* stream);

/* ---- Setup stage 2: the negative eigenpairs that define M_mr ----
 *
 * The paper's scheme computes the k negative eigenvalues of A and an
 * approximate basis of their invariant subspace once, before the solves
 * (Sec. 2, stage two of the three-stage summary; the experiments use a
 * Krylov eigensolver, Sec. 4), and amortises that cost over many solves.
 * mrcg_negative_eigenpairs does this on the GPU with the library's own block
 * SpMV: Chebyshev-filtered subspace iteration on a block of `block` vectors,
 * Rayleigh-Ritz (FP64) between filters; the filter steps run in FP32 while
 * the lowest Ritz pairs' residuals exceed 1e-5 ||A||_gersh and in FP64 from
 * then on (MRCG_EIG_FP32=0: FP64 throughout), until every Ritz value below zero
 * has a residual ||A v - lambda v||_2 <= tol * ||A||_gersh (the Gershgorin
 * bound of the spectral radius) and the first nonnegative Ritz value of the
 * block has settled to sqrt(tol) * ||A||_gersh.  Its output is ready for
 * mrcg_create_args (V column-major, lambda ascending, all < 0). */
typedef struct {
  int32_t negative_found;      /* negative Ritz values in the block at exit */
  int32_t rayleigh_ritz_steps;
  int64_t block_spmvs;         /* products A X with the n x block matrix X */
  double max_residual;         /* max ||A v - lambda v||_2 over the negative pairs at exit */
  double spectrum_lo;          /* Gershgorin bounds of the spectrum of A */
  double spectrum_hi;
  double seconds;              /* wall time of the call */
  int32_t status;              /* mrcg_status of the call */
} mrcg_eig_info;

/* CSR A as for mrcg_create_args (host or device arrays, full symmetric
 * storage).  block: 2..64 vectors, more than the number of negative
 * eigenvalues (a guard of 8 or more speeds convergence).  tol > 0 (1e-11 gives
 * subspaces that pass mrcg_solver_create's validation with a wide margin).
 * max_spmv: cap on block SpMVs.  seed: the start block's counter-based hash.
 * Outputs: *k (the number of negative eigenvalues found), V (capacity n x
 * block doubles, column-major; the first k columns written, orthonormal) and
 * lambda (capacity block; the first k written, ascending), host or device.
 * Allocates its own device work space (about 4 n x 64 doubles at most) on the
 * current device and frees it before returning.  info may be NULL.
 * Errors: MRCG_ERR_INVALID (bad sizes or CSR), MRCG_ERR_NONFINITE,
 * MRCG_ERR_MAXITER (not converged within max_spmv: most often the block holds
 * no nonnegative Ritz value, i.e. `block` is too small for A's negative
 * eigenvalues; info->negative_found says how many it saw), MRCG_ERR_BREAKDOWN
 * (the block lost rank), MRCG_ERR_OOM, MRCG_ERR_CUDA. */
mrcg_status mrcg_negative_eigenpairs(int64_t n, const int64_t* rowptr, const int32_t* colind, const double* val,
                                     int32_t block, double tol, int64_t max_spmv, uint64_t seed, int32_t* k,
                                     double* V, double* lambda, mrcg_eig_info* info);

/* ---- Complex shifted systems of the disk-brake application (Sec. 3) ----
 *
 * For a quadratic pencil lambda^2 Mass + lambda D + K (Mass: lumped, i.e.
 * diagonal, positive; K, D general sparse) with companion linearisation
 * A = [[0, I], [-K, -D]], B = [[I, 0], [0, Mass]], solve
 *     (gamma B - A) (x + i y) = f + i g        (x, y, f, g of length 2n)
 * through the double-size real system of Sec. 3 with its preconditioner M
 * built from the symmetric positive definite stiffness KE (K without its
 * general part) and no damping: flexible GMRES on the real system, M applied
 * by its block LU, the Schur complement S = S1 S2 (Sec. 3), S2 solved by
 * flexible GMRES preconditioned with its block lower triangular part, whose
 * diagonal solves are with KE - |gamma|^2 Mass: the symmetric indefinite
 * inner level, solved by this library's MINRES-CG.  That inner matrix depends
 * on |gamma| only, so one handle serves every gamma of the same modulus (the
 * reuse Sec. 3 points out): its negative eigenpairs are given or computed once
 * at create by mrcg_negative_eigenpairs. */
typedef struct mrcg_complex* mrcg_complex_handle; /* opaque */

typedef struct {
  int64_t n;                                  /* mechanical unknowns (the real system has 4n) */
  const int64_t* ke_rowptr;                   /* KE: symmetric positive definite stiffness, CSR (its diagonal stored) */
  const int32_t* ke_colind;
  const double* ke_val;
  const int64_t* k_rowptr;                    /* K (K_Omega of Sec. 3): general sparse, CSR */
  const int32_t* k_colind;
  const double* k_val;
  const int64_t* d_rowptr;                    /* D (D_Omega): general sparse, CSR */
  const int32_t* d_colind;
  const double* d_val;
  const double* mass;                         /* [n] lumped mass, all > 0 */
  double gamma_abs;                           /* |gamma| > 0 */
  int32_t k;                                  /* negative eigenpairs of KE - |gamma|^2 Mass given in V, lambda
                                                 (0 <= k <= 32), or -1: computed at create */
  const double* V;                            /* [n*k] column-major, orthonormal */
  const double* lambda;                       /* [k], all < 0 */
  int32_t eig_block;                          /* k = -1: block size of the eigensolver (0 selects 32) */
  int32_t precision;                          /* mrcg_precision of the inner CG */
  int32_t inner_prec;                         /* mrcg_inner_prec of the inner CG */
  int32_t reserved;                           /* set to 0 */
  void* stream;                               /* cudaStream_t, or NULL for a stream of its own */
} mrcg_complex_args;

typedef struct {
  int32_t outer_iters;       /* flexible GMRES iterations on the real-equivalent system */
  int32_t s2_iters_total;    /* flexible GMRES iterations on S2, over all applications of M */
  int64_t inner_solves;      /* MINRES-CG solves of the inner level */
  int64_t inner_cg_iters;    /* CG iterations inside them */
  double true_relres;        /* ||f + i g - C (x + i y)|| / ||f + i g|| at exit */
  double solve_ms;
  int32_t status;
} mrcg_complex_info;

/* Copies every input (host or device arrays).  Errors: MRCG_ERR_INVALID (sizes,
 * CSR, a mass entry <= 0, a KE row without its diagonal, k > 32), the errors of
 * mrcg_negative_eigenpairs and mrcg_solver_create for the inner level,
 * MRCG_ERR_OOM, MRCG_ERR_CUDA. */
mrcg_status mrcg_complex_create(const mrcg_complex_args* args, mrcg_complex_handle* out);

/* Negative eigenvalues of the handle's inner-level matrix (-1 for NULL). */
int32_t mrcg_complex_negative_count(mrcg_complex_handle h);

/* Solve for one shift gamma = gamma_re + i gamma_im with |gamma| equal to the
 * handle's (relative 1e-10) and gamma_im > 0, from x + i y = 0.  f, g (inputs)
 * and x, y (outputs) hold 2n values each, host or device.  Outer flexible
 * GMRES(restart) to the relative residual tol (at most max_iters iterations,
 * restart <= 120); each application of M solves S2 by one cycle of flexible
 * GMRES to s2_tol (at most s2_max <= 120 iterations); each inner-level solve is
 * MINRES-CG to the true relative residual inner_tol with inner CG tolerance
 * cg_tol.  Allocates its work space (about (restart + 2) 4n + (s2_max + 2) 2n
 * doubles) for the call.  Returns MRCG_OK, MRCG_ERR_MAXITER (info valid, x, y
 * the last iterate), MRCG_ERR_INVALID, or an inner-level failure. */
mrcg_status mrcg_complex_solve(mrcg_complex_handle h, double gamma_re, double gamma_im, const double* f,
                               const double* g, double* x, double* y, double tol, int32_t restart,
                               int32_t max_iters, double s2_tol, int32_t s2_max, double inner_tol, double cg_tol,
                               mrcg_complex_info* info);

/* Release the handle and its inner-level solver (NULL is a no-op). */
void mrcg_complex_destroy(mrcg_complex_handle h);

/* Release every device and host resource of the handle (NULL is a no-op). */
void mrcg_solver_destroy(mrcg_handle h);

/* Static, human-readable name of a status code. */
const char* mrcg_status_string(mrcg_status s);

#ifdef __cplusplus
}
#endif
#endif /* MRCG_H */
