/* Plain FP64 CPU oracle for MINRES-CG (Manguoglu & Mehrmann, "A robust
 * iterative scheme for symmetric indefinite systems").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header or constant with the CUDA path.
 *
 * Conventions: CSR with int64 row pointers and int32 column indices, full
 * symmetric storage.  V_hat is a column-major n x k block (column j starts at
 * V + j*n).  lam holds the k (negative) eigenvalues Lambda_hat.
 */
#ifndef MRCG_ORACLE_H
#define MRCG_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  ORC_OK = 0,
  ORC_ERR_INVALID = 1,
  ORC_ERR_NOT_SPD = 2,
  ORC_ERR_BREAKDOWN = 3,
  ORC_ERR_MAXITER = 4,
  ORC_ERR_NONFINITE = 5
};

/* inner preconditioner M_cg: identity; Jacobi with diag(M_mr); the
 * MINRES-CG* preconditioner of Sec. 2.1, M_cg^{-1} = diag(A)^{-1} - 2 V Lambda^{-1} V^T;
 * the incomplete factorisation ILU(0) of A (Sec. 4), block-Jacobi: factored on
 * the diagonal blocks of `block` consecutive rows; or MINRES-CG* with that
 * factorisation as Atilde: M_cg^{-1} = (L U)^{-1} - 2 V Lambda^{-1} V^T */
enum { ORC_MCG_IDENTITY = 0, ORC_MCG_JACOBI = 1, ORC_MCG_SMW = 2, ORC_MCG_ILU0 = 3, ORC_MCG_SMW_ILU0 = 4 };

/* ILU(0) factors: L strictly lower (unit diagonal implied) and U upper with
 * its diagonal, both on the pattern of A restricted to the diagonal blocks
 * (CSR, column-sorted). */
typedef struct orc_ilu {
  int64_t n, block;
  int64_t *lrow, *urow;
  int32_t *lcol, *ucol;
  double *lval, *uval;
} orc_ilu;

typedef struct {
  int64_t n;
  const int64_t* rowptr;
  const int32_t* colind;
  const double* val;
  int32_t k;
  const double* V;   /* n x k column-major */
  const double* lam; /* k eigenvalues (negative) */
  const orc_ilu* ilu; /* factors for ORC_MCG_ILU0 / ORC_MCG_SMW_ILU0, else NULL */
} orc_system;

/* ILU(0) of A on its diagonal blocks of `block` rows (block >= n: the whole
 * matrix): Gaussian elimination in row order keeping only the positions of
 * A's pattern inside the block (Saad, Iterative Methods, Alg. 10.4).
 * ORC_ERR_BREAKDOWN on a zero or non-finite pivot.  Free with orc_ilu0_free. */
int orc_ilu0_factor(const orc_system* s, int64_t block, orc_ilu* out);
void orc_ilu0_free(orc_ilu* f);
/* out = U^{-1} (L^{-1} r): forward then backward substitution */
void orc_ilu0_apply(const orc_ilu* f, const double* r, double* out);

/* y = A x (the products with A that Alg. 1 takes). */
void orc_csr_spmv(const orc_system* s, const double* x, double* y);

/* out = M_mr u = A u + 2 V (|Lambda| (V^T u))   (Sec. 2, the product
 * procedure following the definition of M_mr).  work: k doubles.
 * If flops != NULL the number of floating-point operations performed is
 * added to *flops. */
void orc_mmr_apply(const orc_system* s, const double* u, double* out, double* work, int64_t* flops);

/* diag(M_mr)_i = A_ii + 2 sum_j |lam_j| V_ij^2 */
void orc_mmr_diag(const orc_system* s, double* d);

/* out = M_cg^{-1} r for the preconditioner mcg selects.  work: n + k
 * doubles.  ORC_ERR_INVALID for ORC_MCG_SMW when a diagonal entry of A is
 * zero or not finite. */
int orc_mcg_apply(const orc_system* s, int mcg, const double* r, double* out, double* work);

/* Inner CG on M_mr z = y (Eq. 2; Alg. 1 inner block), x0 = 0, stopping on
 * the recursive residual ||r|| <= tol ||y||.  mcg selects M_cg.
 * iters: number of M_mr products done.  work: 5n + k doubles.
 * Returns ORC_OK, ORC_ERR_NOT_SPD (p^T M p <= 0), ORC_ERR_NONFINITE,
 * ORC_ERR_INVALID (ORC_MCG_SMW with a zero diagonal entry of A),
 * ORC_ERR_BREAKDOWN (r^T M_cg^{-1} r = 0 before convergence, possible only
 * with an indefinite M_cg) or ORC_ERR_MAXITER (z holds the last iterate). */
int orc_cg(const orc_system* s, int mcg, const double* y, double* z, double tol, int64_t maxit,
           int64_t* iters, double* work);

/* Preconditioner callback for the generic MINRES below: z = P^{-1} v.
 * budget: iterations it may spend; *iters: iterations it spent. */
typedef int (*orc_prec_fn)(void* ctx, int64_t n, const double* v, double* z, int64_t budget,
                           int64_t* iters);

typedef struct {
  int32_t outer_iters;      /* outer MINRES iterations over all cycles */
  int32_t restarts;         /* restart cycles started after the first */
  int64_t inner_iters_total;
  int64_t prec_calls;
  double true_relres;       /* ||b - A x|| / ||b|| at exit */
  int32_t history_len;      /* entries written to the history arrays */
  int32_t status;
} orc_info;

/* Preconditioned MINRES (Paige-Saunders, in the unnormalised-Lanczos form
 * with Givens QR), stopping on the true relative residual.  On entry x holds
 * x0, on exit the last iterate.  hist_relres[j] = true relative residual after
 * outer step j, hist_eta[j] = |eta| after step j (may be NULL).
 * Restart rule: a new cycle starts from the current x when, within a cycle,
 * relres_j > restart_factor * relres_{j-3} (j >= 4 within the cycle;
 * restart_factor <= 0 disables this test), or
 * when gamma_{j+1} underflows to zero without convergence.
 * max_inner_total bounds the preconditioner's total iterations. */
int orc_minres(const orc_system* s, const double* b, double* x, orc_prec_fn prec, void* prec_ctx,
               double outer_tol, int32_t max_outer, int64_t max_inner_total, double restart_factor,
               double* hist_relres, double* hist_eta, int32_t hist_cap, orc_info* info);

/* MINRES-CG: orc_minres with P = the inner CG on M_mr (Alg. 1). */
int orc_minres_cg(const orc_system* s, int mcg, const double* b, double* x, double outer_tol,
                  double inner_tol, int64_t max_iters, int32_t max_outer, double restart_factor,
                  double* hist_relres, double* hist_eta, int32_t hist_cap, orc_info* info);

/* 2x2 block spectral replacement (Sec. 1): the symmetric block
 * [[a, b], [b, c]] = R diag(l1, l2) R with R = [[cs, sn], [sn, -cs]] is
 * replaced by R diag(|l1|, |l2|) R.  out = {a~, b~, c~}; eig = {l1, l2};
 * rot = {cs, sn} (any of these may be NULL). */
void orc_abs_2x2(double a, double b, double c, double* out, double* eig, double* rot);

/* ||b - A x||_2 / ||b||_2 */
double orc_true_relres(const orc_system* s, const double* b, const double* x, double* work);

#ifdef __cplusplus
}
#endif
#endif
