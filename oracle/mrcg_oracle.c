/* Plain FP64 CPU oracle for MINRES-CG.
 *
 * TEST INFRASTRUCTURE ONLY: serial, unblocked, unfused, written to be checked
 * against the paper by eye.  Each function cites the passage it follows.
 * Nothing here is shared with, or called by, the CUDA library; the tests, the
 * smoke check and the benchmark's CPU-baseline and reference legs load it.
 *
 * Every function's results are pinned by the CPU tests (closed forms, dense
 * linear algebra, textbook properties of CG and MINRES, hand-derived 2x2
 * fixtures).  The iteration counts it reports (outer, inner, restarts) are
 * parity unpinned: nothing in the paper fixes them for these matrices.
 */
#include "mrcg_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* The same source builds twice: serially (the pinned oracle) and with
 * -fopenmp for the all-core CPU baseline, where these markers split the
 * length-n loops over the cores (the reductions then sum in another order).
 * Without OpenMP they expand to nothing. */
#ifdef _OPENMP
#define ORC_FOR _Pragma("omp parallel for schedule(static)")
#define ORC_FOR_SUM _Pragma("omp parallel for schedule(static) reduction(+ : s)")
#else
#define ORC_FOR
#define ORC_FOR_SUM
#endif

static double dot(int64_t n, const double* a, const double* b) {
  double s = 0.0;
  ORC_FOR_SUM
  for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

static double nrm2(int64_t n, const double* a) { return sqrt(dot(n, a, a)); }

/* Alg. 1: products with the sparse coefficient matrix A. */
void orc_csr_spmv(const orc_system* s, const double* x, double* y) {
  ORC_FOR
  for (int64_t i = 0; i < s->n; ++i) {
    double acc = 0.0;
    for (int64_t p = s->rowptr[i]; p < s->rowptr[i + 1]; ++p) acc += s->val[p] * x[s->colind[p]];
    y[i] = acc;
  }
}

/* Sec. 2: M_mr u = A u + 2 (V (|Lambda| (V^T u))), cost O(nnz + kn).
 * Steps in the paper's order: t = V^T u; t <- 2|Lambda| t; out = A u + V t. */
void orc_mmr_apply(const orc_system* s, const double* u, double* out, double* t, int64_t* flops) {
  const int64_t n = s->n;
  const int32_t k = s->k;
  for (int32_t j = 0; j < k; ++j) t[j] = dot(n, s->V + (int64_t)j * n, u); /* 2n flops each */
  for (int32_t j = 0; j < k; ++j) t[j] *= 2.0 * fabs(s->lam[j]);           /* 1 flop each: the factor 2|lam| is data */
  ORC_FOR
  for (int64_t i = 0; i < n; ++i) {
    double acc = 0.0;
    for (int64_t p = s->rowptr[i]; p < s->rowptr[i + 1]; ++p) acc += s->val[p] * u[s->colind[p]];
    for (int32_t j = 0; j < k; ++j) acc += s->V[(int64_t)j * n + i] * t[j];
    out[i] = acc;
  }
  if (flops) *flops += 2 * s->rowptr[n] + 4 * (int64_t)k * n + k;
}

void orc_mmr_diag(const orc_system* s, double* d) {
  for (int64_t i = 0; i < s->n; ++i) {
    double a = 0.0;
    for (int64_t p = s->rowptr[i]; p < s->rowptr[i + 1]; ++p)
      if (s->colind[p] == i) a += s->val[p];
    for (int32_t j = 0; j < s->k; ++j) {
      double v = s->V[(int64_t)j * s->n + i];
      a += 2.0 * fabs(s->lam[j]) * v * v;
    }
    d[i] = a;
  }
}

/* Sec. 2.1 (MINRES-CG*): the inner CG's preconditioner taken from the
 * Sherman-Morrison-Woodbury form of M_mr^{-1}, with the action of A^{-1}
 * approximated:  M_cg^{-1} r = Atilde^{-1} r - 2 V (Lambda^{-1} (V^T r)).
 * Here Atilde = diag(A).  Steps in the formula's order: t = V^T r;
 * t <- -2 Lambda^{-1} t; out = diag(A)^{-1} r + V t.  dainv holds 1/diag(A). */
static void smw_apply(const orc_system* s, const double* dainv, const double* r, double* out, double* t) {
  const int64_t n = s->n;
  for (int32_t j = 0; j < s->k; ++j) t[j] = dot(n, s->V + (int64_t)j * n, r);
  for (int32_t j = 0; j < s->k; ++j) t[j] = -2.0 * t[j] / s->lam[j];
  for (int64_t i = 0; i < n; ++i) {
    double acc = dainv[i] * r[i];
    for (int32_t j = 0; j < s->k; ++j) acc += s->V[(int64_t)j * n + i] * t[j];
    out[i] = acc;
  }
}

/* 1 / diag(A); ORC_ERR_INVALID when a diagonal entry is zero or not finite
 * (Atilde = diag(A) must be invertible).  Sec. 2.1 notes that with an
 * approximate Atilde the preconditioner need not be positive definite; it is
 * positive definite whenever diag(A) > 0. */
static int diag_a_inverse(const orc_system* s, double* dainv) {
  for (int64_t i = 0; i < s->n; ++i) {
    double a = 0.0;
    for (int64_t p = s->rowptr[i]; p < s->rowptr[i + 1]; ++p)
      if (s->colind[p] == i) a += s->val[p];
    if (a == 0.0 || !isfinite(a)) return ORC_ERR_INVALID;
    dainv[i] = 1.0 / a;
  }
  return ORC_OK;
}

/* Sec. 4 (the experiments' inner preconditioner): ILU(0).  Row i of the
 * working copy w (A's entries of row i inside its block) is reduced by the
 * rows k < i it holds, in increasing k: w_ik <- w_ik / u_kk, then
 * w_ij <- w_ij - w_ik u_kj for every j > k that is in row i's pattern.  The
 * reduced row is split into L (j < i) and U (j >= i). */
int orc_ilu0_factor(const orc_system* s, int64_t block, orc_ilu* f) {
  const int64_t n = s->n;
  memset(f, 0, sizeof(*f));
  if (block < 1) return ORC_ERR_INVALID;
  f->n = n;
  f->block = block;
  f->lrow = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  f->urow = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  const int64_t nnz = s->rowptr[n];
  f->lcol = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz + 1));
  f->ucol = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz + 1));
  f->lval = (double*)malloc(sizeof(double) * (size_t)(nnz + 1));
  f->uval = (double*)malloc(sizeof(double) * (size_t)(nnz + 1));
  double* w = (double*)calloc((size_t)n, sizeof(double));       /* dense scatter of the current row */
  int64_t* upos = (int64_t*)malloc(sizeof(int64_t) * (size_t)n); /* row k -> position of u_kk */
  if (!f->lrow || !f->urow || !f->lcol || !f->ucol || !f->lval || !f->uval || !w || !upos) {
    free(w); free(upos); orc_ilu0_free(f);
    return ORC_ERR_INVALID;
  }
  int64_t nl = 0, nu = 0;
  int rc = ORC_OK;
  for (int64_t i = 0; i < n && rc == ORC_OK; ++i) {
    const int64_t b0 = (i / block) * block, b1 = b0 + block < n ? b0 + block : n;
    /* scatter row i's in-block entries */
    for (int64_t p = s->rowptr[i]; p < s->rowptr[i + 1]; ++p) {
      const int64_t j = s->colind[p];
      if (j >= b0 && j < b1) w[j] = s->val[p];
    }
    /* eliminate with the rows k < i of the pattern, in increasing k */
    for (int64_t p = s->rowptr[i]; p < s->rowptr[i + 1]; ++p) {
      const int64_t kk = s->colind[p];
      if (kk < b0 || kk >= i) continue;
      const double piv = f->uval[upos[kk]];
      const double lik = w[kk] / piv;
      w[kk] = lik;
      for (int64_t q = upos[kk] + 1; q < f->urow[kk + 1]; ++q) {
        const int64_t j = f->ucol[q];
        /* only positions of row i's pattern are kept (level 0 fill) */
        int in_pattern = 0;
        for (int64_t r = s->rowptr[i]; r < s->rowptr[i + 1]; ++r)
          if (s->colind[r] == j) { in_pattern = 1; break; }
        if (in_pattern) w[j] -= lik * f->uval[q];
      }
    }
    /* gather: L (j < i), U (j >= i) */
    f->lrow[i] = nl;
    f->urow[i] = nu;
    int have_diag = 0;
    for (int64_t p = s->rowptr[i]; p < s->rowptr[i + 1]; ++p) {
      const int64_t j = s->colind[p];
      if (j < b0 || j >= b1) continue;
      if (j < i) {
        f->lcol[nl] = (int32_t)j;
        f->lval[nl++] = w[j];
      } else {
        if (j == i) { upos[i] = nu; have_diag = 1; }
        f->ucol[nu] = (int32_t)j;
        f->uval[nu++] = w[j];
      }
      w[j] = 0.0;
    }
    if (!have_diag || f->uval[upos[i]] == 0.0 || !isfinite(f->uval[upos[i]])) rc = ORC_ERR_BREAKDOWN;
    f->lrow[i + 1] = nl;
    f->urow[i + 1] = nu;
  }
  free(w);
  free(upos);
  if (rc != ORC_OK) orc_ilu0_free(f);
  return rc;
}

void orc_ilu0_free(orc_ilu* f) {
  free(f->lrow); free(f->urow); free(f->lcol); free(f->ucol); free(f->lval); free(f->uval);
  memset(f, 0, sizeof(*f));
}

void orc_ilu0_apply(const orc_ilu* f, const double* r, double* out) {
  const int64_t n = f->n;
  for (int64_t i = 0; i < n; ++i) { /* L y = r (unit diagonal) */
    double acc = r[i];
    for (int64_t p = f->lrow[i]; p < f->lrow[i + 1]; ++p) acc -= f->lval[p] * out[f->lcol[p]];
    out[i] = acc;
  }
  for (int64_t i = n - 1; i >= 0; --i) { /* U x = y; u_ii is the row's first U entry */
    double acc = out[i];
    const int64_t p0 = f->urow[i];
    for (int64_t p = p0 + 1; p < f->urow[i + 1]; ++p) acc -= f->uval[p] * out[f->ucol[p]];
    out[i] = acc / f->uval[p0];
  }
}

/* Sec. 2.1 with Atilde = the ILU(0) factors: (L U)^{-1} r - 2 V (Lambda^{-1} (V^T r)) */
static void smw_ilu_apply(const orc_system* s, const double* r, double* out, double* t) {
  const int64_t n = s->n;
  for (int32_t j = 0; j < s->k; ++j) t[j] = dot(n, s->V + (int64_t)j * n, r);
  for (int32_t j = 0; j < s->k; ++j) t[j] = -2.0 * t[j] / s->lam[j];
  orc_ilu0_apply(s->ilu, r, out);
  for (int64_t i = 0; i < n; ++i)
    for (int32_t j = 0; j < s->k; ++j) out[i] += s->V[(int64_t)j * n + i] * t[j];
}

int orc_mcg_apply(const orc_system* s, int mcg, const double* r, double* out, double* work) {
  const int64_t n = s->n;
  double* d = work;
  double* t = work + n;
  if (mcg == ORC_MCG_ILU0 || mcg == ORC_MCG_SMW_ILU0) {
    if (!s->ilu) return ORC_ERR_INVALID;
    if (mcg == ORC_MCG_ILU0) orc_ilu0_apply(s->ilu, r, out);
    else smw_ilu_apply(s, r, out, t);
    return ORC_OK;
  }
  if (mcg == ORC_MCG_SMW) {
    const int rc = diag_a_inverse(s, d);
    if (rc != ORC_OK) return rc;
    smw_apply(s, d, r, out, t);
    return ORC_OK;
  }
  if (mcg == ORC_MCG_JACOBI) {
    orc_mmr_diag(s, d);
    for (int64_t i = 0; i < n; ++i) out[i] = r[i] / d[i];
    return ORC_OK;
  }
  for (int64_t i = 0; i < n; ++i) out[i] = r[i];
  return ORC_OK;
}

/* Preconditioned CG (Hestenes-Stiefel) on the SPD system M_mr z = y, Eq. 2,
 * with M_cg = I, Jacobi, or the MINRES-CG* preconditioner of Sec. 2.1.
 * Start z = 0, stop when ||r|| <= tol ||y||. */
int orc_cg(const orc_system* s, int mcg, const double* y, double* z, double tol, int64_t maxit,
           int64_t* iters, double* work) {
  const int64_t n = s->n;
  double* r = work;
  double* p = work + n;
  double* q = work + 2 * n;
  double* sv = work + 3 * n; /* M_cg^{-1} r */
  double* dinv = work + 4 * n;
  double* t = work + 5 * n;
  *iters = 0;
  const int fact = mcg == ORC_MCG_ILU0 || mcg == ORC_MCG_SMW_ILU0; /* M_cg^{-1} through the ILU(0) factors */
  if (fact && !s->ilu) return ORC_ERR_INVALID;
  if (mcg == ORC_MCG_SMW) {
    const int rc = diag_a_inverse(s, dinv);
    if (rc != ORC_OK) return rc;
  } else if (mcg == ORC_MCG_JACOBI) {
    orc_mmr_diag(s, dinv);
    for (int64_t i = 0; i < n; ++i) dinv[i] = 1.0 / dinv[i];
  } else {
    for (int64_t i = 0; i < n; ++i) dinv[i] = 1.0;
  }
  for (int64_t i = 0; i < n; ++i) {
    z[i] = 0.0;
    r[i] = y[i];
  }
  if (mcg == ORC_MCG_SMW) {
    smw_apply(s, dinv, r, sv, t);
  } else if (fact) {
    orc_mcg_apply(s, mcg, r, sv, dinv); /* dinv: scratch of n + k doubles here */
  } else {
    for (int64_t i = 0; i < n; ++i) sv[i] = dinv[i] * r[i];
  }
  for (int64_t i = 0; i < n; ++i) p[i] = sv[i];
  const double ynorm = nrm2(n, y);
  if (!isfinite(ynorm)) return ORC_ERR_NONFINITE;
  if (ynorm == 0.0) return ORC_OK;
  double rho = dot(n, r, sv);
  for (int64_t it = 0; it < maxit; ++it) {
    orc_mmr_apply(s, p, q, t, NULL);
    const double kappa = dot(n, p, q);
    if (!isfinite(kappa)) return ORC_ERR_NONFINITE;
    if (kappa <= 0.0) return ORC_ERR_NOT_SPD;
    const double alpha = rho / kappa;
    ORC_FOR
    for (int64_t i = 0; i < n; ++i) {
      z[i] += alpha * p[i];
      r[i] -= alpha * q[i];
    }
    *iters = it + 1;
    const double rnorm = nrm2(n, r);
    if (!isfinite(rnorm)) return ORC_ERR_NONFINITE;
    if (rnorm <= tol * ynorm) return ORC_OK;
    if (mcg == ORC_MCG_SMW) {
      smw_apply(s, dinv, r, sv, t);
    } else if (fact) {
      orc_mcg_apply(s, mcg, r, sv, dinv);
    } else {
      ORC_FOR
      for (int64_t i = 0; i < n; ++i) sv[i] = dinv[i] * r[i];
    }
    const double rho_new = dot(n, r, sv);
    if (!isfinite(rho_new)) return ORC_ERR_NONFINITE;
    if (rho_new == 0.0) return ORC_ERR_BREAKDOWN; /* r^T M_cg^{-1} r = 0 with r != 0: indefinite M_cg */
    const double beta = rho_new / rho;
    rho = rho_new;
    ORC_FOR
    for (int64_t i = 0; i < n; ++i) p[i] = sv[i] + beta * p[i];
  }
  return ORC_ERR_MAXITER;
}

double orc_true_relres(const orc_system* s, const double* b, const double* x, double* work) {
  orc_csr_spmv(s, x, work);
  for (int64_t i = 0; i < s->n; ++i) work[i] = b[i] - work[i];
  const double bn = nrm2(s->n, b);
  return bn == 0.0 ? nrm2(s->n, work) : nrm2(s->n, work) / bn;
}

/* Preconditioned MINRES [PaiS75], the outer iteration of Alg. 1.  Lanczos in
 * the P^{-1} inner product with unnormalised vectors v (z = P^{-1} v,
 * gamma = sqrt(z^T v)), QR of the tridiagonal by Givens rotations, and the
 * short recurrence for the search directions w.  Stopping test: the true
 * relative residual against the tolerance (Sec. 4.2). */
int orc_minres(const orc_system* s, const double* b, double* x, orc_prec_fn prec, void* prec_ctx,
               double outer_tol, int32_t max_outer, int64_t max_inner_total, double restart_factor,
               double* hist_relres, double* hist_eta, int32_t hist_cap, orc_info* info) {
  const int64_t n = s->n;
  memset(info, 0, sizeof(*info));
  double* mem = (double*)calloc((size_t)(9 * n + 1), sizeof(double));
  if (!mem) return ORC_ERR_INVALID;
  double* v_old = mem;
  double* v = mem + n;
  double* v_new = mem + 2 * n;
  double* z = mem + 3 * n;
  double* z_new = mem + 4 * n;
  double* w_old = mem + 5 * n;
  double* w = mem + 6 * n;
  double* az = mem + 7 * n; /* also used as the residual */
  double* w_new = mem + 8 * n;

  int status = ORC_ERR_MAXITER;
  const double bnorm = nrm2(n, b);
  if (!isfinite(bnorm)) { free(mem); info->status = ORC_ERR_NONFINITE; return ORC_ERR_NONFINITE; }
  if (bnorm == 0.0) {
    for (int64_t i = 0; i < n; ++i) x[i] = 0.0;
    free(mem);
    info->status = ORC_OK;
    return ORC_OK;
  }
  /* residual of the start vector */
  orc_csr_spmv(s, x, az);
  for (int64_t i = 0; i < n; ++i) az[i] = b[i] - az[i];
  double relres = nrm2(n, az) / bnorm;
  info->true_relres = relres;
  if (relres <= outer_tol) { free(mem); info->status = ORC_OK; return ORC_OK; }

  int32_t hist_n = 0;
  for (;;) { /* one restart cycle */
    double cyc_relres[4096];
    int32_t cyc_n = 0;
    /* v_1 = b - A x0, z_1 = P^{-1} v_1, gamma_1 = sqrt(z_1^T v_1) */
    for (int64_t i = 0; i < n; ++i) { v[i] = az[i]; v_old[i] = 0.0; w[i] = 0.0; w_old[i] = 0.0; }
    int64_t used = 0;
    int rc = prec(prec_ctx, n, v, z, max_inner_total - info->inner_iters_total, &used);
    info->inner_iters_total += used;
    info->prec_calls += 1;
    if (rc != ORC_OK) { status = rc; goto done; }
    double gamma2 = dot(n, z, v);
    if (!isfinite(gamma2)) { status = ORC_ERR_NONFINITE; goto done; }
    if (gamma2 <= 0.0) { status = ORC_ERR_BREAKDOWN; goto done; }
    double gamma = sqrt(gamma2), gamma_old = 1.0;
    double eta = gamma;
    double s_old = 0.0, s_cur = 0.0, c_old = 1.0, c_cur = 1.0;
    int restart = 0;
    while (!restart) {
      if (info->outer_iters >= max_outer) { status = ORC_ERR_MAXITER; goto done; }
      /* Lanczos step */
      ORC_FOR
      for (int64_t i = 0; i < n; ++i) z[i] /= gamma;
      orc_csr_spmv(s, z, az);
      const double delta = dot(n, z, az);
      ORC_FOR
      for (int64_t i = 0; i < n; ++i)
        v_new[i] = az[i] - (delta / gamma) * v[i] - (gamma / gamma_old) * v_old[i];
      rc = prec(prec_ctx, n, v_new, z_new, max_inner_total - info->inner_iters_total, &used);
      info->inner_iters_total += used;
      info->prec_calls += 1;
      if (rc != ORC_OK) { status = rc; goto done; }
      const double gamma_new2 = dot(n, z_new, v_new);
      if (!isfinite(gamma_new2)) { status = ORC_ERR_NONFINITE; goto done; }
      if (gamma_new2 < 0.0) { status = ORC_ERR_BREAKDOWN; goto done; }
      const double gamma_new = sqrt(gamma_new2);
      /* Givens rotations on the new column of the tridiagonal */
      const double a0 = c_cur * delta - c_old * s_cur * gamma;
      const double a1 = sqrt(a0 * a0 + gamma_new * gamma_new);
      const double a2 = s_cur * delta + c_old * c_cur * gamma;
      const double a3 = s_old * gamma;
      if (!(a1 > 0.0)) { status = ORC_ERR_BREAKDOWN; goto done; }
      const double c_new = a0 / a1;
      const double s_new = gamma_new / a1;
      /* direction and solution update */
      ORC_FOR
      for (int64_t i = 0; i < n; ++i) {
        w_new[i] = (z[i] - a3 * w_old[i] - a2 * w[i]) / a1;
        x[i] += c_new * eta * w_new[i];
      }
      eta = -s_new * eta;
      info->outer_iters += 1;
      /* true relative residual */
      orc_csr_spmv(s, x, az);
      for (int64_t i = 0; i < n; ++i) az[i] = b[i] - az[i];
      relres = nrm2(n, az) / bnorm;
      info->true_relres = relres;
      if (hist_n < hist_cap) {
        if (hist_relres) hist_relres[hist_n] = relres;
        if (hist_eta) hist_eta[hist_n] = fabs(eta);
      }
      hist_n++;
      if (!isfinite(relres)) { status = ORC_ERR_NONFINITE; goto done; }
      if (relres <= outer_tol) { status = ORC_OK; goto done; }
      if (cyc_n < 4096) cyc_relres[cyc_n] = relres;
      cyc_n++;
      if (restart_factor > 0.0 && cyc_n >= 4 && cyc_n <= 4096 &&
          relres > restart_factor * cyc_relres[cyc_n - 4])
        restart = 1;
      if (gamma_new == 0.0) restart = 1;
      /* shift the recurrences */
      double* tp;
      tp = v_old; v_old = v; v = v_new; v_new = tp;
      tp = z; z = z_new; z_new = tp;
      tp = w_old; w_old = w; w = w_new; w_new = tp;
      gamma_old = gamma; gamma = gamma_new;
      c_old = c_cur; c_cur = c_new;
      s_old = s_cur; s_cur = s_new;
    }
    info->restarts += 1; /* az holds b - A x: the next cycle starts from it */
  }
done:
  info->history_len = hist_n < hist_cap ? hist_n : hist_cap;
  info->status = status;
  free(mem);
  return status;
}

typedef struct {
  const orc_system* s;
  int mcg;
  double tol;
  double* work;
} cg_ctx;

static int cg_prec(void* ctx, int64_t n, const double* v, double* z, int64_t budget, int64_t* iters) {
  (void)n;
  cg_ctx* c = (cg_ctx*)ctx;
  if (budget <= 0) { *iters = 0; return ORC_ERR_MAXITER; }
  return orc_cg(c->s, c->mcg, v, z, c->tol, budget, iters, c->work);
}

/* Alg. 1: MINRES on A x = b with preconditioner M_mr, each application of
 * M_mr^{-1} done approximately by the inner CG. */
int orc_minres_cg(const orc_system* s, int mcg, const double* b, double* x, double outer_tol,
                  double inner_tol, int64_t max_iters, int32_t max_outer, double restart_factor,
                  double* hist_relres, double* hist_eta, int32_t hist_cap, orc_info* info) {
  cg_ctx c;
  c.s = s;
  c.mcg = mcg;
  c.tol = inner_tol;
  c.work = (double*)malloc(sizeof(double) * (size_t)(5 * s->n + s->k + 1));
  if (!c.work) return ORC_ERR_INVALID;
  int rc = orc_minres(s, b, x, cg_prec, &c, outer_tol, max_outer, max_iters, restart_factor,
                      hist_relres, hist_eta, hist_cap, info);
  free(c.work);
  return rc;
}

/* Sec. 1, 2x2 pivot blocks of the Bunch-Parlett factor: spectral
 * decomposition with the reflector R = [[c, s], [s, -c]] and replacement of
 * the eigenvalues by their absolute values. */
void orc_abs_2x2(double a, double b, double c, double* out, double* eig, double* rot) {
  double cs, sn, l1, l2;
  if (b == 0.0) {
    cs = 1.0; sn = 0.0; l1 = a; l2 = c;
  } else {
    const double mid = 0.5 * (a + c);
    const double rad = hypot(0.5 * (a - c), b);
    l1 = mid + rad;
    l2 = mid - rad;
    /* eigenvector of l1: the larger of the two row-based candidates */
    double x1 = b, y1 = l1 - a;   /* from row 1: (a-l1) x + b y = 0 */
    double x2 = l1 - c, y2 = b;   /* from row 2: b x + (c-l1) y = 0 */
    double n1 = hypot(x1, y1), n2 = hypot(x2, y2);
    if (n1 >= n2) { cs = x1 / n1; sn = y1 / n1; }
    else { cs = x2 / n2; sn = y2 / n2; }
  }
  const double m1 = fabs(l1), m2 = fabs(l2);
  /* R diag(m1, m2) R, R = [[cs, sn], [sn, -cs]] */
  out[0] = cs * cs * m1 + sn * sn * m2;
  out[1] = cs * sn * m1 - sn * cs * m2;
  out[2] = sn * sn * m1 + cs * cs * m2;
  if (eig) { eig[0] = l1; eig[1] = l2; }
  if (rot) { rot[0] = cs; rot[1] = sn; }
}
