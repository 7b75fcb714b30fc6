// Inner CG on M_mr z = y (Eq. 2, the inner block of Algorithm 1), one
// application of the preconditioner of the outer MINRES.
//
// One CG iteration is two streaming kernels (one grid-wide reduction each):
//   step_a: p' = s + beta p ; q = A p' + V c ; partials p'^T q and
//           V^T M_cg^{-1} (A p')  (the direction update is fused into the
//           SpMV gathers, so p' is never re-read; c = 2|Lambda| (V^T p')
//           arrives as scalars)
//   step_b: z += alpha p' ; r -= alpha q ; s = M_cg^{-1} r ;
//           partials r^T s (and r^T r when M_cg is Jacobi)
// The k numbers V^T s, V^T p' that the low-rank term needs come from exact
// recurrences instead of passes over V_hat:
//   V^T M_cg^{-1} q = V^T M_cg^{-1} (A p') + G c      (G = V^T M_cg^{-1} V)
//   V^T s_{i+1}    = V^T s_i - alpha V^T M_cg^{-1} q_i (s = M_cg^{-1} r)
//   V^T p'_{i+1}   = V^T s_{i+1} + beta V^T p'_i
// so V_hat is read once per iteration (in step a, for both V c and the
// partials) where the paper's M_mr product reads it twice (V^T u, then V t).
// All scalar recurrences (alpha, beta, the stopping test) run in FP64 in the
// last block of each kernel, which also publishes FP32 copies for the FP32
// kernels.  Per-thread sums and the block reductions run in the kernel's own
// precision (FP32 in mixed mode), the cross-block sum in FP64.
//
// The whole preconditioner application is one CUDA graph:
//   norm(v) -> init -> while(not done) { U x (step_a, step_b), ctl } -> finish
// The while loop is a conditional graph node: the inner iteration never
// returns to the host.
#pragma once

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace mrcg {

template <typename T>
struct CgArgs {
  DevState* st;
  double* partials;
  // SELL A in the inner precision
  const int64_t* slice_ptr;
  const int32_t* col;
  const int16_t* col16;  // col - row (16 bit) when it fits, else nullptr
  const T* val;
  int64_t nslices, n_pad;
  // low-rank term
  const T* V;  // n_pad x k column-major
  const uint16_t* Vbf;  // the same values as BF16 bits, streamed by variant 14 (else null)
  int k;
  // Jacobi: dinv != nullptr, s is a separate vector; identity: s == r
  const T* dinv;
  // MINRES-CG* (Sec. 2.1): 1 / diag(A) != nullptr, s = diag(A)^{-1} r - 2 V Lambda^{-1} V^T r
  // is a separate vector, and dinv is nullptr (step a then forms V^T (A p'))
  const T* dsmw;
  const double* gram;  // k x k V^T M_cg^{-1} V (row-major) of the kernels' V
  // staged step a: ring of shared-memory stages (bytes; region offsets inside a stage)
  int stages, stage_bytes, off_col, off_v, off_s, off_p, off_d, off_z;
  int stall_test;  // test hook: the producer stops after the first tile (waits then run out)
  // one-gather family: step b's partials (step a's are `partials`), the grids
  // that wrote them, and the parity of the iteration this launch belongs to
  double* partials_b;
  const double* partials_o;  // step a's partials of the other parity (the previous iteration's)
  int grid_a, grid_b, par;
  // one-kernel iteration: r and q ping-pong (r = r_{i-1} read, r_new written; q = q_i written, q_old read)
  T* r_new;
  T* q_old;
  // vectors
  T* z;
  T* r;
  T* s;
  T* p_old;
  T* p_new;
  T* q;
};

// ------------------------------------------------------------------ small helpers

template <typename T>
__device__ __forceinline__ T ld_stream(const T* p) {
  return __ldcs(p);
}

// ------------------------------------------------------------------ norm of v

static __global__ void __launch_bounds__(kThreads) cg_vnorm_kernel(DevState* st, double* partials, int64_t n_pad) {
  CgState& S = st->cg;
  const double* v = S.vin;
  double acc[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n_pad; i += (int64_t)gridDim.x * kThreads) {
    const double x = v[i];
    acc[0] += x * x;
  }
  block_partials<1>(acc, 1, partials);
  if (last_block_after_partials(&st->ticket)) {
    __shared__ double tot[1];
    final_sums(partials, 1, tot);
    if (threadIdx.x == 0) S.vnorm = sqrt(tot[0]);
  }
}

// ------------------------------------------------------------------ init

// Scalars of a new inner solve, once rho = r^T s, ||r|| and S.u = V^T s are known.
__device__ __forceinline__ void start_cg(CgState& S, int k, double vn, double rho, double rnorm) {
  S.rho = rho;
  S.alpha = 0.0;
  S.alpha32 = 0.0f;
  S.beta = 0.0;
  S.beta32 = 0.0f;
  S.fused_pending = 0;
  S.iters = 0;
  S.tol_abs = S.inner_tol * rnorm;
  S.maxit = S.budget;
  S.ctl_count = 0;
  {
    const long long per = S.unroll > 0 ? S.unroll : 1;
    const long long lim = (S.maxit > 0 ? S.maxit : 0) / per + 2;
    S.ctl_limit = (int)(lim < 0x7fffffffLL ? lim : 0x7fffffffLL);
  }
  S.done = kRunning;
  S.rho_s[0] = rho;
  S.it_s[0] = 0;
  S.bp_s[0] = S.bp_s[1] = 0;
  if (!isfinite(vn) || !isfinite(rho)) {
    S.done = kNonFinite;
  } else if (vn == 0.0 || rnorm == 0.0) {
    S.done = kConverged;
  } else if (S.maxit <= 0) {
    S.done = kMaxIter;
  }
  for (int l = 0; l < k; ++l) S.t[l] = S.u[l];
  publish_c(S, k);
  for (int l = 0; l < k; ++l) {  // iteration 0 of the one-gather family
    S.u_s[0][l] = S.u[l];
    S.t_s[0][l] = S.t[l];
    S.c_s[0][l] = S.c[l];
  }
}

template <typename T, int KB>
__global__ void __launch_bounds__(kThreads) cg_init_kernel(CgArgs<T> a) {
  constexpr int W = V16<T>::W;
  constexpr int KS = KB > 0 ? KB : 1;
  CgState& S = a.st->cg;
  const double vn = S.vnorm;
  const double scale = (vn > 0.0 && isfinite(vn)) ? 1.0 / vn : 0.0;
  const double* v = S.vin;
  const bool jac = a.dinv != nullptr;
  T rs = 0, rr = 0;
  T u[KS];
#pragma unroll
  for (int l = 0; l < KS; ++l) u[l] = 0;
  const T zero[W] = {};
  const int64_t nvec = a.n_pad / W;
  for (int64_t iv = blockIdx.x * (int64_t)kThreads + threadIdx.x; iv < nvec; iv += (int64_t)gridDim.x * kThreads) {
    const int64_t i = iv * W;
    T r[W], s[W];
#pragma unroll
    for (int e = 0; e < W; ++e) r[e] = (T)(v[i + e] * scale);
    st16(a.r + i, r);
    st16(a.z + i, zero);
    if (a.q_old) st16(a.q_old + i, zero);  // one-kernel iteration: q_{-1} = 0
    if (jac) {
      T d[W];
      ld16(a.dinv + i, d);
#pragma unroll
      for (int e = 0; e < W; ++e) s[e] = d[e] * r[e];
      if (a.s != a.r) st16(a.s + i, s);
    } else {
#pragma unroll
      for (int e = 0; e < W; ++e) s[e] = r[e];
    }
    // p_0 = s_0: variants 9-11 use it as their first direction; the others
    // form s + beta p with beta = 0, which is s again
    st16(a.p_old + i, s);
#pragma unroll
    for (int e = 0; e < W; ++e) {
      rs += r[e] * s[e];
      rr += r[e] * r[e];
    }
#pragma unroll
    for (int l = 0; l < KB; ++l)
      if (l < a.k) {
        T vv[W];
        ld16_stream(a.V + (size_t)l * a.n_pad + i, vv);
#pragma unroll
        for (int e = 0; e < W; ++e) u[l] += vv[e] * s[e];
      }
  }
  T acc[KB + 2];
  pack_slots<T, KB>(acc, rs, u, rr, a.k, jac);
  const int nv = a.k + 1 + (jac ? 1 : 0);
  block_partials_t<T, KB + 2>(acc, nv, a.partials);
  if (last_block_after_partials(&a.st->ticket)) {
    __shared__ double tot[KB + 2];
    final_sums(a.partials, nv, tot);
    if (threadIdx.x == 0) {
      const double rho = tot[0], rnorm = sqrt(jac ? tot[a.k + 1] : tot[0]);
      for (int l = 0; l < a.k; ++l) S.u[l] = tot[l + 1];
      start_cg(S, a.k, vn, rho, rnorm);
    }
  }
}

// ------------------------------------------------------------------ MINRES-CG* inner preconditioner
//
// Sec. 2.1: M_cg^{-1} = Atilde^{-1} - 2 V Lambda^{-1} V^T with Atilde = diag(A),
// so s = M_cg^{-1} r = diag(A)^{-1} r + V e,  e = -2 Lambda^{-1} (V^T r)
// = 4 (V^T r) / (2|lambda|).  V^T r follows the recurrence
// V^T r_{i+1} = V^T r_i - alpha V^T q_i (V^T q from step a), and
// V^T s = V^T diag(A)^{-1} r + (V^T V) e, so each V_hat entry is read once per
// iteration (in step b, which must form s explicitly for the next SpMV).

// e = 4 vr / lam2 in the kernel's precision, shared by the block
template <typename T, int KS>
__device__ __forceinline__ void smw_coeffs(const CgState& S, const double* vr, int k, T (&es)[KS]) {
  if ((int)threadIdx.x < KS) es[threadIdx.x] = ((int)threadIdx.x < k) ? (T)(4.0 * vr[threadIdx.x] / S.lam2[threadIdx.x]) : (T)0;
  __syncthreads();
}

// init, pass 1: r = v / ||v||, z = p = 0, and S.vr = V^T r
template <typename T, int KB>
__global__ void __launch_bounds__(kThreads) cg_init_smw_vr_kernel(CgArgs<T> a) {
  constexpr int W = V16<T>::W;
  constexpr int KS = KB > 0 ? KB : 1;
  CgState& S = a.st->cg;
  const double vn = S.vnorm;
  const double scale = (vn > 0.0 && isfinite(vn)) ? 1.0 / vn : 0.0;
  const double* v = S.vin;
  T u[KS];
#pragma unroll
  for (int l = 0; l < KS; ++l) u[l] = 0;
  const T zero[W] = {};
  const int64_t nvec = a.n_pad / W;
  for (int64_t iv = blockIdx.x * (int64_t)kThreads + threadIdx.x; iv < nvec; iv += (int64_t)gridDim.x * kThreads) {
    const int64_t i = iv * W;
    T r[W];
#pragma unroll
    for (int e = 0; e < W; ++e) r[e] = (T)(v[i + e] * scale);
    st16(a.r + i, r);
    st16(a.z + i, zero);
    st16(a.p_old + i, zero);
#pragma unroll
    for (int l = 0; l < KB; ++l)
      if (l < a.k) {
        T vv[W];
        ld16_stream(a.V + (size_t)l * a.n_pad + i, vv);
#pragma unroll
        for (int e = 0; e < W; ++e) u[l] += vv[e] * r[e];
      }
  }
  T acc[KS];
#pragma unroll
  for (int l = 0; l < KS; ++l) acc[l] = u[l];
  const int nv = a.k > 0 ? a.k : 1;
  block_partials_t<T, KS>(acc, nv, a.partials);
  if (last_block_after_partials(&a.st->ticket)) {
    __shared__ double tot[KS];
    final_sums(a.partials, nv, tot);
    if ((int)threadIdx.x < a.k) S.vr[threadIdx.x] = tot[threadIdx.x];
  }
}

// One pass over rows [i, i + W): s = diag(A)^{-1} r + V e, accumulating
// r^T s, r^T r and wd = V^T (diag(A)^{-1} r).
template <typename T, int KB, int W>
__device__ __forceinline__ void smw_rows(const CgArgs<T>& a, int64_t i, const T (&r)[W], const T* es, T& rs, T& rr,
                                         T (&wd)[KB > 0 ? KB : 1]) {
  T d[W], dr[W], s[W];
  ld16(a.dsmw + i, d);
#pragma unroll
  for (int e = 0; e < W; ++e) {
    dr[e] = d[e] * r[e];
    s[e] = dr[e];
  }
  // V rows in groups of G (FP64: four, the loads of a group in flight together)
  constexpr int G = sizeof(T) == 8 ? 4 : 1;
#pragma unroll
  for (int l0 = 0; l0 < KB; l0 += G) {
    T vv[G][W];
#pragma unroll
    for (int j = 0; j < G; ++j)
      if (l0 + j < KB && l0 + j < a.k) ld16_stream(a.V + (size_t)(l0 + j) * a.n_pad + i, vv[j]);
#pragma unroll
    for (int j = 0; j < G; ++j)
      if (l0 + j < KB && l0 + j < a.k) {
#pragma unroll
        for (int e = 0; e < W; ++e) {
          s[e] += vv[j][e] * es[l0 + j];
          wd[l0 + j] += vv[j][e] * dr[e];
        }
      }
  }
  st16(a.s + i, s);
#pragma unroll
  for (int e = 0; e < W; ++e) {
    rs += r[e] * s[e];
    rr += r[e] * r[e];
  }
}

// u = V^T s = wd + (V^T V) e: thread l of the last block, after final_sums
// left wd in tot[1 .. k] (G = V^T V is symmetric: column l)
__device__ __forceinline__ void smw_u(CgState& S, const double* gram, const double* tot, int k, const double* e) {
  const int l = threadIdx.x;
  if (l < k) {
    double u = tot[l + 1];
    for (int m = 0; m < k; ++m) u += gram[(size_t)m * k + l] * e[m];
    S.u[l] = u;
  }
}

// init, pass 2: s = M_cg^{-1} r and the scalars of the new solve
template <typename T, int KB>
__global__ void __launch_bounds__(kThreads) cg_init_smw_kernel(CgArgs<T> a) {
  constexpr int W = V16<T>::W;
  constexpr int KS = KB > 0 ? KB : 1;
  CgState& S = a.st->cg;
  __shared__ T es[KS];
  smw_coeffs<T, KS>(S, S.vr, a.k, es);
  T rs = 0, rr = 0;
  T wd[KS];
#pragma unroll
  for (int l = 0; l < KS; ++l) wd[l] = 0;
  const int64_t nvec = a.n_pad / W;
  for (int64_t iv = blockIdx.x * (int64_t)kThreads + threadIdx.x; iv < nvec; iv += (int64_t)gridDim.x * kThreads) {
    const int64_t i = iv * W;
    T r[W];
    ld16(a.r + i, r);
    smw_rows<T, KB, W>(a, i, r, es, rs, rr, wd);
  }
  T acc[KB + 2];
  pack_slots<T, KB>(acc, rs, wd, rr, a.k, true);
  const int nv = a.k + 2;
  block_partials_t<T, KB + 2>(acc, nv, a.partials);
  if (last_block_after_partials(&a.st->ticket)) {
    __shared__ double tot[KB + 2];
    __shared__ double ed[KS];
    final_sums(a.partials, nv, tot);
    if ((int)threadIdx.x < a.k) ed[threadIdx.x] = 4.0 * S.vr[threadIdx.x] / S.lam2[threadIdx.x];
    __syncthreads();
    smw_u(S, a.gram, tot, a.k, ed);
    __syncthreads();
    if (threadIdx.x == 0) start_cg(S, a.k, S.vnorm, tot[0], sqrt(tot[a.k + 1]));
  }
}

// step b with the MINRES-CG* M_cg: z += alpha p', r -= alpha q, s = M_cg^{-1} r
template <typename T, int KB>
__global__ void __launch_bounds__(kThreads) cg_step_b_smw_kernel(CgArgs<T> a) {
  constexpr int W = V16<T>::W;
  constexpr int KS = KB > 0 ? KB : 1;
  CgState& S = a.st->cg;
  if (S.done != kRunning) return;
  const T alpha = alpha_of(S, T(0));
  // V^T r_{i+1} = V^T r_i - alpha V^T q_i, formed alike in every block
  __shared__ double vr_new[KS];
  __shared__ T es[KS];
  if ((int)threadIdx.x < KS) vr_new[threadIdx.x] = ((int)threadIdx.x < a.k) ? S.vr[threadIdx.x] - S.alpha * S.vq[threadIdx.x] : 0.0;
  __syncthreads();
  smw_coeffs<T, KS>(S, vr_new, a.k, es);
  T rs = 0, rr = 0;
  T wd[KS];
#pragma unroll
  for (int l = 0; l < KS; ++l) wd[l] = 0;
  const int64_t nvec = a.n_pad / W;
  const int64_t stride = (int64_t)gridDim.x * kThreads;
  // FP64: two grid-stride chunks per trip, their vector loads issued together
  // (measured faster there; in FP32 one chunk per trip keeps more blocks resident)
  constexpr int U = sizeof(T) == 8 ? 2 : 1;
  for (int64_t iv0 = blockIdx.x * (int64_t)kThreads + threadIdx.x; iv0 < nvec; iv0 += U * stride) {
    T pn[U][W], qv[U][W], zv[U][W], rv[U][W];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t iv = iv0 + u * stride;
      if (iv < nvec) {
        const int64_t i = iv * W;
        ld16(a.p_new + i, pn[u]);
        ld16(a.q + i, qv[u]);
        ld16(a.z + i, zv[u]);
        ld16(a.r + i, rv[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t iv = iv0 + u * stride;
      if (iv >= nvec) continue;
      const int64_t i = iv * W;
#pragma unroll
      for (int e = 0; e < W; ++e) {
        zv[u][e] += alpha * pn[u][e];
        rv[u][e] -= alpha * qv[u][e];
      }
      st16(a.z + i, zv[u]);
      st16(a.r + i, rv[u]);
      smw_rows<T, KB, W>(a, i, rv[u], es, rs, rr, wd);
    }
  }
  T acc[KB + 2];
  pack_slots<T, KB>(acc, rs, wd, rr, a.k, true);
  const int nv = a.k + 2;
  block_partials_t<T, KB + 2>(acc, nv, a.partials);
  if (last_block_after_partials(&a.st->ticket)) {
    __shared__ double tot[KB + 2];
    __shared__ double ed[KS];
    final_sums(a.partials, nv, tot);
    if ((int)threadIdx.x < a.k) {
      S.vr[threadIdx.x] = vr_new[threadIdx.x];
      ed[threadIdx.x] = 4.0 * vr_new[threadIdx.x] / S.lam2[threadIdx.x];
    }
    __syncthreads();
    smw_u(S, a.gram, tot, a.k, ed);
    __syncthreads();
    if (threadIdx.x == 0) {
      const double rho_new = tot[0], rnorm = sqrt(tot[a.k + 1]);
      S.iters += 1;
      if (!isfinite(rho_new) || !isfinite(rnorm)) {
        S.done = kNonFinite;
      } else if (rnorm <= S.tol_abs) {
        S.done = kConverged;
      } else if (S.iters >= S.maxit) {
        S.done = kMaxIter;
      } else if (rho_new == 0.0) {
        S.done = kBreakdown;
      } else {
        const double beta = rho_new / S.rho;
        S.beta = beta;
        S.beta32 = (float)beta;
        S.rho = rho_new;
        for (int l = 0; l < a.k; ++l) S.t[l] = S.u[l] + beta * S.t[l];
        publish_c(S, a.k);
      }
    }
  }
}

// shared memory of one warp of the ILU(0) step b: the block's values, then the
// largest sweep image (when staged)
template <typename T>
__host__ __device__ inline size_t ilu_warp_bytes(const IluArgs& f) {
  return (size_t)f.bs * sizeof(T) + (size_t)f.img_bytes;
}

// ------------------------------------------------------------------ step b with the block-Jacobi ILU(0) M_cg
//
// The inner preconditioner of the paper's experiments (Sec. 4) is an
// incomplete LU factorisation of A; here its block-Jacobi form (ilu.cu): the
// factors of A's diagonal blocks of bs consecutive rows.  One warp owns a
// block: it applies the CG updates z += alpha p', r -= alpha q to the block's
// rows, solves L U s = r by a forward and a backward sweep over the block's
// levels with the block's values of r / s in shared memory (a warp barrier
// between levels), and stores s with the partials r^T s, r^T r and
// V^T (L U)^{-1} r.  V^T s is then direct (no recurrence): with M_cg^{-1} not
// diagonal, step a cannot form its share row by row.  With f.smw (MINRES-CG*,
// Sec. 2.1, Atilde = L U) s = (L U)^{-1} r + V e, e = -2 Lambda^{-1} V^T r,
// with V^T r by its recurrence and V^T s = V^T (L U)^{-1} r + (V^T V) e as in
// the diag(A) form.  init = 1: the first residual (alpha = 0) and start_cg.
// Launched with kThreads threads per CTA; warps 0 .. f.wpc-1 own blocks
// blockIdx.x * f.wpc + warp, the others only join the reduction.
template <typename T, int KB>
__global__ void __launch_bounds__(kThreads) cg_step_b_ilu_kernel(CgArgs<T> a, IluArgs f, int init) {
  constexpr int KS = KB > 0 ? KB : 1;
  extern __shared__ __align__(16) unsigned char ilu_smem[];
  CgState& S = a.st->cg;
  if (!init && S.done != kRunning) return;
  const T alpha = init ? (T)0 : alpha_of(S, T(0));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __shared__ double vr_new[KS];
  __shared__ T es[KS];
  if (f.smw) {
    if ((int)threadIdx.x < KS)
      vr_new[threadIdx.x] = ((int)threadIdx.x < a.k)
                                ? (init ? S.vr[threadIdx.x] : S.vr[threadIdx.x] - S.alpha * S.vq[threadIdx.x])
                                : 0.0;
    __syncthreads();
    smw_coeffs<T, KS>(S, vr_new, a.k, es);
  }
  T rs = 0, rr = 0;
  T wd[KS];
#pragma unroll
  for (int l = 0; l < KS; ++l) wd[l] = 0;
  const int blk = blockIdx.x * f.wpc + warp;
  if (warp < f.wpc && blk < f.nblk) {
    unsigned char* wmem = ilu_smem + (size_t)warp * ilu_warp_bytes<T>(f);
    T* x = reinterpret_cast<T*>(wmem);
    const int64_t b0 = (int64_t)blk * f.bs;
    const int m = (int)min((int64_t)f.bs, a.n_pad - b0);
    // CG updates of the block's rows; x = r, the right-hand side of the solve
    // (eight rows per lane in flight: one warp streams the whole block)
    constexpr int UR = 8;
    for (int r0 = lane; r0 < m; r0 += 32 * UR) {
      T rv[UR], zv[UR], pw[UR], qv[UR];
#pragma unroll
      for (int u = 0; u < UR; ++u) {
        const int r = r0 + 32 * u;
        if (r < m) {
          const int64_t i = b0 + r;
          rv[u] = a.r[i];
          if (!init) {
            zv[u] = a.z[i];
            pw[u] = a.p_new[i];
            qv[u] = a.q[i];
          }
        }
      }
#pragma unroll
      for (int u = 0; u < UR; ++u) {
        const int r = r0 + 32 * u;
        if (r < m) {
          const int64_t i = b0 + r;
          if (!init) {
            a.z[i] = zv[u] + alpha * pw[u];
            rv[u] -= alpha * qv[u];
            a.r[i] = rv[u];
          }
          x[r] = rv[u];
        }
      }
    }
    __syncwarp();
    if (f.img_bytes > 0) {  // sweeps from this block's images, copied into shared memory
      unsigned char* im = wmem + (size_t)f.bs * sizeof(T);
      for (int back = 0; back < 2; ++back) {
        const uint4* src = reinterpret_cast<const uint4*>(f.img + f.img_off[2 * (int64_t)blk + back]);
        const int4 hdr = __ldg(reinterpret_cast<const int4*>(src));
        const IluImage g = ilu_image_layout(hdr.x, hdr.y, hdr.z, (int)sizeof(T), back != 0);
        uint4* dst = reinterpret_cast<uint4*>(im);
        for (int c = lane; c < g.bytes / 16; c += 32) dst[c] = __ldg(src + c);
        __syncwarp();
        const uint16_t* lv = reinterpret_cast<const uint16_t*>(im + g.lv);
        const uint16_t* rw = reinterpret_cast<const uint16_t*>(im + g.rows);
        const uint16_t* en = reinterpret_cast<const uint16_t*>(im + g.ent);
        const uint16_t* cl = reinterpret_cast<const uint16_t*>(im + g.cols);
        const T* vl = reinterpret_cast<const T*>(im + g.vals);
        const T* di = reinterpret_cast<const T*>(im + g.dinv);
        for (int l = 0; l < hdr.y; ++l) {  // L y = r (unit diagonal), then U s = y
          for (int pos = lv[l] + lane; pos < lv[l + 1]; pos += 32) {
            const int row = rw[pos];
            T acc = x[row];
            for (int e = en[pos]; e < en[pos + 1]; ++e) acc -= vl[e] * x[cl[e]];
            x[row] = back ? acc * di[pos] : acc;
          }
          __syncwarp();
        }
      }
    } else {
      const T* fval = reinterpret_cast<const T*>(f.fval);
      for (int lv = f.fblk[blk]; lv < f.fblk[blk + 1]; ++lv) {  // L y = r (unit diagonal)
        for (int pos = f.flvl[lv] + lane; pos < f.flvl[lv + 1]; pos += 32) {
          const int row = f.frow[pos];
          T acc = x[row];
          for (int e = f.fent[pos]; e < f.fent[pos + 1]; ++e) acc -= fval[e] * x[f.fcol[e]];
          x[row] = acc;
        }
        __syncwarp();
      }
      const T* bval = reinterpret_cast<const T*>(f.bval);
      const T* bdinv = reinterpret_cast<const T*>(f.bdinv);
      for (int lv = f.bblk[blk]; lv < f.bblk[blk + 1]; ++lv) {  // U s = y
        for (int pos = f.blvl[lv] + lane; pos < f.blvl[lv + 1]; pos += 32) {
          const int row = f.brow[pos];
          T acc = x[row];
          for (int e = f.bent[pos]; e < f.bent[pos + 1]; ++e) acc -= bval[e] * x[f.bcol[e]];
          x[row] = acc * bdinv[pos];
        }
        __syncwarp();
      }
    }
    // s, its V_hat projections and the dot products (each lane rereads the
    // residual rows it wrote itself; UV rows per lane in flight)
    constexpr int UV = KB <= 12 ? 4 : (KB <= 24 ? 2 : 1);
    for (int r0 = lane; r0 < m; r0 += 32 * UV) {
      T rv[UV], vv[UV][KS];
#pragma unroll
      for (int u = 0; u < UV; ++u) {
        const int r = r0 + 32 * u;
        const int64_t i = b0 + (r < m ? r : 0);
        rv[u] = r < m ? a.r[i] : (T)0;
#pragma unroll
        for (int l = 0; l < KB; ++l) vv[u][l] = (r < m && l < a.k) ? a.V[(size_t)l * a.n_pad + i] : (T)0;
      }
#pragma unroll
      for (int u = 0; u < UV; ++u) {
        const int r = r0 + 32 * u;
        if (r < m) {
          const T xr = x[r];
          T sv = xr;
#pragma unroll
          for (int l = 0; l < KB; ++l)
            if (l < a.k) {
              wd[l] += vv[u][l] * xr;
              if (f.smw) sv += vv[u][l] * es[l];
            }
          a.s[b0 + r] = sv;
          rs += rv[u] * sv;
          rr += rv[u] * rv[u];
        }
      }
    }
  }
  T acc[KB + 2];
  pack_slots<T, KB>(acc, rs, wd, rr, a.k, true);
  const int nv = a.k + 2;
  block_partials_t<T, KB + 2>(acc, nv, a.partials);
  if (last_block_after_partials(&a.st->ticket)) {
    __shared__ double tot[KB + 2];
    __shared__ double ed[KS];
    final_sums(a.partials, nv, tot);
    if (f.smw) {
      if ((int)threadIdx.x < a.k) {
        S.vr[threadIdx.x] = vr_new[threadIdx.x];
        ed[threadIdx.x] = 4.0 * vr_new[threadIdx.x] / S.lam2[threadIdx.x];
      }
      __syncthreads();
      smw_u(S, a.gram, tot, a.k, ed);
    } else if ((int)threadIdx.x < a.k) {
      S.u[threadIdx.x] = tot[threadIdx.x + 1];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      const double rho_new = tot[0], rnorm = sqrt(tot[a.k + 1]);
      if (init) {
        start_cg(S, a.k, S.vnorm, rho_new, rnorm);
      } else {
        S.iters += 1;
        if (!isfinite(rho_new) || !isfinite(rnorm)) {
          S.done = kNonFinite;
        } else if (rnorm <= S.tol_abs) {
          S.done = kConverged;
        } else if (S.iters >= S.maxit) {
          S.done = kMaxIter;
        } else if (rho_new == 0.0) {
          S.done = kBreakdown;
        } else {
          const double beta = rho_new / S.rho;
          S.beta = beta;
          S.beta32 = (float)beta;
          S.rho = rho_new;
          for (int l = 0; l < a.k; ++l) S.t[l] = S.u[l] + beta * S.t[l];
          publish_c(S, a.k);
        }
      }
    }
  }
}

// ------------------------------------------------------------------ step a

// The entries of one slice row, 8 at a time: all value / index loads of a
// group are in flight before the gathers that depend on them.
template <typename T>
__device__ __forceinline__ T slice_row(const T* vp, const int32_t* cp, int w, const T* __restrict__ sv,
                                       const T* __restrict__ po, T beta) {
  T acc = 0;
  for (int j0 = 0; j0 < w; j0 += 8) {
    T av[8];
    int cc[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      av[j] = (j0 + j < w) ? ld_stream(vp + (size_t)(j0 + j) * kSlice) : (T)0;
      cc[j] = (j0 + j < w) ? ld_stream(cp + (size_t)(j0 + j) * kSlice) : 0;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (j0 + j < w) acc += av[j] * (__ldg(sv + cc[j]) + beta * __ldg(po + cc[j]));
  }
  return acc;
}

// The same with 16-bit column deltas (col = row + delta): half the index bytes.
template <typename T>
__device__ __forceinline__ T slice_row16(const T* vp, const int16_t* cp, int row, int w, const T* __restrict__ sv,
                                         const T* __restrict__ po, T beta) {
  T acc = 0;
  for (int j0 = 0; j0 < w; j0 += 8) {
    T av[8];
    int cc[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      av[j] = (j0 + j < w) ? ld_stream(vp + (size_t)(j0 + j) * kSlice) : (T)0;
      cc[j] = (j0 + j < w) ? row + (int)ld_stream(cp + (size_t)(j0 + j) * kSlice) : row;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (j0 + j < w) acc += av[j] * (__ldg(sv + cc[j]) + beta * __ldg(po + cc[j]));
  }
  return acc;
}

// Block partials of p'^T q and V^T M_cg^{-1} (A p'), then in the last block:
// kappa = p'^T q, alpha = rho / kappa and vq = V^T M_cg^{-1} (A p') + G c with
// the c the kernels applied.  G is fetched (all loads independent) before the
// cross-block sums, so its L2 latency overlaps theirs.  A block that met a
// stalled copy has set S.done already; the last block then leaves alpha alone.
template <typename T, int KB, int NW = kThreads / 32>
__device__ __forceinline__ void step_a_reduce(const CgArgs<T>& a, CgState& S, T dot, const T (&wq)[KB > 0 ? KB : 1],
                                              const T* cl) {
  constexpr int KS = KB > 0 ? KB : 1;
  T part[KB + 1];
  part[0] = dot;
#pragma unroll
  for (int l = 0; l < KB; ++l) part[l + 1] = wq[l];
  block_partials_t<T, KB + 1, NW>(part, a.k + 1, a.partials);
  if (last_block_after_partials(&a.st->ticket)) {
    constexpr int KK = KS * KS;
    constexpr int NT = NW * 32;
    constexpr int GPT = (KK + NT - 1) / NT;
    __shared__ double gs[KK];
    double greg[GPT];
    const int kk = a.k * a.k;
#pragma unroll
    for (int j = 0; j < GPT; ++j) {
      const int e = threadIdx.x + j * NT;
      greg[j] = (e < kk) ? __ldcg(a.gram + e) : 0.0;
    }
    __shared__ double tot[KB + 1];
    final_sums(a.partials, a.k + 1, tot);
#pragma unroll
    for (int j = 0; j < GPT; ++j) {
      const int e = threadIdx.x + j * NT;
      if (e < kk) gs[e] = greg[j];
    }
    __syncthreads();
    const int l = threadIdx.x;
    if (l < a.k) {
      // G is symmetric: column l, conflict-free shared reads
      double g = tot[l + 1];
#pragma unroll 8
      for (int m = 0; m < KB; ++m)
        if (m < a.k) g += gs[m * a.k + l] * (double)cl[m];
      S.vq[l] = g;
    }
    if (threadIdx.x == 0 && *(volatile int*)&S.done == kRunning) {
      const double kappa = tot[0];
      S.kappa = kappa;
      if (!isfinite(kappa)) {
        S.done = kNonFinite;
      } else if (kappa <= 0.0) {
        S.done = kNotSpd;
      } else {
        S.alpha = S.rho / kappa;
        S.alpha32 = (float)S.alpha;
      }
    }
  }
}

// Variants (picked per handle by the launch-shape autotuner):
//   VAR 0: V_hat row loads issued before the SpMV (more bytes in flight)
//   VAR 1: V_hat read after the SpMV (fewer registers: no V_hat row is kept)
//   VAR 2: two slices per warp per trip, V_hat early (more independent work)
//   VAR 3, 4: as VAR 1 with registers capped for 6 and 8 resident blocks per SM
//   (VAR 5, 6, 7: cg_step_a_staged_kernel below, registers capped for 2 / 4 blocks
//   per SM; 7 issues each warp's gathers one tile ahead)
//
// V^T M_cg^{-1} q splits exactly as V^T M_cg^{-1} (A p') + G c with the
// k x k Gram matrix G = V^T M_cg^{-1} V of the kernels' own V and M_cg^{-1}
// (formed once per handle).  The kernel therefore accumulates only
// V^T M_cg^{-1} (A p'), which is known before any V_hat entry of the row is
// touched, and each V_hat entry is used once and dropped; the last block
// adds G c.
template <typename T, int KB, int VAR>
__global__ void __launch_bounds__(kThreads, VAR == 3 ? 6 : (VAR == 4 ? 8 : 4)) cg_step_a_kernel(CgArgs<T> a) {
  constexpr int KS = KB > 0 ? KB : 1;
  constexpr int NSL = VAR == 2 ? 2 : 1;
  constexpr bool kEarlyV = VAR == 0 || VAR == 2;
  constexpr int VS = kEarlyV ? KS : 1;
  CgState& S = a.st->cg;
  if (S.done != kRunning) return;
  const T beta = beta_of(S, T(0));
  // c = 2|Lambda| (V^T p') staged in shared memory (broadcast reads, no registers)
  __shared__ T cl[KS];
  if (threadIdx.x < KS) cl[threadIdx.x] = ((int)threadIdx.x < a.k) ? c_of(S, threadIdx.x, T(0)) : (T)0;
  __syncthreads();
  const T* __restrict__ sv = a.s;
  const T* __restrict__ po = a.p_old;
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = (blockIdx.x * (int64_t)kThreads + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
  const bool jac = a.dinv != nullptr;
  T dot = 0;
  // wq[l] = (V^T M_cg^{-1} A p')_l: with this step b needs no pass over V (see step b)
  T wq[KS];
#pragma unroll
  for (int l = 0; l < KS; ++l) wq[l] = 0;
  for (int64_t sl0 = warp0 * NSL; sl0 < a.nslices; sl0 += nwarps * NSL) {
    T vrow[NSL][VS], srow[NSL], prow[NSL], drow[NSL], acc[NSL];
    int64_t rowv[NSL];
    bool ok[NSL];
#pragma unroll
    for (int h = 0; h < NSL; ++h) {
      const int64_t sl = sl0 + h;
      ok[h] = sl < a.nslices;
      rowv[h] = (ok[h] ? sl : sl0) * kSlice + lane;
      if constexpr (kEarlyV) {
#pragma unroll
        for (int l = 0; l < KS; ++l)
          vrow[h][l] = (ok[h] && l < a.k) ? ld_stream(a.V + (size_t)l * a.n_pad + rowv[h]) : (T)0;
      }
      srow[h] = sv[rowv[h]];
      prow[h] = po[rowv[h]];
      drow[h] = jac ? a.dinv[rowv[h]] : (T)1;
    }
#pragma unroll
    for (int h = 0; h < NSL; ++h) {
      if (!ok[h]) {
        acc[h] = 0;
        continue;
      }
      const int64_t sl = sl0 + h;
      const int64_t base = a.slice_ptr[sl];
      const int w = (int)((a.slice_ptr[sl + 1] - base) >> 5);
      acc[h] = a.col16 ? slice_row16<T>(a.val + base + lane, a.col16 + base + lane, (int)rowv[h], w, sv, po, beta)
                       : slice_row<T>(a.val + base + lane, a.col + base + lane, w, sv, po, beta);
    }
#pragma unroll
    for (int h = 0; h < NSL; ++h) {
      if (!ok[h]) continue;
      const int64_t row = rowv[h];
      const T pn = srow[h] + beta * prow[h];
      const T ap = acc[h];
      const T aps = jac ? drow[h] * ap : ap;  // (M_cg^{-1} A p')_row
      T q = ap;
      T vv[KS];  // this row of V_hat (the late loads are all issued before their first use)
#pragma unroll
      for (int l = 0; l < KS; ++l) {
        if constexpr (kEarlyV) vv[l] = vrow[h][l < VS ? l : 0];
        else vv[l] = (l < a.k) ? ld_stream(a.V + (size_t)l * a.n_pad + row) : (T)0;
      }
#pragma unroll
      for (int l = 0; l < KB; ++l)
        if (l < a.k) q += vv[l] * cl[l];
#pragma unroll
      for (int l = 0; l < KB; ++l)
        if (l < a.k) wq[l] += vv[l] * aps;
      a.q[row] = q;
      a.p_new[row] = pn;
      dot += pn * q;
    }
  }
  step_a_reduce<T, KB>(a, S, dot, wq, cl);
}

// ------------------------------------------------------------------ step a, staged
//
// The arithmetic of cg_step_a_kernel, with every streamed operand of a tile
// of 8 slices (256 rows) -- the tile's SELL values and indices, its rows of
// each V_hat column, of s, p and (Jacobi) M_cg^{-1} -- brought into shared
// memory by bulk copies (TMA), several tiles ahead: a ring of `stages`
// buffers, each with a "full" mbarrier (copies landed) and an "empty" one
// (every consumer warp has left it).  A producer warp issues the copies;
// eight consumer warps take one slice of each tile and never wait on each
// other.  Only the gathers s[col], p[col] of the SpMV go through the caches.
// The grid is persistent: block b takes tiles b, b + grid, ...
constexpr int kTileSlices = kThreads / 32;       // one consumer warp per slice
constexpr int kTileRows = kTileSlices * kSlice;
constexpr int kStagedThreads = kThreads + 32;    // consumer warps + one producer warp
constexpr int kMaxStages = 8;

template <typename T, bool FUSED, int TSL = kTileSlices>
__device__ __forceinline__ void issue_tile(const CgArgs<T>& a, unsigned char* b, uint64_t* bar, int64_t t, int64_t e0,
                                           int64_t e1, uint64_t stream_pol) {
  constexpr int TR = TSL * kSlice;  // rows of a tile
  const bool jac = !FUSED && a.dinv != nullptr;
  const int ib = a.col16 ? 2 : 4;
  const char* idx = a.col16 ? (const char*)a.col16 : (const char*)a.col;
  const int64_t s0 = t * TSL, s1 = min(s0 + TSL, a.nslices);
  const int64_t row0 = s0 * kSlice;
  const uint32_t rb = (uint32_t)((s1 - s0) * kSlice * (int64_t)sizeof(T));
  const uint32_t ne = (uint32_t)(e1 - e0);
  const int own = FUSED ? 4 : 2 + (jac ? 1 : 0);  // own-row vectors staged per tile
  mbar_arrive_expect_tx(bar, ne * (uint32_t)(sizeof(T) + ib) + (uint32_t)(a.k + own) * rb);
  // the matrix and V_hat are read once per pass: evict-first in L2
  if (ne > 0) {
    bulk_g2s_hint(b, a.val + e0, ne * (uint32_t)sizeof(T), bar, stream_pol);
    bulk_g2s_hint(b + a.off_col, idx + e0 * ib, ne * (uint32_t)ib, bar, stream_pol);
  }
  for (int l = 0; l < a.k; ++l)
    bulk_g2s_hint(b + a.off_v + (size_t)l * TR * sizeof(T), a.V + (size_t)l * a.n_pad + row0, rb, bar,
                  stream_pol);
  if constexpr (FUSED) {
    bulk_g2s(b + a.off_s, a.r + row0, rb, bar);
    bulk_g2s(b + a.off_p, a.p_old + row0, rb, bar);
    bulk_g2s(b + a.off_d, a.q_old + row0, rb, bar);
    bulk_g2s(b + a.off_z, a.z + row0, rb, bar);
  } else {
    bulk_g2s(b + a.off_s, a.s + row0, rb, bar);
    bulk_g2s(b + a.off_p, a.p_old + row0, rb, bar);
    if (jac) bulk_g2s(b + a.off_d, a.dinv + row0, rb, bar);
  }
}

// The producer lane of a staged kernel: refills a stage as soon as every
// consumer warp has left it (tile offsets fetched one tile ahead), then waits
// (bounded) until no copy it issued is still writing this block's shared
// memory.  Tile i of this block is tile blockIdx.x + i * gridDim.x.
template <typename T, bool FUSED, int TSL = kTileSlices>
__device__ __forceinline__ void stage_producer(const CgArgs<T>& a, unsigned char* stage_mem, uint64_t* full,
                                               uint64_t* empty, int* stalled, int64_t ntl, int nst) {
  const int64_t G = gridDim.x;
  const uint64_t stream_pol = l2_evict_first_policy();
  int64_t issued = 0;
  int64_t e0 = 0, e1 = 0;
  if (ntl > 0) {
    e0 = a.slice_ptr[(int64_t)blockIdx.x * TSL];
    e1 = a.slice_ptr[min((int64_t)(blockIdx.x + 1) * TSL, a.nslices)];
  }
  // stage st of tile i = i mod nst, and the parity of its use (i / nst) & 1,
  // kept incrementally (no integer division in the loop)
  int st = 0;
  uint32_t ph = 0;
  int64_t t = blockIdx.x;
  for (int64_t i = 0; i < ntl; ++i, t += G) {
    if (a.stall_test && i >= 1) break;
    if (i >= nst && !mbar_wait_or_abort(&empty[st], ph ^ 1u, stalled)) break;
    const int64_t c0 = e0, c1 = e1;
    if (i + 1 < ntl) {
      e0 = a.slice_ptr[(t + G) * TSL];
      e1 = a.slice_ptr[min((t + G + 1) * TSL, a.nslices)];
    }
    fence_proxy_async_smem();
    issue_tile<T, FUSED, TSL>(a, stage_mem + (size_t)st * a.stage_bytes, &full[st], t, c0, c1, stream_pol);
    ++issued;
    if (++st == nst) {
      st = 0;
      ph ^= 1u;
    }
  }
  for (int64_t j = issued > nst ? issued - nst : 0; j < issued; ++j)
    mbar_wait(&full[j % nst], (uint32_t)((j / nst) & 1));
}

// ------------------------------------------------------------------ one-kernel CG iteration (variant 8)
//
// With M_cg = I the two kernels of a CG iteration fold into one.  Iteration i
// starts from alpha_{i-1}, beta_{i-1} and c_i (set by the last block of
// iteration i-1) and forms, for its own rows,
//   r_i = r_{i-1} - alpha_{i-1} q_{i-1},  z_i = z_{i-1} + alpha_{i-1} p_{i-1},
//   p_i = r_i + beta_{i-1} p_{i-1},
// while its SpMV rebuilds p_i at every column it gathers from r_{i-1},
// q_{i-1} and p_{i-1}, so no grid-wide step separates the vector updates from
// the product q_i = A p_i + V c_i.  The reduction gives p_i^T q_i,
// r_i^T q_i, q_i^T q_i, rho_i = r_i^T r_i and V^T A p_i; the last block sets
// alpha_i = rho_i / p_i^T q_i and
//   rho_{i+1} = ||r_i - alpha_i q_i||^2 = rho_i - 2 alpha_i r_i^T q_i + alpha_i^2 q_i^T q_i
// (exact algebra from fresh dot products, so rounding does not carry from one
// estimate to the next) for the stopping test and beta_i.  r and q ping-pong
// between two buffers (they are gathered while rewritten); the last z update
// is left to the finish kernel.

// A p_i of a slice row for the one-kernel iteration: p_i at each column is
// rebuilt from the gathered r_{i-1}, q_{i-1}, p_{i-1} (8 entries in flight)
template <typename T, typename I>
__device__ __forceinline__ T fused_row(const T* vp, const I* cp, int row, bool delta, int w, const T* __restrict__ ro,
                                       const T* __restrict__ qo, const T* __restrict__ po, T alpha, T beta) {
  T acc = 0;
  for (int j0 = 0; j0 < w; j0 += 8) {
    T av[8];
    int cc[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      av[j] = (j0 + j < w) ? vp[(j0 + j) * kSlice] : (T)0;
      cc[j] = (j0 + j < w) ? (delta ? row : 0) + (int)cp[(j0 + j) * kSlice] : row;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (j0 + j < w) {
        const T rn = __ldg(ro + cc[j]) - alpha * __ldg(qo + cc[j]);
        acc += av[j] * (rn + beta * __ldg(po + cc[j]));
      }
  }
  return acc;
}

// Last block of the one-kernel iteration (M_cg = I: s = r).  rho_i = r_i^T r_i
// is the fresh dot product of this iteration (it sets alpha_i and is the base
// of the expansion, so the expansion's rounding never accumulates); rho_{i+1}
// by expansion gives the stopping test and beta_i; then the V^T recurrences.
template <typename T, int KB, int NW>
__device__ __forceinline__ void fused_reduce(const CgArgs<T>& a, CgState& S, T pq, T rq, T qq, T rr,
                                             const T (&wq)[KB > 0 ? KB : 1], const T* cl) {
  constexpr int KS = KB > 0 ? KB : 1;
  T part[KB + 4];
  part[0] = pq;
  part[1] = rq;
  part[2] = qq;
  part[3] = rr;
#pragma unroll
  for (int l = 0; l < KB; ++l) part[l + 4] = wq[l];
  block_partials_t<T, KB + 4, NW>(part, a.k + 4, a.partials);
  if (last_block_after_partials(&a.st->ticket)) {
    constexpr int KK = KS * KS;
    constexpr int NT = NW * 32;
    constexpr int GPT = (KK + NT - 1) / NT;
    __shared__ double gs[KK];
    double greg[GPT];
    const int kk = a.k * a.k;
#pragma unroll
    for (int j = 0; j < GPT; ++j) {
      const int e = threadIdx.x + j * NT;
      greg[j] = (e < kk) ? __ldcg(a.gram + e) : 0.0;
    }
    __shared__ double tot[KB + 4];
    final_sums(a.partials, a.k + 4, tot);
#pragma unroll
    for (int j = 0; j < GPT; ++j) {
      const int e = threadIdx.x + j * NT;
      if (e < kk) gs[e] = greg[j];
    }
    __syncthreads();
    const int l = threadIdx.x;
    if (l < a.k) {  // V^T q_i = V^T A p_i + (V^T V) c_i
      double g = tot[l + 4];
#pragma unroll 8
      for (int m = 0; m < KB; ++m)
        if (m < a.k) g += gs[m * a.k + l] * (double)cl[m];
      S.vq[l] = g;
    }
    __syncthreads();
    if (threadIdx.x == 0 && *(volatile int*)&S.done == kRunning) {
      const double kappa = tot[0], rho = tot[3];
      S.kappa = kappa;
      if (!isfinite(kappa) || !isfinite(rho)) {
        S.done = kNonFinite;
      } else if (sqrt(rho) <= S.tol_abs) {
        // the fresh ||r_i|| already meets the test (the previous iteration's
        // expansion was below its rounding floor, so it did not stop there):
        // z_i is complete, nothing is pending
        S.done = kConverged;
      } else if (kappa <= 0.0) {
        S.done = kNotSpd;
      } else {
        const double alpha = rho / kappa;
        const double aqq = alpha * alpha * tot[2];
        const double rho_new = rho - 2.0 * alpha * tot[1] + aqq;
        // the expansion cancels O(rho + alpha^2 q^T q) terms computed in the
        // kernel's precision; below this floor its value (and its sign) is
        // rounding noise and must not end the solve
        constexpr double kEpsT = sizeof(T) == 4 ? 5.9604644775390625e-08 : 1.1102230246251565e-16;
        const bool reliable = rho_new > 32.0 * kEpsT * (rho + aqq);
        S.alpha = alpha;
        S.alpha32 = (float)alpha;
        S.iters += 1;
        // z_{i+1} = z_i + alpha_i p_i is done by the next iteration, or by
        // the finish kernel when this one ends the solve
        S.fused_pending = 1;
        S.p_last = a.p_new;
        const double rnorm = sqrt(rho_new > 0.0 ? rho_new : 0.0);
        if (!isfinite(rho_new)) {
          S.done = kNonFinite;
        } else if (reliable && rnorm <= S.tol_abs) {
          S.done = kConverged;
        } else if (S.iters >= S.maxit) {
          S.done = kMaxIter;
        } else {
          // an unreliable expansion continues with beta >= 0 near zero (a
          // steepest-descent step); the next iteration tests its fresh ||r||
          S.fused_pending = 0;
          const double beta = (rho_new > 0.0 ? rho_new : 0.0) / rho;
          S.beta = beta;
          S.beta32 = (float)beta;
          S.rho = rho_new;
          for (int m = 0; m < a.k; ++m) {
            S.u[m] -= alpha * S.vq[m];
            S.t[m] = S.u[m] + beta * S.t[m];
          }
          publish_c(S, a.k);
        }
      }
    }
  }
}

// entries of one slice row from a staged tile: values and indices in shared
// memory, the gathered s, p from global memory (8 gathers in flight)
template <typename T, typename I>
__device__ __forceinline__ T staged_row(const T* vp, const I* cp, int row, bool delta, int w,
                                        const T* __restrict__ sv, const T* __restrict__ po, T beta) {
  T acc = 0;
  for (int j0 = 0; j0 < w; j0 += 8) {
    T av[8];
    int cc[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      av[j] = (j0 + j < w) ? vp[(j0 + j) * kSlice] : (T)0;
      cc[j] = (j0 + j < w) ? (delta ? row : 0) + (int)cp[(j0 + j) * kSlice] : row;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (j0 + j < w) acc += av[j] * (__ldg(sv + cc[j]) + beta * __ldg(po + cc[j]));
  }
  return acc;
}

// The first eight entries of a slice row: gathers s[col], p[col] issued into
// registers (the pipelined consumers issue them one tile ahead of their use).
template <typename T, typename I>
__device__ __forceinline__ void gather8(const I* cp, int row, bool delta, int w, const T* __restrict__ sv,
                                        const T* __restrict__ po, T (&gs)[8], T (&gp)[8]) {
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int c = (j < w) ? (delta ? row : 0) + (int)cp[j * kSlice] : row;
    gs[j] = (j < w) ? __ldg(sv + c) : (T)0;
    gp[j] = (j < w) ? __ldg(po + c) : (T)0;
  }
}

// A p' of a slice row from its first eight gathered pairs plus the rest of the row
template <typename T, typename I>
__device__ __forceinline__ T finish_row(const T* vp, const I* cp, int row, bool delta, int w, const T (&gs)[8],
                                        const T (&gp)[8], const T* __restrict__ sv, const T* __restrict__ po, T beta) {
  T acc = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j)
    if (j < w) acc += vp[j * kSlice] * (gs[j] + beta * gp[j]);
  if (w > 8) acc += staged_row<T, I>(vp + 8 * kSlice, cp + 8 * kSlice, row, delta, w - 8, sv, po, beta);
  return acc;
}

template <typename T, int KB, int MB, bool PIPE, bool FUSED = false>
__global__ void __launch_bounds__(kStagedThreads, MB) cg_step_a_staged_kernel(CgArgs<T> a) {
  constexpr int KS = KB > 0 ? KB : 1;
  extern __shared__ __align__(128) unsigned char stage_mem[];
  __shared__ __align__(8) uint64_t full[kMaxStages];   // tile landed (1 arrival + bytes)
  __shared__ __align__(8) uint64_t empty[kMaxStages];  // all consumer warps left the tile
  __shared__ int stalled;
  __shared__ T cl[KS];
  CgState& S = a.st->cg;
  if (S.done != kRunning) return;
  const T beta = beta_of(S, T(0));
  if (threadIdx.x < KS) cl[threadIdx.x] = ((int)threadIdx.x < a.k) ? c_of(S, threadIdx.x, T(0)) : (T)0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool jac = a.dinv != nullptr;
  const int nst = a.stages;
  const int64_t ntiles = (a.nslices + kTileSlices - 1) / kTileSlices;
  const int64_t ntl = (int64_t)blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t G = gridDim.x;
  if (threadIdx.x == 0) {
    for (int i = 0; i < nst; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], kTileSlices);
    }
    stalled = 0;
    mbar_init_fence();
  }
  __syncthreads();
  T dot = 0, rq = 0, qq = 0, rr = 0;
  T wq[KS];
#pragma unroll
  for (int l = 0; l < KS; ++l) wq[l] = 0;
  if (warp == kTileSlices) {
    if (lane == 0) stage_producer<T, FUSED>(a, stage_mem, full, empty, &stalled, ntl, nst);
  } else if constexpr (FUSED) {
    // consumer warps of the one-kernel iteration (M_cg = I): warp w takes slice w of every tile
    const T alpha = alpha_of(S, T(0));
    const T* __restrict__ ro = a.r;
    const T* __restrict__ qo = a.q_old;
    const T* __restrict__ po = a.p_old;
    int64_t c_t0 = 0, c_s0 = 0, c_s1 = 0;
    if (ntl > 0) {
      const int64_t sl = blockIdx.x * (int64_t)kTileSlices + warp;
      c_t0 = a.slice_ptr[blockIdx.x * (int64_t)kTileSlices];
      if (sl < a.nslices) {
        c_s0 = a.slice_ptr[sl];
        c_s1 = a.slice_ptr[sl + 1];
      }
    }
    int st = 0;
    uint32_t ph = 0;
    int64_t t = blockIdx.x;
    for (int64_t i = 0; i < ntl; ++i, t += G) {
      const int64_t sl = t * kTileSlices + warp;
      const int64_t t0 = c_t0, s0 = c_s0, s1 = c_s1;
      if (i + 1 < ntl) {
        const int64_t tn = t + G, sln = tn * kTileSlices + warp;
        c_t0 = a.slice_ptr[tn * kTileSlices];
        if (sln < a.nslices) {
          c_s0 = a.slice_ptr[sln];
          c_s1 = a.slice_ptr[sln + 1];
        }
      }
      if (!mbar_wait_or_abort(&full[st], ph, &stalled)) break;
      if (sl < a.nslices) {
        const unsigned char* b = stage_mem + (size_t)st * a.stage_bytes;
        const int off = (int)(s0 - t0) + lane;
        const int w = (int)((s1 - s0) >> 5);
        const int r = warp * kSlice + lane;
        const int64_t row = sl * kSlice + lane;
        const T* vp = reinterpret_cast<const T*>(b) + off;
        const T ap = a.col16 ? fused_row<T, int16_t>(vp, reinterpret_cast<const int16_t*>(b + a.off_col) + off,
                                                     (int)row, true, w, ro, qo, po, alpha, beta)
                             : fused_row<T, int32_t>(vp, reinterpret_cast<const int32_t*>(b + a.off_col) + off,
                                                     (int)row, false, w, ro, qo, po, alpha, beta);
        const T r_old = reinterpret_cast<const T*>(b + a.off_s)[r];
        const T p_old = reinterpret_cast<const T*>(b + a.off_p)[r];
        const T q_old = reinterpret_cast<const T*>(b + a.off_d)[r];
        const T z_old = reinterpret_cast<const T*>(b + a.off_z)[r];
        const T rn = r_old - alpha * q_old;  // r_i
        const T pn = rn + beta * p_old;      // p_i
        const T* vt = reinterpret_cast<const T*>(b + a.off_v) + r;
        T q = ap;
#pragma unroll
        for (int l = 0; l < KB; ++l)
          if (l < a.k) {
            const T v = vt[l * kTileRows];
            q += v * cl[l];
            wq[l] += v * ap;
          }
        a.q[row] = q;
        a.p_new[row] = pn;
        a.r_new[row] = rn;
        a.z[row] = z_old + alpha * p_old;
        dot += pn * q;
        rq += rn * q;
        qq += q * q;
        rr += rn * rn;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[st]);
      if (++st == nst) {
        st = 0;
        ph ^= 1u;
      }
    }
  } else if constexpr (PIPE) {
    // consumer warps, software-pipelined: while a warp finishes its slice of
    // tile i it already has the gathers of its slice of tile i + 1 in flight
    // (the tile's stage is waited for first), so gather latency overlaps
    // the V_hat products, stores and sums of the tile before
    const T* __restrict__ sv = a.s;
    const T* __restrict__ po = a.p_old;
    const bool d16 = a.col16 != nullptr;
    int st = 0;
    uint32_t ph = 0;
    int64_t t = blockIdx.x;
    // offsets of this warp's slice: tile i (cur_*) and the next tile (c_*, fetched ahead)
    int cur_off = 0, cur_w = 0;
    int64_t c_t0 = 0, c_s0 = 0, c_s1 = 0;
    T gs[8], gp[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) gs[j] = gp[j] = 0;
    auto offsets = [&](int64_t tt) {
      const int64_t sl = tt * kTileSlices + warp;
      c_t0 = a.slice_ptr[tt * kTileSlices];
      if (sl < a.nslices) {
        c_s0 = a.slice_ptr[sl];
        c_s1 = a.slice_ptr[sl + 1];
      } else {
        c_s0 = c_s1 = c_t0;
      }
    };
    // the gathers of this warp's slice of tile tt (stage sst, landed)
    auto start = [&](int64_t tt, int sst, T (&g1)[8], T (&g2)[8]) {
      const int64_t sl = tt * kTileSlices + warp;
      cur_off = (int)(c_s0 - c_t0) + lane;
      cur_w = (int)((c_s1 - c_s0) >> 5);
      if (sl < a.nslices) {
        const unsigned char* b = stage_mem + (size_t)sst * a.stage_bytes;
        const int row = (int)(sl * kSlice + lane);
        if (d16) gather8<T, int16_t>(reinterpret_cast<const int16_t*>(b + a.off_col) + cur_off, row, true, cur_w, sv,
                                     po, g1, g2);
        else gather8<T, int32_t>(reinterpret_cast<const int32_t*>(b + a.off_col) + cur_off, row, false, cur_w, sv, po,
                                 g1, g2);
      }
    };
    bool alive = true;
    if (ntl > 0) {
      offsets(t);
      alive = mbar_wait_or_abort(&full[0], 0u, &stalled);
      if (alive) start(t, 0, gs, gp);
      if (ntl > 1) offsets(t + G);
    }
    for (int64_t i = 0; alive && i < ntl; ++i, t += G) {
      const int off = cur_off, w = cur_w;
      const int stn = st + 1 == nst ? 0 : st + 1;
      const uint32_t phn = st + 1 == nst ? ph ^ 1u : ph;
      T gsn[8], gpn[8];
      if (i + 1 < ntl) {
        if (!mbar_wait_or_abort(&full[stn], phn, &stalled)) break;
        start(t + G, stn, gsn, gpn);
        if (i + 2 < ntl) offsets(t + 2 * G);
      }
      const int64_t sl = t * kTileSlices + warp;
      if (sl < a.nslices) {
        const unsigned char* b = stage_mem + (size_t)st * a.stage_bytes;
        const int r = warp * kSlice + lane;
        const int64_t row = sl * kSlice + lane;
        const T* vp = reinterpret_cast<const T*>(b) + off;
        const T ap = d16 ? finish_row<T, int16_t>(vp, reinterpret_cast<const int16_t*>(b + a.off_col) + off, (int)row,
                                                  true, w, gs, gp, sv, po, beta)
                         : finish_row<T, int32_t>(vp, reinterpret_cast<const int32_t*>(b + a.off_col) + off, (int)row,
                                                  false, w, gs, gp, sv, po, beta);
        const T pn =
            reinterpret_cast<const T*>(b + a.off_s)[r] + beta * reinterpret_cast<const T*>(b + a.off_p)[r];
        const T aps = jac ? reinterpret_cast<const T*>(b + a.off_d)[r] * ap : ap;
        const T* vt = reinterpret_cast<const T*>(b + a.off_v) + r;
        T q = ap;
#pragma unroll
        for (int l = 0; l < KB; ++l)
          if (l < a.k) {
            const T v = vt[l * kTileRows];
            q += v * cl[l];
            wq[l] += v * aps;
          }
        a.q[row] = q;
        a.p_new[row] = pn;
        dot += pn * q;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[st]);
      if (i + 1 < ntl) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          gs[j] = gsn[j];
          gp[j] = gpn[j];
        }
      }
      st = stn;
      ph = phn;
    }
  } else {
    // consumer warps: warp w takes slice w of every tile
    int64_t c_t0 = 0, c_s0 = 0, c_s1 = 0;
    if (ntl > 0) {
      const int64_t sl = blockIdx.x * (int64_t)kTileSlices + warp;
      c_t0 = a.slice_ptr[blockIdx.x * (int64_t)kTileSlices];
      if (sl < a.nslices) {
        c_s0 = a.slice_ptr[sl];
        c_s1 = a.slice_ptr[sl + 1];
      }
    }
    const T* __restrict__ sv = a.s;
    const T* __restrict__ po = a.p_old;
    int st = 0;
    uint32_t ph = 0;
    int64_t t = blockIdx.x;
    for (int64_t i = 0; i < ntl; ++i, t += G) {
      const int64_t sl = t * kTileSlices + warp;
      const int64_t t0 = c_t0, s0 = c_s0, s1 = c_s1;
      if (i + 1 < ntl) {
        const int64_t tn = t + G, sln = tn * kTileSlices + warp;
        c_t0 = a.slice_ptr[tn * kTileSlices];
        if (sln < a.nslices) {
          c_s0 = a.slice_ptr[sln];
          c_s1 = a.slice_ptr[sln + 1];
        }
      }
      if (!mbar_wait_or_abort(&full[st], ph, &stalled)) break;
      if (sl < a.nslices) {
        const unsigned char* b = stage_mem + (size_t)st * a.stage_bytes;
        const int off = (int)(s0 - t0) + lane;
        const int w = (int)((s1 - s0) >> 5);
        const int r = warp * kSlice + lane;
        const int64_t row = sl * kSlice + lane;
        const T* vp = reinterpret_cast<const T*>(b) + off;
        const T ap = a.col16 ? staged_row<T, int16_t>(vp, reinterpret_cast<const int16_t*>(b + a.off_col) + off,
                                                      (int)row, true, w, sv, po, beta)
                             : staged_row<T, int32_t>(vp, reinterpret_cast<const int32_t*>(b + a.off_col) + off,
                                                      (int)row, false, w, sv, po, beta);
        const T pn =
            reinterpret_cast<const T*>(b + a.off_s)[r] + beta * reinterpret_cast<const T*>(b + a.off_p)[r];
        const T aps = jac ? reinterpret_cast<const T*>(b + a.off_d)[r] * ap : ap;  // (M_cg^{-1} A p')_row
        const T* vt = reinterpret_cast<const T*>(b + a.off_v) + r;
        T q = ap;
#pragma unroll
        for (int l = 0; l < KB; ++l)
          if (l < a.k) {
            const T v = vt[l * kTileRows];
            q += v * cl[l];
            wq[l] += v * aps;
          }
        a.q[row] = q;
        a.p_new[row] = pn;
        dot += pn * q;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[st]);
      if (++st == nst) {
        st = 0;
        ph ^= 1u;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && stalled) *(volatile int*)&S.done = kStall;
  if constexpr (FUSED) fused_reduce<T, KB, kStagedThreads / 32>(a, S, dot, rq, qq, rr, wq, cl);
  else step_a_reduce<T, KB, kStagedThreads / 32>(a, S, dot, wq, cl);
}

// ------------------------------------------------------------------ step a / step b with one gather per entry
//
// Variants 9-11 (M_cg = I or Jacobi) keep the next direction p explicit so
// that the SpMV gathers one vector instead of rebuilding p' = s + beta p at
// every gathered column.  That needs beta before step b, and step a has it:
// its reduction also forms s^T q and q^T M_cg^{-1} q, and with the fresh
// rho_i = r_i^T s_i of step b
//   rho_{i+1} = (r - alpha q)^T M_cg^{-1} (r - alpha q)
//             = rho_i - 2 alpha s^T q + alpha^2 q^T M_cg^{-1} q
// (exact algebra; the base rho_i and all three dot products are of this
// iteration, so the expansion's rounding does not carry over).  So
//   step a: q = A p + V c ; partials p^T q, s^T q, q^T M_cg^{-1} q and
//           V^T M_cg^{-1} (A p); last block: alpha, beta and the k-vector
//           recurrences (V^T s_{i+1}, V^T p_{i+1}, c_{i+1})
//   step b: z += alpha p ; r -= alpha q ; s = M_cg^{-1} r ; p = s + beta p
//           (in place) ; partials r^T s (the fresh rho_{i+1}), r^T r;
//           last block: the stopping test on the fresh values.
// The stopping test and alpha use freshly reduced values; only beta comes
// from the expansion.  Per row and iteration the two kernels stream as many
// vector bytes as variants 0-7 (p, r read and q written in step a; p, q, z, r
// read and z, r, p written in step b) and one gather per matrix entry fewer.

// A p of a slice row: entries in groups of 8, every gather p[col] of a group
// in flight before the products (vp, cp: column-major slice, stride 32)
template <typename T, typename I, bool GLOBAL>
__device__ __forceinline__ T pg_row(const T* vp, const I* cp, int row, bool delta, int w, const T* __restrict__ pv) {
  T acc = 0;
  for (int j0 = 0; j0 < w; j0 += 8) {
    T av[8];
    int cc[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (GLOBAL) {
        av[j] = (j0 + j < w) ? ld_stream(vp + (size_t)(j0 + j) * kSlice) : (T)0;
        cc[j] = (j0 + j < w) ? (delta ? row : 0) + (int)ld_stream(cp + (size_t)(j0 + j) * kSlice) : row;
      } else {
        av[j] = (j0 + j < w) ? vp[(j0 + j) * kSlice] : (T)0;
        cc[j] = (j0 + j < w) ? (delta ? row : 0) + (int)cp[(j0 + j) * kSlice] : row;
      }
    }
    T g[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) g[j] = (j0 + j < w) ? __ldg(pv + cc[j]) : (T)0;
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (j0 + j < w) acc += av[j] * g[j];
  }
  return acc;
}

// Reductions of the one-gather iteration (variants 9-15).  No last block:
// every block of a kernel finishes its predecessor's reduction itself (the
// partials are visible once the predecessor has completed) and all blocks
// take the same decisions from the same sums; block 0 alone writes the state
// (into slots its own kernel does not read; see CgState).
//
// pg_begin, step a of iteration j (all threads, after the grid dependency
// wait): for j >= 1 the sums r^T s (and r^T r) of step b of iteration j - 1:
// rho_j, the iteration count j, and the stopping test on the fresh values.
// Returns false (in every block) when the solve is over.
template <typename T, int KB, int NT = 0>
__device__ __forceinline__ bool pg_begin(const CgArgs<T>& a, CgState& S, T* cls) {
  constexpr int KS = KB > 0 ? KB : 1;
  constexpr int KK = KS * KS;
  constexpr int GPT = (KK + kThreads - 1) / kThreads;
  __shared__ int go;
  __shared__ double tot[KB + 2];
  __shared__ double gs[KK];
  __shared__ double cprev[KS];
  const int P = a.par, l = threadIdx.x, k = a.k;
  const bool jac = a.dinv != nullptr;
  const int nb = jac ? 2 : 1;
  // one round of loads: the status and the slots, step b's partials (rho_j)
  // and the previous step a's projections, whether or not they are pending
  // (iteration 0 takes its slot from the init kernel and uses neither)
  // (no load depends on another: both slots are read, the pending flag picks one)
  const int running = *(volatile int*)&S.done == kRunning;
  const int pending = S.bp_s[P];
  const double alpha = S.alpha, beta = S.beta;
  long long it = 0, maxit = 0;
  double tol = 0.0, u_l = 0.0, t_l = 0.0, lam_l = 0.0, c_l = 0.0, u_o = 0.0, t_o = 0.0, c_o = 0.0;
  double greg[GPT];
  if (l == 0) {
    it = S.it_s[P ^ 1] + 1;
    maxit = S.maxit;
    tol = S.tol_abs;
  }
  if (l < k) {
    u_l = S.u_s[P][l];
    t_l = S.t_s[P][l];
    c_l = S.c_s[P][l];
    u_o = S.u_s[P ^ 1][l];
    t_o = S.t_s[P ^ 1][l];
    c_o = S.c_s[P ^ 1][l];
    lam_l = S.lam2[l];
  }
#pragma unroll
  for (int j = 0; j < GPT; ++j) {
    const int e = l + j * kThreads;
    greg[j] = e < k * k ? __ldcg(a.gram + e) : 0.0;
  }
  if (pending) {  // iteration j - 1's slot
    u_l = u_o;
    t_l = t_o;
    c_l = c_o;
  }
  if (l < k) cprev[l] = (double)(T)c_l;  // the coefficient the previous step a applied
  final_sums_2<NT>(a.partials_b, a.grid_b, nb, a.partials_o + (size_t)3 * a.grid_a, a.grid_a, k, tot);
#pragma unroll
  for (int j = 0; j < GPT; ++j) {
    const int e = l + j * kThreads;
    if (e < k * k) gs[e] = greg[j];
  }
  if (l == 0) {
    int st = running ? kRunning : kConverged;  // (an earlier status stands; only its "not running" is used here)
    if (running && pending) {
      const double rho = tot[0], rnorm = sqrt(jac ? tot[1] : tot[0]);
      if (!isfinite(rho) || !isfinite(rnorm)) st = kNonFinite;
      else if (rnorm <= tol) st = kConverged;
      else if (it >= maxit) st = kMaxIter;
      else if (rho <= 0.0) st = kBreakdown;
      if (blockIdx.x == 0) {
        S.it_s[P] = it;
        S.iters = it;
        if (st == kRunning) {
          S.rho_s[P] = rho;
          S.rho = rho;
        } else {
          S.done = st;
        }
      }
    }
    go = st == kRunning ? 1 : 0;
  }
  group_sync<NT>();
  if (l < KS) {
    double c = c_l;
    if (pending && l < k) {
      // iteration j - 1's recurrences: V^T M_cg^{-1} q = V^T M_cg^{-1} A p + G c,
      // V^T s -= alpha V^T M_cg^{-1} q, V^T p = V^T s + beta V^T p, c = 2|lambda| V^T p
      double vq = tot[nb + l];
#pragma unroll 8
      for (int m = 0; m < KB; ++m)
        if (m < k) vq += gs[m * k + l] * cprev[m];
      u_l -= alpha * vq;
      t_l = u_l + beta * t_l;
      c = lam_l * t_l;
      if (blockIdx.x == 0 && running) {
        S.vq[l] = vq;
        S.u_s[P][l] = u_l;
        S.t_s[P][l] = t_l;
        S.c_s[P][l] = c;
      }
    }
    cls[l] = l < k ? (T)c : (T)0;
  }
  group_sync<NT>();
  return go != 0;
}

// pg_end, step a: this block's partials p^T q, s^T q, q^T M_cg^{-1} q and
// V^T M_cg^{-1} A p (finished by step b).
template <typename T, int KB, int NW>
__device__ __forceinline__ void pg_end(const CgArgs<T>& a, T pq, T sq, T qdq, const T (&wq)[KB > 0 ? KB : 1]) {
  T part[KB + 3];
  part[0] = pq;
  part[1] = sq;
  part[2] = qdq;
#pragma unroll
  for (int l = 0; l < KB; ++l) part[l + 3] = wq[l];
  block_partials_t<T, KB + 3, NW, false>(part, a.k + 3, a.partials);
}

// pg_b_begin, step b of iteration j (all threads, after the grid dependency
// wait): step a's sums give kappa = p^T q, alpha = rho_j / kappa and beta from
// the expansion rho_j - 2 alpha s^T q + alpha^2 q^T M_cg^{-1} q; block 0 also
// advances V^T s, V^T p and c = 2|Lambda| V^T p with
// V^T M_cg^{-1} q = V^T M_cg^{-1} A p + G c (G = V^T M_cg^{-1} V, c the
// coefficients step a applied).  Returns false when the solve is over.
template <typename T, int KB>
__device__ __forceinline__ bool pg_b_begin(const CgArgs<T>& a, CgState& S, T& alpha_t, T& beta_t) {
  __shared__ int go;
  __shared__ double ab[2];
  __shared__ double tot[3];
  const int P = a.par;
  double rho = 0.0;
  int running = 0;
  if (threadIdx.x == 0) {  // one round of loads: these and step a's sums
    running = *(volatile int*)&S.done == kRunning;
    rho = S.rho_s[P];
  }
  final_sums_g(a.partials, a.grid_a, 3, tot);
  if (threadIdx.x == 0) {
    int st = kRunning;
    double alpha = 0.0, beta = 0.0;
    const double kappa = tot[0];
    if (!running) {
      st = kConverged;  // over already (its status stands)
    } else if (!isfinite(kappa)) {
      st = kNonFinite;
    } else if (kappa <= 0.0) {
      st = kNotSpd;
    } else {
      alpha = rho / kappa;
      const double rho_e = rho - 2.0 * alpha * tot[1] + alpha * alpha * tot[2];
      // below its rounding floor the expansion is noise around a true
      // rho_{i+1} << rho_i: beta is then ~0 either way (>= 0 is kept)
      beta = (rho_e > 0.0 ? rho_e : 0.0) / rho;
      if (!isfinite(rho_e)) st = kNonFinite;
    }
    if (blockIdx.x == 0 && running) {
      S.kappa = kappa;
      if (st == kRunning) {
        S.alpha = alpha;
        S.alpha32 = (float)alpha;
        S.beta = beta;
        S.beta32 = (float)beta;
        S.bp_s[P ^ 1] = 1;
      } else {
        S.done = st;
      }
    }
    ab[0] = alpha;
    ab[1] = beta;
    go = st == kRunning ? 1 : 0;
  }
  __syncthreads();
  if (!go) return false;
  alpha_t = (T)ab[0];
  beta_t = (T)ab[1];
  return true;
}

// per-row part of step a (variants 9-11): q = A p + V c and the row's terms of the partials
template <typename T, int KB, int VSTRIDE>
__device__ __forceinline__ void pg_row_update(const CgArgs<T>& a, int64_t row, T ap, T pv, T rv, T d, bool jac,
                                              const T* vrow, const T* cl, T& pq, T& sq, T& qdq,
                                              T (&wq)[KB > 0 ? KB : 1]) {
  const T aps = jac ? d * ap : ap;  // (M_cg^{-1} A p)_row
  T q = ap;
#pragma unroll
  for (int l = 0; l < KB; ++l)
    if (l < a.k) {
      const T v = vrow[l * VSTRIDE];
      q += v * cl[l];
      wq[l] += v * aps;
    }
  a.q[row] = q;
  const T sv = jac ? d * rv : rv;
  pq += pv * q;
  sq += sv * q;
  qdq += jac ? d * q * q : q * q;
}

// Variants 9 / 10: operands staged by bulk copies as in variants 5 / 6 (the
// "s" region of a stage holds r), registers capped for MB = 2 / 3 blocks per
// SM (at 4 the three extra accumulators spill); 12 / 13: the same with each
// warp's gathers issued one tile ahead (PIPE).
template <typename T, int KB, int MB, bool PIPE>
__global__ void __launch_bounds__(kStagedThreads, MB) cg_step_a_pg_staged_kernel(CgArgs<T> a) {
  constexpr int KS = KB > 0 ? KB : 1;
  extern __shared__ __align__(128) unsigned char stage_mem[];
  __shared__ __align__(8) uint64_t full[kMaxStages];
  __shared__ __align__(8) uint64_t empty[kMaxStages];
  __shared__ int stalled;
  __shared__ T cl[KS];
  CgState& S = a.st->cg;
  grid_dependency_wait();
  if (!pg_begin<T, KB>(a, S, cl)) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool jac = a.dinv != nullptr;
  const int nst = a.stages;
  const int64_t ntiles = (a.nslices + kTileSlices - 1) / kTileSlices;
  const int64_t ntl = (int64_t)blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t G = gridDim.x;
  if (threadIdx.x == 0) {
    for (int i = 0; i < nst; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], kTileSlices);
    }
    stalled = 0;
    mbar_init_fence();
  }
  __syncthreads();
  T pq = 0, sq = 0, qdq = 0;
  T wq[KS];
#pragma unroll
  for (int l = 0; l < KS; ++l) wq[l] = 0;
  if (warp == kTileSlices) {
    if (lane == 0) stage_producer<T, false>(a, stage_mem, full, empty, &stalled, ntl, nst);
  } else if constexpr (PIPE) {
    // software-pipelined consumers: the gathers of this warp's slice of tile
    // i + 1 are in flight while it finishes tile i, so two L2 round trips
    // overlap per warp
    const T* __restrict__ pv = a.p_old;
    const bool d16 = a.col16 != nullptr;
    int st = 0;
    uint32_t ph = 0;
    int64_t t = blockIdx.x;
    int cur_off = 0, cur_w = 0;                 // this warp's slice of the tile being finished
    int64_t c_t0 = 0, c_s0 = 0, c_s1 = 0;       // offsets of the next tile (fetched ahead)
    T gc[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) gc[j] = 0;
    auto offsets = [&](int64_t tt) {
      const int64_t sl = tt * kTileSlices + warp;
      c_t0 = a.slice_ptr[tt * kTileSlices];
      if (sl < a.nslices) {
        c_s0 = a.slice_ptr[sl];
        c_s1 = a.slice_ptr[sl + 1];
      } else {
        c_s0 = c_s1 = c_t0;
      }
    };
    // issue the gathers p[col] of the first eight entries of this warp's slice of tile tt (stage sst, landed)
    auto start = [&](int64_t tt, int sst, T (&g)[8]) {
      const int64_t sl = tt * kTileSlices + warp;
      cur_off = (int)(c_s0 - c_t0) + lane;
      cur_w = (int)((c_s1 - c_s0) >> 5);
      if (sl < a.nslices) {
        const unsigned char* b = stage_mem + (size_t)sst * a.stage_bytes;
        const int row = (int)(sl * kSlice + lane);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const int c = j < cur_w ? (d16 ? row + (int)reinterpret_cast<const int16_t*>(b + a.off_col)[cur_off + j * kSlice]
                                         : reinterpret_cast<const int32_t*>(b + a.off_col)[cur_off + j * kSlice])
                                  : row;
          g[j] = j < cur_w ? __ldg(pv + c) : (T)0;
        }
      }
    };
    bool alive = true;
    if (ntl > 0) {
      offsets(t);
      alive = mbar_wait_or_abort(&full[0], 0u, &stalled);
      if (alive) start(t, 0, gc);
      if (ntl > 1) offsets(t + G);
    }
    for (int64_t i = 0; alive && i < ntl; ++i, t += G) {
      const int off = cur_off, w = cur_w;
      const int stn = st + 1 == nst ? 0 : st + 1;
      const uint32_t phn = st + 1 == nst ? ph ^ 1u : ph;
      T gn[8];
      if (i + 1 < ntl) {
        if (!mbar_wait_or_abort(&full[stn], phn, &stalled)) break;
        start(t + G, stn, gn);
        if (i + 2 < ntl) offsets(t + 2 * G);
      }
      const int64_t sl = t * kTileSlices + warp;
      if (sl < a.nslices) {
        const unsigned char* b = stage_mem + (size_t)st * a.stage_bytes;
        const int r = warp * kSlice + lane;
        const int64_t row = sl * kSlice + lane;
        const T* vp = reinterpret_cast<const T*>(b) + off;
        T ap = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (j < w) ap += vp[j * kSlice] * gc[j];
        if (w > 8)
          ap += d16 ? pg_row<T, int16_t, false>(vp + 8 * kSlice,
                                                reinterpret_cast<const int16_t*>(b + a.off_col) + off + 8 * kSlice,
                                                (int)row, true, w - 8, pv)
                    : pg_row<T, int32_t, false>(vp + 8 * kSlice,
                                                reinterpret_cast<const int32_t*>(b + a.off_col) + off + 8 * kSlice,
                                                (int)row, false, w - 8, pv);
        const T pr = reinterpret_cast<const T*>(b + a.off_p)[r];
        const T rr = reinterpret_cast<const T*>(b + a.off_s)[r];
        const T d = jac ? reinterpret_cast<const T*>(b + a.off_d)[r] : (T)1;
        pg_row_update<T, KB, kTileRows>(a, row, ap, pr, rr, d, jac, reinterpret_cast<const T*>(b + a.off_v) + r, cl,
                                        pq, sq, qdq, wq);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[st]);
      if (i + 1 < ntl) {
#pragma unroll
        for (int j = 0; j < 8; ++j) gc[j] = gn[j];
      }
      st = stn;
      ph = phn;
    }
  } else {
    const T* __restrict__ pv = a.p_old;
    int64_t c_t0 = 0, c_s0 = 0, c_s1 = 0;
    if (ntl > 0) {
      const int64_t sl = blockIdx.x * (int64_t)kTileSlices + warp;
      c_t0 = a.slice_ptr[blockIdx.x * (int64_t)kTileSlices];
      if (sl < a.nslices) {
        c_s0 = a.slice_ptr[sl];
        c_s1 = a.slice_ptr[sl + 1];
      }
    }
    int st = 0;
    uint32_t ph = 0;
    int64_t t = blockIdx.x;
    for (int64_t i = 0; i < ntl; ++i, t += G) {
      const int64_t sl = t * kTileSlices + warp;
      const int64_t t0 = c_t0, s0 = c_s0, s1 = c_s1;
      if (i + 1 < ntl) {
        const int64_t tn = t + G, sln = tn * kTileSlices + warp;
        c_t0 = a.slice_ptr[tn * kTileSlices];
        if (sln < a.nslices) {
          c_s0 = a.slice_ptr[sln];
          c_s1 = a.slice_ptr[sln + 1];
        }
      }
      if (!mbar_wait_or_abort(&full[st], ph, &stalled)) break;
      if (sl < a.nslices) {
        const unsigned char* b = stage_mem + (size_t)st * a.stage_bytes;
        const int off = (int)(s0 - t0) + lane;
        const int w = (int)((s1 - s0) >> 5);
        const int r = warp * kSlice + lane;
        const int64_t row = sl * kSlice + lane;
        const T* vp = reinterpret_cast<const T*>(b) + off;
        const T ap = a.col16 ? pg_row<T, int16_t, false>(vp, reinterpret_cast<const int16_t*>(b + a.off_col) + off,
                                                         (int)row, true, w, pv)
                             : pg_row<T, int32_t, false>(vp, reinterpret_cast<const int32_t*>(b + a.off_col) + off,
                                                         (int)row, false, w, pv);
        const T pr = reinterpret_cast<const T*>(b + a.off_p)[r];
        const T rr = reinterpret_cast<const T*>(b + a.off_s)[r];
        const T d = jac ? reinterpret_cast<const T*>(b + a.off_d)[r] : (T)1;
        pg_row_update<T, KB, kTileRows>(a, row, ap, pr, rr, d, jac, reinterpret_cast<const T*>(b + a.off_v) + r, cl,
                                        pq, sq, qdq, wq);
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[st]);
      if (++st == nst) {
        st = 0;
        ph ^= 1u;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && stalled) *(volatile int*)&S.done = kStall;
  pg_end<T, KB, kStagedThreads / 32>(a, pq, sq, qdq, wq);
}

// Variants 14 / 15: the one-gather step a on tiles of 16 slices (512 rows),
// each consumer warp taking two adjacent slices of every tile.  A warp's
// per-tile work (the stage wait and release, the tile offsets) is shared by
// two slices, the gathers of both slices are in flight together, and the
// coefficients c stay in registers.  Registers capped for MB = 2 / 1 blocks
// per SM (FP32 with two stages of about 46 KB; FP64, or deeper rings).

// A p of two slice rows (entries in groups of 8, the 16 gathers of a group in
// flight before the products; missing entries contribute 0 * 0)
template <typename T, typename I>
__device__ __forceinline__ void pg_row_pair(const T* va, const I* ca, int rowa, int wa, const T* vb, const I* cb,
                                            int rowb, int wb, bool delta, const T* __restrict__ pv, T& apa, T& apb) {
  const int w = wa > wb ? wa : wb;
  for (int j0 = 0; j0 < w; j0 += 8) {
    T xa[8], xb[8];
    int ja[8], jb[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const bool ia = j0 + j < wa, ib = j0 + j < wb;
      xa[j] = ia ? va[(j0 + j) * kSlice] : (T)0;
      ja[j] = ia ? (delta ? rowa : 0) + (int)ca[(j0 + j) * kSlice] : rowa;
      xb[j] = ib ? vb[(j0 + j) * kSlice] : (T)0;
      jb[j] = ib ? (delta ? rowb : 0) + (int)cb[(j0 + j) * kSlice] : rowb;
    }
    T ga[8], gb[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      ga[j] = (j0 + j < wa) ? __ldg(pv + ja[j]) : (T)0;
      gb[j] = (j0 + j < wb) ? __ldg(pv + jb[j]) : (T)0;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      apa += xa[j] * ga[j];
      apb += xb[j] * gb[j];
    }
  }
}

// Producer of variants 14 / 15.  A stage is filled in two parts: the static
// operands (A's values and indices, V_hat's rows, the Jacobi diagonal), which
// no kernel of the iteration writes, and the Krylov vectors of the own rows
// (s, p).  The static parts of the first stages are issued before the grid
// dependency wait, so behind a programmatic edge they stream in while the
// previous step b still runs.
template <typename T, int TSL>
__device__ __forceinline__ void pg2_issue_static(const CgArgs<T>& a, unsigned char* b, uint64_t* bar, int64_t t,
                                                 int64_t e0, int64_t e1, uint64_t pol) {
  constexpr int TR = TSL * kSlice;
  const int ib = a.col16 ? 2 : 4;
  const char* idx = a.col16 ? (const char*)a.col16 : (const char*)a.col;
  const int64_t s0 = t * TSL, s1 = min(s0 + TSL, a.nslices);
  const int64_t row0 = s0 * kSlice;
  const uint32_t rb = (uint32_t)((s1 - s0) * kSlice * (int64_t)sizeof(T));
  const uint32_t ne = (uint32_t)(e1 - e0);
  const bool jac = a.dinv != nullptr;
  const bool vbf = a.Vbf != nullptr;
  const uint32_t rbv = vbf ? rb / (uint32_t)(sizeof(T) / 2) : rb;  // bytes of one V_hat column's rows
  mbar_arrive_expect_tx(bar, ne * (uint32_t)(sizeof(T) + ib) + (uint32_t)(2 + (jac ? 1 : 0)) * rb +
                                 (uint32_t)a.k * rbv);
  if (ne > 0) {
    bulk_g2s_hint(b, a.val + e0, ne * (uint32_t)sizeof(T), bar, pol);
    bulk_g2s_hint(b + a.off_col, idx + e0 * ib, ne * (uint32_t)ib, bar, pol);
  }
  for (int l = 0; l < a.k; ++l) {
    if (vbf)
      bulk_g2s_hint(b + a.off_v + (size_t)l * TR * 2, a.Vbf + (size_t)l * a.n_pad + row0, rbv, bar, pol);
    else
      bulk_g2s_hint(b + a.off_v + (size_t)l * TR * sizeof(T), a.V + (size_t)l * a.n_pad + row0, rb, bar, pol);
  }
  if (jac) bulk_g2s(b + a.off_d, a.dinv + row0, rb, bar);
}

// The same copies spread over the producer warp's lanes (the kernel's
// prologue, where a single lane's issue loop would hold the whole block at
// the begin phase's barrier): lane 0 arms the barrier with the tile's bytes,
// then lane c issues copy c (A's values, its indices, V_hat column c - 2, the
// Jacobi diagonal).
template <typename T, int TSL>
__device__ __forceinline__ void pg2_issue_static_warp(const CgArgs<T>& a, unsigned char* b, uint64_t* bar, int64_t t,
                                                      int64_t e0, int64_t e1, uint64_t pol, int lane) {
  constexpr int TR = TSL * kSlice;
  const int ib = a.col16 ? 2 : 4;
  const char* idx = a.col16 ? (const char*)a.col16 : (const char*)a.col;
  const int64_t s0 = t * TSL, s1 = min(s0 + TSL, a.nslices);
  const int64_t row0 = s0 * kSlice;
  const uint32_t rb = (uint32_t)((s1 - s0) * kSlice * (int64_t)sizeof(T));
  const uint32_t ne = (uint32_t)(e1 - e0);
  const bool jac = a.dinv != nullptr;
  const bool vbf = a.Vbf != nullptr;
  const uint32_t rbv = vbf ? rb / (uint32_t)(sizeof(T) / 2) : rb;  // bytes of one V_hat column's rows
  if (lane == 0)
    mbar_arrive_expect_tx(bar, ne * (uint32_t)(sizeof(T) + ib) + (uint32_t)(2 + (jac ? 1 : 0)) * rb +
                                   (uint32_t)a.k * rbv);
  __syncwarp();
  const int nc = 2 + a.k + (jac ? 1 : 0);
  for (int c = lane; c < nc; c += 32) {
    if (c == 0) {
      if (ne > 0) bulk_g2s_hint(b, a.val + e0, ne * (uint32_t)sizeof(T), bar, pol);
    } else if (c == 1) {
      if (ne > 0) bulk_g2s_hint(b + a.off_col, idx + e0 * ib, ne * (uint32_t)ib, bar, pol);
    } else if (c < 2 + a.k) {
      const int l = c - 2;
      if (vbf)
        bulk_g2s_hint(b + a.off_v + (size_t)l * TR * 2, a.Vbf + (size_t)l * a.n_pad + row0, rbv, bar, pol);
      else
        bulk_g2s_hint(b + a.off_v + (size_t)l * TR * sizeof(T), a.V + (size_t)l * a.n_pad + row0, rb, bar, pol);
    } else {
      bulk_g2s(b + a.off_d, a.dinv + row0, rb, bar);
    }
  }
}

template <typename T, int TSL>
__device__ __forceinline__ void pg2_issue_vectors(const CgArgs<T>& a, unsigned char* b, uint64_t* bar, int64_t t) {
  const int64_t s0 = t * TSL, s1 = min(s0 + TSL, a.nslices);
  const int64_t row0 = s0 * kSlice;
  const uint32_t rb = (uint32_t)((s1 - s0) * kSlice * (int64_t)sizeof(T));
  bulk_g2s(b + a.off_s, a.s + row0, rb, bar);
  bulk_g2s(b + a.off_p, a.p_old + row0, rb, bar);
}

// The stages before `pre` were issued whole by the kernel's prologue; with
// run == false the producer only waits until their copies have landed.
template <typename T, int TSL>
__device__ __forceinline__ void pg2_producer(const CgArgs<T>& a, unsigned char* stage_mem, uint64_t* full,
                                             uint64_t* empty, int* stalled, int64_t ntl, int nst, bool run) {
  const int64_t G = gridDim.x;
  const uint64_t pol = l2_evict_first_policy();
  const int64_t pre = min(ntl, (int64_t)(a.stall_test ? 1 : nst));  // stages issued before the loop
  int64_t issued = pre;
  if (run) {
    int st = (int)(pre % nst);
    uint32_t ph = (uint32_t)((pre / nst) & 1);
    int64_t t = blockIdx.x + pre * G;
    int64_t e0 = 0, e1 = 0;
    if (pre < ntl) {
      e0 = a.slice_ptr[t * TSL];
      e1 = a.slice_ptr[min((t + 1) * TSL, a.nslices)];
    }
    for (int64_t i = pre; i < ntl; ++i, t += G) {
      if (a.stall_test) break;
      if (!mbar_wait_or_abort(&empty[st], ph ^ 1u, stalled)) break;
      const int64_t c0 = e0, c1 = e1;
      if (i + 1 < ntl) {
        e0 = a.slice_ptr[(t + G) * TSL];
        e1 = a.slice_ptr[min((t + G + 1) * TSL, a.nslices)];
      }
      fence_proxy_async_smem();
      unsigned char* b = stage_mem + (size_t)st * a.stage_bytes;
      pg2_issue_static<T, TSL>(a, b, &full[st], t, c0, c1, pol);
      pg2_issue_vectors<T, TSL>(a, b, &full[st], t);
      ++issued;
      if (++st == nst) {
        st = 0;
        ph ^= 1u;
      }
    }
  }
  for (int64_t j = issued > nst ? issued - nst : 0; j < issued; ++j)
    mbar_wait(&full[j % nst], (uint32_t)((j / nst) & 1));
}

template <typename T, int KB, int MB>
__global__ void __launch_bounds__(kStagedThreads, MB) cg_step_a_pg2_kernel(CgArgs<T> a) {
  constexpr int KS = KB > 0 ? KB : 1;
  constexpr int TSL = 2 * kTileSlices;  // slices of a tile
  constexpr int TR = TSL * kSlice;      // rows of a tile
  extern __shared__ __align__(128) unsigned char stage_mem[];
  __shared__ __align__(8) uint64_t full[kMaxStages];
  __shared__ __align__(8) uint64_t empty[kMaxStages];
  __shared__ int stalled;
  __shared__ T cls[KS];
  __shared__ int run_flag;
  CgState& S = a.st->cg;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool jac = a.dinv != nullptr;
  const int nst = a.stages;
  const int64_t ntiles = (a.nslices + TSL - 1) / TSL;
  const int64_t ntl = (int64_t)blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int64_t G = gridDim.x;
  if (threadIdx.x == 0) {
    for (int i = 0; i < nst; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], kTileSlices);
    }
    stalled = 0;
    mbar_init_fence();
  }
  __syncthreads();
  if (warp == kTileSlices) {  // static operands of the first stages, issued by the whole producer warp
    const uint64_t pol = l2_evict_first_policy();
    const int64_t pre = min(ntl, (int64_t)(a.stall_test ? 1 : nst));
    int64_t e0[kMaxStages], e1[kMaxStages];  // their entry ranges, all loads in flight together
#pragma unroll
    for (int i = 0; i < kMaxStages; ++i) {
      const int64_t t = blockIdx.x + i * G;
      e0[i] = i < pre ? a.slice_ptr[t * TSL] : 0;
      e1[i] = i < pre ? a.slice_ptr[min((t + 1) * TSL, a.nslices)] : 0;
    }
#pragma unroll
    for (int i = 0; i < kMaxStages; ++i)
      if (i < pre)
        pg2_issue_static_warp<T, TSL>(a, stage_mem + (size_t)i * a.stage_bytes, &full[i], blockIdx.x + i * G, e0[i],
                                      e1[i], pol, lane);
  }
  // entry offsets of the tile and of a consumer warp's slices 2 warp,
  // 2 warp + 1 (fetched one tile ahead; the first before the dependency
  // wait, as the matrix is static); a slice past the end has no entries
  int64_t c_t0 = 0, c_a0 = 0, c_a1 = 0, c_b1 = 0;
  auto fetch = [&](int64_t tt) {
    const int64_t sa = tt * TSL + 2 * warp;
    c_t0 = a.slice_ptr[tt * TSL];
    c_a0 = a.slice_ptr[min(sa, a.nslices)];
    c_a1 = a.slice_ptr[min(sa + 1, a.nslices)];
    c_b1 = a.slice_ptr[min(sa + 2, a.nslices)];
  };
  if (warp < kTileSlices && ntl > 0) fetch(blockIdx.x);
  grid_dependency_wait();  // the previous step b's p, s, c and partials are visible from here on
  // The consumer warps run the begin phase among themselves (named barrier
  // 1), so that the producer, whose bulk copies can block while the memory
  // system drains the first stages, does not hold them; the producer learns
  // the outcome at barrier 2, where the consumers only arrive.
  bool run;
  if (warp == kTileSlices) {  // the Krylov vectors of those stages, lane i issuing stage i's
    const int64_t pre = min(ntl, (int64_t)(a.stall_test ? 1 : nst));
    if (lane < pre)
      pg2_issue_vectors<T, TSL>(a, stage_mem + (size_t)lane * a.stage_bytes, &full[lane], blockIdx.x + lane * G);
    asm volatile("bar.sync 2, %0;" ::"n"(kStagedThreads) : "memory");
    run = run_flag != 0;
  } else {
    run = pg_begin<T, KB, kThreads>(a, S, cls);
    if (threadIdx.x == 0) run_flag = run ? 1 : 0;
    asm volatile("bar.arrive 2, %0;" ::"n"(kStagedThreads) : "memory");
  }
  if (!run) {  // the producer lets its copies land before the block leaves
    if (warp == kTileSlices && lane == 0) pg2_producer<T, TSL>(a, stage_mem, full, empty, &stalled, ntl, nst, false);
    return;
  }
  T cl[KS];
#pragma unroll
  for (int l = 0; l < KS; ++l) cl[l] = cls[l];
  T pq = 0, sq = 0, qdq = 0;
  T wq[KS];
#pragma unroll
  for (int l = 0; l < KS; ++l) wq[l] = 0;
  if (warp == kTileSlices) {
    if (lane == 0) pg2_producer<T, TSL>(a, stage_mem, full, empty, &stalled, ntl, nst, true);
  } else {
    const T* __restrict__ pv = a.p_old;
    const bool d16 = a.col16 != nullptr;
    const bool vbf = a.Vbf != nullptr;
    int st = 0;
    uint32_t ph = 0;
    int64_t t = blockIdx.x;
    for (int64_t i = 0; i < ntl; ++i, t += G) {
      const int64_t t0 = c_t0, a0 = c_a0, a1 = c_a1, b1 = c_b1;
      if (i + 1 < ntl) fetch(t + G);
      if (!mbar_wait_or_abort(&full[st], ph, &stalled)) break;
      const int64_t sla = t * TSL + 2 * warp;
      if (sla < a.nslices) {
        const unsigned char* b = stage_mem + (size_t)st * a.stage_bytes;
        const bool has_b = sla + 1 < a.nslices;
        const int wa = (int)((a1 - a0) >> 5), wb = (int)((b1 - a1) >> 5);
        const int offa = (int)(a0 - t0) + lane, offb = (int)(a1 - t0) + lane;
        const int ra = 2 * warp * kSlice + lane, rb = ra + kSlice;  // rows within the tile
        const int rowa = (int)(sla * kSlice) + lane, rowb = rowa + kSlice;
        const T* vals = reinterpret_cast<const T*>(b);
        const T* ps = reinterpret_cast<const T*>(b + a.off_p);
        const T* rs = reinterpret_cast<const T*>(b + a.off_s);
        const T* ds = reinterpret_cast<const T*>(b + a.off_d);
        const T* vt = reinterpret_cast<const T*>(b + a.off_v);
        T apa = 0, apb = 0;
        if (d16) {
          const int16_t* cc = reinterpret_cast<const int16_t*>(b + a.off_col);
          pg_row_pair<T, int16_t>(vals + offa, cc + offa, rowa, wa, vals + offb, cc + offb, rowb, wb, true, pv, apa,
                                  apb);
        } else {
          const int32_t* cc = reinterpret_cast<const int32_t*>(b + a.off_col);
          pg_row_pair<T, int32_t>(vals + offa, cc + offa, rowa, wa, vals + offb, cc + offb, rowb, wb, false, pv, apa,
                                  apb);
        }
        const T pa = ps[ra], rva = rs[ra];
        const T pb = has_b ? ps[rb] : (T)0, rvb = has_b ? rs[rb] : (T)0;
        const T da = jac ? ds[ra] : (T)1;
        const T db = (jac && has_b) ? ds[rb] : (T)1;
        const T apsa = jac ? da * apa : apa;  // (M_cg^{-1} A p)_row
        const T apsb = has_b ? (jac ? db * apb : apb) : (T)0;
        T qa = apa, qb = apb;
        if (vbf) {  // V_hat's rows as BF16: the FP32 value is the BF16 bits shifted up
          const uint16_t* vh = reinterpret_cast<const uint16_t*>(b + a.off_v);
#pragma unroll
          for (int l = 0; l < KB; ++l)
            if (l < a.k) {
              const T v1 = (T)__uint_as_float((uint32_t)vh[l * TR + ra] << 16);
              const T v2 = has_b ? (T)__uint_as_float((uint32_t)vh[l * TR + rb] << 16) : (T)0;
              qa += v1 * cl[l];
              qb += v2 * cl[l];
              wq[l] += v1 * apsa;
              wq[l] += v2 * apsb;
            }
        } else {
#pragma unroll
          for (int l = 0; l < KB; ++l)
            if (l < a.k) {
              const T v1 = vt[l * TR + ra];
              const T v2 = has_b ? vt[l * TR + rb] : (T)0;
              qa += v1 * cl[l];
              qb += v2 * cl[l];
              wq[l] += v1 * apsa;
              wq[l] += v2 * apsb;
            }
        }
        a.q[rowa] = qa;
        pq += pa * qa;
        sq += (jac ? da * rva : rva) * qa;
        qdq += jac ? da * qa * qa : qa * qa;
        if (has_b) {
          a.q[rowb] = qb;
          pq += pb * qb;
          sq += (jac ? db * rvb : rvb) * qb;
          qdq += jac ? db * qb * qb : qb * qb;
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[st]);
      if (++st == nst) {
        st = 0;
        ph ^= 1u;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && stalled) *(volatile int*)&S.done = kStall;
  pg_end<T, KB, kStagedThreads / 32>(a, pq, sq, qdq, wq);
}

// Variant 11: the same arithmetic with plain loads, one warp per SELL slice,
// grid-stride (matrices whose tiles do not fit two shared-memory stages);
// registers capped for 4 blocks per SM in FP32, 2 in FP64 (no spills)
template <typename T, int KB>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 8 ? 2 : 4) cg_step_a_pg_kernel(CgArgs<T> a) {
  constexpr int KS = KB > 0 ? KB : 1;
  CgState& S = a.st->cg;
  grid_dependency_wait();
  __shared__ T cl[KS];
  if (!pg_begin<T, KB>(a, S, cl)) return;
  const T* __restrict__ pv = a.p_old;
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = (blockIdx.x * (int64_t)kThreads + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
  const bool jac = a.dinv != nullptr;
  T pq = 0, sq = 0, qdq = 0;
  T wq[KS];
#pragma unroll
  for (int l = 0; l < KS; ++l) wq[l] = 0;
  for (int64_t sl = warp0; sl < a.nslices; sl += nwarps) {
    const int64_t row = sl * kSlice + lane;
    const T pr = pv[row];
    const T rr = a.r[row];
    const T d = jac ? a.dinv[row] : (T)1;
    const int64_t base = a.slice_ptr[sl];
    const int w = (int)((a.slice_ptr[sl + 1] - base) >> 5);
    const T ap = a.col16 ? pg_row<T, int16_t, true>(a.val + base + lane, a.col16 + base + lane, (int)row, true, w, pv)
                         : pg_row<T, int32_t, true>(a.val + base + lane, a.col + base + lane, (int)row, false, w, pv);
    T vv[KS];  // this row of V_hat, all loads issued before the first use
#pragma unroll
    for (int l = 0; l < KS; ++l) vv[l] = (l < a.k) ? ld_stream(a.V + (size_t)l * a.n_pad + row) : (T)0;
    pg_row_update<T, KB, 1>(a, row, ap, pr, rr, d, jac, vv, cl, pq, sq, qdq, wq);
  }
  pg_end<T, KB, kThreads / 32>(a, pq, sq, qdq, wq);
}

// step b of variants 9-11: z += alpha p, r -= alpha q, s = M_cg^{-1} r,
// p = s + beta p in place, and the stopping test on the fresh r^T s, r^T r
template <typename T, int KB>
__global__ void __launch_bounds__(kThreads) cg_step_b_pg_kernel(CgArgs<T> a) {
  constexpr int W = V16<T>::W;
  CgState& S = a.st->cg;
  grid_dependency_wait();  // step a's q and partials (launched early behind a programmatic edge)
  T alpha, beta;
  if (!pg_b_begin<T, KB>(a, S, alpha, beta)) return;
  const bool jac = a.dinv != nullptr;
  T rs = 0, rr = 0;
  const int64_t nvec = a.n_pad / W;
  const int64_t stride = (int64_t)gridDim.x * kThreads;
  constexpr int U = 4;
  for (int64_t iv0 = blockIdx.x * (int64_t)kThreads + threadIdx.x; iv0 < nvec; iv0 += stride * U) {
    T pv[U][W], qv[U][W], zv[U][W], rv[U][W], d[U][W];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t iv = iv0 + u * stride;
      if (iv < nvec) {
        const int64_t i = iv * W;
        ld16(a.p_old + i, pv[u]);
        ld16(a.q + i, qv[u]);
        ld16(a.z + i, zv[u]);
        ld16(a.r + i, rv[u]);
        if (jac) ld16(a.dinv + i, d[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t iv = iv0 + u * stride;
      if (iv >= nvec) continue;
      const int64_t i = iv * W;
#pragma unroll
      for (int e = 0; e < W; ++e) {
        zv[u][e] += alpha * pv[u][e];
        rv[u][e] -= alpha * qv[u][e];
        const T s = jac ? d[u][e] * rv[u][e] : rv[u][e];
        pv[u][e] = s + beta * pv[u][e];
        rs += rv[u][e] * s;
        if (jac) rr += rv[u][e] * rv[u][e];
      }
      st16(a.z + i, zv[u]);
      st16(a.r + i, rv[u]);
      st16(a.p_old + i, pv[u]);
    }
  }
  T acc[2] = {rs, rr};
  block_partials_t<T, 2, kThreads / 32, false>(acc, jac ? 2 : 1, a.partials_b);  // finished by the next step a
}

// G = V^T M_cg^{-1} V (k x k, both triangles) from the kernels' own V and
// M_cg^{-1} in FP64: one block per pair l <= m.
template <typename T>
__global__ void __launch_bounds__(kThreads) cg_gram_kernel(const T* V, const T* dinv, int64_t n_pad, int k,
                                                          double* G) {
  int p = blockIdx.x, l = 0;
  while (l < k && p >= k - l) {
    p -= k - l;
    ++l;
  }
  if (l >= k) return;
  const int m = l + p;
  const T* vl = V + (size_t)l * n_pad;
  const T* vm = V + (size_t)m * n_pad;
  double s[1] = {0.0};
  for (int64_t i = threadIdx.x; i < n_pad; i += kThreads) {
    const double d = dinv ? (double)dinv[i] : 1.0;
    s[0] += (double)vl[i] * d * (double)vm[i];
  }
  __shared__ double sm[kThreads / 32];
  const double w = warp_sum(s[0]);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = w;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < kThreads / 32; ++i) t += sm[i];
    G[(size_t)l * k + m] = t;
    G[(size_t)m * k + l] = t;
  }
}

// ------------------------------------------------------------------ step b

// V^T s_{i+1} = V^T s_i - alpha V^T (M_cg^{-1} q_i) follows from what step a
// already formed (exact algebra, the same recurrence CG uses for r itself),
// so this kernel streams only the four CG vectors.
template <typename T, int KB>
__global__ void __launch_bounds__(kThreads) cg_step_b_kernel(CgArgs<T> a) {
  constexpr int W = V16<T>::W;
  CgState& S = a.st->cg;
  if (S.done != kRunning) return;
  const T alpha = alpha_of(S, T(0));
  const bool jac = a.dinv != nullptr;
  T rs = 0, rr = 0;
  const int64_t nvec = a.n_pad / W;
  const int64_t stride = (int64_t)gridDim.x * kThreads;
  // U grid-stride chunks per trip, all their loads issued before any use
  // (the kernel is latency-bound: more bytes in flight per thread)
  constexpr int U = 4;
  for (int64_t iv0 = blockIdx.x * (int64_t)kThreads + threadIdx.x; iv0 < nvec; iv0 += stride * U) {
    T pn[U][W], qv[U][W], zv[U][W], rv[U][W], d[U][W];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t iv = iv0 + u * stride;
      if (iv < nvec) {
        const int64_t i = iv * W;
        ld16(a.p_new + i, pn[u]);
        ld16(a.q + i, qv[u]);
        ld16(a.z + i, zv[u]);
        ld16(a.r + i, rv[u]);
        if (jac) ld16(a.dinv + i, d[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t iv = iv0 + u * stride;
      if (iv >= nvec) continue;
      const int64_t i = iv * W;
      T s[W];
#pragma unroll
      for (int e = 0; e < W; ++e) {
        zv[u][e] += alpha * pn[u][e];
        rv[u][e] -= alpha * qv[u][e];
      }
      st16(a.z + i, zv[u]);
      st16(a.r + i, rv[u]);
      if (jac) {
#pragma unroll
        for (int e = 0; e < W; ++e) {
          s[e] = d[u][e] * rv[u][e];
          rr += rv[u][e] * rv[u][e];
        }
        st16(a.s + i, s);
      } else {
#pragma unroll
        for (int e = 0; e < W; ++e) s[e] = rv[u][e];
      }
#pragma unroll
      for (int e = 0; e < W; ++e) rs += rv[u][e] * s[e];
    }
  }
  T acc[2] = {rs, rr};
  const int nv = jac ? 2 : 1;
  block_partials_t<T, 2>(acc, nv, a.partials);
  if (last_block_after_partials(&a.st->ticket)) {
    __shared__ double tot[2];
    final_sums(a.partials, nv, tot);
    if (threadIdx.x == 0) {
      const double rho_new = tot[0], rnorm = sqrt(jac ? tot[1] : tot[0]);
      const double alpha_d = S.alpha;
      for (int l = 0; l < a.k; ++l) S.u[l] -= alpha_d * S.vq[l];
      S.iters += 1;
      if (!isfinite(rho_new) || !isfinite(rnorm)) {
        S.done = kNonFinite;
      } else if (rnorm <= S.tol_abs) {
        S.done = kConverged;
      } else if (S.iters >= S.maxit) {
        S.done = kMaxIter;
      } else if (rho_new == 0.0) {
        S.done = kBreakdown;
      } else {
        const double beta = rho_new / S.rho;
        S.beta = beta;
        S.beta32 = (float)beta;
        S.rho = rho_new;
        for (int l = 0; l < a.k; ++l) S.t[l] = S.u[l] + beta * S.t[l];
        publish_c(S, a.k);
      }
    }
  }
}

// ------------------------------------------------------------------ loop control

static __global__ void cg_ctl_kernel(DevState* st, cudaGraphConditionalHandle handle) {
  CgState& S = st->cg;
  S.ctl_count += 1;
  if (S.done == kRunning && S.ctl_count >= S.ctl_limit) S.done = kLoopCap;
  cudaGraphSetConditional(handle, S.done == kRunning ? 1u : 0u);
}

// the same bookkeeping for the host-driven loop (no graph condition)
static __global__ void cg_ctl_host_kernel(DevState* st) {
  CgState& S = st->cg;
  S.ctl_count += 1;
  if (S.done == kRunning && S.ctl_count >= S.ctl_limit) S.done = kLoopCap;
}

// ------------------------------------------------------------------ finish

template <typename T>
__global__ void __launch_bounds__(kThreads) cg_finish_kernel(DevState* st, const T* z, int64_t n_pad) {
  CgState& S = st->cg;
  const double vn = (S.vnorm > 0.0 && isfinite(S.vnorm)) ? S.vnorm : 0.0;
  double* out = S.zout;
  // the one-kernel iteration leaves its last z update z += alpha p to this kernel
  const T* pl = S.fused_pending ? reinterpret_cast<const T*>(S.p_last) : nullptr;
  const T alpha = alpha_of(S, T(0));
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n_pad; i += (int64_t)gridDim.x * kThreads)
    out[i] = vn * (double)(pl ? z[i] + alpha * pl[i] : z[i]);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    S.budget -= S.iters;
    OuterState& O = st->out;
    O.inner_total += S.iters;
    O.prec_calls += 1;
    O.bodies += S.ctl_count;
    if (O.status == MRCG_OK) {
      if (S.done == kNotSpd) O.status = MRCG_ERR_NOT_SPD;
      else if (S.done == kNonFinite) O.status = MRCG_ERR_NONFINITE;
      else if (S.done == kMaxIter || S.done == kLoopCap) O.status = MRCG_ERR_MAXITER;
      else if (S.done == kBreakdown) O.status = MRCG_ERR_BREAKDOWN;
      else if (S.done == kStall) O.status = MRCG_ERR_CUDA;
    }
  }
}

static __global__ void fill_pattern_kernel(double* v, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads)
    v[i] = 1.0 + 0.125 * (double)(i % 7) - 0.0625 * (double)(i % 3);
}

// ------------------------------------------------------------------ host side

namespace {

// stage layout of the staged step a (128-byte aligned regions)
struct StageGeo {
  int off_col, off_v, off_s, off_p, off_d, off_z, bytes;
};

// V_hat streamed as BF16: FP32 one-gather step a on 16-slice tiles (variant 14)
inline bool bf16_stream(const InnerGraphSpec& spec) { return spec.Vbf != nullptr && spec.fp32 && spec.var_a == 14; }

StageGeo stage_geo(const InnerGraphSpec& spec) {
  auto up = [](int64_t x) { return (x + 127) / 128 * 128; };
  const int64_t w = spec.fp32 ? 4 : 8, ib = spec.A.col16 ? 2 : 4;
  const int64_t TR = (int64_t)tile_slices(spec.var_a) * kSlice;  // rows of the variant's tile
  const int64_t E = tile_slices(spec.var_a) == 16 ? spec.tile_entries16 : spec.tile_entries;
  StageGeo g;
  int64_t o = up(E * w);
  g.off_col = (int)o;
  o += up(E * ib);
  g.off_v = (int)o;
  o += up((int64_t)spec.k * TR * (bf16_stream(spec) ? 2 : w));
  g.off_s = (int)o;
  o += TR * w;
  g.off_p = (int)o;
  o += TR * w;
  g.off_d = (int)o;
  if (spec.dinv || spec.var_a == 8) o += TR * w;  // M_cg^{-1} (Jacobi) or q_{i-1} (one-kernel iteration)
  g.off_z = (int)o;
  if (spec.var_a == 8) o += TR * w;  // z (one-kernel iteration)
  g.bytes = o > (1 << 30) ? (1 << 30) : (int)o;
  return g;
}

constexpr int kMaxDynSmem = 227 * 1024 - 16 * 1024;  // leaves room for the kernel's static shared memory

template <typename T>
void make_args(const InnerGraphSpec& spec, CgArgs<T> (&a)[2]) {
  const StageGeo geo = stage_geo(spec);
  for (int par = 0; par < 2; ++par) {
    CgArgs<T>& x = a[par];
    x.stages = spec.stages;
    x.stall_test = spec.stall_test ? 1 : 0;
    x.stage_bytes = geo.bytes;
    x.off_col = geo.off_col;
    x.off_v = geo.off_v;
    x.off_s = geo.off_s;
    x.off_p = geo.off_p;
    x.off_d = geo.off_d;
    x.off_z = geo.off_z;
    x.st = spec.st;
    // rows of kMaxBlocks: [0, kMaxNV) and [kMaxNV, 2 kMaxNV) step a's partials by
    // the parity of the iteration (a step a reads the other parity's while its
    // own blocks write theirs), then two rows of step b's
    x.partials = spec.partials + (size_t)par * kMaxNV * kMaxBlocks;
    x.partials_o = spec.partials + (size_t)(par ^ 1) * kMaxNV * kMaxBlocks;
    x.partials_b = spec.partials + (size_t)2 * kMaxNV * kMaxBlocks;
    x.grid_a = spec.grid_spmv;
    x.grid_b = spec.grid_stream_b;
    x.par = par;
    x.slice_ptr = spec.A.slice_ptr;
    x.col = spec.A.col;
    x.col16 = spec.A.col16;
    x.val = reinterpret_cast<const T*>(sizeof(T) == 8 ? (const void*)spec.A.val64 : (const void*)spec.A.val32);
    x.nslices = spec.A.nslices;
    x.n_pad = spec.A.n_pad;
    x.V = reinterpret_cast<const T*>(spec.V);
    x.Vbf = bf16_stream(spec) ? reinterpret_cast<const uint16_t*>(spec.Vbf) : nullptr;
    x.k = spec.k;
    x.dinv = reinterpret_cast<const T*>(spec.dinv);
    x.dsmw = reinterpret_cast<const T*>(spec.dsmw);
    x.gram = spec.gram;
    x.z = reinterpret_cast<T*>(spec.z);
    x.r = reinterpret_cast<T*>(spec.r);
    x.s = (spec.dinv || spec.dsmw || spec.ilu.nblk > 0) ? reinterpret_cast<T*>(spec.s) : reinterpret_cast<T*>(spec.r);
    x.q = reinterpret_cast<T*>(spec.q);
    x.p_old = reinterpret_cast<T*>(par == 0 ? spec.p0 : spec.p1);
    x.p_new = reinterpret_cast<T*>(par == 0 ? spec.p1 : spec.p0);
    x.r_new = nullptr;
    x.q_old = nullptr;
    if (spec.var_a == 8) {  // one-kernel iteration: r and q ping-pong as p does
      x.r = reinterpret_cast<T*>(par == 0 ? spec.r : spec.r2);
      x.r_new = reinterpret_cast<T*>(par == 0 ? spec.r2 : spec.r);
      x.q = reinterpret_cast<T*>(par == 0 ? spec.q : spec.q2);
      x.q_old = reinterpret_cast<T*>(par == 0 ? spec.q2 : spec.q);
      x.s = x.r;
    }
    if (is_pg_variant(spec.var_a)) {  // one p updated in place; s = M_cg^{-1} r formed where it is used
      x.p_old = x.p_new = reinterpret_cast<T*>(spec.p0);
      x.s = x.r;
    }
  }
}

cudaError_t add_kernel(cudaGraph_t g, cudaGraphNode_t* node, const cudaGraphNode_t* deps, size_t ndeps,
                       const void* fn, int grid, int block, void** args, unsigned smem = 0) {
  cudaKernelNodeParams p = {};
  p.func = const_cast<void*>(fn);
  p.gridDim = dim3(grid);
  p.blockDim = dim3(block);
  p.sharedMemBytes = smem;
  p.kernelParams = args;
  p.extra = nullptr;
  return cudaGraphAddKernelNode(node, g, deps, ndeps, &p);
}

template <typename T, int KB>
const void* step_a_fn(int var) {
  switch (var) {
    case 9: return (const void*)cg_step_a_pg_staged_kernel<T, KB, 2, false>;
    case 10: return (const void*)cg_step_a_pg_staged_kernel<T, KB, 3, false>;
    case 11: return (const void*)cg_step_a_pg_kernel<T, KB>;
    case 12: return (const void*)cg_step_a_pg_staged_kernel<T, KB, 2, true>;
    case 13: return (const void*)cg_step_a_pg_staged_kernel<T, KB, 3, true>;
    case 14: return (const void*)cg_step_a_pg2_kernel<T, KB, 2>;
    case 15: return (const void*)cg_step_a_pg2_kernel<T, KB, 1>;
    case 1: return (const void*)cg_step_a_kernel<T, KB, 1>;
    case 2: return (const void*)cg_step_a_kernel<T, KB, 2>;
    case 3: return (const void*)cg_step_a_kernel<T, KB, 3>;
    case 4: return (const void*)cg_step_a_kernel<T, KB, 4>;
    case 5: return (const void*)cg_step_a_staged_kernel<T, KB, 2, false>;
    case 6: return (const void*)cg_step_a_staged_kernel<T, KB, 4, false>;
    case 7: return (const void*)cg_step_a_staged_kernel<T, KB, 2, true>;
    case 8: return (const void*)cg_step_a_staged_kernel<T, KB, 3, false, true>;
    default: return (const void*)cg_step_a_kernel<T, KB, 0>;
  }
}

// dynamic shared memory of the step-a launch (opting the staged kernel in above 48 KB)
template <typename T, int KB>
unsigned step_a_smem(const InnerGraphSpec& spec) {
  if (!is_staged_variant(spec.var_a)) return 0;
  const int bytes = stage_geo(spec).bytes * spec.stages;
  cudaFuncSetAttribute(step_a_fn<T, KB>(spec.var_a), cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  return (unsigned)bytes;
}

// threads per block of the step-a launch
int step_a_block(const InnerGraphSpec& spec) { return is_staged_variant(spec.var_a) ? kStagedThreads : kThreads; }

template <typename T>
cudaError_t launch_a(const void* fn, int grid, int block, cudaStream_t stream, CgArgs<T>& a, unsigned smem) {
  void* args[] = {&a};
  return cudaLaunchKernel(fn, dim3(grid), dim3(block), args, smem, stream);
}

// step b of the spec's inner preconditioner
template <typename T, int KB>
const void* step_b_fn(const InnerGraphSpec& spec) {
  if (is_pg_variant(spec.var_a)) return (const void*)cg_step_b_pg_kernel<T, KB>;
  return spec.dsmw ? (const void*)cg_step_b_smw_kernel<T, KB> : (const void*)cg_step_b_kernel<T, KB>;
}

// the ILU step b: grid, dynamic shared memory (one block's values per owning warp)
inline int ilu_grid(const InnerGraphSpec& spec) { return (spec.ilu.nblk + spec.ilu.wpc - 1) / spec.ilu.wpc; }
template <typename T>
unsigned ilu_smem(const InnerGraphSpec& spec) {
  return (unsigned)((size_t)spec.ilu.wpc * ilu_warp_bytes<T>(spec.ilu));
}

template <typename T, int KB>
void launch_b(const InnerGraphSpec& spec, cudaStream_t stream, CgArgs<T>& a) {
  if (spec.ilu.nblk > 0) {
    cudaFuncSetAttribute((const void*)cg_step_b_ilu_kernel<T, KB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)ilu_smem<T>(spec));
    IluArgs f = spec.ilu;
    int init = 0;
    void* args[] = {&a, &f, &init};
    cudaLaunchKernel((const void*)cg_step_b_ilu_kernel<T, KB>, dim3(ilu_grid(spec)), dim3(kThreads), args,
                     ilu_smem<T>(spec), stream);
    return;
  }
  void* args[] = {&a};
  cudaLaunchKernel(step_b_fn<T, KB>(spec), dim3(spec.grid_stream_b), dim3(kThreads), args, 0, stream);
}

// the first residual and its preconditioned form (two passes for the MINRES-CG* M_cg)
template <typename T, int KB>
void launch_init(const InnerGraphSpec& spec, cudaStream_t stream, CgArgs<T>& a) {
  if (spec.ilu.nblk > 0) {
    cudaFuncSetAttribute((const void*)cg_step_b_ilu_kernel<T, KB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)ilu_smem<T>(spec));
    cg_init_smw_vr_kernel<T, KB><<<spec.grid_stream, kThreads, 0, stream>>>(a);
    IluArgs f = spec.ilu;
    int init = 1;
    void* args[] = {&a, &f, &init};
    cudaLaunchKernel((const void*)cg_step_b_ilu_kernel<T, KB>, dim3(ilu_grid(spec)), dim3(kThreads), args,
                     ilu_smem<T>(spec), stream);
    return;
  }
  if (spec.dsmw) {
    cg_init_smw_vr_kernel<T, KB><<<spec.grid_stream, kThreads, 0, stream>>>(a);
    cg_init_smw_kernel<T, KB><<<spec.grid_stream, kThreads, 0, stream>>>(a);
  } else {
    cg_init_kernel<T, KB><<<spec.grid_stream, kThreads, 0, stream>>>(a);
  }
}

template <typename T, int KB>
cudaError_t build_graph_t(const InnerGraphSpec& spec, cudaGraph_t* out_graph) {
  cudaError_t e;
  cudaGraph_t g;
  if ((e = cudaGraphCreate(&g, 0)) != cudaSuccess) return e;
  CgArgs<T> a[2];
  make_args(spec, a);
  DevState* st = spec.st;
  double* partials = spec.partials;
  int64_t n_pad = spec.A.n_pad;
  const T* zc = reinterpret_cast<const T*>(spec.z);
  const unsigned smem_a = step_a_smem<T, KB>(spec);
  IluArgs ilu_f = spec.ilu;
  int ilu_init1 = 1, ilu_init0 = 0;
  const unsigned smem_ilu = spec.ilu.nblk > 0 ? ilu_smem<T>(spec) : 0;
  if (spec.ilu.nblk > 0)
    cudaFuncSetAttribute((const void*)cg_step_b_ilu_kernel<T, KB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem_ilu);

  cudaGraphNode_t n_norm, n_init, n_loop, n_fin;
  void* norm_args[] = {&st, &partials, &n_pad};
  if ((e = add_kernel(g, &n_norm, nullptr, 0, (const void*)cg_vnorm_kernel, spec.grid_stream, kThreads, norm_args)))
    goto fail;
  {
    void* init_args[] = {&a[0]};
    if (spec.ilu.nblk > 0) {
      cudaGraphNode_t n_vr;
      void* ilu_args[] = {&a[0], &ilu_f, &ilu_init1};
      if ((e = add_kernel(g, &n_vr, &n_norm, 1, (const void*)cg_init_smw_vr_kernel<T, KB>, spec.grid_stream,
                          kThreads, init_args)))
        goto fail;
      if ((e = add_kernel(g, &n_init, &n_vr, 1, (const void*)cg_step_b_ilu_kernel<T, KB>, ilu_grid(spec), kThreads,
                          ilu_args, smem_ilu)))
        goto fail;
    } else if (spec.dsmw) {
      cudaGraphNode_t n_vr;
      if ((e = add_kernel(g, &n_vr, &n_norm, 1, (const void*)cg_init_smw_vr_kernel<T, KB>, spec.grid_stream,
                          kThreads, init_args)))
        goto fail;
      if ((e = add_kernel(g, &n_init, &n_vr, 1, (const void*)cg_init_smw_kernel<T, KB>, spec.grid_stream, kThreads,
                          init_args)))
        goto fail;
    } else if ((e = add_kernel(g, &n_init, &n_norm, 1, (const void*)cg_init_kernel<T, KB>, spec.grid_stream,
                               kThreads, init_args))) {
      goto fail;
    }
  }
  {
    cudaGraphConditionalHandle h;
    if ((e = cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault))) goto fail;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    if ((e = cudaGraphAddNode(&n_loop, g, &n_init, nullptr, 1, &cp))) goto fail;
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    cudaGraphNode_t prev = nullptr;
    // variants 14 / 15 with the one-gather step b: programmatic edges (the
    // successor may start once every block of its predecessor has started; it
    // waits for the predecessor's results with grid_dependency_wait), so a
    // step a streams its static operands while the previous step b finishes
    const bool pdl = spec.pdl != 0 && (spec.var_a == 14 || spec.var_a == 15) && spec.ilu.nblk == 0 && !spec.dsmw;
    cudaGraphEdgeData ed = {}, ed_plain = {};
    ed.from_port = cudaGraphKernelNodePortLaunchCompletion;
    ed.type = cudaGraphDependencyTypeProgrammatic;
    // pdl 1: both edges programmatic; 2 (default): only step b -> step a, whose
    // static prefetch then overlaps step b's tail (an early step b slowed its
    // own streaming, measured); 3: only step a -> step b
    const cudaGraphEdgeData& e_ba = (spec.pdl == 1 || spec.pdl == 2) ? ed : ed_plain;
    const cudaGraphEdgeData& e_ab = (spec.pdl == 1 || spec.pdl == 3) ? ed : ed_plain;
    for (int it = 0; it < spec.unroll; ++it) {
      void* aa[] = {&a[it & 1]};
      cudaGraphNode_t na, nb;
      if (pdl) {
        if ((e = add_kernel(body, &na, nullptr, 0, step_a_fn<T, KB>(spec.var_a), spec.grid_spmv,
                            step_a_block(spec), aa, smem_a)))
          goto fail;
        if (prev && (e = cudaGraphAddDependencies(body, &prev, &na, &e_ba, 1))) goto fail;
        if ((e = add_kernel(body, &nb, nullptr, 0, step_b_fn<T, KB>(spec), spec.grid_stream_b, kThreads, aa)))
          goto fail;
        if ((e = cudaGraphAddDependencies(body, &na, &nb, &e_ab, 1))) goto fail;
        prev = nb;
        continue;
      }
      if ((e = add_kernel(body, &na, prev ? &prev : nullptr, prev ? 1 : 0, step_a_fn<T, KB>(spec.var_a),
                          spec.grid_spmv, step_a_block(spec), aa, smem_a)))
        goto fail;
      if (spec.var_a == 8) {  // the one-kernel iteration has no step b
        prev = na;
        continue;
      }
      if (spec.ilu.nblk > 0) {
        void* ba[] = {&a[it & 1], &ilu_f, &ilu_init0};
        if ((e = add_kernel(body, &nb, &na, 1, (const void*)cg_step_b_ilu_kernel<T, KB>, ilu_grid(spec), kThreads,
                            ba, smem_ilu)))
          goto fail;
      } else if ((e = add_kernel(body, &nb, &na, 1, step_b_fn<T, KB>(spec), spec.grid_stream_b, kThreads,
                                 aa))) {
        goto fail;
      }
      prev = nb;
    }
    cudaGraphNode_t nc;
    void* ctl_args[] = {&st, &h};
    if ((e = add_kernel(body, &nc, &prev, 1, (const void*)cg_ctl_kernel, 1, 1, ctl_args))) goto fail;
  }
  {
    void* fin_args[] = {&st, (void*)&zc, &n_pad};
    if ((e = add_kernel(g, &n_fin, &n_loop, 1, (const void*)cg_finish_kernel<T>, spec.grid_stream, kThreads,
                        fin_args)))
      goto fail;
  }
  *out_graph = g;
  return cudaSuccess;
fail:
  cudaGraphDestroy(g);
  return e;
}

// The same launch sequence as the graph, driven from the host: after every U
// iterations the host reads the `done` word.  Used when a profiler must see
// the individual kernels (kernel nodes under a conditional node cannot be
// profiled).
template <typename T, int KB>
cudaError_t run_host_t(const InnerGraphSpec& spec, cudaStream_t stream, int* h_done) {
  CgArgs<T> a[2];
  make_args(spec, a);
  const unsigned smem_a = step_a_smem<T, KB>(spec);
  cg_vnorm_kernel<<<spec.grid_stream, kThreads, 0, stream>>>(spec.st, spec.partials, spec.A.n_pad);
  launch_init<T, KB>(spec, stream, a[0]);
  cudaError_t e = cudaSuccess;
  for (;;) {
    for (int it = 0; it < spec.unroll; ++it) {
      launch_a<T>(step_a_fn<T, KB>(spec.var_a), spec.grid_spmv, step_a_block(spec), stream, a[it & 1], smem_a);
      if (spec.var_a != 8) launch_b<T, KB>(spec, stream, a[it & 1]);
    }
    cg_ctl_host_kernel<<<1, 1, 0, stream>>>(spec.st);
    if ((e = cudaMemcpyAsync(h_done, &spec.st->cg.done, sizeof(int), cudaMemcpyDeviceToHost, stream))) return e;
    if ((e = cudaStreamSynchronize(stream))) return e;
    if (*h_done != kRunning) break;
  }
  cg_finish_kernel<T><<<spec.grid_stream, kThreads, 0, stream>>>(spec.st, reinterpret_cast<const T*>(spec.z),
                                                                  spec.A.n_pad);
  return cudaGetLastError();
}

template <typename T, int KB>
cudaError_t time_t(const InnerGraphSpec& spec, int iters, cudaStream_t stream, double* vin, int64_t n,
                   double* ms) {
  CgArgs<T> a[2];
  make_args(spec, a);
  const unsigned smem_a = step_a_smem<T, KB>(spec);
  fill_pattern_kernel<<<spec.grid_stream, kThreads, 0, stream>>>(vin, n);
  cg_vnorm_kernel<<<spec.grid_stream, kThreads, 0, stream>>>(spec.st, spec.partials, spec.A.n_pad);
  launch_init<T, KB>(spec, stream, a[0]);
  std::vector<cudaEvent_t> ev(2 * (size_t)iters + 1);
  for (auto& e : ev) cudaEventCreate(&e);
  cudaEventRecord(ev[0], stream);
  for (int it = 0; it < iters; ++it) {
    launch_a<T>(step_a_fn<T, KB>(spec.var_a), spec.grid_spmv, step_a_block(spec), stream, a[it & 1], smem_a);
    cudaEventRecord(ev[2 * it + 1], stream);
    if (spec.var_a != 8) launch_b<T, KB>(spec, stream, a[it & 1]);
    cudaEventRecord(ev[2 * it + 2], stream);
  }
  cudaError_t e = cudaStreamSynchronize(stream);
  // ms[0], ms[1]: medians over the iterations (robust against a stray slow
  // launch; the autotuner's measure); ms[2], ms[3]: means
  std::vector<float> ta(iters, 0.f), tb(iters, 0.f);
  double sa = 0.0, sb = 0.0;
  for (int it = 0; it < iters && e == cudaSuccess; ++it) {
    cudaEventElapsedTime(&ta[it], ev[2 * it], ev[2 * it + 1]);
    cudaEventElapsedTime(&tb[it], ev[2 * it + 1], ev[2 * it + 2]);
    sa += ta[it];
    sb += tb[it];
  }
  for (auto& ee : ev) cudaEventDestroy(ee);
  std::sort(ta.begin(), ta.end());
  std::sort(tb.begin(), tb.end());
  ms[0] = iters > 0 ? ta[iters / 2] : 0.0;
  ms[1] = iters > 0 ? tb[iters / 2] : 0.0;
  ms[2] = iters > 0 ? sa / iters : 0.0;
  ms[3] = iters > 0 ? sb / iters : 0.0;
  if (e == cudaSuccess) e = cudaGetLastError();
  return e;
}

template <typename T, int KB>
void occupancy_t(const InnerGraphSpec& spec, int* a_blocks, int* b_blocks) {
  const unsigned smem = step_a_smem<T, KB>(spec);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(a_blocks, step_a_fn<T, KB>(spec.var_a), step_a_block(spec), smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(b_blocks, step_b_fn<T, KB>(spec), kThreads, 0);
}

// dispatch on the k bucket of the kernels (one precision per translation unit)
template <typename T, template <typename, int> class F, typename... Args>
cudaError_t dispatch_k(const InnerGraphSpec& spec, Args... args) {
  if (spec.k == 0) return F<T, 0>::run(spec, args...);
  if (spec.k <= 8) return F<T, 8>::run(spec, args...);
  if (spec.k <= 12) return F<T, 12>::run(spec, args...);
  if (spec.k <= 16) return F<T, 16>::run(spec, args...);
  if (spec.k <= 24) return F<T, 24>::run(spec, args...);
  return F<T, 32>::run(spec, args...);
}

template <typename T, int KB>
struct BuildF {
  static cudaError_t run(const InnerGraphSpec& s, cudaGraph_t* g) { return build_graph_t<T, KB>(s, g); }
};
template <typename T, int KB>
struct HostF {
  static cudaError_t run(const InnerGraphSpec& s, cudaStream_t st, int* d) { return run_host_t<T, KB>(s, st, d); }
};
template <typename T, int KB>
struct TimeF {
  static cudaError_t run(const InnerGraphSpec& s, int it, cudaStream_t st, double* v, int64_t n, double* ms) {
    return time_t<T, KB>(s, it, st, v, n, ms);
  }
};
template <typename T, int KB>
struct OccF {
  static cudaError_t run(const InnerGraphSpec& s, int* a, int* b) {
    occupancy_t<T, KB>(s, a, b);
    return cudaSuccess;
  }
};

template <typename T>
cudaError_t launch_gram_t(const InnerGraphSpec& spec, cudaStream_t stream, double* gram) {
  if (spec.k <= 0) return cudaSuccess;
  const int pairs = spec.k * (spec.k + 1) / 2;
  cg_gram_kernel<T><<<pairs, kThreads, 0, stream>>>(reinterpret_cast<const T*>(spec.V),
                                                     reinterpret_cast<const T*>(spec.dinv), spec.A.n_pad, spec.k, gram);
  return cudaGetLastError();
}

}  // namespace

// the entry points of one precision, defined by cg_f32.cu and cg_f64.cu
#define MRCG_CG_PRECISION_ENTRY_POINTS(T, SUFFIX)                                                                \
  cudaError_t build_inner_graph_##SUFFIX(const InnerGraphSpec& spec, cudaGraph_t* graph) {                      \
    return dispatch_k<T, BuildF>(spec, graph);                                                                   \
  }                                                                                                              \
  cudaError_t run_inner_host_##SUFFIX(const InnerGraphSpec& spec, cudaStream_t stream, int* h_done) {           \
    return dispatch_k<T, HostF>(spec, stream, h_done);                                                           \
  }                                                                                                              \
  cudaError_t time_inner_kernels_##SUFFIX(const InnerGraphSpec& spec, int iters, cudaStream_t stream,           \
                                          double* vin, int64_t n, double* ms) {                                  \
    return dispatch_k<T, TimeF>(spec, iters, stream, vin, n, ms);                                                \
  }                                                                                                              \
  cudaError_t launch_gram_##SUFFIX(const InnerGraphSpec& spec, cudaStream_t stream, double* gram) {             \
    return launch_gram_t<T>(spec, stream, gram);                                                                 \
  }                                                                                                              \
  void inner_occupancy_##SUFFIX(const InnerGraphSpec& spec, int* a, int* b) { dispatch_k<T, OccF>(spec, a, b); }

}  // namespace mrcg
