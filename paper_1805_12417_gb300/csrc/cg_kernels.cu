// Inner CG on M_mr z = y (Eq. 2, the inner block of Algorithm 1), one
// application of the preconditioner of the outer MINRES.
//
// One CG iteration is two streaming kernels (one grid-wide reduction each):
//   step_a: p' = s + beta p ; q = A p' + V c ; partial p'^T q
//           (the direction update is fused into the SpMV gathers, so p' is
//           never re-read; c = 2|Lambda| (V^T p') arrives as scalars)
//   step_b: z += alpha p' ; r -= alpha q ; s = M_cg^{-1} r ;
//           partials r^T s, V^T s (and r^T r when M_cg is Jacobi)
// V^T p' for the next step follows from V^T p' = V^T s + beta V^T p, so the
// paper's two passes over V_hat per M_mr product (V^T u, then V t) stay two
// and no third kernel is needed.  All scalar recurrences (alpha, beta, the
// stopping test) run in FP64 in the last block of each kernel, which also
// publishes FP32 copies for the FP32 kernels.  Per-thread sums and the block
// reductions run in the kernel's own precision (FP32 in mixed mode), the
// cross-block sum in FP64.
//
// The whole preconditioner application is one CUDA graph:
//   norm(v) -> init -> while(not done) { U x (step_a, step_b), ctl } -> finish
// The while loop is a conditional graph node: the inner iteration never
// returns to the host.
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
  int k;
  // Jacobi: dinv != nullptr, s is a separate vector; identity: s == r
  const T* dinv;
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

template <typename T>
struct V16;
template <>
struct V16<float> {
  using type = float4;
  static constexpr int W = 4;
};
template <>
struct V16<double> {
  using type = double2;
  static constexpr int W = 2;
};

// 16-byte vector load / store into a register array
template <typename T>
__device__ __forceinline__ void ld16(const T* p, T (&x)[V16<T>::W]) {
  const typename V16<T>::type v = *reinterpret_cast<const typename V16<T>::type*>(p);
  memcpy(x, &v, 16);
}
template <typename T>
__device__ __forceinline__ void ld16_stream(const T* p, T (&x)[V16<T>::W]) {
  const typename V16<T>::type v = __ldcs(reinterpret_cast<const typename V16<T>::type*>(p));
  memcpy(x, &v, 16);
}
template <typename T>
__device__ __forceinline__ void st16(T* p, const T (&x)[V16<T>::W]) {
  typename V16<T>::type v;
  memcpy(&v, x, 16);
  *reinterpret_cast<typename V16<T>::type*>(p) = v;
}

// broadcast scalars in the kernel's precision
__device__ __forceinline__ float alpha_of(const CgState& S, float) { return S.alpha32; }
__device__ __forceinline__ double alpha_of(const CgState& S, double) { return S.alpha; }
__device__ __forceinline__ float beta_of(const CgState& S, float) { return S.beta32; }
__device__ __forceinline__ double beta_of(const CgState& S, double) { return S.beta; }
__device__ __forceinline__ float c_of(const CgState& S, int l, float) { return S.c32[l]; }
__device__ __forceinline__ double c_of(const CgState& S, int l, double) { return S.c[l]; }

// set c = 2|lambda| t (FP64 and FP32 copies)
__device__ __forceinline__ void publish_c(CgState& S, int k) {
  for (int l = 0; l < k; ++l) {
    S.c[l] = S.lam2[l] * S.t[l];
    S.c32[l] = (float)S.c[l];
  }
}

// ------------------------------------------------------------------ norm of v

__global__ void __launch_bounds__(kThreads) cg_vnorm_kernel(DevState* st, double* partials, int64_t n_pad) {
  CgState& S = st->cg;
  const double* v = S.vin;
  double acc[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n_pad; i += (int64_t)gridDim.x * kThreads) {
    const double x = v[i];
    acc[0] += x * x;
  }
  block_partials<1>(acc, 1, partials);
  if (last_block(&st->ticket)) {
    __shared__ double tot[1];
    final_sums(partials, 1, tot);
    if (threadIdx.x == 0) S.vnorm = sqrt(tot[0]);
  }
}

// Reduction slots of init / step_b:  [0] = r^T s, [1 .. k] = V^T s,
// [k + 1] = r^T r (Jacobi only; with M_cg = I, r^T s is r^T r).  Indices are
// compile-time after unrolling, so the slot array stays in registers.
template <typename T, int KB>
__device__ __forceinline__ void pack_slots(T (&acc)[KB + 2], T rs, const T (&u)[KB > 0 ? KB : 1], T rr, int k,
                                           bool jac) {
  constexpr int KS = KB > 0 ? KB : 1;
#pragma unroll
  for (int l = 0; l < KB + 2; ++l) {
    T val = (T)0;
    if (l == 0) val = rs;
    else if (l - 1 < KB && l - 1 < k) val = u[(l - 1 < KS) ? l - 1 : 0];
    else if (jac && l == k + 1) val = rr;
    acc[l] = val;
  }
}

// ------------------------------------------------------------------ init

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
    st16(a.p_old + i, zero);
    if (jac) {
      T d[W];
      ld16(a.dinv + i, d);
#pragma unroll
      for (int e = 0; e < W; ++e) s[e] = d[e] * r[e];
      st16(a.s + i, s);
    } else {
#pragma unroll
      for (int e = 0; e < W; ++e) s[e] = r[e];
    }
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
  if (last_block(&a.st->ticket)) {
    __shared__ double tot[KB + 2];
    final_sums(a.partials, nv, tot);
    if (threadIdx.x == 0) {
      const double rho = tot[0], rnorm = sqrt(jac ? tot[a.k + 1] : tot[0]);
      S.rho = rho;
      S.beta = 0.0;
      S.beta32 = 0.0f;
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
      if (!isfinite(vn) || !isfinite(rho)) {
        S.done = kNonFinite;
      } else if (vn == 0.0 || rnorm == 0.0) {
        S.done = kConverged;
      } else if (S.maxit <= 0) {
        S.done = kMaxIter;
      }
      for (int l = 0; l < a.k; ++l) S.t[l] = S.u[l] = tot[l + 1];
      publish_c(S, a.k);
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

// Variants (picked per handle by the launch-shape autotuner):
//   VAR 0: V_hat row loads issued before the SpMV (more bytes in flight)
//   VAR 1: V_hat read after the SpMV (fewer registers)
//   VAR 2: two slices per warp per trip, V_hat early (more independent work)
template <typename T, int KB, int VAR>
__global__ void __launch_bounds__(kThreads, 4) cg_step_a_kernel(CgArgs<T> a) {
  constexpr int KS = KB > 0 ? KB : 1;
  constexpr int NSL = VAR == 2 ? 2 : 1;
  constexpr bool kEarlyV = VAR != 1;
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
  // wq[l] = (V^T M_cg^{-1} q)_l: with this step b needs no pass over V (see step b)
  T wq[KS];
#pragma unroll
  for (int l = 0; l < KS; ++l) wq[l] = 0;
  for (int64_t sl0 = warp0 * NSL; sl0 < a.nslices; sl0 += nwarps * NSL) {
    T vrow[NSL][KS], srow[NSL], prow[NSL], acc[NSL];
    int64_t rowv[NSL];
    bool ok[NSL];
#pragma unroll
    for (int h = 0; h < NSL; ++h) {
      const int64_t sl = sl0 + h;
      ok[h] = sl < a.nslices;
      rowv[h] = (ok[h] ? sl : sl0) * kSlice + lane;
      if (kEarlyV) {
#pragma unroll
        for (int l = 0; l < KS; ++l)
          vrow[h][l] = (ok[h] && l < a.k) ? ld_stream(a.V + (size_t)l * a.n_pad + rowv[h]) : (T)0;
      }
      srow[h] = sv[rowv[h]];
      prow[h] = po[rowv[h]];
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
      T q = acc[h];
      if (!kEarlyV) {
#pragma unroll
        for (int l = 0; l < KS; ++l)
          vrow[h][l] = (l < a.k) ? ld_stream(a.V + (size_t)l * a.n_pad + row) : (T)0;
      }
#pragma unroll
      for (int l = 0; l < KB; ++l)
        if (l < a.k) q += vrow[h][l] * cl[l];
      a.q[row] = q;
      a.p_new[row] = pn;
      dot += pn * q;
      const T qs = jac ? a.dinv[row] * q : q;
#pragma unroll
      for (int l = 0; l < KB; ++l)
        if (l < a.k) wq[l] += vrow[h][l] * qs;
    }
  }
  T part[KB + 1];
  part[0] = dot;
#pragma unroll
  for (int l = 0; l < KB; ++l) part[l + 1] = wq[l];
  block_partials_t<T, KB + 1>(part, a.k + 1, a.partials);
  if (last_block(&a.st->ticket)) {
    __shared__ double tot[KB + 1];
    final_sums(a.partials, a.k + 1, tot);
    if (threadIdx.x == 0) {
      const double kappa = tot[0];
      S.kappa = kappa;
      for (int l = 0; l < a.k; ++l) S.vq[l] = tot[l + 1];
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

// ------------------------------------------------------------------ step b

// V^T s_{i+1} = V^T s_i - alpha V^T (M_cg^{-1} q_i) follows from the
// partials step a already formed (exact algebra, the same recurrence CG uses
// for r itself), so this kernel streams only the four CG vectors.
template <typename T, int KB>
__global__ void __launch_bounds__(kThreads) cg_step_b_kernel(CgArgs<T> a) {
  constexpr int W = V16<T>::W;
  CgState& S = a.st->cg;
  if (S.done != kRunning) return;
  const T alpha = alpha_of(S, T(0));
  const bool jac = a.dinv != nullptr;
  T rs = 0, rr = 0;
  const int64_t nvec = a.n_pad / W;
  for (int64_t iv = blockIdx.x * (int64_t)kThreads + threadIdx.x; iv < nvec; iv += (int64_t)gridDim.x * kThreads) {
    const int64_t i = iv * W;
    T pn[W], qv[W], zv[W], rv[W], s[W];
    ld16(a.p_new + i, pn);
    ld16(a.q + i, qv);
    ld16(a.z + i, zv);
    ld16(a.r + i, rv);
#pragma unroll
    for (int e = 0; e < W; ++e) {
      zv[e] += alpha * pn[e];
      rv[e] -= alpha * qv[e];
    }
    st16(a.z + i, zv);
    st16(a.r + i, rv);
    if (jac) {
      T d[W];
      ld16(a.dinv + i, d);
#pragma unroll
      for (int e = 0; e < W; ++e) {
        s[e] = d[e] * rv[e];
        rr += rv[e] * rv[e];
      }
      st16(a.s + i, s);
    } else {
#pragma unroll
      for (int e = 0; e < W; ++e) s[e] = rv[e];
    }
#pragma unroll
    for (int e = 0; e < W; ++e) rs += rv[e] * s[e];
  }
  T acc[2] = {rs, rr};
  const int nv = jac ? 2 : 1;
  block_partials_t<T, 2>(acc, nv, a.partials);
  if (last_block(&a.st->ticket)) {
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

__global__ void cg_ctl_kernel(DevState* st, cudaGraphConditionalHandle handle) {
  CgState& S = st->cg;
  S.ctl_count += 1;
  if (S.done == kRunning && S.ctl_count >= S.ctl_limit) S.done = kLoopCap;
  cudaGraphSetConditional(handle, S.done == kRunning ? 1u : 0u);
}

// the same bookkeeping for the host-driven loop (no graph condition)
__global__ void cg_ctl_host_kernel(DevState* st) {
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
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n_pad; i += (int64_t)gridDim.x * kThreads)
    out[i] = vn * (double)z[i];
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
    }
  }
}

__global__ void fill_pattern_kernel(double* v, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads)
    v[i] = 1.0 + 0.125 * (double)(i % 7) - 0.0625 * (double)(i % 3);
}

// ------------------------------------------------------------------ host side

namespace {

template <typename T>
void make_args(const InnerGraphSpec& spec, CgArgs<T> (&a)[2]) {
  for (int par = 0; par < 2; ++par) {
    CgArgs<T>& x = a[par];
    x.st = spec.st;
    x.partials = spec.partials;
    x.slice_ptr = spec.A.slice_ptr;
    x.col = spec.A.col;
    x.col16 = spec.A.col16;
    x.val = reinterpret_cast<const T*>(sizeof(T) == 8 ? (const void*)spec.A.val64 : (const void*)spec.A.val32);
    x.nslices = spec.A.nslices;
    x.n_pad = spec.A.n_pad;
    x.V = reinterpret_cast<const T*>(spec.V);
    x.k = spec.k;
    x.dinv = reinterpret_cast<const T*>(spec.dinv);
    x.z = reinterpret_cast<T*>(spec.z);
    x.r = reinterpret_cast<T*>(spec.r);
    x.s = spec.dinv ? reinterpret_cast<T*>(spec.s) : reinterpret_cast<T*>(spec.r);
    x.q = reinterpret_cast<T*>(spec.q);
    x.p_old = reinterpret_cast<T*>(par == 0 ? spec.p0 : spec.p1);
    x.p_new = reinterpret_cast<T*>(par == 0 ? spec.p1 : spec.p0);
  }
}

cudaError_t add_kernel(cudaGraph_t g, cudaGraphNode_t* node, const cudaGraphNode_t* deps, size_t ndeps,
                       const void* fn, int grid, int block, void** args) {
  cudaKernelNodeParams p = {};
  p.func = const_cast<void*>(fn);
  p.gridDim = dim3(grid);
  p.blockDim = dim3(block);
  p.sharedMemBytes = 0;
  p.kernelParams = args;
  p.extra = nullptr;
  return cudaGraphAddKernelNode(node, g, deps, ndeps, &p);
}

template <typename T, int KB>
const void* step_a_fn(int var) {
  switch (var) {
    case 1: return (const void*)cg_step_a_kernel<T, KB, 1>;
    case 2: return (const void*)cg_step_a_kernel<T, KB, 2>;
    default: return (const void*)cg_step_a_kernel<T, KB, 0>;
  }
}

template <typename T>
cudaError_t launch_a(const void* fn, int grid, cudaStream_t stream, CgArgs<T>& a) {
  void* args[] = {&a};
  return cudaLaunchKernel(fn, dim3(grid), dim3(kThreads), args, 0, stream);
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

  cudaGraphNode_t n_norm, n_init, n_loop, n_fin;
  void* norm_args[] = {&st, &partials, &n_pad};
  if ((e = add_kernel(g, &n_norm, nullptr, 0, (const void*)cg_vnorm_kernel, spec.grid_stream, kThreads, norm_args)))
    goto fail;
  {
    void* init_args[] = {&a[0]};
    if ((e = add_kernel(g, &n_init, &n_norm, 1, (const void*)cg_init_kernel<T, KB>, spec.grid_stream, kThreads,
                        init_args)))
      goto fail;
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
    for (int it = 0; it < spec.unroll; ++it) {
      void* aa[] = {&a[it & 1]};
      cudaGraphNode_t na, nb;
      if ((e = add_kernel(body, &na, prev ? &prev : nullptr, prev ? 1 : 0, step_a_fn<T, KB>(spec.var_a),
                          spec.grid_spmv, kThreads, aa)))
        goto fail;
      if ((e = add_kernel(body, &nb, &na, 1, (const void*)cg_step_b_kernel<T, KB>, spec.grid_stream_b, kThreads,
                          aa)))
        goto fail;
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
  cg_vnorm_kernel<<<spec.grid_stream, kThreads, 0, stream>>>(spec.st, spec.partials, spec.A.n_pad);
  cg_init_kernel<T, KB><<<spec.grid_stream, kThreads, 0, stream>>>(a[0]);
  cudaError_t e = cudaSuccess;
  for (;;) {
    for (int it = 0; it < spec.unroll; ++it) {
      launch_a<T>(step_a_fn<T, KB>(spec.var_a), spec.grid_spmv, stream, a[it & 1]);
      cg_step_b_kernel<T, KB><<<spec.grid_stream_b, kThreads, 0, stream>>>(a[it & 1]);
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
  fill_pattern_kernel<<<spec.grid_stream, kThreads, 0, stream>>>(vin, n);
  cg_vnorm_kernel<<<spec.grid_stream, kThreads, 0, stream>>>(spec.st, spec.partials, spec.A.n_pad);
  cg_init_kernel<T, KB><<<spec.grid_stream, kThreads, 0, stream>>>(a[0]);
  std::vector<cudaEvent_t> ev(2 * (size_t)iters + 1);
  for (auto& e : ev) cudaEventCreate(&e);
  cudaEventRecord(ev[0], stream);
  for (int it = 0; it < iters; ++it) {
    launch_a<T>(step_a_fn<T, KB>(spec.var_a), spec.grid_spmv, stream, a[it & 1]);
    cudaEventRecord(ev[2 * it + 1], stream);
    cg_step_b_kernel<T, KB><<<spec.grid_stream_b, kThreads, 0, stream>>>(a[it & 1]);
    cudaEventRecord(ev[2 * it + 2], stream);
  }
  cudaError_t e = cudaStreamSynchronize(stream);
  double ta = 0.0, tb = 0.0;
  for (int it = 0; it < iters && e == cudaSuccess; ++it) {
    float x = 0.f, y = 0.f;
    cudaEventElapsedTime(&x, ev[2 * it], ev[2 * it + 1]);
    cudaEventElapsedTime(&y, ev[2 * it + 1], ev[2 * it + 2]);
    ta += x;
    tb += y;
  }
  for (auto& ee : ev) cudaEventDestroy(ee);
  ms[0] = ta / iters;
  ms[1] = tb / iters;
  if (e == cudaSuccess) e = cudaGetLastError();
  return e;
}

template <typename T, int KB>
void occupancy_t(int* a_blocks, int* b_blocks) {
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(a_blocks, step_a_fn<T, KB>(0), kThreads, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(b_blocks, (const void*)cg_step_b_kernel<T, KB>, kThreads, 0);
}

// dispatch on (precision, k bucket)
template <template <typename, int> class F, typename... Args>
cudaError_t dispatch(const InnerGraphSpec& spec, Args... args) {
  if (spec.fp32) {
    if (spec.k == 0) return F<float, 0>::run(spec, args...);
    if (spec.k <= 8) return F<float, 8>::run(spec, args...);
    if (spec.k <= 16) return F<float, 16>::run(spec, args...);
    if (spec.k <= 24) return F<float, 24>::run(spec, args...);
    return F<float, 32>::run(spec, args...);
  }
  if (spec.k == 0) return F<double, 0>::run(spec, args...);
  if (spec.k <= 8) return F<double, 8>::run(spec, args...);
  if (spec.k <= 16) return F<double, 16>::run(spec, args...);
  if (spec.k <= 24) return F<double, 24>::run(spec, args...);
  return F<double, 32>::run(spec, args...);
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
  static cudaError_t run(const InnerGraphSpec&, int* a, int* b) {
    occupancy_t<T, KB>(a, b);
    return cudaSuccess;
  }
};

}  // namespace

cudaError_t build_inner_graph(const InnerGraphSpec& spec, cudaGraph_t* graph) {
  return dispatch<BuildF>(spec, graph);
}

cudaError_t run_inner_host(const InnerGraphSpec& spec, cudaStream_t stream, int* h_done) {
  return dispatch<HostF>(spec, stream, h_done);
}

cudaError_t time_inner_kernels(const InnerGraphSpec& spec, int iters, cudaStream_t stream, double* vin, int64_t n,
                               double* ms) {
  return dispatch<TimeF>(spec, iters, stream, vin, n, ms);
}

void inner_occupancy(bool fp32, int k, int* spmv_blocks_per_sm, int* stream_blocks_per_sm) {
  *spmv_blocks_per_sm = 1;
  *stream_blocks_per_sm = 1;
  InnerGraphSpec s;
  s.fp32 = fp32;
  s.k = k;
  dispatch<OccF>(s, spmv_blocks_per_sm, stream_blocks_per_sm);
}

}  // namespace mrcg
