// Inner CG on M_mr z = y (Eq. 2, the inner block of Algorithm 1), one
// application of the preconditioner of the outer MINRES.
//
// One CG iteration is two streaming kernels (one grid-wide reduction each):
//   step_a: p' = s + beta p ; q = A p' + V c ; partial p'^T q
//           (the direction update is fused into the SpMV gathers, so p' is
//           never re-read; c = 2|Lambda| (V^T p') arrives as scalars)
//   step_b: z += alpha p' ; r -= alpha q ; s = M_cg^{-1} r ;
//           partials r^T s, r^T r, V^T s
// V^T p' for the next step follows from V^T p' = V^T s + beta V^T p, so the
// paper's two passes over V_hat per M_mr product (V^T u, then V t) stay two
// and no third kernel is needed.  All scalar recurrences (alpha, beta, the
// stopping test) run in FP64 in the last block of each kernel.
//
// The whole preconditioner application is one CUDA graph:
//   norm(v) -> init -> while(not done) { U x (step_a, step_b), ctl } -> finish
// The while loop is a conditional graph node: the inner iteration never
// returns to the host.
#include <cstdio>
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

template <typename T>
__device__ __forceinline__ T ld_stream(const T* p) {
  return __ldcs(p);
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

// ------------------------------------------------------------------ init

template <typename T, int KB>
__global__ void __launch_bounds__(kThreads) cg_init_kernel(CgArgs<T> a) {
  CgState& S = a.st->cg;
  const double vn = S.vnorm;
  const double scale = (vn > 0.0 && isfinite(vn)) ? 1.0 / vn : 0.0;
  const double* v = S.vin;
  T rs = 0, rr = 0;
  T u[KB > 0 ? KB : 1];
#pragma unroll
  for (int l = 0; l < (KB > 0 ? KB : 1); ++l) u[l] = 0;
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < a.n_pad; i += (int64_t)gridDim.x * kThreads) {
    const T r = (T)(v[i] * scale);
    a.r[i] = r;
    a.z[i] = 0;
    a.p_old[i] = 0;
    T s = r;
    if (a.dinv) {
      s = a.dinv[i] * r;
      a.s[i] = s;
    }
    rs += r * s;
    rr += r * r;
#pragma unroll
    for (int l = 0; l < KB; ++l)
      if (l < a.k) u[l] += ld_stream(a.V + (size_t)l * a.n_pad + i) * s;
  }
  double acc[KB + 2];
  acc[0] = (double)rs;
  acc[1] = (double)rr;
#pragma unroll
  for (int l = 0; l < KB; ++l) acc[l + 2] = (double)u[l];
  block_partials<KB + 2>(acc, a.k + 2, a.partials);
  if (last_block(&a.st->ticket)) {
    __shared__ double tot[KB + 2];
    final_sums(a.partials, a.k + 2, tot);
    if (threadIdx.x == 0) {
      const double rho = tot[0], rnorm = sqrt(tot[1]);
      S.rho = rho;
      S.beta = 0.0;
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
      for (int l = 0; l < a.k; ++l) {
        S.t[l] = tot[l + 2];
        S.c[l] = S.lam2[l] * tot[l + 2];
      }
    }
  }
}

// ------------------------------------------------------------------ step a

template <typename T, int KB>
__global__ void __launch_bounds__(kThreads) cg_step_a_kernel(CgArgs<T> a) {
  CgState& S = a.st->cg;
  if (S.done != kRunning) return;
  const T beta = (T)S.beta;
  T cl[KB > 0 ? KB : 1];
#pragma unroll
  for (int l = 0; l < KB; ++l) cl[l] = (l < a.k) ? (T)S.c[l] : (T)0;
  const T* __restrict__ sv = a.s;
  const T* __restrict__ po = a.p_old;
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = (blockIdx.x * (int64_t)kThreads + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
  T dot = 0;
  for (int64_t sl = warp0; sl < a.nslices; sl += nwarps) {
    const int64_t base = a.slice_ptr[sl];
    const int w = (int)((a.slice_ptr[sl + 1] - base) >> 5);
    const T* vp = a.val + base + lane;
    const int32_t* cp = a.col + base + lane;
    T acc = 0;
#pragma unroll 4
    for (int j = 0; j < w; ++j) {
      const T av = ld_stream(vp + (size_t)j * kSlice);
      const int c = ld_stream(cp + (size_t)j * kSlice);
      acc += av * (__ldg(sv + c) + beta * __ldg(po + c));
    }
    const int64_t row = sl * kSlice + lane;
    const T pn = sv[row] + beta * po[row];
#pragma unroll
    for (int l = 0; l < KB; ++l)
      if (l < a.k) acc += ld_stream(a.V + (size_t)l * a.n_pad + row) * cl[l];
    a.q[row] = acc;
    a.p_new[row] = pn;
    dot += pn * acc;
  }
  double part[1] = {(double)dot};
  block_partials<1>(part, 1, a.partials);
  if (last_block(&a.st->ticket)) {
    __shared__ double tot[1];
    final_sums(a.partials, 1, tot);
    if (threadIdx.x == 0) {
      const double kappa = tot[0];
      S.kappa = kappa;
      if (!isfinite(kappa)) {
        S.done = kNonFinite;
      } else if (kappa <= 0.0) {
        S.done = kNotSpd;
      } else {
        S.alpha = S.rho / kappa;
      }
    }
  }
}

// ------------------------------------------------------------------ step b

template <typename T, int KB>
__global__ void __launch_bounds__(kThreads) cg_step_b_kernel(CgArgs<T> a) {
  CgState& S = a.st->cg;
  if (S.done != kRunning) return;
  const T alpha = (T)S.alpha;
  T rs = 0, rr = 0;
  T u[KB > 0 ? KB : 1];
#pragma unroll
  for (int l = 0; l < (KB > 0 ? KB : 1); ++l) u[l] = 0;
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < a.n_pad; i += (int64_t)gridDim.x * kThreads) {
    const T pn = a.p_new[i];
    const T qi = a.q[i];
    a.z[i] = a.z[i] + alpha * pn;
    const T r = a.r[i] - alpha * qi;
    a.r[i] = r;
    T s = r;
    if (a.dinv) {
      s = a.dinv[i] * r;
      a.s[i] = s;
    }
    rs += r * s;
    rr += r * r;
#pragma unroll
    for (int l = 0; l < KB; ++l)
      if (l < a.k) u[l] += ld_stream(a.V + (size_t)l * a.n_pad + i) * s;
  }
  double acc[KB + 2];
  acc[0] = (double)rs;
  acc[1] = (double)rr;
#pragma unroll
  for (int l = 0; l < KB; ++l) acc[l + 2] = (double)u[l];
  block_partials<KB + 2>(acc, a.k + 2, a.partials);
  if (last_block(&a.st->ticket)) {
    __shared__ double tot[KB + 2];
    final_sums(a.partials, a.k + 2, tot);
    if (threadIdx.x == 0) {
      const double rho_new = tot[0], rnorm = sqrt(tot[1]);
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
        S.rho = rho_new;
        for (int l = 0; l < a.k; ++l) {
          const double t = tot[l + 2] + beta * S.t[l];
          S.t[l] = t;
          S.c[l] = S.lam2[l] * t;
        }
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

// ------------------------------------------------------------------ graph assembly

namespace {

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
cudaError_t build_graph_t(const InnerGraphSpec& spec, cudaGraph_t* out_graph) {
  cudaError_t e;
  cudaGraph_t g;
  if ((e = cudaGraphCreate(&g, 0)) != cudaSuccess) return e;
  CgArgs<T> a[2];
  for (int par = 0; par < 2; ++par) {
    CgArgs<T>& x = a[par];
    x.st = spec.st;
    x.partials = spec.partials;
    x.slice_ptr = spec.A.slice_ptr;
    x.col = spec.A.col;
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
      if ((e = add_kernel(body, &na, prev ? &prev : nullptr, prev ? 1 : 0, (const void*)cg_step_a_kernel<T, KB>,
                          spec.grid_spmv, kThreads, aa)))
        goto fail;
      if ((e = add_kernel(body, &nb, &na, 1, (const void*)cg_step_b_kernel<T, KB>, spec.grid_stream, kThreads, aa)))
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

template <typename T>
cudaError_t build_graph_k(const InnerGraphSpec& spec, cudaGraph_t* g) {
  if (spec.k == 0) return build_graph_t<T, 0>(spec, g);
  if (spec.k <= 8) return build_graph_t<T, 8>(spec, g);
  if (spec.k <= 16) return build_graph_t<T, 16>(spec, g);
  return build_graph_t<T, 32>(spec, g);
}

__global__ void fill_pattern_kernel(double* v, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads)
    v[i] = 1.0 + 0.125 * (double)(i % 7) - 0.0625 * (double)(i % 3);
}

template <typename T, int KB>
cudaError_t time_t(const InnerGraphSpec& spec, int iters, cudaStream_t stream, double* vin, int64_t n,
                   double* ms) {
  CgArgs<T> a[2];
  for (int par = 0; par < 2; ++par) {
    CgArgs<T>& x = a[par];
    x.st = spec.st;
    x.partials = spec.partials;
    x.slice_ptr = spec.A.slice_ptr;
    x.col = spec.A.col;
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
  fill_pattern_kernel<<<spec.grid_stream, kThreads, 0, stream>>>(vin, n);
  cg_vnorm_kernel<<<spec.grid_stream, kThreads, 0, stream>>>(spec.st, spec.partials, spec.A.n_pad);
  cg_init_kernel<T, KB><<<spec.grid_stream, kThreads, 0, stream>>>(a[0]);
  std::vector<cudaEvent_t> ev(2 * (size_t)iters + 1);
  for (auto& e : ev) cudaEventCreate(&e);
  cudaEventRecord(ev[0], stream);
  for (int it = 0; it < iters; ++it) {
    cg_step_a_kernel<T, KB><<<spec.grid_spmv, kThreads, 0, stream>>>(a[it & 1]);
    cudaEventRecord(ev[2 * it + 1], stream);
    cg_step_b_kernel<T, KB><<<spec.grid_stream, kThreads, 0, stream>>>(a[it & 1]);
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

template <typename T>
cudaError_t time_k(const InnerGraphSpec& spec, int iters, cudaStream_t stream, double* vin, int64_t n, double* ms) {
  if (spec.k == 0) return time_t<T, 0>(spec, iters, stream, vin, n, ms);
  if (spec.k <= 8) return time_t<T, 8>(spec, iters, stream, vin, n, ms);
  if (spec.k <= 16) return time_t<T, 16>(spec, iters, stream, vin, n, ms);
  return time_t<T, 32>(spec, iters, stream, vin, n, ms);
}

template <typename T, int KB>
void occupancy_t(int* a_blocks, int* b_blocks) {
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(a_blocks, (const void*)cg_step_a_kernel<T, KB>, kThreads, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(b_blocks, (const void*)cg_step_b_kernel<T, KB>, kThreads, 0);
}

}  // namespace

cudaError_t time_inner_kernels(const InnerGraphSpec& spec, int iters, cudaStream_t stream, double* vin, int64_t n,
                               double* ms) {
  if (spec.fp32) return time_k<float>(spec, iters, stream, vin, n, ms);
  return time_k<double>(spec, iters, stream, vin, n, ms);
}

cudaError_t build_inner_graph(const InnerGraphSpec& spec, cudaGraph_t* graph) {
  if (spec.fp32) return build_graph_k<float>(spec, graph);
  return build_graph_k<double>(spec, graph);
}

void inner_occupancy(bool fp32, int k, int* spmv_blocks_per_sm, int* stream_blocks_per_sm) {
  *spmv_blocks_per_sm = 1;
  *stream_blocks_per_sm = 1;
  if (fp32) {
    if (k == 0) occupancy_t<float, 0>(spmv_blocks_per_sm, stream_blocks_per_sm);
    else if (k <= 8) occupancy_t<float, 8>(spmv_blocks_per_sm, stream_blocks_per_sm);
    else if (k <= 16) occupancy_t<float, 16>(spmv_blocks_per_sm, stream_blocks_per_sm);
    else occupancy_t<float, 32>(spmv_blocks_per_sm, stream_blocks_per_sm);
  } else {
    if (k == 0) occupancy_t<double, 0>(spmv_blocks_per_sm, stream_blocks_per_sm);
    else if (k <= 8) occupancy_t<double, 8>(spmv_blocks_per_sm, stream_blocks_per_sm);
    else if (k <= 16) occupancy_t<double, 16>(spmv_blocks_per_sm, stream_blocks_per_sm);
    else occupancy_t<double, 32>(spmv_blocks_per_sm, stream_blocks_per_sm);
  }
}

}  // namespace mrcg
