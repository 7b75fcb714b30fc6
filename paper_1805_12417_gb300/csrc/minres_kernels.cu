// Outer preconditioned MINRES (Algorithm 1, outer level) in FP64, plus the
// SpMV with A, setup kernels and the operator kernels of the C ABI.
//
// One outer step j (Lanczos in the P^{-1} inner product with unnormalised
// vectors, Givens QR of the tridiagonal, short recurrence for w):
//   lanczos_spmv    zn = z_j / gamma_j ; az = A zn ; delta_j = zn^T az
//   lanczos_update  v_{j+1} = az - (delta_j/gamma_j) v_j - (gamma_j/gamma_{j-1}) v_{j-1}
//   inner CG graph  z_{j+1} ~ M_mr^{-1} v_{j+1}
//   gamma_givens    gamma_{j+1} = sqrt(z_{j+1}^T v_{j+1}); rotation (c, s); eta
//   minres_update   w_{j+1} = (zn - a3 w_{j-1} - a2 w_j) / a1 ; x += c eta w_{j+1}
//   residual        r = b - A x ; true relative residual (the stopping test)
// Each kernel streams its vectors once; reductions finish in the last block.
#include "common.cuh"
#include "kernels.h"

namespace mrcg {

namespace {

__device__ __forceinline__ bool failed(const DevState* st) { return st->out.status != MRCG_OK; }

// sum over the stored entries of one row of a SELL slice (lane = row in slice)
template <typename T, typename F>
__device__ __forceinline__ T sell_row_dot(const int64_t* __restrict__ slice_ptr, const int32_t* __restrict__ col,
                                          const T* __restrict__ val, int64_t sl, int lane, F gather) {
  const int64_t base = slice_ptr[sl];
  const int w = (int)((slice_ptr[sl + 1] - base) >> 5);
  const T* vp = val + base + lane;
  const int32_t* cp = col + base + lane;
  T acc = 0;
#pragma unroll 4
  for (int j = 0; j < w; ++j) {
    const T av = __ldcs(vp + (size_t)j * kSlice);
    const int c = __ldcs(cp + (size_t)j * kSlice);
    acc += av * gather(c);
  }
  return acc;
}

#define SLICE_LOOP(A)                                                                    \
  const int lane = threadIdx.x & 31;                                                     \
  const int64_t warp0 = (blockIdx.x * (int64_t)kThreads + threadIdx.x) >> 5;            \
  const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;                           \
  for (int64_t sl = warp0; sl < (A).nslices; sl += nwarps)

#define ROW_LOOP(i, n)                                                                          \
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < (n); i += (int64_t)gridDim.x * kThreads)

// ------------------------------------------------------------------ plain SpMV

__global__ void __launch_bounds__(kThreads) spmv_kernel(Sell A, const double* __restrict__ x, double* __restrict__ y) {
  SLICE_LOOP(A) {
    const double acc = sell_row_dot<double>(A.slice_ptr, A.col, A.val64, sl, lane, [&](int c) { return __ldg(x + c); });
    y[sl * kSlice + lane] = acc;
  }
}

// ------------------------------------------------------------------ M_mr product (operator entry point)

template <typename T, int KB>
__global__ void __launch_bounds__(kThreads) vtu_kernel(DevState* st, double* partials, const T* __restrict__ V, int k,
                                                         int64_t n_pad, const T* __restrict__ u) {
  T acc[KB];
#pragma unroll
  for (int l = 0; l < KB; ++l) acc[l] = 0;
  ROW_LOOP(i, n_pad) {
    const T ui = u[i];
#pragma unroll
    for (int l = 0; l < KB; ++l)
      if (l < k) acc[l] += __ldcs(V + (size_t)l * n_pad + i) * ui;
  }
  double d[KB];
#pragma unroll
  for (int l = 0; l < KB; ++l) d[l] = (double)acc[l];
  block_partials<KB>(d, k, partials);
  if (last_block(&st->ticket)) {
    __shared__ double tot[KB];
    final_sums(partials, k, tot);
    if (threadIdx.x < k) st->cg.c[threadIdx.x] = st->cg.lam2[threadIdx.x] * tot[threadIdx.x];
  }
}

template <typename T, int KB>
__global__ void __launch_bounds__(kThreads) mmr_kernel(const DevState* st, Sell A, const T* __restrict__ val,
                                                         const T* __restrict__ V, int k, const T* __restrict__ u,
                                                         T* __restrict__ out) {
  T cl[KB > 0 ? KB : 1];
#pragma unroll
  for (int l = 0; l < KB; ++l) cl[l] = (l < k) ? (T)st->cg.c[l] : (T)0;
  SLICE_LOOP(A) {
    T acc = sell_row_dot<T>(A.slice_ptr, A.col, val, sl, lane, [&](int c) { return __ldg(u + c); });
    const int64_t row = sl * kSlice + lane;
#pragma unroll
    for (int l = 0; l < KB; ++l)
      if (l < k) acc += __ldcs(V + (size_t)l * A.n_pad + row) * cl[l];
    out[row] = acc;
  }
}

// ------------------------------------------------------------------ norms and residual

__global__ void __launch_bounds__(kThreads) bnorm_kernel(DevState* st, double* partials, const double* __restrict__ b,
                                                           int64_t n_pad) {
  double acc[1] = {0.0};
  ROW_LOOP(i, n_pad) {
    const double x = b[i];
    acc[0] += x * x;
  }
  block_partials<1>(acc, 1, partials);
  if (last_block(&st->ticket)) {
    __shared__ double tot[1];
    final_sums(partials, 1, tot);
    if (threadIdx.x == 0) st->out.bnorm = sqrt(tot[0]);
  }
}

__global__ void __launch_bounds__(kThreads) residual_kernel(DevState* st, double* partials, Sell A,
                                                              const double* __restrict__ b,
                                                              const double* __restrict__ x, double* __restrict__ res) {
  if (failed(st)) return;
  double acc[1] = {0.0};
  SLICE_LOOP(A) {
    const double ax = sell_row_dot<double>(A.slice_ptr, A.col, A.val64, sl, lane, [&](int c) { return __ldg(x + c); });
    const int64_t row = sl * kSlice + lane;
    const double r = b[row] - ax;
    res[row] = r;
    acc[0] += r * r;
  }
  block_partials<1>(acc, 1, partials);
  if (last_block(&st->ticket)) {
    __shared__ double tot[1];
    final_sums(partials, 1, tot);
    if (threadIdx.x == 0) {
      OuterState& O = st->out;
      O.rnorm2 = tot[0];
      const double rn = sqrt(tot[0]);
      O.relres = O.bnorm > 0.0 ? rn / O.bnorm : rn;
      if (!isfinite(O.relres)) O.status = MRCG_ERR_NONFINITE;
    }
  }
}

// ------------------------------------------------------------------ cycle start

__global__ void __launch_bounds__(kThreads) cycle_start_kernel(DevState* st, int64_t n_pad, const double* __restrict__ res,
                                                                 double* v_cur, double* v_prev, double* w_cur,
                                                                 double* w_prev, double* zraw) {
  if (failed(st)) return;
  ROW_LOOP(i, n_pad) {
    v_cur[i] = res[i];
    v_prev[i] = 0.0;
    w_cur[i] = 0.0;
    w_prev[i] = 0.0;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->cg.vin = v_cur;
    st->cg.zout = zraw;
  }
}

__global__ void __launch_bounds__(kThreads) gamma_first_kernel(DevState* st, double* partials, int64_t n_pad,
                                                                 const double* __restrict__ z,
                                                                 const double* __restrict__ v) {
  if (failed(st)) return;
  double acc[1] = {0.0};
  ROW_LOOP(i, n_pad) acc[0] += z[i] * v[i];
  block_partials<1>(acc, 1, partials);
  if (last_block(&st->ticket)) {
    __shared__ double tot[1];
    final_sums(partials, 1, tot);
    if (threadIdx.x == 0) {
      OuterState& O = st->out;
      const double g2 = tot[0];
      if (!isfinite(g2)) {
        O.status = MRCG_ERR_NONFINITE;
      } else if (g2 <= 0.0) {
        O.status = MRCG_ERR_BREAKDOWN;
      } else {
        O.gamma = sqrt(g2);
        O.gamma_old = 1.0;
        O.gamma_new = O.gamma;
        O.eta = O.gamma;
        O.s = O.s_old = 0.0;
        O.c = O.c_old = 1.0;
      }
    }
  }
}

// ------------------------------------------------------------------ Lanczos step

__global__ void __launch_bounds__(kThreads) lanczos_spmv_kernel(DevState* st, double* partials, Sell A,
                                                                  const double* __restrict__ zraw,
                                                                  double* __restrict__ zn, double* __restrict__ az) {
  if (failed(st)) return;
  const double inv_gamma = 1.0 / st->out.gamma;
  double acc[1] = {0.0};
  SLICE_LOOP(A) {
    const double a =
        sell_row_dot<double>(A.slice_ptr, A.col, A.val64, sl, lane, [&](int c) { return __ldg(zraw + c); });
    const int64_t row = sl * kSlice + lane;
    const double zi = zraw[row] * inv_gamma;
    const double ai = a * inv_gamma;
    zn[row] = zi;
    az[row] = ai;
    acc[0] += zi * ai;
  }
  block_partials<1>(acc, 1, partials);
  if (last_block(&st->ticket)) {
    __shared__ double tot[1];
    final_sums(partials, 1, tot);
    if (threadIdx.x == 0) {
      st->out.delta = tot[0];
      if (!isfinite(tot[0])) st->out.status = MRCG_ERR_NONFINITE;
    }
  }
}

__global__ void __launch_bounds__(kThreads) lanczos_update_kernel(DevState* st, int64_t n_pad,
                                                                    const double* __restrict__ az,
                                                                    const double* __restrict__ v,
                                                                    const double* v_old, double* v_new,
                                                                    double* zraw) {
  if (failed(st)) return;
  const OuterState& O = st->out;
  const double f1 = O.delta / O.gamma, f2 = O.gamma / O.gamma_old;
  ROW_LOOP(i, n_pad) v_new[i] = az[i] - f1 * v[i] - f2 * v_old[i];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->cg.vin = v_new;
    st->cg.zout = zraw;
  }
}

__global__ void __launch_bounds__(kThreads) gamma_givens_kernel(DevState* st, double* partials, int64_t n_pad,
                                                                  const double* __restrict__ z,
                                                                  const double* __restrict__ v) {
  if (failed(st)) return;
  double acc[1] = {0.0};
  ROW_LOOP(i, n_pad) acc[0] += z[i] * v[i];
  block_partials<1>(acc, 1, partials);
  if (last_block(&st->ticket)) {
    __shared__ double tot[1];
    final_sums(partials, 1, tot);
    if (threadIdx.x == 0) {
      OuterState& O = st->out;
      const double g2 = tot[0];
      if (!isfinite(g2)) {
        O.status = MRCG_ERR_NONFINITE;
        return;
      }
      if (g2 < 0.0) {
        O.status = MRCG_ERR_BREAKDOWN;
        return;
      }
      const double gnew = sqrt(g2);
      const double a0 = O.c * O.delta - O.c_old * O.s * O.gamma;
      const double a1 = sqrt(a0 * a0 + gnew * gnew);
      const double a2 = O.s * O.delta + O.c_old * O.c * O.gamma;
      const double a3 = O.s_old * O.gamma;
      if (!(a1 > 0.0)) {
        O.status = MRCG_ERR_BREAKDOWN;
        return;
      }
      const double c_new = a0 / a1, s_new = gnew / a1;
      O.a1 = a1;
      O.a2 = a2;
      O.a3 = a3;
      O.ceta = c_new * O.eta;
      O.eta = -s_new * O.eta;
      O.gamma_new = gnew;
      O.c_old = O.c;
      O.c = c_new;
      O.s_old = O.s;
      O.s = s_new;
      O.gamma_old = O.gamma;
      O.gamma = gnew;
    }
  }
}

__global__ void __launch_bounds__(kThreads) minres_update_kernel(const DevState* st, int64_t n_pad,
                                                                   const double* __restrict__ zn, const double* w_old,
                                                                   const double* __restrict__ w, double* w_new,
                                                                   double* __restrict__ x) {
  if (failed(st)) return;
  const OuterState& O = st->out;
  const double a1 = O.a1, a2 = O.a2, a3 = O.a3, ceta = O.ceta;
  ROW_LOOP(i, n_pad) {
    const double wn = (zn[i] - a3 * w_old[i] - a2 * w[i]) / a1;
    w_new[i] = wn;
    x[i] += ceta * wn;
  }
}

// ------------------------------------------------------------------ setup kernels

__global__ void __launch_bounds__(kThreads) sell_fill_kernel(int64_t n, int64_t n_pad, const int64_t* __restrict__ rowptr,
                                                               const int32_t* __restrict__ colind,
                                                               const double* __restrict__ val,
                                                               const int64_t* __restrict__ slice_ptr, int32_t* col,
                                                               double* val64, float* val32) {
  ROW_LOOP(i, n_pad) {
    const int64_t sl = i / kSlice, lane = i % kSlice;
    const int64_t base = slice_ptr[sl];
    const int w = (int)((slice_ptr[sl + 1] - base) / kSlice);
    int len = 0;
    int64_t p0 = 0;
    if (i < n) {
      p0 = rowptr[i];
      len = (int)(rowptr[i + 1] - p0);
    }
    for (int j = 0; j < w; ++j) {
      const int64_t idx = base + (int64_t)j * kSlice + lane;
      if (j < len) {
        col[idx] = colind[p0 + j];
        val64[idx] = val[p0 + j];
        if (val32) val32[idx] = (float)val[p0 + j];
      } else {
        col[idx] = (int32_t)i;
        val64[idx] = 0.0;
        if (val32) val32[idx] = 0.0f;
      }
    }
  }
}

__global__ void __launch_bounds__(kThreads) mmr_diag_kernel(int64_t n, int64_t n_pad, const int64_t* __restrict__ rowptr,
                                                              const int32_t* __restrict__ colind,
                                                              const double* __restrict__ val,
                                                              const double* __restrict__ V, int k,
                                                              const double* __restrict__ lam2, bool fp32, void* dinv) {
  ROW_LOOP(i, n_pad) {
    double inv = 0.0;
    if (i < n) {
      double d = 0.0;
      for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p)
        if (colind[p] == i) d += val[p];
      for (int l = 0; l < k; ++l) {
        const double v = V[(size_t)l * n_pad + i];
        d += lam2[l] * v * v;
      }
      inv = 1.0 / d;
    }
    if (fp32) reinterpret_cast<float*>(dinv)[i] = (float)inv;
    else reinterpret_cast<double*>(dinv)[i] = inv;
  }
}

// col16 = col - row for every stored SELL entry (the caller checked that it fits)
__global__ void sell_delta16_kernel(int64_t n_pad, const int64_t* __restrict__ slice_ptr,
                                    const int32_t* __restrict__ col, int16_t* __restrict__ col16) {
  ROW_LOOP(i, n_pad) {
    const int64_t sl = i / kSlice, lane = i % kSlice;
    const int64_t base = slice_ptr[sl];
    const int w = (int)((slice_ptr[sl + 1] - base) / kSlice);
    for (int j = 0; j < w; ++j) {
      const int64_t idx = base + (int64_t)j * kSlice + lane;
      col16[idx] = (int16_t)(col[idx] - i);
    }
  }
}

__global__ void to_f32_kernel(const double* __restrict__ in, float* __restrict__ out, int64_t n) {
  ROW_LOOP(i, n) out[i] = (float)in[i];
}

__global__ void to_f64_kernel(const float* __restrict__ in, double* __restrict__ out, int64_t n) {
  ROW_LOOP(i, n) out[i] = (double)in[i];
}

inline int grid_for(int64_t n, int cap) {
  int64_t g = (n + kThreads - 1) / kThreads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

template <typename T, int KB>
cudaError_t mmr_t(const OuterArgs& a, const T* val, const T* V, int k, const T* u, T* out) {
  if (k > 0) {
    vtu_kernel<T, KB><<<a.grid_stream, kThreads, 0, a.stream>>>(a.st, a.partials, V, k, a.A.n_pad, u);
  }
  mmr_kernel<T, KB><<<a.grid_spmv, kThreads, 0, a.stream>>>(a.st, a.A, val, V, k, u, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t mmr_k(const OuterArgs& a, const T* val, const T* V, int k, const T* u, T* out) {
  if (k <= 8) return mmr_t<T, 8>(a, val, V, k, u, out);
  if (k <= 16) return mmr_t<T, 16>(a, val, V, k, u, out);
  return mmr_t<T, 32>(a, val, V, k, u, out);
}

}  // namespace

cudaError_t launch_spmv(const OuterArgs& a, const double* x, double* y) {
  spmv_kernel<<<a.grid_spmv, kThreads, 0, a.stream>>>(a.A, x, y);
  return cudaGetLastError();
}

cudaError_t launch_mmr(const OuterArgs& a, bool fp32, const void* val, const void* V, int k, const double* lam2,
                       const double* u, double* out, void* tmp_in, void* tmp_out) {
  (void)lam2;
  const int g = grid_for(a.A.n_pad, kMaxBlocks);
  if (fp32) {
    to_f32_kernel<<<g, kThreads, 0, a.stream>>>(u, (float*)tmp_in, a.A.n_pad);
    cudaError_t e = mmr_k<float>(a, (const float*)val, (const float*)V, k, (const float*)tmp_in, (float*)tmp_out);
    if (e != cudaSuccess) return e;
    to_f64_kernel<<<g, kThreads, 0, a.stream>>>((const float*)tmp_out, out, a.A.n_pad);
    return cudaGetLastError();
  }
  return mmr_k<double>(a, (const double*)val, (const double*)V, k, u, out);
}

cudaError_t launch_bnorm(const OuterArgs& a, const double* b) {
  bnorm_kernel<<<a.grid_stream, kThreads, 0, a.stream>>>(a.st, a.partials, b, a.A.n_pad);
  return cudaGetLastError();
}

cudaError_t launch_residual(const OuterArgs& a, const double* b, const double* x, double* res) {
  residual_kernel<<<a.grid_spmv, kThreads, 0, a.stream>>>(a.st, a.partials, a.A, b, x, res);
  return cudaGetLastError();
}

cudaError_t launch_cycle_start(const OuterArgs& a, const double* res, double* v_cur, double* v_prev, double* w_cur,
                               double* w_prev, double* zraw) {
  cycle_start_kernel<<<a.grid_stream, kThreads, 0, a.stream>>>(a.st, a.A.n_pad, res, v_cur, v_prev, w_cur, w_prev,
                                                               zraw);
  return cudaGetLastError();
}

cudaError_t launch_gamma_first(const OuterArgs& a, const double* zraw, const double* v) {
  gamma_first_kernel<<<a.grid_stream, kThreads, 0, a.stream>>>(a.st, a.partials, a.A.n_pad, zraw, v);
  return cudaGetLastError();
}

cudaError_t launch_lanczos_spmv(const OuterArgs& a, const double* zraw, double* zn, double* az) {
  lanczos_spmv_kernel<<<a.grid_spmv, kThreads, 0, a.stream>>>(a.st, a.partials, a.A, zraw, zn, az);
  return cudaGetLastError();
}

cudaError_t launch_lanczos_update(const OuterArgs& a, const double* az, const double* v, const double* v_old,
                                  double* v_new, double* zraw) {
  lanczos_update_kernel<<<a.grid_stream, kThreads, 0, a.stream>>>(a.st, a.A.n_pad, az, v, v_old, v_new, zraw);
  return cudaGetLastError();
}

cudaError_t launch_gamma_givens(const OuterArgs& a, const double* zraw, const double* v_new) {
  gamma_givens_kernel<<<a.grid_stream, kThreads, 0, a.stream>>>(a.st, a.partials, a.A.n_pad, zraw, v_new);
  return cudaGetLastError();
}

cudaError_t launch_minres_update(const OuterArgs& a, const double* zn, const double* w_old, const double* w,
                                 double* w_new, double* x) {
  minres_update_kernel<<<a.grid_stream, kThreads, 0, a.stream>>>(a.st, a.A.n_pad, zn, w_old, w, w_new, x);
  return cudaGetLastError();
}

cudaError_t launch_mmr_diag(cudaStream_t stream, int64_t n, int64_t n_pad, const int64_t* rowptr,
                            const int32_t* colind, const double* val, const double* V64, int k, const double* lam2,
                            bool fp32, void* dinv) {
  mmr_diag_kernel<<<grid_for(n_pad, kMaxBlocks), kThreads, 0, stream>>>(n, n_pad, rowptr, colind, val, V64, k, lam2,
                                                                        fp32, dinv);
  return cudaGetLastError();
}

cudaError_t launch_sell_fill(cudaStream_t stream, int64_t n, const int64_t* rowptr, const int32_t* colind,
                             const double* val, const int64_t* slice_ptr, int32_t* col, double* val64, float* val32) {
  const int64_t n_pad = ((n + kSlice - 1) / kSlice) * kSlice;
  sell_fill_kernel<<<grid_for(n_pad, kMaxBlocks), kThreads, 0, stream>>>(n, n_pad, rowptr, colind, val, slice_ptr,
                                                                         col, val64, val32);
  return cudaGetLastError();
}

cudaError_t launch_sell_delta16(cudaStream_t stream, int64_t n_pad, const int64_t* slice_ptr, const int32_t* col,
                                int16_t* col16) {
  sell_delta16_kernel<<<grid_for(n_pad, kMaxBlocks), kThreads, 0, stream>>>(n_pad, slice_ptr, col, col16);
  return cudaGetLastError();
}

cudaError_t launch_to_f32(cudaStream_t stream, const double* in, float* out, int64_t n) {
  to_f32_kernel<<<grid_for(n, kMaxBlocks), kThreads, 0, stream>>>(in, out, n);
  return cudaGetLastError();
}

cudaError_t launch_to_f64(cudaStream_t stream, const float* in, double* out, int64_t n) {
  to_f64_kernel<<<grid_for(n, kMaxBlocks), kThreads, 0, stream>>>(in, out, n);
  return cudaGetLastError();
}

}  // namespace mrcg
