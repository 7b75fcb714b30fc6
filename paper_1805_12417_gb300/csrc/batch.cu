// Batched MINRES-CG: many independent systems of uneven size in one launch
// sequence (the paper's many-systems-after-one-setup use, Sec. 2-3).
//
// The systems are concatenated block-diagonally: one SELL-32 matrix with
// global column indices, every system padded to whole slices, each with its
// own V_hat block (column-major, n_pad_i x k_i) and its own scalar state.
// Work is cut into chunks of at most kChunkRows rows that never straddle two
// systems; blocks loop over chunks, so a block's partial sums always belong
// to one system.  Each kernel reduces per system: the block that finishes the
// last chunk of system i (per-system ticket) sums that system's chunk
// partials in a fixed order and updates its FP64 scalars.  Systems whose
// inner solve has converged skip their chunks (per-system convergence mask);
// the device-side while loop runs until every system in the round is done.
//
// The outer MINRES steps of all systems advance in rounds driven by the host:
// in a round each system is idle (mode 0), starts a cycle (mode 1: v_1 = r,
// z_1 = P v_1, gamma_1) or takes one step (mode 2: Lanczos, P, Givens, x, true
// residual); the host then reads every system's state and applies the
// stopping and restart rules per system.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "mrcg.h"
#include "trace.h"

namespace mrcg {
namespace batch {

constexpr int kChunkRows = 4096;  // default rows per chunk
constexpr int kChunkMin = 1024;   // smallest chunk height the autotuner tries
constexpr int kMaxSystems = 4096;

struct SysDesc {
  int64_t row0, n, n_pad, slice0, voff;
  int k, chunk0, nchunks, pad;
};

struct Chunk {
  int64_t row0, row1;
  int sys, pad;
};

template <typename T>
struct BArgs {
  DevState* st;  // [S]
  const SysDesc* sys;
  const Chunk* chunks;
  int nchunks;
  double* partials;  // [kMaxNV][nchunks]
  const int64_t* slice_ptr;
  const int32_t* col;
  const T* val;
  const T* V;
  const T* dinv;
  T* z;
  T* r;
  T* s;
  T* p_old;
  T* p_new;
  T* q;
};

// ------------------------------------------------------------------ helpers

// block reduction of NV values into partials[i * nc + c]
template <typename T, int NV>
__device__ __forceinline__ void chunk_partials(T (&v)[NV], int nv, double* partials, int nc, int c) {
  __shared__ T smt[kThreads / 32][NV];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < NV; ++i)
    if (i < nv) v[i] = warp_sum<T>(v[i]);
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i)
      if (i < nv) smt[warp][i] = v[i];
  }
  __syncthreads();
  if (threadIdx.x < nv) {
    T s = 0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) s += smt[w][threadIdx.x];
    partials[(size_t)threadIdx.x * nc + c] = (double)s;
  }
}

// the block that finishes the last chunk of a system
__device__ __forceinline__ bool system_last(unsigned int* ticket, int nchunks_sys) {
  __shared__ bool is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int prev = atomicAdd(ticket, 1u);
    is_last = (prev == (unsigned int)nchunks_sys - 1u);
    if (is_last) *ticket = 0u;
  }
  __syncthreads();
  if (is_last) __threadfence();
  return is_last;
}

// fixed-order sum of the partials of chunks [c0, c0 + ncs) of one system
__device__ __forceinline__ void system_sums(const double* partials, int nc, int c0, int ncs, int nv, double* out) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = warp; i < nv; i += kThreads / 32) {
    double s = 0.0;
    s = lane_sum8(partials + (size_t)i * nc + c0, ncs, lane);
    s = warp_sum(s);
    if (lane == 0) out[i] = s;
  }
  __syncthreads();
}


#define CHUNK_LOOP(nc) for (int c = blockIdx.x; c < (nc); c += gridDim.x)

// ------------------------------------------------------------------ inner CG kernels

// mode of a system for the inner solve: participates when the outer step of
// this round needs P (mode 1 or 2)
__device__ __forceinline__ bool in_round(const DevState& d) { return d.out.mode == 1 || d.out.mode == 2; }

__global__ void __launch_bounds__(kThreads) b_vnorm_kernel(DevState* st, const SysDesc* sys, const Chunk* chunks,
                                                             int nc, double* partials) {
  CHUNK_LOOP(nc) {
    const Chunk ch = chunks[c];
    DevState& D = st[ch.sys];
    if (!in_round(D)) continue;
    const double* v = D.cg.vin;
    double acc[1] = {0.0};
    for (int64_t i = ch.row0 + threadIdx.x; i < ch.row1; i += kThreads) acc[0] += v[i] * v[i];
    chunk_partials<double, 1>(acc, 1, partials, nc, c);
    const SysDesc sd = sys[ch.sys];
    if (system_last(&D.ticket, sd.nchunks)) {
      __shared__ double tot[1];
      system_sums(partials, nc, sd.chunk0, sd.nchunks, 1, tot);
      if (threadIdx.x == 0) D.cg.vnorm = sqrt(tot[0]);
    }
  }
}

// CTAs per SM the V_hat-width buckets are compiled for (register budgets)
constexpr int b_min_blocks(int kb) { return kb >= 24 ? 2 : kb >= 16 ? 3 : 4; }
template <typename T>
constexpr int b_min_blocks_a(int kb) { return kb >= 24 ? 3 : 4; }

template <typename T, int KB>
__global__ void __launch_bounds__(kThreads, b_min_blocks(KB)) b_init_kernel(BArgs<T> a) {
  constexpr int W = V16<T>::W;
  constexpr int KS = KB > 0 ? KB : 1;
  const bool jac = a.dinv != nullptr;
  CHUNK_LOOP(a.nchunks) {
    const Chunk ch = a.chunks[c];
    DevState& D = a.st[ch.sys];
    if (!in_round(D)) continue;
    const SysDesc sd = a.sys[ch.sys];
    CgState& S = D.cg;
    const double vn = S.vnorm;
    const double scale = (vn > 0.0 && isfinite(vn)) ? 1.0 / vn : 0.0;
    const double* v = S.vin;
    T rs = 0, rr = 0;
    T u[KS];
#pragma unroll
    for (int l = 0; l < KS; ++l) u[l] = 0;
    const T zero[W] = {};
    for (int64_t i = ch.row0 + (int64_t)threadIdx.x * W; i < ch.row1; i += (int64_t)kThreads * W) {
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
      const int64_t li = i - sd.row0;
#pragma unroll
      for (int l = 0; l < KB; ++l)
        if (l < sd.k) {
          T vv[W];
          ld16_stream(a.V + sd.voff + (size_t)l * sd.n_pad + li, vv);
#pragma unroll
          for (int e = 0; e < W; ++e) u[l] += vv[e] * s[e];
        }
    }
    T acc[KB + 2];
    pack_slots<T, KB>(acc, rs, u, rr, sd.k, jac);
    const int nv = sd.k + 1 + (jac ? 1 : 0);
    chunk_partials<T, KB + 2>(acc, nv, a.partials, a.nchunks, c);
    if (system_last(&D.ticket, sd.nchunks)) {
      __shared__ double tot[KB + 2];
      system_sums(a.partials, a.nchunks, sd.chunk0, sd.nchunks, nv, tot);
      if (threadIdx.x == 0) {
        const double rho = tot[0], rnorm = sqrt(jac ? tot[sd.k + 1] : tot[0]);
        S.rho = rho;
        S.beta = 0.0;
        S.beta32 = 0.0f;
        S.iters = 0;
        S.tol_abs = S.inner_tol * rnorm;
        S.maxit = S.budget;
        S.done = kRunning;
        if (!isfinite(vn) || !isfinite(rho)) S.done = kNonFinite;
        else if (vn == 0.0 || rnorm == 0.0) S.done = kConverged;
        else if (S.maxit <= 0) S.done = kMaxIter;
        for (int l = 0; l < sd.k; ++l) S.t[l] = tot[l + 1];
        publish_c(S, sd.k);
      }
    }
  }
}

template <typename T, int KB>
__global__ void __launch_bounds__(kThreads, b_min_blocks_a<T>(KB)) b_step_a_kernel(BArgs<T> a) {
  constexpr int KS = KB > 0 ? KB : 1;
  __shared__ T cl[KS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  CHUNK_LOOP(a.nchunks) {
    const Chunk ch = a.chunks[c];
    DevState& D = a.st[ch.sys];
    CgState& S = D.cg;
    if (!in_round(D) || S.done != kRunning) continue;
    const SysDesc sd = a.sys[ch.sys];
    __syncthreads();
    if (threadIdx.x < KS) cl[threadIdx.x] = ((int)threadIdx.x < sd.k) ? c_of(S, threadIdx.x, T(0)) : (T)0;
    __syncthreads();
    const T beta = beta_of(S, T(0));
    const T* __restrict__ sv = a.s;
    const T* __restrict__ po = a.p_old;
    T dot = 0;
    constexpr int NW = kThreads / 32;
    const int64_t s_end = ch.row1 / kSlice;
    for (int64_t g0 = ch.row0 / kSlice + warp; g0 < s_end; g0 += 32 * NW) {
      // FP32: the slice pointers of the warp's next (up to) 32 slices in one
      // round trip, lane t holding those of slice g0 + t * NW (FP64 keeps the
      // per-slice loads: the two registers would spill at its register budget)
      constexpr bool PF = sizeof(T) == 4;
      const int64_t my_sl = g0 + (int64_t)lane * NW;
      const int64_t my_b = (PF && my_sl < s_end) ? a.slice_ptr[my_sl] : 0;
      const int my_w = (PF && my_sl < s_end) ? (int)((a.slice_ptr[my_sl + 1] - my_b) >> 5) : 0;
      const int cnt = (int)min((int64_t)32, (s_end - g0 + NW - 1) / NW);
      for (int t = 0; t < cnt; ++t) {
        const int64_t sl = g0 + (int64_t)t * NW;
        const int64_t row = sl * kSlice + lane;
        const int64_t li = row - sd.row0;
        T vrow[KS];
#pragma unroll
        for (int l = 0; l < KS; ++l)
          vrow[l] = (l < sd.k) ? __ldcs(a.V + sd.voff + (size_t)l * sd.n_pad + li) : (T)0;
        const T srow = sv[row], prow = po[row];
        const int64_t base = PF ? __shfl_sync(0xffffffffu, my_b, t) : a.slice_ptr[sl];
        const int w = PF ? __shfl_sync(0xffffffffu, my_w, t) : (int)((a.slice_ptr[sl + 1] - base) >> 5);
        const T* vp = a.val + base + lane;
        const int32_t* cp = a.col + base + lane;
        T acc = 0;
        if (w <= 8) {
          T av[8];
          int cc[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            av[j] = (j < w) ? __ldcs(vp + (size_t)j * kSlice) : (T)0;
            cc[j] = (j < w) ? __ldcs(cp + (size_t)j * kSlice) : 0;
          }
#pragma unroll
          for (int j = 0; j < 8; ++j)
            if (j < w) acc += av[j] * (__ldg(sv + cc[j]) + beta * __ldg(po + cc[j]));
        } else {
#pragma unroll 4
          for (int j = 0; j < w; ++j) {
            const T av = __ldcs(vp + (size_t)j * kSlice);
            const int cj = __ldcs(cp + (size_t)j * kSlice);
            acc += av * (__ldg(sv + cj) + beta * __ldg(po + cj));
          }
        }
        const T pn = srow + beta * prow;
#pragma unroll
        for (int l = 0; l < KB; ++l)
          if (l < sd.k) acc += vrow[l] * cl[l];
        a.q[row] = acc;
        a.p_new[row] = pn;
        dot += pn * acc;
      }
    }
    T part[1] = {dot};
    chunk_partials<T, 1>(part, 1, a.partials, a.nchunks, c);
    if (system_last(&D.ticket, sd.nchunks)) {
      __shared__ double tot[1];
      system_sums(a.partials, a.nchunks, sd.chunk0, sd.nchunks, 1, tot);
      if (threadIdx.x == 0) {
        const double kappa = tot[0];
        S.kappa = kappa;
        if (!isfinite(kappa)) S.done = kNonFinite;
        else if (kappa <= 0.0) S.done = kNotSpd;
        else {
          S.alpha = S.rho / kappa;
          S.alpha32 = (float)S.alpha;
        }
      }
    }
  }
}

template <typename T, int KB>
__global__ void __launch_bounds__(kThreads, b_min_blocks(KB)) b_step_b_kernel(BArgs<T> a) {
  constexpr int W = V16<T>::W;
  constexpr int KS = KB > 0 ? KB : 1;
  const bool jac = a.dinv != nullptr;
  CHUNK_LOOP(a.nchunks) {
    const Chunk ch = a.chunks[c];
    DevState& D = a.st[ch.sys];
    CgState& S = D.cg;
    if (!in_round(D) || S.done != kRunning) continue;
    const SysDesc sd = a.sys[ch.sys];
    const T alpha = alpha_of(S, T(0));
    T rs = 0, rr = 0;
    T u[KS];
#pragma unroll
    for (int l = 0; l < KS; ++l) u[l] = 0;
    for (int64_t i = ch.row0 + (int64_t)threadIdx.x * W; i < ch.row1; i += (int64_t)kThreads * W) {
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
      // V_hat^T s: the columns in groups of 8, each group's loads issued
      // together before its FMAs (k is uniform over the block)
      const int64_t li = i - sd.row0;
#pragma unroll
      for (int l0 = 0; l0 < KB; l0 += 8) {
        if (l0 >= sd.k) break;
        T vv[8][W];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if (l0 + j < sd.k) {
            ld16_stream(a.V + sd.voff + (size_t)(l0 + j) * sd.n_pad + li, vv[j]);
          } else {
#pragma unroll
            for (int e = 0; e < W; ++e) vv[j][e] = 0;
          }
        }
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
          for (int e = 0; e < W; ++e) u[l0 + j] += vv[j][e] * s[e];
      }
    }
    T acc[KB + 2];
    pack_slots<T, KB>(acc, rs, u, rr, sd.k, jac);
    const int nv = sd.k + 1 + (jac ? 1 : 0);
    chunk_partials<T, KB + 2>(acc, nv, a.partials, a.nchunks, c);
    if (system_last(&D.ticket, sd.nchunks)) {
      __shared__ double tot[KB + 2];
      system_sums(a.partials, a.nchunks, sd.chunk0, sd.nchunks, nv, tot);
      if (threadIdx.x == 0) {
        const double rho_new = tot[0], rnorm = sqrt(jac ? tot[sd.k + 1] : tot[0]);
        S.iters += 1;
        if (!isfinite(rho_new) || !isfinite(rnorm)) S.done = kNonFinite;
        else if (rnorm <= S.tol_abs) S.done = kConverged;
        else if (S.iters >= S.maxit) S.done = kMaxIter;
        else {
          const double beta = rho_new / S.rho;
          S.beta = beta;
          S.beta32 = (float)beta;
          S.rho = rho_new;
          for (int l = 0; l < sd.k; ++l) S.t[l] = tot[l + 1] + beta * S.t[l];
          publish_c(S, sd.k);
        }
      }
    }
  }
}

// loop control: continue while any system of the round is still iterating
// ctl[0]: executed loop bodies of this inner solve, ctl[1]: their limit
__global__ void b_ctl_kernel(DevState* st, int nsys, int* ctl, cudaGraphConditionalHandle handle) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < nsys; i += blockDim.x)
    if (in_round(st[i]) && st[i].cg.done == kRunning) atomicOr(&any, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    ctl[0] += 1;
    int go = any;
    if (go && ctl[0] >= ctl[1]) {
      go = 0;
      for (int i = 0; i < nsys; ++i)
        if (in_round(st[i]) && st[i].cg.done == kRunning) st[i].cg.done = kLoopCap;
    }
    cudaGraphSetConditional(handle, go ? 1u : 0u);
  }
}

// the same loop control for the host-driven loop (profiling mode): the
// decision goes to ctl[2] for the host to read instead of a graph condition
__global__ void b_ctl_host_kernel(DevState* st, int nsys, int* ctl) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < nsys; i += blockDim.x)
    if (in_round(st[i]) && st[i].cg.done == kRunning) atomicOr(&any, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    ctl[0] += 1;
    int go = any;
    if (go && ctl[0] >= ctl[1]) {
      go = 0;
      for (int i = 0; i < nsys; ++i)
        if (in_round(st[i]) && st[i].cg.done == kRunning) st[i].cg.done = kLoopCap;
    }
    ctl[2] = go;
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) b_finish_kernel(DevState* st, const SysDesc* sys, const Chunk* chunks,
                                                              int nc, const T* z) {
  CHUNK_LOOP(nc) {
    const Chunk ch = chunks[c];
    DevState& D = st[ch.sys];
    if (!in_round(D)) continue;
    CgState& S = D.cg;
    const double vn = (S.vnorm > 0.0 && isfinite(S.vnorm)) ? S.vnorm : 0.0;
    double* out = S.zout;
    for (int64_t i = ch.row0 + threadIdx.x; i < ch.row1; i += kThreads) out[i] = vn * (double)z[i];
    if (c == sys[ch.sys].chunk0 && threadIdx.x == 0) {
      S.budget -= S.iters;
      OuterState& O = D.out;
      O.inner_total += S.iters;
      O.prec_calls += 1;
      if (O.status == MRCG_OK) {
        if (S.done == kNotSpd) O.status = MRCG_ERR_NOT_SPD;
        else if (S.done == kNonFinite) O.status = MRCG_ERR_NONFINITE;
        else if (S.done == kMaxIter || S.done == kLoopCap) O.status = MRCG_ERR_MAXITER;
      }
    }
  }
}

// ------------------------------------------------------------------ outer MINRES kernels (FP64)

struct OArgs {
  DevState* st;
  const SysDesc* sys;
  const Chunk* chunks;
  int nc;
  double* partials;
  const int64_t* slice_ptr;
  const int32_t* col;
  const double* val;
  double *x, *b, *res, *zraw, *zn, *v0, *v1, *w0, *w1;
};

__device__ __forceinline__ double sell_dot(const OArgs& a, int64_t sl, int lane, const double* x) {
  const int64_t base = a.slice_ptr[sl];
  const int w = (int)((a.slice_ptr[sl + 1] - base) >> 5);
  const double* vp = a.val + base + lane;
  const int32_t* cp = a.col + base + lane;
  double acc = 0.0;
#pragma unroll 4
  for (int j = 0; j < w; ++j) acc += __ldcs(vp + (size_t)j * kSlice) * __ldg(x + __ldcs(cp + (size_t)j * kSlice));
  return acc;
}

#define SYS_SCALAR_FINISH(D, sd, nv, ...)                                      \
  if (system_last(&(D).ticket, (sd).nchunks)) {                                \
    __shared__ double tot[(nv)];                                               \
    system_sums(a.partials, a.nc, (sd).chunk0, (sd).nchunks, (nv), tot);       \
    if (threadIdx.x == 0) {                                                    \
      __VA_ARGS__                                                              \
    }                                                                          \
  }

// all systems with mode >= 0 flagged by `which` (0: every system, 2: mode 2)
__global__ void __launch_bounds__(kThreads) b_bnorm_kernel(OArgs a) {
  CHUNK_LOOP(a.nc) {
    const Chunk ch = a.chunks[c];
    DevState& D = a.st[ch.sys];
    double acc[1] = {0.0};
    for (int64_t i = ch.row0 + threadIdx.x; i < ch.row1; i += kThreads) acc[0] += a.b[i] * a.b[i];
    chunk_partials<double, 1>(acc, 1, a.partials, a.nc, c);
    const SysDesc sd = a.sys[ch.sys];
    SYS_SCALAR_FINISH(D, sd, 1, D.out.bnorm = sqrt(tot[0]);)
  }
}

// res = b - A x and the true relative residual; mode 2 systems (or all when all != 0)
__global__ void __launch_bounds__(kThreads) b_residual_kernel(OArgs a, int all) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  CHUNK_LOOP(a.nc) {
    const Chunk ch = a.chunks[c];
    DevState& D = a.st[ch.sys];
    if (!all && (D.out.mode != 2 || D.out.status != MRCG_OK)) continue;
    double acc[1] = {0.0};
    for (int64_t sl = ch.row0 / kSlice + warp; sl < ch.row1 / kSlice; sl += kThreads / 32) {
      const int64_t row = sl * kSlice + lane;
      const double r = a.b[row] - sell_dot(a, sl, lane, a.x);
      a.res[row] = r;
      acc[0] += r * r;
    }
    chunk_partials<double, 1>(acc, 1, a.partials, a.nc, c);
    const SysDesc sd = a.sys[ch.sys];
    SYS_SCALAR_FINISH(D, sd, 1, {
      OuterState& O = D.out;
      O.rnorm2 = tot[0];
      const double rn = sqrt(tot[0]);
      O.relres = O.bnorm > 0.0 ? rn / O.bnorm : rn;
      if (!isfinite(O.relres)) O.status = MRCG_ERR_NONFINITE;
      if (!all) O.cur ^= 1;
    })
  }
}

__global__ void __launch_bounds__(kThreads) b_cycle_start_kernel(OArgs a) {
  CHUNK_LOOP(a.nc) {
    const Chunk ch = a.chunks[c];
    DevState& D = a.st[ch.sys];
    if (D.out.mode != 1) continue;
    double* vc = D.out.cur ? a.v1 : a.v0;
    double* vp = D.out.cur ? a.v0 : a.v1;
    double* wc = D.out.cur ? a.w1 : a.w0;
    double* wp = D.out.cur ? a.w0 : a.w1;
    for (int64_t i = ch.row0 + threadIdx.x; i < ch.row1; i += kThreads) {
      vc[i] = a.res[i];
      vp[i] = 0.0;
      wc[i] = 0.0;
      wp[i] = 0.0;
    }
    if (c == a.sys[ch.sys].chunk0 && threadIdx.x == 0) {
      D.cg.vin = vc;
      D.cg.zout = a.zraw;
    }
  }
}

// z^T v per system: gamma_1 (mode 1) or gamma_{j+1} with the Givens rotation (mode 2)
__global__ void __launch_bounds__(kThreads) b_gamma_kernel(OArgs a) {
  CHUNK_LOOP(a.nc) {
    const Chunk ch = a.chunks[c];
    DevState& D = a.st[ch.sys];
    const int mode = D.out.mode;
    if ((mode != 1 && mode != 2) || D.out.status != MRCG_OK) continue;
    const double* v = D.cg.vin;
    double acc[1] = {0.0};
    for (int64_t i = ch.row0 + threadIdx.x; i < ch.row1; i += kThreads) acc[0] += a.zraw[i] * v[i];
    chunk_partials<double, 1>(acc, 1, a.partials, a.nc, c);
    const SysDesc sd = a.sys[ch.sys];
    SYS_SCALAR_FINISH(D, sd, 1, {
      OuterState& O = D.out;
      const double g2 = tot[0];
      if (!isfinite(g2)) {
        O.status = MRCG_ERR_NONFINITE;
      } else if (mode == 1) {
        if (g2 <= 0.0) {
          O.status = MRCG_ERR_BREAKDOWN;
        } else {
          O.gamma = sqrt(g2);
          O.gamma_old = 1.0;
          O.gamma_new = O.gamma;
          O.eta = O.gamma;
          O.s = O.s_old = 0.0;
          O.c = O.c_old = 1.0;
        }
      } else if (g2 < 0.0) {
        O.status = MRCG_ERR_BREAKDOWN;
      } else {
        const double gnew = sqrt(g2);
        const double a0 = O.c * O.delta - O.c_old * O.s * O.gamma;
        const double a1 = sqrt(a0 * a0 + gnew * gnew);
        const double a2 = O.s * O.delta + O.c_old * O.c * O.gamma;
        const double a3 = O.s_old * O.gamma;
        if (!(a1 > 0.0)) {
          O.status = MRCG_ERR_BREAKDOWN;
        } else {
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
    })
  }
}

// zn = zraw / gamma ; az = A zn ; delta = zn^T az   (az kept in res)
__global__ void __launch_bounds__(kThreads) b_lanczos_spmv_kernel(OArgs a) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  CHUNK_LOOP(a.nc) {
    const Chunk ch = a.chunks[c];
    DevState& D = a.st[ch.sys];
    if (D.out.mode != 2 || D.out.status != MRCG_OK) continue;
    const double inv_gamma = 1.0 / D.out.gamma;
    double acc[1] = {0.0};
    for (int64_t sl = ch.row0 / kSlice + warp; sl < ch.row1 / kSlice; sl += kThreads / 32) {
      const int64_t row = sl * kSlice + lane;
      const double zi = a.zraw[row] * inv_gamma;
      const double ai = sell_dot(a, sl, lane, a.zraw) * inv_gamma;
      a.zn[row] = zi;
      a.res[row] = ai;
      acc[0] += zi * ai;
    }
    chunk_partials<double, 1>(acc, 1, a.partials, a.nc, c);
    const SysDesc sd = a.sys[ch.sys];
    SYS_SCALAR_FINISH(D, sd, 1, {
      D.out.delta = tot[0];
      if (!isfinite(tot[0])) D.out.status = MRCG_ERR_NONFINITE;
    })
  }
}

// v_{j+1} = az - (delta/gamma) v_j - (gamma/gamma_old) v_{j-1}, written over v_{j-1}
__global__ void __launch_bounds__(kThreads) b_lanczos_update_kernel(OArgs a) {
  CHUNK_LOOP(a.nc) {
    const Chunk ch = a.chunks[c];
    DevState& D = a.st[ch.sys];
    if (D.out.mode != 2 || D.out.status != MRCG_OK) continue;
    const OuterState& O = D.out;
    const double* v = O.cur ? a.v1 : a.v0;
    double* vo = O.cur ? a.v0 : a.v1;
    const double f1 = O.delta / O.gamma, f2 = O.gamma / O.gamma_old;
    for (int64_t i = ch.row0 + threadIdx.x; i < ch.row1; i += kThreads) vo[i] = a.res[i] - f1 * v[i] - f2 * vo[i];
    if (c == a.sys[ch.sys].chunk0 && threadIdx.x == 0) {
      D.cg.vin = vo;
      D.cg.zout = a.zraw;
    }
  }
}

// w_{j+1} = (zn - a3 w_{j-1} - a2 w_j) / a1 over w_{j-1}; x += c eta w_{j+1}
__global__ void __launch_bounds__(kThreads) b_minres_update_kernel(OArgs a) {
  CHUNK_LOOP(a.nc) {
    const Chunk ch = a.chunks[c];
    DevState& D = a.st[ch.sys];
    if (D.out.mode != 2 || D.out.status != MRCG_OK) continue;
    const OuterState& O = D.out;
    const double* w = O.cur ? a.w1 : a.w0;
    double* wo = O.cur ? a.w0 : a.w1;
    const double a1 = O.a1, a2 = O.a2, a3 = O.a3, ceta = O.ceta;
    for (int64_t i = ch.row0 + threadIdx.x; i < ch.row1; i += kThreads) {
      const double wn = (a.zn[i] - a3 * wo[i] - a2 * w[i]) / a1;
      wo[i] = wn;
      a.x[i] += ceta * wn;
    }
  }
}

__global__ void b_set_modes_kernel(DevState* st, const int* modes, int nsys) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nsys; i += gridDim.x * blockDim.x) st[i].out.mode = modes[i];
}

// ------------------------------------------------------------------ graph

cudaError_t add_kernel(cudaGraph_t g, cudaGraphNode_t* node, const cudaGraphNode_t* deps, size_t ndeps,
                       const void* fn, int grid, int block, void** args) {
  cudaKernelNodeParams p = {};
  p.func = const_cast<void*>(fn);
  p.gridDim = dim3(grid);
  p.blockDim = dim3(block);
  p.kernelParams = args;
  return cudaGraphAddKernelNode(node, g, deps, ndeps, &p);
}

struct GraphSpec {
  bool fp32;
  int kb;  // k bucket of the batch
  int nsys, nc;
  DevState* st;
  const SysDesc* sys;
  const Chunk* chunks;
  double* partials;
  Sell A;
  const void* V;
  const void* dinv;
  void *z, *r, *s, *p0, *p1, *q;
  int* ctl;
  int grid, grid_b, unroll;  // grid of step a and the other kernels, grid of step b
};

template <typename T>
void make_bargs(const GraphSpec& g, BArgs<T> (&a)[2]) {
  for (int par = 0; par < 2; ++par) {
    BArgs<T>& x = a[par];
    x.st = g.st;
    x.sys = g.sys;
    x.chunks = g.chunks;
    x.nchunks = g.nc;
    x.partials = g.partials;
    x.slice_ptr = g.A.slice_ptr;
    x.col = g.A.col;
    x.val = reinterpret_cast<const T*>(sizeof(T) == 8 ? (const void*)g.A.val64 : (const void*)g.A.val32);
    x.V = reinterpret_cast<const T*>(g.V);
    x.dinv = reinterpret_cast<const T*>(g.dinv);
    x.z = reinterpret_cast<T*>(g.z);
    x.r = reinterpret_cast<T*>(g.r);
    x.s = g.dinv ? reinterpret_cast<T*>(g.s) : reinterpret_cast<T*>(g.r);
    x.q = reinterpret_cast<T*>(g.q);
    x.p_old = reinterpret_cast<T*>(par == 0 ? g.p0 : g.p1);
    x.p_new = reinterpret_cast<T*>(par == 0 ? g.p1 : g.p0);
  }
}

__global__ void b_ctl_reset_kernel(int* ctl) { ctl[0] = 0; }

template <typename T, int KB>
cudaError_t build_graph(const GraphSpec& gs, cudaGraph_t* out) {
  cudaError_t e;
  cudaGraph_t g;
  if ((e = cudaGraphCreate(&g, 0))) return e;
  BArgs<T> a[2];
  make_bargs(gs, a);
  DevState* st = gs.st;
  const SysDesc* sys = gs.sys;
  const Chunk* chunks = gs.chunks;
  int nc = gs.nc, nsys = gs.nsys;
  double* partials = gs.partials;
  int* ctl = gs.ctl;
  const T* zc = reinterpret_cast<const T*>(gs.z);
  cudaGraphNode_t n0, n1, n2, nl, nf;
  void* r_args[] = {&ctl};
  void* vn_args[] = {&st, (void*)&sys, (void*)&chunks, &nc, &partials};
  void* in_args[] = {&a[0]};
  if ((e = add_kernel(g, &n0, nullptr, 0, (const void*)b_ctl_reset_kernel, 1, 1, r_args))) goto fail;
  if ((e = add_kernel(g, &n1, &n0, 1, (const void*)b_vnorm_kernel, gs.grid, kThreads, vn_args))) goto fail;
  if ((e = add_kernel(g, &n2, &n1, 1, (const void*)b_init_kernel<T, KB>, gs.grid, kThreads, in_args))) goto fail;
  {
    cudaGraphConditionalHandle h;
    if ((e = cudaGraphConditionalHandleCreate(&h, g, 1u, cudaGraphCondAssignDefault))) goto fail;
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    if ((e = cudaGraphAddNode(&nl, g, &n2, nullptr, 1, &cp))) goto fail;
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    cudaGraphNode_t prev = nullptr;
    for (int it = 0; it < gs.unroll; ++it) {
      void* aa[] = {&a[it & 1]};
      cudaGraphNode_t na, nb;
      if ((e = add_kernel(body, &na, prev ? &prev : nullptr, prev ? 1 : 0, (const void*)b_step_a_kernel<T, KB>,
                          gs.grid, kThreads, aa)))
        goto fail;
      if ((e = add_kernel(body, &nb, &na, 1, (const void*)b_step_b_kernel<T, KB>, gs.grid_b, kThreads, aa)))
        goto fail;
      prev = nb;
    }
    cudaGraphNode_t nctl;
    void* ctl_args[] = {&st, &nsys, &ctl, &h};
    if ((e = add_kernel(body, &nctl, &prev, 1, (const void*)b_ctl_kernel, 1, 256, ctl_args))) goto fail;
  }
  {
    void* f_args[] = {&st, (void*)&sys, (void*)&chunks, &nc, (void*)&zc};
    if ((e = add_kernel(g, &nf, &nl, 1, (const void*)b_finish_kernel<T>, gs.grid, kThreads, f_args))) goto fail;
  }
  *out = g;
  return cudaSuccess;
fail:
  cudaGraphDestroy(g);
  return e;
}

// The graph's launch sequence driven from the host: after every U iterations
// the host reads the loop decision.  Used when a profiler must see the
// individual kernels (kernel nodes under a conditional node cannot be profiled).
template <typename T, int KB>
cudaError_t run_host(const GraphSpec& gs, cudaStream_t stream) {
  BArgs<T> a[2];
  make_bargs(gs, a);
  const T* zc = reinterpret_cast<const T*>(gs.z);
  b_ctl_reset_kernel<<<1, 1, 0, stream>>>(gs.ctl);
  b_vnorm_kernel<<<gs.grid, kThreads, 0, stream>>>(gs.st, gs.sys, gs.chunks, gs.nc, gs.partials);
  b_init_kernel<T, KB><<<gs.grid, kThreads, 0, stream>>>(a[0]);
  cudaError_t e = cudaSuccess;
  for (;;) {
    for (int it = 0; it < gs.unroll; ++it) {
      b_step_a_kernel<T, KB><<<gs.grid, kThreads, 0, stream>>>(a[it & 1]);
      b_step_b_kernel<T, KB><<<gs.grid_b, kThreads, 0, stream>>>(a[it & 1]);
    }
    b_ctl_host_kernel<<<1, 256, 0, stream>>>(gs.st, gs.nsys, gs.ctl);
    int go = 0;
    if ((e = cudaMemcpyAsync(&go, gs.ctl + 2, sizeof(int), cudaMemcpyDeviceToHost, stream))) return e;
    if ((e = cudaStreamSynchronize(stream))) return e;
    if (!go) break;
  }
  b_finish_kernel<T><<<gs.grid, kThreads, 0, stream>>>(gs.st, gs.sys, gs.chunks, gs.nc, zc);
  return cudaGetLastError();
}

cudaError_t run_host_any(const GraphSpec& gs, cudaStream_t stream) {
  if (gs.fp32) {
    if (gs.kb == 0) return run_host<float, 0>(gs, stream);
    if (gs.kb == 8) return run_host<float, 8>(gs, stream);
    if (gs.kb == 16) return run_host<float, 16>(gs, stream);
    if (gs.kb == 24) return run_host<float, 24>(gs, stream);
    return run_host<float, 32>(gs, stream);
  }
  if (gs.kb == 0) return run_host<double, 0>(gs, stream);
  if (gs.kb == 8) return run_host<double, 8>(gs, stream);
  if (gs.kb == 16) return run_host<double, 16>(gs, stream);
  if (gs.kb == 24) return run_host<double, 24>(gs, stream);
  return run_host<double, 32>(gs, stream);
}

cudaError_t build_graph_any(const GraphSpec& gs, cudaGraph_t* out) {
  if (gs.fp32) {
    if (gs.kb == 0) return build_graph<float, 0>(gs, out);
    if (gs.kb == 8) return build_graph<float, 8>(gs, out);
    if (gs.kb == 16) return build_graph<float, 16>(gs, out);
    if (gs.kb == 24) return build_graph<float, 24>(gs, out);
    return build_graph<float, 32>(gs, out);
  }
  if (gs.kb == 0) return build_graph<double, 0>(gs, out);
  if (gs.kb == 8) return build_graph<double, 8>(gs, out);
  if (gs.kb == 16) return build_graph<double, 16>(gs, out);
  if (gs.kb == 24) return build_graph<double, 24>(gs, out);
  return build_graph<double, 32>(gs, out);
}

// resident blocks per SM of step a (returned) and step b (*occ_b)
int occupancy(bool fp32, int kb, int* occ_b) {
  int a = 1, b = 1;
  const void* fa;
  const void* fb;
  if (fp32) {
    fa = kb == 0 ? (const void*)b_step_a_kernel<float, 0>
       : kb == 8 ? (const void*)b_step_a_kernel<float, 8>
       : kb == 16 ? (const void*)b_step_a_kernel<float, 16>
       : kb == 24 ? (const void*)b_step_a_kernel<float, 24> : (const void*)b_step_a_kernel<float, 32>;
    fb = kb == 0 ? (const void*)b_step_b_kernel<float, 0>
       : kb == 8 ? (const void*)b_step_b_kernel<float, 8>
       : kb == 16 ? (const void*)b_step_b_kernel<float, 16>
       : kb == 24 ? (const void*)b_step_b_kernel<float, 24> : (const void*)b_step_b_kernel<float, 32>;
  } else {
    fa = kb == 0 ? (const void*)b_step_a_kernel<double, 0>
       : kb == 8 ? (const void*)b_step_a_kernel<double, 8>
       : kb == 16 ? (const void*)b_step_a_kernel<double, 16>
       : kb == 24 ? (const void*)b_step_a_kernel<double, 24> : (const void*)b_step_a_kernel<double, 32>;
    fb = kb == 0 ? (const void*)b_step_b_kernel<double, 0>
       : kb == 8 ? (const void*)b_step_b_kernel<double, 8>
       : kb == 16 ? (const void*)b_step_b_kernel<double, 16>
       : kb == 24 ? (const void*)b_step_b_kernel<double, 24> : (const void*)b_step_b_kernel<double, 32>;
  }
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, fa, kThreads, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fb, kThreads, 0);
  *occ_b = std::max(1, b);
  return std::max(1, a);
}

}  // namespace batch
}  // namespace mrcg

// ====================================================================== host side

using namespace mrcg;
using namespace mrcg::batch;

struct mrcg_batch {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int nsys = 0, nc = 0, kmax = 0, kb = 0;
  bool fp32 = false;
  int mcg = MRCG_MCG_IDENTITY;
  int max_outer = 200;
  double restart_factor = 0.5;
  int64_t n_total = 0;  // sum of padded rows
  std::vector<SysDesc> h_sys;
  std::vector<Chunk> h_chunks;
  std::vector<double> lam2;  // [nsys][kMaxK]
  SysDesc* d_sys = nullptr;
  Chunk* d_chunks = nullptr;
  DevState* d_st = nullptr;
  DevState* h_st = nullptr;  // pinned
  DevState* h_init = nullptr;
  int* h_modes = nullptr;    // pinned
  int* d_modes = nullptr;
  int* d_ctl = nullptr;
  double* d_partials = nullptr;
  Sell A;
  double *d_V64 = nullptr, *d_dinv64 = nullptr;
  float* d_V32 = nullptr;
  void* d_dinv = nullptr;
  double *x = nullptr, *b = nullptr, *res = nullptr, *zraw = nullptr, *zn = nullptr;
  double *v0 = nullptr, *v1 = nullptr, *w0 = nullptr, *w1 = nullptr;
  void *iz = nullptr, *ir = nullptr, *is = nullptr, *ip0 = nullptr, *ip1 = nullptr, *iq = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int grid = 1, grid_b = 1, unroll = 4;
  int chunk_rows = 0, nc_cap = 0;  // rows per chunk (autotuned), chunk capacity of the device arrays
  int occ_a = 1, occ_b = 1;        // occupancy limits of step a / step b (blocks per SM)
  bool host_loop = false;  // MRCG_INNER_LOOP=host: inner loop driven from the host (for profilers)
  GraphSpec gs;
  std::vector<void*> allocs;
};

namespace {

#define BCK(call)                                                                                 \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess) {                                                                      \
      if (getenv("MRCG_DEBUG")) fprintf(stderr, "mrcg batch: %s failed: %s (%s:%d)\n", #call,     \
                                        cudaGetErrorString(e_), __FILE__, __LINE__);              \
      return e_ == cudaErrorMemoryAllocation ? MRCG_ERR_OOM : MRCG_ERR_CUDA;                      \
    }                                                                                             \
  } while (0)
#define BST(call)                   \
  do {                              \
    mrcg_status s_ = (call);        \
    if (s_ != MRCG_OK) return s_;   \
  } while (0)

bool dev_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

template <typename T>
mrcg_status balloc(mrcg_batch* h, T** p, size_t count) {
  void* q = nullptr;
  if (cudaMalloc(&q, count * sizeof(T) + 16) != cudaSuccess) {
    cudaGetLastError();
    return MRCG_ERR_OOM;
  }
  h->allocs.push_back(q);
  *p = reinterpret_cast<T*>(q);
  return MRCG_OK;
}

template <typename T>
mrcg_status fetch(const T* src, size_t count, std::vector<T>& dst) {
  dst.resize(count);
  if (!count) return MRCG_OK;
  if (dev_ptr(src)) BCK(cudaMemcpy(dst.data(), src, count * sizeof(T), cudaMemcpyDeviceToHost));
  else std::memcpy(dst.data(), src, count * sizeof(T));
  return MRCG_OK;
}

// cut every system into chunks of at most `rows` rows (never straddling two
// systems); chunk0 / nchunks of each system follow
void make_chunks(mrcg_batch* h, int rows) {
  h->chunk_rows = rows;
  h->h_chunks.clear();
  int chunk0 = 0;
  for (int i = 0; i < (int)h->h_sys.size(); ++i) {
    SysDesc& sd = h->h_sys[i];
    sd.chunk0 = chunk0;
    sd.nchunks = (int)((sd.n_pad + rows - 1) / rows);
    for (int c = 0; c < sd.nchunks; ++c) {
      Chunk ch = {};
      ch.row0 = sd.row0 + (int64_t)c * rows;
      ch.row1 = std::min<int64_t>(sd.row0 + sd.n_pad, ch.row0 + rows);
      ch.sys = i;
      h->h_chunks.push_back(ch);
    }
    chunk0 += sd.nchunks;
  }
  h->nc = chunk0;
}

mrcg_status upload_chunks(mrcg_batch* h) {
  BCK(cudaMemcpyAsync(h->d_sys, h->h_sys.data(), h->h_sys.size() * sizeof(SysDesc), cudaMemcpyHostToDevice,
                      h->stream));
  BCK(cudaMemcpyAsync(h->d_chunks, h->h_chunks.data(), h->nc * sizeof(Chunk), cudaMemcpyHostToDevice, h->stream));
  BCK(cudaStreamSynchronize(h->stream));  // the host vectors may change next
  return MRCG_OK;
}

mrcg_status batched_solve_impl(mrcg_batch* h, const double* B, double* X, double outer_tol, double inner_tol,
                               int64_t max_iters, mrcg_info* infos, int64_t* launches_out);

__global__ void b_pattern_kernel(double* v, int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < count; i += (int64_t)gridDim.x * kThreads)
    v[i] = 1.0 + 0.125 * (double)(i % 7) - 0.0625 * (double)(i % 5);
}

// host time of one calibration solve: each system's first inner solve runs
// exactly `iters` iterations (tolerance 1e-300, budget iters) on a fixed
// right-hand side, then every system stops (iteration budget)
mrcg_status b_calib(mrcg_batch* h, long long iters, double* ms) {
  b_pattern_kernel<<<256, kThreads, 0, h->stream>>>(h->zn, h->n_total);
  BCK(cudaGetLastError());
  BCK(cudaStreamSynchronize(h->stream));
  const auto t0 = std::chrono::steady_clock::now();
  const mrcg_status st = batched_solve_impl(h, h->zn, h->w0, 0.0, 1e-300, iters, nullptr, nullptr);
  *ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return (st == MRCG_OK || st == MRCG_ERR_MAXITER) ? MRCG_OK : st;
}

mrcg_status b_rebuild(mrcg_batch* h, int nsm, int rows, int bps_a, int bps_b) {
  make_chunks(h, rows);
  BST(upload_chunks(h));
  h->grid = std::max(1, std::min(h->nc, nsm * bps_a));
  h->grid_b = std::max(1, std::min(h->nc, nsm * bps_b));
  h->gs.nc = h->nc;
  h->gs.grid = h->grid;
  h->gs.grid_b = h->grid_b;
  if (h->exec) cudaGraphExecDestroy(h->exec);
  if (h->graph) cudaGraphDestroy(h->graph);
  h->exec = nullptr;
  h->graph = nullptr;
  BCK(build_graph_any(h->gs, &h->graph));
  BCK(cudaGraphInstantiate(&h->exec, h->graph, 0));
  return MRCG_OK;
}

// Launch-shape autotuner of the batch engine: rows per chunk (the unit a
// block reduces and a converged system skips) and blocks per SM of step a,
// then blocks per SM of step b, each candidate timed by the difference of two
// calibration solves (8 and 40 inner iterations per system)
mrcg_status batch_autotune(mrcg_batch* h, int nsm) {
  auto per_iter = [&](double* out) -> mrcg_status {
    double t1 = 0.0, t2 = 0.0;
    BST(b_calib(h, 8, &t1));
    BST(b_calib(h, 40, &t2));
    *out = (t2 - t1) / 32.0;
    return MRCG_OK;
  };
  double best = 1e300;
  int best_rows = kChunkRows, best_a = h->occ_a, best_b = h->occ_b;
  for (int rows : {1024, 2048, 4096, 8192}) {
    for (int bps = 1; bps <= h->occ_a; ++bps) {
      BST(b_rebuild(h, nsm, rows, bps, h->occ_b));
      double t = 0.0;
      BST(per_iter(&t));
      if (getenv("MRCG_DEBUG"))
        fprintf(stderr, "mrcg batch autotune: chunk %d rows, step a %d blocks/SM: %.4f ms per iteration\n", rows,
                bps, t);
      if (t < best) {
        best = t;
        best_rows = rows;
        best_a = bps;
      }
    }
  }
  for (int bps = 1; bps <= h->occ_b; ++bps) {
    if (bps == h->occ_b) continue;  // timed above
    BST(b_rebuild(h, nsm, best_rows, best_a, bps));
    double t = 0.0;
    BST(per_iter(&t));
    if (getenv("MRCG_DEBUG"))
      fprintf(stderr, "mrcg batch autotune: step b %d blocks/SM: %.4f ms per iteration\n", bps, t);
    if (t < best) {
      best = t;
      best_b = bps;
    }
  }
  BST(b_rebuild(h, nsm, best_rows, best_a, best_b));
  BCK(cudaStreamSynchronize(h->stream));
  return MRCG_OK;
}

mrcg_status batch_create_impl(int32_t nsys, const mrcg_create_args* args, mrcg_batch* h) {
  h->nsys = nsys;
  h->fp32 = args[0].precision == MRCG_MIXED_FP32;
  h->mcg = args[0].inner_prec;
  h->max_outer = args[0].max_outer > 0 ? args[0].max_outer : 200;
  h->restart_factor = args[0].restart_factor == 0.0 ? 0.5 : args[0].restart_factor;
  if (args[0].stream) {
    h->stream = (cudaStream_t)args[0].stream;
  } else {
    BCK(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    h->own_stream = true;
  }
  // ---- host copies, validation, layout
  std::vector<std::vector<int64_t>> rps(nsys);
  std::vector<std::vector<int32_t>> cis(nsys);
  std::vector<std::vector<double>> vas(nsys), Vs(nsys), lams(nsys);
  h->lam2.assign((size_t)nsys * kMaxK, 0.0);
  int64_t row0 = 0, voff = 0, slices = 0;

  for (int i = 0; i < nsys; ++i) {
    const mrcg_create_args& a = args[i];
    if (a.n < 1 || a.nnz < 0 || a.k < 0 || a.k > kMaxK || !a.rowptr || (a.nnz > 0 && (!a.colind || !a.val)) ||
        (a.k > 0 && (!a.V || !a.lambda)))
      return MRCG_ERR_INVALID;
    if (a.precision != args[0].precision || a.inner_prec != args[0].inner_prec) return MRCG_ERR_INVALID;
    if (a.inner_prec != MRCG_MCG_IDENTITY && a.inner_prec != MRCG_MCG_JACOBI) return MRCG_ERR_INVALID;
    if (a.precision != MRCG_FP64 && a.precision != MRCG_MIXED_FP32) return MRCG_ERR_INVALID;
    BST(fetch(a.rowptr, (size_t)a.n + 1, rps[i]));
    BST(fetch(a.colind, (size_t)a.nnz, cis[i]));
    BST(fetch(a.val, (size_t)a.nnz, vas[i]));
    BST(fetch(a.lambda, (size_t)a.k, lams[i]));
    BST(fetch(a.V, (size_t)a.n * a.k, Vs[i]));
    const auto& rp = rps[i];
    const auto& ci = cis[i];
    if (rp[0] != 0 || rp[a.n] != a.nnz) return MRCG_ERR_INVALID;
    for (int64_t r = 0; r < a.n; ++r) {
      if (rp[r + 1] < rp[r]) return MRCG_ERR_INVALID;
      for (int64_t p = rp[r]; p < rp[r + 1]; ++p) {
        if (ci[p] < 0 || ci[p] >= a.n || (p > rp[r] && ci[p] <= ci[p - 1])) return MRCG_ERR_INVALID;
        if (!std::isfinite(vas[i][p])) return MRCG_ERR_NONFINITE;
      }
    }
    for (int l = 0; l < a.k; ++l) {
      if (!(lams[i][l] < 0.0) || !std::isfinite(lams[i][l])) return MRCG_ERR_INVALID;
      h->lam2[(size_t)i * kMaxK + l] = 2.0 * std::fabs(lams[i][l]);
    }
    SysDesc sd = {};
    sd.row0 = row0;
    sd.n = a.n;
    sd.n_pad = (a.n + kSlice - 1) / kSlice * kSlice;
    sd.slice0 = slices;
    sd.voff = voff;
    sd.k = a.k;
    h->h_sys.push_back(sd);
    row0 += sd.n_pad;
    slices += sd.n_pad / kSlice;
    voff += sd.n_pad * a.k;
    h->kmax = std::max(h->kmax, a.k);
  }
  if (row0 > (int64_t)0x7fffff00) return MRCG_ERR_INVALID;
  h->n_total = row0;
  // chunk capacity: the smallest chunk height the autotuner tries
  h->nc_cap = 0;
  for (const SysDesc& sd : h->h_sys) h->nc_cap += (int)((sd.n_pad + kChunkMin - 1) / kChunkMin);
  make_chunks(h, kChunkRows);
  h->kb = h->kmax == 0 ? 0 : h->kmax <= 8 ? 8 : h->kmax <= 16 ? 16 : h->kmax <= 24 ? 24 : 32;
  // ---- block-diagonal SELL-32 with global columns
  const int64_t nslices = slices;
  std::vector<int64_t> sp((size_t)nslices + 1, 0);
  for (int i = 0; i < nsys; ++i) {
    const SysDesc& sd = h->h_sys[i];
    const auto& rp = rps[i];
    for (int64_t s = 0; s < sd.n_pad / kSlice; ++s) {
      int64_t w = 0;
      for (int64_t r = s * kSlice; r < std::min<int64_t>(sd.n, (s + 1) * kSlice); ++r) w = std::max(w, rp[r + 1] - rp[r]);
      sp[sd.slice0 + s + 1] = w * kSlice;
    }
  }
  for (int64_t s = 0; s < nslices; ++s) sp[s + 1] += sp[s];
  const int64_t total = sp[nslices];
  std::vector<int32_t> col((size_t)total);
  std::vector<double> val((size_t)total, 0.0);
  for (int i = 0; i < nsys; ++i) {
    const SysDesc& sd = h->h_sys[i];
    const auto& rp = rps[i];
    for (int64_t r = 0; r < sd.n_pad; ++r) {
      const int64_t s = sd.slice0 + r / kSlice, lane = r % kSlice;
      const int64_t w = (sp[s + 1] - sp[s]) / kSlice;
      const int64_t len = r < sd.n ? rp[r + 1] - rp[r] : 0;
      for (int64_t j = 0; j < w; ++j) {
        const int64_t idx = sp[s] + j * kSlice + lane;
        if (j < len) {
          col[idx] = (int32_t)(sd.row0 + cis[i][rp[r] + j]);
          val[idx] = vas[i][rp[r] + j];
        } else {
          col[idx] = (int32_t)(sd.row0 + r);
          val[idx] = 0.0;
        }
      }
    }
  }
  int64_t* d_sp;
  int32_t* d_col;
  double* d_val;
  float* d_val32 = nullptr;
  BST(balloc(h, &d_sp, sp.size()));
  BST(balloc(h, &d_col, col.size() + 1));
  BST(balloc(h, &d_val, val.size() + 1));
  BCK(cudaMemcpyAsync(d_sp, sp.data(), sp.size() * 8, cudaMemcpyHostToDevice, h->stream));
  BCK(cudaMemcpyAsync(d_col, col.data(), col.size() * 4, cudaMemcpyHostToDevice, h->stream));
  BCK(cudaMemcpyAsync(d_val, val.data(), val.size() * 8, cudaMemcpyHostToDevice, h->stream));
  if (h->fp32) {
    BST(balloc(h, &d_val32, val.size() + 1));
    if (launch_to_f32(h->stream, d_val, d_val32, (int64_t)val.size()) != cudaSuccess) return MRCG_ERR_CUDA;
  }
  h->A.n = h->n_total;
  h->A.n_pad = h->n_total;
  h->A.nslices = nslices;
  h->A.total = total;
  h->A.slice_ptr = d_sp;
  h->A.col = d_col;
  h->A.val64 = d_val;
  h->A.val32 = d_val32;
  // ---- V_hat blocks (zero padded rows) and Jacobi diagonal
  const size_t vtot = (size_t)std::max<int64_t>(voff, 1);
  std::vector<double> Vh(vtot, 0.0), dinv((size_t)h->n_total, 0.0);
  for (int i = 0; i < nsys; ++i) {
    const SysDesc& sd = h->h_sys[i];
    for (int l = 0; l < sd.k; ++l)
      std::memcpy(&Vh[sd.voff + (size_t)l * sd.n_pad], &Vs[i][(size_t)l * sd.n], sd.n * sizeof(double));
    for (int64_t r = 0; r < sd.n; ++r) {
      double d = 0.0;
      for (int64_t p = rps[i][r]; p < rps[i][r + 1]; ++p)
        if (cis[i][p] == r) d += vas[i][p];
      for (int l = 0; l < sd.k; ++l) {
        const double vv = Vs[i][(size_t)l * sd.n + r];
        d += h->lam2[(size_t)i * kMaxK + l] * vv * vv;
      }
      dinv[sd.row0 + r] = 1.0 / d;
    }
  }
  BST(balloc(h, &h->d_V64, vtot));
  BCK(cudaMemcpyAsync(h->d_V64, Vh.data(), vtot * 8, cudaMemcpyHostToDevice, h->stream));
  if (h->fp32) {
    BST(balloc(h, &h->d_V32, vtot));
    if (launch_to_f32(h->stream, h->d_V64, h->d_V32, (int64_t)vtot) != cudaSuccess) return MRCG_ERR_CUDA;
  }
  const size_t esz = h->fp32 ? 4 : 8;
  if (h->mcg == MRCG_MCG_JACOBI) {
    BST(balloc(h, &h->d_dinv64, (size_t)h->n_total));
    BCK(cudaMemcpyAsync(h->d_dinv64, dinv.data(), dinv.size() * 8, cudaMemcpyHostToDevice, h->stream));
    if (h->fp32) {
      float* d32;
      BST(balloc(h, &d32, (size_t)h->n_total));
      if (launch_to_f32(h->stream, h->d_dinv64, d32, h->n_total) != cudaSuccess) return MRCG_ERR_CUDA;
      h->d_dinv = d32;
    } else {
      h->d_dinv = h->d_dinv64;
    }
  }
  // ---- vectors and state
  double** f64[] = {&h->x, &h->b, &h->res, &h->zraw, &h->zn, &h->v0, &h->v1, &h->w0, &h->w1};
  for (double** p : f64) {
    BST(balloc(h, p, (size_t)h->n_total));
    BCK(cudaMemsetAsync(*p, 0, (size_t)h->n_total * 8, h->stream));
  }
  void** inner[] = {&h->iz, &h->ir, &h->is, &h->ip0, &h->ip1, &h->iq};
  for (void** p : inner) {
    if (p == &h->is && h->mcg != MRCG_MCG_JACOBI) continue;
    char* q;
    BST(balloc(h, &q, (size_t)h->n_total * esz));
    BCK(cudaMemsetAsync(q, 0, (size_t)h->n_total * esz, h->stream));
    *p = q;
  }
  BST(balloc(h, &h->d_sys, (size_t)nsys));
  BST(balloc(h, &h->d_chunks, (size_t)h->nc_cap));
  BST(balloc(h, &h->d_st, (size_t)nsys));
  BST(balloc(h, &h->d_partials, (size_t)kMaxNV * h->nc_cap));
  BST(balloc(h, &h->d_modes, (size_t)nsys));
  BST(balloc(h, &h->d_ctl, 3));
  BST(upload_chunks(h));
  BCK(cudaMemsetAsync(h->d_st, 0, nsys * sizeof(DevState), h->stream));
  BCK(cudaMallocHost(&h->h_st, nsys * sizeof(DevState)));
  BCK(cudaMallocHost(&h->h_init, nsys * sizeof(DevState)));
  BCK(cudaMallocHost(&h->h_modes, nsys * sizeof(int)));
  // ---- geometry and graph
  int nsm = 1;
  BCK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device));
  int occ_b = 1;
  const int occ = occupancy(h->fp32, h->kb, &occ_b);
  h->occ_a = occ;
  h->occ_b = occ_b;
  h->grid = std::max(1, std::min(h->nc, nsm * occ));
  h->grid_b = std::max(1, std::min(h->nc, nsm * occ_b));
  if (const char* u = getenv("MRCG_UNROLL")) h->unroll = std::max(2, atoi(u) & ~1);
  GraphSpec gs = {};
  gs.fp32 = h->fp32;
  gs.kb = h->kb;
  gs.nsys = nsys;
  gs.nc = h->nc;
  gs.st = h->d_st;
  gs.sys = h->d_sys;
  gs.chunks = h->d_chunks;
  gs.partials = h->d_partials;
  gs.A = h->A;
  gs.V = h->fp32 ? (const void*)h->d_V32 : (const void*)h->d_V64;
  gs.dinv = h->d_dinv;
  gs.z = h->iz;
  gs.r = h->ir;
  gs.s = h->is;
  gs.p0 = h->ip0;
  gs.p1 = h->ip1;
  gs.q = h->iq;
  gs.ctl = h->d_ctl;
  gs.grid = h->grid;
  gs.grid_b = h->grid_b;
  gs.unroll = h->unroll;
  h->gs = gs;
  if (const char* m = getenv("MRCG_INNER_LOOP")) h->host_loop = std::strcmp(m, "host") == 0;
  BCK(build_graph_any(gs, &h->graph));
  BCK(cudaGraphInstantiate(&h->exec, h->graph, 0));
  BCK(cudaStreamSynchronize(h->stream));
  const char* at = getenv("MRCG_AUTOTUNE");
  // MRCG_AUTOTUNE=2 tunes whatever the size (tests)
  if ((!at || atoi(at) != 0) && (h->n_total >= (1 << 20) || (at && atoi(at) == 2))) BST(batch_autotune(h, nsm));
  return MRCG_OK;
}

void batch_destroy_impl(mrcg_batch* h) {
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->exec) cudaGraphExecDestroy(h->exec);
  if (h->graph) cudaGraphDestroy(h->graph);
  for (void* p : h->allocs) cudaFree(p);
  if (h->h_st) cudaFreeHost(h->h_st);
  if (h->h_init) cudaFreeHost(h->h_init);
  if (h->h_modes) cudaFreeHost(h->h_modes);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  cudaGetLastError();
  delete h;
}

OArgs oargs(mrcg_batch* h) {
  OArgs a;
  a.st = h->d_st;
  a.sys = h->d_sys;
  a.chunks = h->d_chunks;
  a.nc = h->nc;
  a.partials = h->d_partials;
  a.slice_ptr = h->A.slice_ptr;
  a.col = h->A.col;
  a.val = h->A.val64;
  a.x = h->x;
  a.b = h->b;
  a.res = h->res;
  a.zraw = h->zraw;
  a.zn = h->zn;
  a.v0 = h->v0;
  a.v1 = h->v1;
  a.w0 = h->w0;
  a.w1 = h->w1;
  return a;
}

mrcg_status set_modes(mrcg_batch* h) {
  BCK(cudaMemcpyAsync(h->d_modes, h->h_modes, h->nsys * sizeof(int), cudaMemcpyHostToDevice, h->stream));
  b_set_modes_kernel<<<(h->nsys + 255) / 256, 256, 0, h->stream>>>(h->d_st, h->d_modes, h->nsys);
  BCK(cudaGetLastError());
  return MRCG_OK;
}

mrcg_status read_states(mrcg_batch* h) {
  BCK(cudaMemcpyAsync(h->h_st, h->d_st, h->nsys * sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
  BCK(cudaStreamSynchronize(h->stream));
  return MRCG_OK;
}

// copy the systems' n rows between a user array of sum(n_i) entries and the padded device layout
mrcg_status stage(mrcg_batch* h, const double* user, double* dev, bool to_dev) {
  const bool ud = dev_ptr(user);
  int64_t off = 0;
  for (int i = 0; i < h->nsys; ++i) {
    const SysDesc& sd = h->h_sys[i];
    if (to_dev)
      BCK(cudaMemcpyAsync(dev + sd.row0, user + off, sd.n * 8, ud ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                          h->stream));
    else
      BCK(cudaMemcpyAsync(const_cast<double*>(user) + off, dev + sd.row0, sd.n * 8,
                          ud ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
    off += sd.n;
  }
  return MRCG_OK;
}

mrcg_status batched_solve_impl(mrcg_batch* h, const double* B, double* X, double outer_tol, double inner_tol,
                               int64_t max_iters, mrcg_info* infos, int64_t* launches_out) {
  const int S = h->nsys;
  const long long budget = max_iters > 0 ? (long long)max_iters : (1LL << 31);
  BST(stage(h, B, h->b, true));
  BST(stage(h, X, h->x, true));
  for (int i = 0; i < S; ++i) {
    DevState& d = h->h_init[i];
    std::memset(&d, 0, sizeof(DevState));
    for (int l = 0; l < kMaxK; ++l) d.cg.lam2[l] = h->lam2[(size_t)i * kMaxK + l];
    d.cg.inner_tol = inner_tol;
    d.cg.budget = budget;
    d.cg.done = kConverged;
    d.out.status = MRCG_OK;
  }
  BCK(cudaMemcpyAsync(h->d_st, h->h_init, S * sizeof(DevState), cudaMemcpyHostToDevice, h->stream));
  {
    const long long lim = budget / h->unroll + 2;
    int ctl_host[2] = {0, (int)std::min<long long>(lim, 0x7fffffffLL)};
    BCK(cudaMemcpyAsync(h->d_ctl, ctl_host, sizeof(ctl_host), cudaMemcpyHostToDevice, h->stream));
    BCK(cudaStreamSynchronize(h->stream));
  }
  OArgs oa = oargs(h);
  long long launches = 0;
  const int g = h->grid;
  b_bnorm_kernel<<<g, kThreads, 0, h->stream>>>(oa);
  b_residual_kernel<<<g, kThreads, 0, h->stream>>>(oa, 1);
  launches += 2;
  BCK(cudaGetLastError());
  BST(read_states(h));
  std::vector<int> mode(S, 0), outer(S, 0), restarts(S, 0), hist_len(S, 0);
  std::vector<mrcg_status> status(S, MRCG_ERR_MAXITER);
  std::vector<double> relres(S, 0.0);
  std::vector<std::vector<double>> cyc(S);
  int active = 0;
  for (int i = 0; i < S; ++i) {
    const OuterState& O = h->h_st[i].out;
    relres[i] = O.relres;
    if (O.status != MRCG_OK || !std::isfinite(O.bnorm)) {
      status[i] = MRCG_ERR_NONFINITE;
    } else if (O.bnorm == 0.0) {
      BCK(cudaMemsetAsync(h->x + h->h_sys[i].row0, 0, h->h_sys[i].n * 8, h->stream));
      relres[i] = 0.0;
      status[i] = MRCG_OK;
    } else if (O.relres <= outer_tol) {
      status[i] = MRCG_OK;
    } else {
      mode[i] = 1;
      ++active;
    }
  }
  while (active > 0) {
    for (int i = 0; i < S; ++i) {
      if (mode[i] == 2 && outer[i] >= h->max_outer) {
        mode[i] = 0;
        status[i] = MRCG_ERR_MAXITER;
        --active;
      }
      h->h_modes[i] = mode[i];
    }
    if (active == 0) break;
    BST(set_modes(h));
    b_cycle_start_kernel<<<g, kThreads, 0, h->stream>>>(oa);
    b_lanczos_spmv_kernel<<<g, kThreads, 0, h->stream>>>(oa);
    b_lanczos_update_kernel<<<g, kThreads, 0, h->stream>>>(oa);
    BCK(cudaGetLastError());
    if (h->host_loop) BCK(run_host_any(h->gs, h->stream));
    else BCK(cudaGraphLaunch(h->exec, h->stream));
    b_gamma_kernel<<<g, kThreads, 0, h->stream>>>(oa);
    b_minres_update_kernel<<<g, kThreads, 0, h->stream>>>(oa);
    b_residual_kernel<<<g, kThreads, 0, h->stream>>>(oa, 0);
    launches += 8;
    BCK(cudaGetLastError());
    BST(read_states(h));
    int ctl = 0;
    BCK(cudaMemcpy(&ctl, h->d_ctl, sizeof(int), cudaMemcpyDeviceToHost));
    launches += 3 + (long long)ctl * (2LL * h->unroll + 1);
    for (int i = 0; i < S; ++i) {
      const OuterState& O = h->h_st[i].out;
      if (mode[i] == 0) continue;
      if (O.status != MRCG_OK) {
        status[i] = (mrcg_status)O.status;
        mode[i] = 0;
        --active;
        continue;
      }
      if (mode[i] == 1) {
        mode[i] = 2;
        cyc[i].clear();
        continue;
      }
      ++outer[i];
      relres[i] = O.relres;
      mrcg_info* inf = infos ? &infos[i] : nullptr;
      if (inf && inf->relres_history && hist_len[i] < inf->history_cap) inf->relres_history[hist_len[i]] = O.relres;
      ++hist_len[i];
      if (O.relres <= outer_tol) {
        status[i] = MRCG_OK;
        mode[i] = 0;
        --active;
        continue;
      }
      cyc[i].push_back(O.relres);
      const size_t m = cyc[i].size();
      if ((h->restart_factor > 0.0 && m >= 4 && O.relres > h->restart_factor * cyc[i][m - 4]) || O.gamma_new == 0.0) {
        ++restarts[i];
        mode[i] = 1;
      }
    }
  }
  BST(stage(h, X, h->x, false));
  BST(read_states(h));
  mrcg_status worst = MRCG_OK;
  for (int i = 0; i < S; ++i) {
    if (infos) {
      mrcg_info& inf = infos[i];
      inf.outer_iters = outer[i];
      inf.restarts = restarts[i];
      inf.inner_iters_total = h->h_st[i].out.inner_total;
      inf.prec_calls = h->h_st[i].out.prec_calls;
      inf.true_relres = relres[i];
      inf.history_len = inf.relres_history ? std::min(hist_len[i], inf.history_cap) : 0;
      inf.status = status[i];
      inf.kernel_launches = launches;
    }
    if (status[i] != MRCG_OK && worst == MRCG_OK) worst = status[i];
  }
  if (launches_out) *launches_out = launches;
  return worst;
}

}  // namespace

extern "C" {

mrcg_status mrcg_batch_create(int32_t nsys, const mrcg_create_args* sys, mrcg_batch_handle* out) {
  if (!sys || !out || nsys < 1 || nsys > kMaxSystems) return MRCG_ERR_INVALID;
  *out = nullptr;
  mrcg_batch* h = new (std::nothrow) mrcg_batch();
  if (!h) return MRCG_ERR_OOM;
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    delete h;
    return MRCG_ERR_CUDA;
  }
  mrcg_status s = batch_create_impl(nsys, sys, h);
  if (s != MRCG_OK) {
    cudaGetLastError();
    batch_destroy_impl(h);
    return s;
  }
  *out = h;
  return MRCG_OK;
}

mrcg_status mrcg_batched_solve(mrcg_batch_handle h, const double* B, double* X, double outer_tol, double inner_tol,
                               int64_t max_iters, mrcg_info* infos) {
  mrcg::TraceRange tr("mrcg_batched_solve");
  if (!h || !B || !X) return MRCG_ERR_INVALID;
  if (!(outer_tol >= 0.0) || !(inner_tol > 0.0) || !(inner_tol < 1.0)) return MRCG_ERR_INVALID;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != h->device) cudaSetDevice(h->device);
  const auto t0 = std::chrono::steady_clock::now();
  mrcg_status s = batched_solve_impl(h, B, X, outer_tol, inner_tol, max_iters, infos, nullptr);
  const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  if (infos)
    for (int i = 0; i < h->nsys; ++i) infos[i].solve_ms = ms;
  if (prev >= 0 && prev != h->device) cudaSetDevice(prev);
  return s;
}

int32_t mrcg_batch_size(mrcg_batch_handle h) { return h ? h->nsys : 0; }

mrcg_status mrcg_batch_launch_config(mrcg_batch_handle h, int32_t* cfg) {
  if (!h || !cfg) return MRCG_ERR_INVALID;
  cfg[0] = h->chunk_rows;
  cfg[1] = h->grid;
  cfg[2] = h->grid_b;
  cfg[3] = h->nc;
  return MRCG_OK;
}

void mrcg_batch_destroy(mrcg_batch_handle h) {
  if (h) batch_destroy_impl(h);
}

}  // extern "C"
