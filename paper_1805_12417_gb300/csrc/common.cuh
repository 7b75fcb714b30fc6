// Shared definitions of the MINRES-CG CUDA library (sm_103a).
//
// Data layout in HBM (one solver handle):
//   A        SELL-32: slices of 32 consecutive rows; inside a slice the j-th
//            stored entry of every row is contiguous (col-major), so lane l of
//            a warp reads entry j of row 32*s + l with one coalesced access.
//            Padded entries carry value 0 and a valid column (the row itself).
//   vectors  length n_pad = 32 * nslices, padding rows held at zero.
//   V_hat    column-major n_pad x k (column j at V + j * n_pad).
//   scalars  one DevState per handle: every scalar of the Krylov recurrences
//            lives on the device, so the inner loop never waits for the host.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstring>

#include "mrcg.h"

namespace mrcg {

constexpr int kSlice = 32;      // SELL slice height = warp width
constexpr int kMaxK = 32;       // maximum columns of V_hat
constexpr int kThreads = 256;   // block size of every streaming kernel
constexpr int kMaxBlocks = 2048;
constexpr int kMaxNV = kMaxK + 4;  // reduction values per block

// inner CG outcome codes (CgState::done)
// (kStall: a staged copy did not arrive within its wait limit; reported as a CUDA error)
// (kBreakdown: r^T M_cg^{-1} r = 0 before convergence, possible only with an indefinite M_cg)
enum : int {
  kRunning = 0,
  kConverged = 1,
  kNotSpd = 2,
  kNonFinite = 3,
  kMaxIter = 4,
  kLoopCap = 5,
  kStall = 6,
  kBreakdown = 7
};

struct CgState {
  double rho;            // r^T s of the current residual (s = M_cg^{-1} r)
  double alpha, beta;
  double tol_abs;        // inner_tol * ||y_normalised||
  double vnorm;          // ||v||: the inner solve runs on v / ||v||
  double kappa;          // last p^T M_mr p
  double lam2[kMaxK];    // 2 |lambda_j|
  double c[kMaxK];       // 2 |lambda_j| (V^T p)_j for the current direction p
  double t[kMaxK];       // (V^T p)_j for the current direction p
  double u[kMaxK];       // V^T s of the current preconditioned residual s (recurrence)
  double vq[kMaxK];      // V^T (M_cg^{-1} q) of the last M_mr product q (V^T q with the MINRES-CG* M_cg)
  double vr[kMaxK];      // V^T r (MINRES-CG* M_cg only, by recurrence)
  float c32[kMaxK];      // FP32 copies of c, alpha, beta for the FP32 kernels
  float alpha32, beta32;
  double inner_tol;      // per-call parameters (uploaded by the host)
  long long budget;      // inner iterations still allowed (total budget)
  long long iters;       // iterations of the current inner solve
  long long maxit;
  int done;
  int ctl_count, ctl_limit;
  int unroll;            // CG iterations per body of the device while loop
  const double* vin;     // right-hand side of the inner solve (FP64)
  double* zout;          // its solution (FP64)
  // one-kernel iteration (identity M_cg): its last z update z += alpha p is
  // left to the finish kernel when the solve stops (fused_pending, p_last)
  int fused_pending;
  int pad_f;
  const void* p_last;
  // one-gather iteration (variants 9-15): each kernel finishes the reduction
  // of its predecessor in every block (no last block).  Slots by the parity of
  // the iteration, so that a kernel never writes a slot its own blocks read:
  // rho_s[j & 1] = rho_j, it_s[j & 1] = j (iterations done when step a of
  // iteration j starts), bp_s[j & 1] = 1 once step b of iteration j - 1 left
  // its partials for step a of iteration j to finish.
  double rho_s[2];
  long long it_s[2];
  int bp_s[2];
  // V^T s, V^T p and c = 2|Lambda| V^T p of the one-gather iteration, slot
  // j & 1 holding their values for iteration j (advanced by step a)
  double u_s[2][kMaxK];
  double t_s[2][kMaxK];
  double c_s[2][kMaxK];
};

struct OuterState {
  double bnorm, relres, rnorm2;
  double gamma, gamma_old, gamma_new;  // Lanczos normalisers gamma_j, gamma_{j-1}, gamma_{j+1}
  double delta;
  double eta, c, c_old, s, s_old;      // Givens state
  double a1, a2, a3, ceta;             // coefficients of the current w / x update
  long long inner_total;               // inner iterations of this solve
  long long prec_calls;
  long long bodies;                    // executed bodies of the inner while loop
  int status;                          // mrcg_status of the solve so far
  int mode;                            // batched solves: 0 idle, 1 cycle start, 2 outer step
  int cur;                             // batched solves: which of the two v / w buffers holds v_j, w_j
  int pad0;
};

struct DevState {
  CgState cg;
  OuterState out;
  unsigned int ticket;  // last-block ticket of the running kernel
  unsigned int pad[3];
};

struct Sell {
  int64_t n = 0, n_pad = 0, nslices = 0, total = 0;
  const int64_t* slice_ptr = nullptr;  // [nslices + 1] element offsets
  const int32_t* col = nullptr;        // [total]
  const double* val64 = nullptr;       // [total]
  const float* val32 = nullptr;        // [total] (mixed precision only)
  const int16_t* col16 = nullptr;      // [total] col - row, when every such delta fits in 16 bits (inner kernels)
};

// ------------------------------------------------------------------ device helpers

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block reduction of NV per-thread values in the threads' own precision T
// (FP32 in the mixed-precision kernels: no FP64 pipe work), stored as this
// block's FP64 partials, value-major: partials[i * gridDim.x + blockIdx.x].
// FENCE = false: the partials are read only by a later kernel (the kernel
// boundary makes them visible), so no block draws a ticket after them.
template <typename T, int NV, int NW = kThreads / 32, bool FENCE = true>
__device__ __forceinline__ void block_partials_t(T (&v)[NV], int nv, double* partials) {
  __shared__ T smt[NW][NV > 0 ? NV : 1];
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
    for (int w = 0; w < NW; ++w) s += smt[w][threadIdx.x];
    partials[threadIdx.x * gridDim.x + blockIdx.x] = (double)s;
    if (FENCE) __threadfence();  // the partial is visible before this block draws its ticket
  }
}

// Reduce NV per-thread values over the block and store them as this block's
// partials, value-major: partials[i * gridDim.x + blockIdx.x].
template <int NV>
__device__ __forceinline__ void block_partials(double (&v)[NV], int nv, double* partials) {
  __shared__ double sm[kThreads / 32][NV > 0 ? NV : 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < NV; ++i)
    if (i < nv) v[i] = warp_sum(v[i]);
  if (lane == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i)
      if (i < nv) sm[warp][i] = v[i];
  }
  __syncthreads();
  if (threadIdx.x < nv) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) s += sm[w][threadIdx.x];
    partials[threadIdx.x * gridDim.x + blockIdx.x] = s;
    __threadfence();  // the partial is visible before this block draws its ticket
  }
}

// Sum of x[lane], x[lane + 32], ... x[< count] with eight independent
// accumulators, so eight L2 loads per lane are in flight at once (a single
// accumulator would serialise on load latency).  The order is fixed by count.
__device__ __forceinline__ double lane_sum8(const double* x, int count, int lane) {
  double s[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  int b = lane;
  for (; b + 7 * 32 < count; b += 8 * 32) {
#pragma unroll
    for (int u = 0; u < 8; ++u) s[u] += __ldcg(x + b + u * 32);
  }
  for (int u = 0; b < count; b += 32, ++u) s[u] += __ldcg(x + b);
  return ((s[0] + s[1]) + (s[2] + s[3])) + ((s[4] + s[5]) + (s[6] + s[7]));
}

// Last-block detection (no waiting): every block publishes its partials,
// fences, and takes a ticket; the block that draws the final ticket sees all
// partials and finishes the reduction.  It also rearms the ticket.
__device__ __forceinline__ bool last_block(unsigned int* ticket) {
  __shared__ bool is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int prev = atomicAdd(ticket, 1u);
    is_last = (prev == gridDim.x - 1);
    if (is_last) *ticket = 0u;
  }
  __syncthreads();
  if (is_last) __threadfence();
  return is_last;
}

// The same for kernels whose partials come from block_partials / block_partials_t
// (their writers fence their own partials): the other threads skip the fence,
// which would make them wait for all of their vector stores to complete.
__device__ __forceinline__ bool last_block_after_partials(unsigned int* ticket) {
  __shared__ bool is_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int prev = atomicAdd(ticket, 1u);
    is_last = (prev == gridDim.x - 1);
    if (is_last) *ticket = 0u;
  }
  __syncthreads();
  if (is_last) __threadfence();
  return is_last;
}

// Sum the partials of nv values over all blocks in a fixed order
// (deterministic).  Result in out[0..nv) (shared memory), valid after return.
// Every thread takes part, so the last block's reduction costs one round trip
// to L2 rather than one per value a warp handles: value i is summed by a group
// of g = blockDim / nv threads, thread j of the group over the partials j,
// j + g, j + 2g, ... (16 loads in flight at a time), and one warp per value
// combines its group's sums (strided lane sums, then a butterfly).
// G: the grid that wrote the partials (this grid for a last block; the
// previous kernel's when a kernel finishes its predecessor's reduction).
constexpr int kFinalSumsThreads = 320;  // threads beyond this count only wait
// NT > 0: only the block's first NT threads take part (named barrier 1);
// the others must not call.
template <int NT>
__device__ __forceinline__ void group_sync() {
  if (NT == 0) __syncthreads();
  else asm volatile("bar.sync 1, %0;" ::"n"(NT) : "memory");
}

template <int NT = 0>
__device__ __forceinline__ void final_sums_2(const double* pa, int ga, int na, const double* pb, int gb, int nb,
                                             double* out) {
  __shared__ double fs[kFinalSumsThreads];
  const int nv = na + nb;
  const int nt = (NT > 0 ? NT : min((int)blockDim.x, kFinalSumsThreads)) & ~31;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = max(1, nt / max(1, nv));  // threads per value
  const int nvr = nt / g;                 // values per round
  for (int i0 = 0; i0 < nv; i0 += nvr) {
    const int i = i0 + tid / g, j = tid - (tid / g) * g;
    double s = 0.0;
    if (tid < nvr * g && i < nv) {
      const int G = i < na ? ga : gb;
      const double* x = i < na ? pa + (size_t)i * ga : pb + (size_t)(i - na) * gb;
      for (int b0 = j; b0 < G; b0 += 16 * g) {
        double v[16];
#pragma unroll
        for (int m = 0; m < 16; ++m) v[m] = b0 + m * g < G ? __ldcg(x + b0 + m * g) : 0.0;
#pragma unroll
        for (int w = 8; w > 0; w >>= 1)
#pragma unroll
          for (int m = 0; m < w; ++m) v[m] += v[m + w];
        s += v[0];
      }
    }
    if (tid < nt) fs[tid] = s;
    group_sync<NT>();
    for (int v = warp; v < nvr && i0 + v < nv; v += nt >> 5) {
      double t = 0.0;
      for (int q = lane; q < g; q += 32) t += fs[v * g + q];
      t = warp_sum(t);
      if (lane == 0) out[i0 + v] = t;
    }
    group_sync<NT>();
  }
}

// the na values of one grid's partials
__device__ __forceinline__ void final_sums_g(const double* partials, int G, int nv, double* out) {
  final_sums_2(partials, G, nv, nullptr, 1, 0, out);
}

__device__ __forceinline__ void final_sums(const double* partials, int nv, double* out) {
  final_sums_g(partials, (int)gridDim.x, nv, out);
}

__device__ __forceinline__ bool finite(double x) { return isfinite(x); }

// ------------------------------------------------------------------ vector and scalar helpers
//
// shared by the single-system inner kernels and the batch engine

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


// ------------------------------------------------------------------ bulk copies (TMA) and mbarriers
//
// cp.async.bulk moves a contiguous global range into shared memory on the
// copy engine and signals an mbarrier with the bytes delivered; waits are
// bounded by a clock limit so a copy that never lands turns into an error
// status instead of a hang.

constexpr long long kWaitCycles = 1ll << 31;  // about one second at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// make mbarrier initialisation visible to the copy engine
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// Programmatic dependent launch: a kernel launched behind a programmatic
// graph edge may start while its predecessor still runs; it waits here (all
// of the predecessor's blocks finished, their memory visible) before reading
// anything the predecessor writes.  Without such an edge this returns at once.
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// order this thread's earlier shared-memory accesses before later bulk copies into shared memory
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

// global -> shared bulk copy; dst, src 16-byte aligned, bytes a positive multiple of 16
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// L2 policy for data read once per pass (the matrix and V_hat): evicted
// first, so the Krylov vectors the kernels gather from and re-read stay in L2
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

// bulk copy with an L2 cache policy for its source lines
__device__ __forceinline__ void bulk_g2s_hint(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                              uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}

// One potentially blocking test of the phase: the thread may be suspended
// until the phase completes or about kSuspendNs pass (hardware wakes it on
// completion), so waiting warps do not spin through issue slots.
constexpr uint32_t kSuspendNs = 1000000;
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity), "r"(kSuspendNs)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// wait for the phase with this parity to complete; false after kWaitCycles
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > kWaitCycles) return false;
  return true;
}

// the same, giving up early once another warp of the block has raised *abort
// (and raising it itself when its own limit runs out)
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t* bar, uint32_t parity, int* abort) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (*(volatile int*)abort) return false;
    if (clock64() - t0 > kWaitCycles) {
      *(volatile int*)abort = 1;
      return false;
    }
  }
  return true;
}

}  // namespace mrcg
