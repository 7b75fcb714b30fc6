// Host-side entry points of the kernel translation units.
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"
#include "ilu.h"

namespace mrcg {

// Everything the inner-CG graph needs.  Vector pointers are device buffers of
// n_pad elements in the inner precision (double or float).
struct InnerGraphSpec {
  bool fp32 = false;
  DevState* st = nullptr;
  double* partials = nullptr;
  Sell A;
  const void* V = nullptr;     // n_pad x k, inner precision
  const void* Vbf = nullptr;   // MRCG_MIXED_BF16M: V's BF16 values (uint16 bits), n_pad x k
  int k = 0;
  const void* dinv = nullptr;  // Jacobi: 1 / diag(M_mr) (inner precision) or nullptr
  const void* dsmw = nullptr;  // MINRES-CG* M_cg: 1 / diag(A) (inner precision; dinv is then nullptr)
  const double* gram = nullptr;  // k x k  V^T M V  of the kernels' V (row-major; M = diag(dinv) or I)
  void* z = nullptr;
  void* r = nullptr;
  void* s = nullptr;
  void* p0 = nullptr;
  void* p1 = nullptr;
  void* q = nullptr;
  void* r2 = nullptr;  // second r and q buffers of the one-kernel iteration (variant 8, M_cg = I)
  void* q2 = nullptr;
  int grid_spmv = 1, grid_stream = 1, grid_stream_b = 1;
  int unroll = 4;  // CG iterations per body of the while loop (even)
  int var_a = 0;   // step-a kernel variant (0: early V loads, 1: late V loads, 2: two slices per warp,
                 // 3 / 4: late V loads with registers capped for 6 / 8 blocks per SM,
                 // 5 / 6: operands staged in shared memory by bulk copies, registers capped for
                 // 2 / 4 blocks per SM; 7: as 5 with the gathers issued one tile ahead;
                 // 8: the whole CG iteration in one staged kernel, M_cg = I only;
                 // 9 / 10: staged as 5 / 6 and 11: plain, all three with one gather per
                 // matrix entry (p explicit, beta by expansion in step a; M_cg = I or Jacobi);
                 // 12 / 13: 9 / 10 with each warp's gathers issued one tile ahead)
  IluArgs ilu;               // block-Jacobi ILU(0) M_cg (ilu.nblk > 0): step b solves with the factors
  int64_t tile_entries = 0;    // most SELL entries in one tile of 8 slices (sizes the staged variants' buffers)
  int64_t tile_entries16 = 0;  // the same for tiles of 16 slices (variants 14, 15)
  int pdl = 2;                 // programmatic edges between the inner kernels of variants 14, 15 (MRCG_PDL)
  int stages = 3;            // staged variant: shared-memory stages per block
  bool stall_test = false;   // test hook: the staged producer issues only the first tile
};

// step-a variants whose operands are staged in shared memory by bulk copies
inline bool is_staged_variant(int var) { return (var >= 5 && var <= 10) || (var >= 12 && var <= 15); }
// step-a variants 9-13: one gather per matrix entry, p kept explicit (their own step b)
inline bool is_pg_variant(int var) { return var >= 9 && var <= 15; }
// slices of a staged variant's tile (variants 14, 15: two per consumer warp)
inline int tile_slices(int var) { return var == 14 || var == 15 ? 16 : 8; }
constexpr int kNumStepAVariants = 16;

cudaError_t build_inner_graph(const InnerGraphSpec& spec, cudaGraph_t* graph);
// the same inner solve with the loop driven from the host (profiling mode)
cudaError_t run_inner_host(const InnerGraphSpec& spec, cudaStream_t stream, int* h_done);
// standalone launches of the two CG iteration kernels, timed with events:
// ms[0..1] median ms of step a, step b; ms[2..3] their means
cudaError_t time_inner_kernels(const InnerGraphSpec& spec, int iters, cudaStream_t stream, double* vin, int64_t n,
                               double* ms);
// dynamic shared memory of the staged step a for this spec (0 when it does not fit in a block)
int staged_smem_bytes(const InnerGraphSpec& spec);
// resident blocks per SM of step-a variant var_a (spec.stages for the staged one) and of step b
void inner_occupancy(const InnerGraphSpec& spec, int* spmv_blocks_per_sm, int* stream_blocks_per_sm);
// gram = V^T M_cg^{-1} V (k x k) from spec.V and spec.dinv, FP64
cudaError_t launch_gram(const InnerGraphSpec& spec, cudaStream_t stream, double* gram);

// ---- outer MINRES kernels (FP64), launched on `stream` ----
struct OuterArgs {
  DevState* st;
  double* partials;
  Sell A;
  int grid_spmv, grid_stream;
  cudaStream_t stream;
};

// y = A x (FP64 SELL)
cudaError_t launch_spmv(const OuterArgs& a, const double* x, double* y);
// out = M_mr u in FP64 or FP32 (inner precision data, rounding u to T)
cudaError_t launch_mmr(const OuterArgs& a, bool fp32, const void* val, const void* V, int k, const double* lam2,
                       const double* u, double* out, void* tmp_in, void* tmp_out);
// O.bnorm = ||b||
cudaError_t launch_bnorm(const OuterArgs& a, const double* b);
// res = b - A x ; O.rnorm2, O.relres = ||res|| / O.bnorm
cudaError_t launch_residual(const OuterArgs& a, const double* b, const double* x, double* res);
// cycle start: v_cur = res, v_prev = w_prev = w_cur = 0, cg.vin = v_cur, cg.zout = zraw
cudaError_t launch_cycle_start(const OuterArgs& a, const double* res, double* v_cur, double* v_prev, double* w_cur,
                               double* w_prev, double* zraw);
// gamma_1 = sqrt(z^T v) and the Givens state of a new cycle
cudaError_t launch_gamma_first(const OuterArgs& a, const double* zraw, const double* v);
// zn = zraw / gamma ; az = A zn ; O.delta = zn^T az
cudaError_t launch_lanczos_spmv(const OuterArgs& a, const double* zraw, double* zn, double* az);
// v_new = az - (delta/gamma) v - (gamma/gamma_old) v_old ; cg.vin = v_new ; cg.zout = zraw
cudaError_t launch_lanczos_update(const OuterArgs& a, const double* az, const double* v, const double* v_old,
                                  double* v_new, double* zraw);
// gamma_{j+1} = sqrt(z^T v_new) and the Givens rotation of step j
cudaError_t launch_gamma_givens(const OuterArgs& a, const double* zraw, const double* v_new);
// w_new = (zn - a3 w_old - a2 w) / a1 ; x += c eta w_new
cudaError_t launch_minres_update(const OuterArgs& a, const double* zn, const double* w_old, const double* w,
                                 double* w_new, double* x);
// diag(M_mr) from CSR (device arrays) into d (n entries), and 1/d in T (n_pad entries)
cudaError_t launch_mmr_diag(cudaStream_t stream, int64_t n, int64_t n_pad, const int64_t* rowptr,
                            const int32_t* colind, const double* val, const double* V64, int k, const double* lam2,
                            bool fp32, void* dinv);
// SELL construction on the device from CSR (device arrays)
cudaError_t launch_sell_fill(cudaStream_t stream, int64_t n, const int64_t* rowptr, const int32_t* colind,
                             const double* val, const int64_t* slice_ptr, int32_t* col, double* val64, float* val32);
// elementwise conversions
cudaError_t launch_to_f32(cudaStream_t stream, const double* in, float* out, int64_t n);
// col16[idx] = col[idx] - row(idx) over the SELL layout
cudaError_t launch_sell_delta16(cudaStream_t stream, int64_t n_pad, const int64_t* slice_ptr, const int32_t* col,
                                int16_t* col16);
cudaError_t launch_to_f64(cudaStream_t stream, const float* in, double* out, int64_t n);

}  // namespace mrcg
