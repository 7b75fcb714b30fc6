// C ABI of the MINRES-CG solver: handle setup (SELL conversion, validation,
// graph instantiation) and the host driver of the outer MINRES loop.
//
// The host takes part once per outer MINRES step: it launches the step's
// kernels and the inner-CG graph, then reads back a ~1 KB state block (true
// residual, status, Givens gamma) to apply the stopping and restart rules.
// The inner CG loop itself runs entirely on the device.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <initializer_list>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "mrcg.h"
#include "trace.h"

using namespace mrcg;

struct mrcg_solver {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int64_t n = 0, n_pad = 0, nnz = 0;
  int k = 0;
  bool fp32 = false;
  int mcg = MRCG_MCG_IDENTITY;
  int max_outer = 200;
  double restart_factor = 0.5;
  double lam2[kMaxK] = {};

  Sell A;
  int64_t* d_slice_ptr = nullptr;
  int32_t* d_col = nullptr;
  double* d_val64 = nullptr;
  float* d_val32 = nullptr;
  double* d_V64 = nullptr;
  float* d_V32 = nullptr;
  uint16_t* d_Vbf = nullptr;  // MRCG_MIXED_BF16M: V_hat's BF16 values (the bits of d_V32's upper halves)
  bool bf16v = false;
  void* d_dinv = nullptr;
  void* d_dsmw = nullptr;    // MINRES-CG* M_cg: 1 / diag(A) in the inner precision
  double* d_gram = nullptr;  // k x k V^T M_cg^{-1} V of the inner kernels' V
  DevState* d_st = nullptr;
  DevState* h_st = nullptr;    // pinned mirror (read back)
  DevState* h_init = nullptr;  // pinned staging (upload)
  double* d_partials = nullptr;

  // FP64 vectors of the outer iteration (n_pad each)
  double *x = nullptr, *b = nullptr, *res = nullptr, *zraw = nullptr, *zn = nullptr;
  double* v[2] = {nullptr, nullptr};
  double* w[2] = {nullptr, nullptr};
  // inner-precision vectors
  void *iz = nullptr, *ir = nullptr, *is = nullptr, *ip0 = nullptr, *ip1 = nullptr, *iq = nullptr;
  void *ir2 = nullptr, *iq2 = nullptr;  // one-kernel iteration (M_cg = I): second r and q buffers
  int64_t ilu_levels = 0;              // ILU(0) M_cg: forward + backward levels over all blocks

  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  int grid_spmv = 1, grid_stream = 1, grid_stream_b = 1, unroll = 4;
  bool host_loop = false;  // MRCG_INNER_LOOP=host: inner loop driven from the host (for profilers)
  OuterArgs oargs;
  InnerGraphSpec spec;
  std::vector<void*> allocations;
};

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

#define CK(call)                                                                                 \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess) {                                                                     \
      if (getenv("MRCG_DEBUG")) fprintf(stderr, "mrcg: %s failed: %s (%s:%d)\n", #call,          \
                                        cudaGetErrorString(e_), __FILE__, __LINE__);             \
      return e_ == cudaErrorMemoryAllocation ? MRCG_ERR_OOM : MRCG_ERR_CUDA;                     \
    }                                                                                            \
  } while (0)

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

template <typename T>
mrcg_status dalloc(mrcg_solver* h, T** p, size_t count) {
  // exact sizes: every kernel stays inside n_pad rows / the SELL arrays, and a
  // guard tail would push a vector of a whole number of 2 MiB pages onto one
  // more page (an empty array still gets a small allocation of its own)
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, std::max<size_t>(count * sizeof(T), 256));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return MRCG_ERR_OOM;
  }
  h->allocations.push_back(q);
  *p = reinterpret_cast<T*>(q);
  return MRCG_OK;
}

// copy `count` elements from a host or device array into a host vector
template <typename T>
mrcg_status fetch(const T* src, size_t count, std::vector<T>& dst) {
  dst.resize(count);
  if (count == 0) return MRCG_OK;
  if (is_device_ptr(src)) {
    CK(cudaMemcpy(dst.data(), src, count * sizeof(T), cudaMemcpyDeviceToHost));
  } else {
    std::memcpy(dst.data(), src, count * sizeof(T));
  }
  return MRCG_OK;
}

// copy n doubles between a user array (host or device) and a device buffer
mrcg_status stage_in(mrcg_solver* h, const double* user, double* dev) {
  const cudaMemcpyKind kind = is_device_ptr(user) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CK(cudaMemcpyAsync(dev, user, (size_t)h->n * sizeof(double), kind, h->stream));
  return MRCG_OK;
}

mrcg_status stage_out(mrcg_solver* h, const double* dev, double* user) {
  const cudaMemcpyKind kind = is_device_ptr(user) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  CK(cudaMemcpyAsync(user, dev, (size_t)h->n * sizeof(double), kind, h->stream));
  return MRCG_OK;
}

void reset_state(mrcg_solver* h, double inner_tol, long long budget) {
  DevState& s = *h->h_init;
  std::memset(&s, 0, sizeof(DevState));
  for (int l = 0; l < kMaxK; ++l) s.cg.lam2[l] = h->lam2[l];
  s.cg.inner_tol = inner_tol;
  s.cg.budget = budget;
  s.cg.ctl_limit = 2;
  s.cg.unroll = h->unroll;
  s.out.status = MRCG_OK;
}

mrcg_status upload_state(mrcg_solver* h) {
  CK(cudaMemcpyAsync(h->d_st, h->h_init, sizeof(DevState), cudaMemcpyHostToDevice, h->stream));
  return MRCG_OK;
}

mrcg_status read_state(mrcg_solver* h) {
  CK(cudaMemcpyAsync(h->h_st, h->d_st, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return MRCG_OK;
}

mrcg_status lerr(cudaError_t e) {
  if (e == cudaSuccess) return MRCG_OK;
  if (getenv("MRCG_DEBUG")) fprintf(stderr, "mrcg: launch failed: %s\n", cudaGetErrorString(e));
  return MRCG_ERR_CUDA;
}

#define LK(call)                          \
  do {                                    \
    mrcg_status s_ = lerr(call);          \
    if (s_ != MRCG_OK) return s_;         \
  } while (0)

#define ST(call)                          \
  do {                                    \
    mrcg_status s_ = (call);              \
    if (s_ != MRCG_OK) return s_;         \
  } while (0)

mrcg_status validate_subspace(const mrcg_create_args* a, const std::vector<int64_t>& rp,
                              const std::vector<int32_t>& ci, const std::vector<double>& va,
                              const std::vector<double>& V, const std::vector<double>& lam) {
  const int64_t n = a->n;
  const int k = a->k;
  // Gram matrix V^T V ~ I
  for (int i = 0; i < k; ++i)
    for (int j = 0; j <= i; ++j) {
      double g = 0.0;
      const double* vi = V.data() + (size_t)i * n;
      const double* vj = V.data() + (size_t)j * n;
      for (int64_t r = 0; r < n; ++r) g += vi[r] * vj[r];
      if (std::fabs(g - (i == j ? 1.0 : 0.0)) > 1e-10) return MRCG_ERR_INVALID;
    }
  // ||A V - V Lambda||_F <= 1e-8 ||A||_F sqrt(k)
  double anorm2 = 0.0;
  for (double x : va) anorm2 += x * x;
  double res2 = 0.0;
  for (int j = 0; j < k; ++j) {
    const double* vj = V.data() + (size_t)j * n;
    for (int64_t r = 0; r < n; ++r) {
      double s = 0.0;
      for (int64_t p = rp[r]; p < rp[r + 1]; ++p) s += va[p] * vj[ci[p]];
      const double d = s - lam[j] * vj[r];
      res2 += d * d;
    }
  }
  if (!(std::sqrt(res2) <= 1e-8 * std::sqrt(anorm2) * std::sqrt((double)k))) return MRCG_ERR_INVALID;
  return MRCG_OK;
}

// BF16 of a finite FP32 value: its upper 16 bits after rounding the lower 16
// to nearest, ties to even (BF16 is FP32 with a 7-bit fraction)
inline uint16_t float_to_bf16_bits(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u += 0x7fffu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}
inline float bf16_bits_to_float(uint16_t b) {
  const uint32_t u = (uint32_t)b << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

mrcg_status create_impl(const mrcg_create_args* a, mrcg_solver* h) {
  const int64_t n = a->n;
  h->n = n;
  h->nnz = a->nnz;
  h->k = a->k;
  h->fp32 = a->precision == MRCG_MIXED_FP32 || a->precision == MRCG_MIXED_BF16M;
  h->bf16v = a->precision == MRCG_MIXED_BF16M;
  h->mcg = a->inner_prec;
  h->max_outer = a->max_outer > 0 ? a->max_outer : 200;
  h->restart_factor = a->restart_factor == 0.0 ? 0.5 : a->restart_factor;
  const int64_t nslices = (n + kSlice - 1) / kSlice;
  const int64_t n_pad = nslices * kSlice;
  h->n_pad = n_pad;

  if (a->stream) {
    h->stream = (cudaStream_t)a->stream;
  } else {
    CK(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    h->own_stream = true;
  }

  // ---- host copies and validation of the CSR input
  std::vector<int64_t> rp;
  std::vector<int32_t> ci;
  std::vector<double> va, V, lam;
  ST(fetch(a->rowptr, (size_t)n + 1, rp));
  if (rp[0] != 0 || rp[n] != a->nnz) return MRCG_ERR_INVALID;
  for (int64_t i = 0; i < n; ++i)
    if (rp[i + 1] < rp[i]) return MRCG_ERR_INVALID;
  ST(fetch(a->colind, (size_t)a->nnz, ci));
  ST(fetch(a->val, (size_t)a->nnz, va));
  for (int64_t i = 0; i < n; ++i)
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      if (ci[p] < 0 || ci[p] >= n) return MRCG_ERR_INVALID;
      if (p > rp[i] && ci[p] <= ci[p - 1]) return MRCG_ERR_INVALID;
      if (!std::isfinite(va[p])) return MRCG_ERR_NONFINITE;
    }
  ST(fetch(a->lambda, (size_t)a->k, lam));
  ST(fetch(a->V, (size_t)n * a->k, V));
  for (int j = 0; j < a->k; ++j) {
    if (!(lam[j] < 0.0) || !std::isfinite(lam[j])) return MRCG_ERR_INVALID;
    h->lam2[j] = 2.0 * std::fabs(lam[j]);
  }
  for (double x : V)
    if (!std::isfinite(x)) return MRCG_ERR_NONFINITE;
  if (a->validate && a->k > 0) ST(validate_subspace(a, rp, ci, va, V, lam));
  // MRCG_MIXED_BF16M: V_hat rounded to BF16 (after the validation of the given
  // pairs), so that every kernel, the Jacobi diagonal and MINRES-CG*'s terms
  // all use one V_hat
  if (h->bf16v)
    for (double& x : V) x = (double)bf16_bits_to_float(float_to_bf16_bits((float)x));
  // MINRES-CG* M_cg: Atilde = diag(A) of Sec. 2.1, every diagonal entry nonzero
  std::vector<double> dd;
  if (h->mcg == MRCG_MCG_SMW) {
    dd.assign((size_t)n_pad, 0.0);
    for (int64_t i = 0; i < n; ++i) {
      double d = 0.0;
      for (int64_t p = rp[i]; p < rp[i + 1]; ++p)
        if (ci[p] == i) d += va[p];
      if (d == 0.0 || !std::isfinite(d)) return MRCG_ERR_INVALID;
      dd[i] = 1.0 / d;
    }
  }

  // ---- SELL-32 layout
  std::vector<int64_t> sp((size_t)nslices + 1, 0);
  for (int64_t s = 0; s < nslices; ++s) {
    int64_t w = 0;
    for (int64_t r = s * kSlice; r < std::min<int64_t>(n, (s + 1) * kSlice); ++r) w = std::max(w, rp[r + 1] - rp[r]);
    sp[s + 1] = sp[s] + w * kSlice;
  }
  const int64_t total = sp[nslices];
  ST(dalloc(h, &h->d_slice_ptr, (size_t)nslices + 1));
  ST(dalloc(h, &h->d_col, (size_t)total));
  ST(dalloc(h, &h->d_val64, (size_t)total));
  if (h->fp32) ST(dalloc(h, &h->d_val32, (size_t)total));
  CK(cudaMemcpyAsync(h->d_slice_ptr, sp.data(), sp.size() * sizeof(int64_t), cudaMemcpyHostToDevice, h->stream));

  int64_t* t_rp = nullptr;
  int32_t* t_ci = nullptr;
  double* t_va = nullptr;
  CK(cudaMalloc(&t_rp, rp.size() * sizeof(int64_t)));
  CK(cudaMalloc(&t_ci, (ci.size() + 1) * sizeof(int32_t)));
  CK(cudaMalloc(&t_va, (va.size() + 1) * sizeof(double)));
  CK(cudaMemcpyAsync(t_rp, rp.data(), rp.size() * sizeof(int64_t), cudaMemcpyHostToDevice, h->stream));
  if (!ci.empty()) {
    CK(cudaMemcpyAsync(t_ci, ci.data(), ci.size() * sizeof(int32_t), cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(t_va, va.data(), va.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  }
  LK(launch_sell_fill(h->stream, n, t_rp, t_ci, t_va, h->d_slice_ptr, h->d_col, h->d_val64, h->d_val32));

  h->A.n = n;
  h->A.n_pad = n_pad;
  h->A.nslices = nslices;
  h->A.total = total;
  h->A.slice_ptr = h->d_slice_ptr;
  h->A.col = h->d_col;
  h->A.val64 = h->d_val64;
  h->A.val32 = h->d_val32;
  // 16-bit column deltas for the inner kernels when every |col - row| fits
  {
    int64_t dmax = 0;
    for (int64_t i = 0; i < n; ++i)
      for (int64_t p = rp[i]; p < rp[i + 1]; ++p) dmax = std::max<int64_t>(dmax, std::llabs((int64_t)ci[p] - i));
    const char* e = getenv("MRCG_IDX16");
    if (dmax <= 32767 && !(e && atoi(e) == 0)) {
      int16_t* c16 = nullptr;
      ST(dalloc(h, &c16, (size_t)total + 1));
      LK(launch_sell_delta16(h->stream, n_pad, h->d_slice_ptr, h->d_col, c16));
      h->A.col16 = c16;
    }
  }

  // ---- V_hat (n_pad rows, zero padded) and its FP32 copy
  const size_t vcount = (size_t)n_pad * (a->k > 0 ? a->k : 1);
  ST(dalloc(h, &h->d_V64, vcount));
  CK(cudaMemsetAsync(h->d_V64, 0, vcount * sizeof(double), h->stream));
  for (int j = 0; j < a->k; ++j)
    CK(cudaMemcpyAsync(h->d_V64 + (size_t)j * n_pad, V.data() + (size_t)j * n, (size_t)n * sizeof(double),
                       cudaMemcpyHostToDevice, h->stream));
  if (h->fp32) {
    ST(dalloc(h, &h->d_V32, vcount));
    LK(launch_to_f32(h->stream, h->d_V64, h->d_V32, (int64_t)vcount));
  }
  if (h->bf16v && a->k > 0) {
    std::vector<uint16_t> vb(vcount, 0);
    for (int j = 0; j < a->k; ++j)
      for (int64_t i = 0; i < n; ++i)
        vb[(size_t)j * n_pad + i] = float_to_bf16_bits((float)V[(size_t)j * n + i]);
    ST(dalloc(h, &h->d_Vbf, vcount));
    CK(cudaMemcpyAsync(h->d_Vbf, vb.data(), vcount * sizeof(uint16_t), cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));  // vb goes out of scope
  }

  // ---- vectors
  double** f64[] = {&h->x, &h->b, &h->res, &h->zraw, &h->zn, &h->v[0], &h->v[1], &h->w[0], &h->w[1]};
  for (double** p : f64) {
    ST(dalloc(h, p, (size_t)n_pad));
    CK(cudaMemsetAsync(*p, 0, (size_t)n_pad * sizeof(double), h->stream));
  }
  const size_t esz = h->fp32 ? sizeof(float) : sizeof(double);
  void** inner[] = {&h->iz, &h->ir, &h->is, &h->ip0, &h->ip1, &h->iq, &h->ir2, &h->iq2};
  for (void** p : inner) {
    if (p == &h->is && h->mcg == MRCG_MCG_IDENTITY) continue;
    if ((p == &h->ir2 || p == &h->iq2) && h->mcg != MRCG_MCG_IDENTITY) continue;
    char* q = nullptr;
    ST(dalloc(h, &q, (size_t)n_pad * esz));
    CK(cudaMemsetAsync(q, 0, (size_t)n_pad * esz, h->stream));
    *p = q;
  }
  ST(dalloc(h, &h->d_partials, (size_t)(2 * kMaxNV + 2) * kMaxBlocks));  // one-gather family: two parities + step b
  ST(dalloc(h, &h->d_st, 1));
  CK(cudaMemsetAsync(h->d_st, 0, sizeof(DevState), h->stream));
  CK(cudaMallocHost(&h->h_st, sizeof(DevState)));
  CK(cudaMallocHost(&h->h_init, sizeof(DevState)));
  std::memset(h->h_st, 0, sizeof(DevState));

  if (h->mcg == MRCG_MCG_JACOBI) {
    double* d_lam2 = nullptr;
    CK(cudaMalloc(&d_lam2, kMaxK * sizeof(double)));
    CK(cudaMemcpyAsync(d_lam2, h->lam2, kMaxK * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    char* q = nullptr;
    ST(dalloc(h, &q, (size_t)n_pad * esz));
    h->d_dinv = q;
    LK(launch_mmr_diag(h->stream, n, n_pad, t_rp, t_ci, t_va, h->d_V64, a->k, d_lam2, h->fp32, h->d_dinv));
    CK(cudaStreamSynchronize(h->stream));
    cudaFree(d_lam2);
  }
  if (h->mcg == MRCG_MCG_SMW) {
    double* d64 = nullptr;
    CK(cudaMalloc(&d64, dd.size() * sizeof(double)));
    CK(cudaMemcpyAsync(d64, dd.data(), dd.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    char* q = nullptr;
    ST(dalloc(h, &q, (size_t)n_pad * esz));
    if (h->fp32) LK(launch_to_f32(h->stream, d64, reinterpret_cast<float*>(q), n_pad));
    else CK(cudaMemcpyAsync(q, d64, dd.size() * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    cudaFree(d64);
    h->d_dsmw = q;
  }
  // ---- block-Jacobi ILU(0) M_cg: host factorisation with level scheduling, device copy
  IluArgs ilu;
  if (h->mcg == MRCG_MCG_ILU0 || h->mcg == MRCG_MCG_SMW_ILU0) {
    const int cap = h->fp32 ? kIluMaxBlock : kIluMaxBlock / 2;  // a block's values in shared memory
    int bs = a->ilu_block > 0 ? a->ilu_block : 1024;  // 1024: 8 x-lines of a 128^3 grid, fastest per solve measured
    if (bs % 32 != 0 || bs > cap) return MRCG_ERR_INVALID;
    bs = (int)std::min<int64_t>(bs, n_pad);
    IluHost fh;
    ST(ilu0_build(n, n_pad, rp, ci, va, bs, fh));
    if (fh.fent.back() < 0 || fh.bent.back() < 0) return MRCG_ERR_INVALID;  // entry offsets beyond int32
    auto up_i32 = [&](const std::vector<int32_t>& v, const int32_t** dst) -> mrcg_status {
      int32_t* d = nullptr;
      ST(dalloc(h, &d, v.size()));
      CK(cudaMemcpyAsync(d, v.data(), v.size() * sizeof(int32_t), cudaMemcpyHostToDevice, h->stream));
      *dst = d;
      return MRCG_OK;
    };
    auto up_u16 = [&](const std::vector<uint16_t>& v, const uint16_t** dst) -> mrcg_status {
      uint16_t* d = nullptr;
      ST(dalloc(h, &d, v.size()));
      if (!v.empty()) CK(cudaMemcpyAsync(d, v.data(), v.size() * sizeof(uint16_t), cudaMemcpyHostToDevice, h->stream));
      *dst = d;
      return MRCG_OK;
    };
    auto up_val = [&](const std::vector<double>& v, const void** dst) -> mrcg_status {
      if (h->fp32) {
        std::vector<float> f(v.begin(), v.end());
        float* d = nullptr;
        ST(dalloc(h, &d, f.size()));
        if (!f.empty()) CK(cudaMemcpyAsync(d, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice, h->stream));
        CK(cudaStreamSynchronize(h->stream));  // f is a temporary
        *dst = d;
      } else {
        double* d = nullptr;
        ST(dalloc(h, &d, v.size()));
        if (!v.empty()) CK(cudaMemcpyAsync(d, v.data(), v.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        *dst = d;
      }
      return MRCG_OK;
    };
    ST(up_i32(fh.fblk, &ilu.fblk));
    ST(up_i32(fh.flvl, &ilu.flvl));
    ST(up_i32(fh.frow, &ilu.frow));
    ST(up_i32(fh.fent, &ilu.fent));
    ST(up_u16(fh.fcol, &ilu.fcol));
    ST(up_val(fh.fval, &ilu.fval));
    ST(up_i32(fh.bblk, &ilu.bblk));
    ST(up_i32(fh.blvl, &ilu.blvl));
    ST(up_i32(fh.brow, &ilu.brow));
    ST(up_i32(fh.bent, &ilu.bent));
    ST(up_u16(fh.bcol, &ilu.bcol));
    ST(up_val(fh.bval, &ilu.bval));
    ST(up_val(fh.bdinv, &ilu.bdinv));
    CK(cudaStreamSynchronize(h->stream));  // the host vectors go out of scope
    ilu.nblk = fh.nblk;
    ilu.bs = fh.bs;
    const size_t esz = h->fp32 ? sizeof(float) : sizeof(double);
    size_t per_warp = (size_t)bs * esz;  // the block's values
    // staged sweeps (FP32): each block's sweep data as one image a warp copies
    // into shared memory next to its values, when an image of every block
    // fits beside them (MRCG_ILU_STAGE=0: off, 1: also in FP64).  In FP64 the
    // images are twice the size and the lost occupancy outweighed the shorter
    // sweeps (measured at 128^3, blocks of 1024 and 2048 rows)
    const char* stg = getenv("MRCG_ILU_STAGE");
    if (stg ? atoi(stg) != 0 : h->fp32) {
      std::vector<unsigned char> img;
      std::vector<int64_t> img_off;
      int img_max = 0;
      if (ilu0_images(fh, esz, img, img_off, &img_max) && per_warp + (size_t)img_max <= (size_t)200 * 1024) {
        unsigned char* d_img = nullptr;
        int64_t* d_off = nullptr;
        ST(dalloc(h, &d_img, img.size()));
        ST(dalloc(h, &d_off, img_off.size()));
        CK(cudaMemcpyAsync(d_img, img.data(), img.size(), cudaMemcpyHostToDevice, h->stream));
        CK(cudaMemcpyAsync(d_off, img_off.data(), img_off.size() * sizeof(int64_t), cudaMemcpyHostToDevice,
                           h->stream));
        CK(cudaStreamSynchronize(h->stream));  // the host vectors go out of scope
        ilu.img = d_img;
        ilu.img_off = d_off;
        ilu.img_bytes = img_max;
        per_warp += (size_t)img_max;
      }
    }
    // blocks (warps) per CTA: two CTAs' worth of shared memory fit an SM
    ilu.wpc = (int)std::max<size_t>(1, std::min<size_t>(kThreads / 32, (size_t)(110 * 1024) / per_warp));
    ilu.smw = h->mcg == MRCG_MCG_SMW_ILU0 ? 1 : 0;
    h->ilu_levels = fh.levels_f + fh.levels_b;
  }
  CK(cudaStreamSynchronize(h->stream));
  cudaFree(t_rp);
  cudaFree(t_ci);
  cudaFree(t_va);

  // ---- launch geometry
  int nsm = 1;
  CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device));
  const int vec_w = h->fp32 ? 4 : 2;  // elements per 16-byte access in step b
  const int64_t want_spmv = (nslices + kThreads / 32 - 1) / (kThreads / 32);
  const int64_t want_stream = (n_pad + kThreads - 1) / kThreads;
  const int64_t want_b = (n_pad / vec_w + kThreads - 1) / kThreads;
  auto clamp_grid = [&](int64_t want, int bp) {
    return (int)std::max<int64_t>(1, std::min<int64_t>({want, (int64_t)nsm * std::max(1, bp), kMaxBlocks}));
  };
  // outer FP64 kernels: four resident 256-thread blocks per SM
  h->grid_spmv = clamp_grid(want_spmv, 4);
  h->grid_stream = clamp_grid(want_stream, 4);
  if (const char* u = getenv("MRCG_UNROLL")) h->unroll = std::max(2, atoi(u) & ~1);
  if (const char* m = getenv("MRCG_INNER_LOOP")) h->host_loop = std::strcmp(m, "host") == 0;

  h->oargs.st = h->d_st;
  h->oargs.partials = h->d_partials;
  h->oargs.A = h->A;
  h->oargs.grid_spmv = h->grid_spmv;
  h->oargs.grid_stream = h->grid_stream;
  h->oargs.stream = h->stream;

  // ---- inner CG graph
  InnerGraphSpec g;
  g.fp32 = h->fp32;
  g.st = h->d_st;
  g.partials = h->d_partials;
  g.A = h->A;
  g.V = h->fp32 ? (const void*)h->d_V32 : (const void*)h->d_V64;
  g.Vbf = h->d_Vbf;
  g.k = a->k;
  g.dinv = h->d_dinv;
  g.dsmw = h->d_dsmw;
  g.ilu = ilu;
  if (a->k > 0) {
    ST(dalloc(h, &h->d_gram, (size_t)a->k * a->k));
    CK(launch_gram(g, h->stream, h->d_gram));
  }
  g.gram = h->d_gram;
  g.z = h->iz;
  g.r = h->ir;
  g.s = h->is;
  g.p0 = h->ip0;
  g.p1 = h->ip1;
  g.q = h->iq;
  g.r2 = h->ir2;
  g.q2 = h->iq2;
  g.grid_stream = h->grid_stream;
  g.unroll = h->unroll;
  // failure-detection test hook: the staged step a stops issuing its copies
  // after the first tile, so its bounded waits run out and the solve reports
  // MRCG_ERR_CUDA (the GPU context stays usable)
  if (const char* e = getenv("MRCG_TEST_STALL")) g.stall_test = atoi(e) != 0;
  if (const char* e = getenv("MRCG_PDL")) g.pdl = std::max(0, std::min(3, atoi(e)));
  // SELL entries of the largest tile of 8 (16) slices (the staged step a's buffers)
  for (int64_t s0 = 0; s0 < nslices; s0 += 8) g.tile_entries = std::max(g.tile_entries, sp[std::min(s0 + 8, nslices)] - sp[s0]);
  for (int64_t s0 = 0; s0 < nslices; s0 += 16)
    g.tile_entries16 = std::max(g.tile_entries16, sp[std::min(s0 + 16, nslices)] - sp[s0]);
  if (const char* e = getenv("MRCG_STAGES")) g.stages = std::max(2, std::min(8, atoi(e)));
  const int64_t ntiles = (nslices + 7) / 8, ntiles16 = (nslices + 15) / 16;
  // step-a grid of a variant at bp blocks per SM (the staged variants are persistent over tiles)
  auto grid_a = [&](const InnerGraphSpec& t, int bp) {
    if (!is_staged_variant(t.var_a)) return clamp_grid(want_spmv, bp);
    return clamp_grid(tile_slices(t.var_a) == 16 ? ntiles16 : ntiles, bp);
  };
  if (const char* va = getenv("MRCG_VAR_A")) g.var_a = std::min(kNumStepAVariants - 1, std::max(0, atoi(va)));
  int occ_a = 1, occ_b = 1;
  inner_occupancy(g, &occ_a, &occ_b);
  if (occ_a < 1) {  // the staged variant does not fit this matrix
    g.var_a = 0;
    inner_occupancy(g, &occ_a, &occ_b);
  }
  occ_a = std::max(1, occ_a);
  occ_b = std::max(1, occ_b);
  // blocks per SM of the two CG kernels: the occupancy limit, optionally
  // capped (MRCG_BPSM_A / MRCG_BPSM_B) for launch-shape sweeps
  if (const char* e = getenv("MRCG_BPSM_A")) occ_a = std::max(1, std::min(occ_a, atoi(e)));
  if (const char* e = getenv("MRCG_BPSM_B")) occ_b = std::max(1, std::min(occ_b, atoi(e)));
  g.grid_spmv = grid_a(g, occ_a);
  g.grid_stream_b = clamp_grid(want_b, occ_b);
  // MRCG_SHAPE_F32 / MRCG_SHAPE_F64 = "variant,stages,grid_a,grid_b" replays a
  // shape a previous run reported (mrcg_launch_config), e.g. under a profiler,
  // whose slowed launches would mislead the timing below
  const char* fixed = getenv(h->fp32 ? "MRCG_SHAPE_F32" : "MRCG_SHAPE_F64");
  if (fixed) {
    int v = 0, nst = 0, ga = 0, gb = 0;
    if (sscanf(fixed, "%d,%d,%d,%d", &v, &nst, &ga, &gb) == 4 && v >= 0 && v < kNumStepAVariants && ga >= 1 && gb >= 1 &&
        ga <= kMaxBlocks && gb <= kMaxBlocks) {
      InnerGraphSpec t = g;
      t.var_a = v;
      if (is_staged_variant(v)) t.stages = std::max(2, std::min(8, nst));
      int occ_t = 0, occ_unused = 0;
      inner_occupancy(t, &occ_t, &occ_unused);
      if (occ_t >= 1) {
        g = t;
        g.grid_spmv = ga;
        g.grid_stream_b = gb;
      }
    }
  }
  // ---- launch-shape autotuner: step-a variant (and stages) with its blocks
  // per SM, then step-b blocks per SM, then the one-kernel iteration against
  // the best pair, timed on this matrix (standalone launches, medians of a few
  // iterations)
  const char* at = getenv("MRCG_AUTOTUNE");
  const bool tune = (!at || atoi(at) != 0) && n_pad >= (1 << 12) && !getenv("MRCG_BPSM_A") &&
                    !getenv("MRCG_BPSM_B") && !getenv("MRCG_VAR_A") && !fixed;
  if (tune) {
    double ms[4] = {0.0, 0.0, 0.0, 0.0};
    auto time_spec = [&](const InnerGraphSpec& t) -> mrcg_status {
      reset_state(h, 1e-300, 64);
      h->h_init->cg.vin = h->v[0];
      h->h_init->cg.zout = h->zraw;
      ST(upload_state(h));
      CK(time_inner_kernels(t, 15, h->stream, h->v[0], n, ms));
      return MRCG_OK;
    };
    // one family of step-a variants sharing a step b: the best step a (variant,
    // stages, blocks per SM), then the best step-b blocks per SM for it;
    // returns the time of a whole iteration (1e30 when none fits)
    auto tune_family = [&](std::initializer_list<int> vars, InnerGraphSpec* out, double* total) -> mrcg_status {
      double best = 1e30;
      InnerGraphSpec bestg = g;
      bool any = false;
      for (int var : vars) {
        for (int nst = 2; nst <= (is_staged_variant(var) ? 4 : 2); ++nst) {
          InnerGraphSpec t = g;
          t.var_a = var;
          t.stages = is_staged_variant(var) ? nst : g.stages;
          int occ_v = 0, occ_unused = 0;
          inner_occupancy(t, &occ_v, &occ_unused);
          if (occ_v < 1) continue;
          // blocks per SM: the occupancy limit and one below; the staged kernels
          // (no waits between blocks) also one wave of blocks above it and two
          std::vector<int> bps = {occ_v};
          if (occ_v > 1) bps.push_back(occ_v - 1);
          if (is_staged_variant(var)) {
            bps.push_back(occ_v + 1);
            bps.push_back(2 * occ_v);
          }
          // grids: bp blocks per SM, and for the staged kernels the smallest grid
          // with the same tiles per block (every block then takes as many
          // tiles, none idles while the last ones finish)
          std::vector<int> grids;
          for (int bp : bps) {
            const int gr = grid_a(t, bp);
            grids.push_back(gr);
            if (is_staged_variant(var)) {
              const int64_t tiles = tile_slices(var) == 16 ? ntiles16 : ntiles;
              const int64_t per = (tiles + gr - 1) / gr;
              const int bal = (int)((tiles + per - 1) / per);
              if (bal != gr) grids.push_back(bal);
            }
          }
          for (int gr : grids) {
            t.grid_spmv = gr;
            ST(time_spec(t));
            if (ms[0] < best) {
              best = ms[0];
              bestg = t;
              any = true;
            }
          }
        }
      }
      *total = 1e30;
      if (!any) return MRCG_OK;
      const double best_a = best;
      best = 1e30;
      int occ_unused = 0, occ_bmax = 1;
      inner_occupancy(bestg, &occ_unused, &occ_bmax);
      for (int bp = 1; bp <= std::max(1, occ_bmax); bp += (bp < 4 ? 1 : 2)) {
        InnerGraphSpec t = bestg;
        t.grid_stream_b = clamp_grid(want_b, bp);
        ST(time_spec(t));
        if (ms[1] < best) {
          best = ms[1];
          bestg.grid_stream_b = t.grid_stream_b;
        }
      }
      *out = bestg;
      *total = best_a + best;
      return MRCG_OK;
    };
    InnerGraphSpec classic = g, onegather = g;
    double t_classic = 1e30, t_onegather = 1e30;
    ST(tune_family({0, 1, 2, 3, 4, 5, 6, 7}, &classic, &t_classic));
    ST(tune_family({9, 10, 11, 12, 13, 14, 15}, &onegather, &t_onegather));
    InnerGraphSpec bestg = t_onegather < t_classic ? onegather : classic;
    const double best_pair = std::min(t_classic, t_onegather);
    // the one-kernel iteration (variant 8, M_cg = I) competes with the best
    // step a + step b pair on the time of a whole iteration
    double best8 = 1e30;
    InnerGraphSpec best8g = bestg;
    for (int nst = 2; nst <= 3; ++nst) {
      InnerGraphSpec t = g;
      t.var_a = 8;
      t.stages = nst;
      int occ_v = 0, occ_unused = 0;
      inner_occupancy(t, &occ_v, &occ_unused);
      if (occ_v < 1) continue;
      for (int bp : {occ_v, occ_v + 1}) {
        t.grid_spmv = grid_a(t, bp);
        ST(time_spec(t));
        if (ms[0] < best8) {
          best8 = ms[0];
          best8g = t;
          best8g.grid_stream_b = bestg.grid_stream_b;
        }
      }
    }
    // standalone launches time the pair without the overlap it gets inside the
    // graph (about 10 % at 128^3), so the one-kernel iteration must win by more
    g = best8 < 0.9 * best_pair ? best8g : bestg;
    if (getenv("MRCG_DEBUG"))
      fprintf(stderr, "mrcg autotune: two-gather pair %.4f ms, one-gather pair %.4f ms, one-kernel %.4f ms\n",
              t_classic, t_onegather, best8);
    if (getenv("MRCG_DEBUG"))
      fprintf(stderr, "mrcg autotune: var_a=%d stages=%d grid_a=%d grid_b=%d\n", g.var_a, g.stages, g.grid_spmv,
              g.grid_stream_b);
  }
  h->grid_stream_b = g.grid_stream_b;
  h->spec = g;
  CK(build_inner_graph(g, &h->graph));
  CK(cudaGraphInstantiate(&h->graph_exec, h->graph, 0));
  CK(cudaStreamSynchronize(h->stream));
  return MRCG_OK;
}

void destroy_impl(mrcg_solver* h) {
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
  if (h->graph) cudaGraphDestroy(h->graph);
  for (void* p : h->allocations) cudaFree(p);
  if (h->h_st) cudaFreeHost(h->h_st);
  if (h->h_init) cudaFreeHost(h->h_init);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  cudaGetLastError();
  delete h;
}

// run the inner-CG graph once (zout = P(vin), pointers already in the state)
mrcg_status run_inner(mrcg_solver* h) {
  TraceRange tr("mrcg inner CG");
  if (h->host_loop) {
    CK(run_inner_host(h->spec, h->stream, &h->h_st->cg.done));
    return MRCG_OK;
  }
  CK(cudaGraphLaunch(h->graph_exec, h->stream));
  return MRCG_OK;
}

mrcg_status solve_impl(mrcg_solver* h, const double* ub, double* ux, double outer_tol, double inner_tol,
                       int64_t max_iters, mrcg_info* info) {
  TraceRange tr("mrcg_solve");
  const long long budget = max_iters > 0 ? (long long)max_iters : (1LL << 31);
  long long launches = 0, graphs = 0;
#define LKC(call)  \
  do {             \
    ++launches;    \
    LK(call);      \
  } while (0)
  ST(stage_in(h, ub, h->b));
  ST(stage_in(h, ux, h->x));
  reset_state(h, inner_tol, budget);
  ST(upload_state(h));
  LKC(launch_bnorm(h->oargs, h->b));
  LKC(launch_residual(h->oargs, h->b, h->x, h->res));
  ST(read_state(h));
  const OuterState& O = h->h_st->out;

  int32_t outer = 0, restarts = 0, hist_len = 0;
  mrcg_status status = MRCG_ERR_MAXITER;
  double relres = O.relres;
  auto record = [&](double rr) {
    if (info && info->relres_history && hist_len < info->history_cap) info->relres_history[hist_len] = rr;
    ++hist_len;
  };

  if (O.status != MRCG_OK || !std::isfinite(O.bnorm)) {
    status = MRCG_ERR_NONFINITE;
  } else if (O.bnorm == 0.0) {
    CK(cudaMemsetAsync(h->x, 0, (size_t)h->n_pad * sizeof(double), h->stream));
    relres = 0.0;
    status = MRCG_OK;
  } else if (relres <= outer_tol) {
    status = MRCG_OK;
  } else {
    int cur = 0;   // v[cur] = v_j, v[cur^1] = v_{j-1}; same for w
    bool finished = false;
    while (!finished) {
      // ---- new cycle from the current residual
      LKC(launch_cycle_start(h->oargs, h->res, h->v[cur], h->v[cur ^ 1], h->w[cur], h->w[cur ^ 1], h->zraw));
      ST(run_inner(h)); graphs += 1;
      LKC(launch_gamma_first(h->oargs, h->zraw, h->v[cur]));
      std::vector<double> cyc;
      for (;;) {
        if (outer >= h->max_outer) {
          ST(read_state(h));
          status = h->h_st->out.status != MRCG_OK ? (mrcg_status)h->h_st->out.status : MRCG_ERR_MAXITER;
          finished = true;
          break;
        }
        const int nxt = cur ^ 1;
        TraceRange step("mrcg outer MINRES step");
        LKC(launch_lanczos_spmv(h->oargs, h->zraw, h->zn, h->res));
        LKC(launch_lanczos_update(h->oargs, h->res, h->v[cur], h->v[nxt], h->v[nxt], h->zraw));
        ST(run_inner(h)); graphs += 1;
        LKC(launch_gamma_givens(h->oargs, h->zraw, h->v[nxt]));
        LKC(launch_minres_update(h->oargs, h->zn, h->w[nxt], h->w[cur], h->w[nxt], h->x));
        LKC(launch_residual(h->oargs, h->b, h->x, h->res));
        ST(read_state(h));
        if (O.status != MRCG_OK) {
          status = (mrcg_status)O.status;
          finished = true;
          break;
        }
        ++outer;
        relres = O.relres;
        record(relres);
        if (relres <= outer_tol) {
          status = MRCG_OK;
          finished = true;
          break;
        }
        cur = nxt;
        cyc.push_back(relres);
        const size_t m = cyc.size();
        bool restart = false;
        if (h->restart_factor > 0.0 && m >= 4 && relres > h->restart_factor * cyc[m - 4]) restart = true;
        if (O.gamma_new == 0.0) restart = true;
        if (restart) {
          ++restarts;
          break;  // res holds b - A x: the next cycle starts from it
        }
      }
    }
  }
  ST(stage_out(h, h->x, ux));
  ST(read_state(h));
  if (info) {
    info->outer_iters = outer;
    info->restarts = restarts;
    info->inner_iters_total = h->h_st->out.inner_total;
    info->prec_calls = h->h_st->out.prec_calls;
    // per inner solve: norm, init (two passes for MINRES-CG*), finish; per body
    // of the while loop: U iterations of one or two kernels, then the control kernel
    const long long per_graph = 3 + (h->mcg == MRCG_MCG_SMW || h->mcg == MRCG_MCG_ILU0 || h->mcg == MRCG_MCG_SMW_ILU0 ? 1 : 0);
    const long long per_body = (h->spec.var_a == 8 ? 1LL : 2LL) * h->unroll + 1;
    info->kernel_launches = launches + per_graph * graphs + h->h_st->out.bodies * per_body;
    info->true_relres = relres;
    info->history_len = info->relres_history ? std::min(hist_len, info->history_cap) : 0;
    info->status = status;
  }
  return status;
}

}  // namespace

extern "C" {

const char* mrcg_status_string(mrcg_status s) {
  switch (s) {
    case MRCG_OK: return "MRCG_OK";
    case MRCG_ERR_INVALID: return "MRCG_ERR_INVALID";
    case MRCG_ERR_NOT_SPD: return "MRCG_ERR_NOT_SPD";
    case MRCG_ERR_BREAKDOWN: return "MRCG_ERR_BREAKDOWN";
    case MRCG_ERR_MAXITER: return "MRCG_ERR_MAXITER";
    case MRCG_ERR_NONFINITE: return "MRCG_ERR_NONFINITE";
    case MRCG_ERR_CUDA: return "MRCG_ERR_CUDA";
    case MRCG_ERR_OOM: return "MRCG_ERR_OOM";
  }
  return "MRCG_ERR_UNKNOWN";
}

mrcg_status mrcg_solver_create(const mrcg_create_args* a, mrcg_handle* out) {
  if (!a || !out) return MRCG_ERR_INVALID;
  *out = nullptr;
  if (a->n < 1 || a->n > (int64_t)0x7fffff00 || a->nnz < 0 || a->k < 0 || a->k > kMaxK) return MRCG_ERR_INVALID;
  if (a->precision != MRCG_FP64 && a->precision != MRCG_MIXED_FP32 && a->precision != MRCG_MIXED_BF16M)
    return MRCG_ERR_INVALID;
  if (a->inner_prec < MRCG_MCG_IDENTITY || a->inner_prec > MRCG_MCG_SMW_ILU0) return MRCG_ERR_INVALID;
  if (!a->rowptr || (a->nnz > 0 && (!a->colind || !a->val))) return MRCG_ERR_INVALID;
  if (a->k > 0 && (!a->V || !a->lambda)) return MRCG_ERR_INVALID;
  if (std::isnan(a->restart_factor)) return MRCG_ERR_INVALID;
  mrcg_solver* h = new (std::nothrow) mrcg_solver();
  if (!h) return MRCG_ERR_OOM;
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    delete h;
    return MRCG_ERR_CUDA;
  }
  mrcg_status s = create_impl(a, h);
  if (s != MRCG_OK) {
    cudaGetLastError();
    destroy_impl(h);
    return s;
  }
  *out = h;
  return MRCG_OK;
}

void mrcg_solver_destroy(mrcg_handle h) {
  if (!h) return;
  DeviceGuard g(h->device);
  destroy_impl(h);
}

mrcg_status mrcg_solve(mrcg_handle h, const double* b, double* x, double outer_tol, double inner_tol,
                       int64_t max_iters, mrcg_info* info) {
  if (!h || !b || !x) return MRCG_ERR_INVALID;
  if (!(outer_tol >= 0.0) || !(inner_tol > 0.0) || !(inner_tol < 1.0)) return MRCG_ERR_INVALID;
  if (info && info->relres_history && info->history_cap < 0) return MRCG_ERR_INVALID;
  DeviceGuard g(h->device);
  const auto t0 = std::chrono::steady_clock::now();
  mrcg_status s = solve_impl(h, b, x, outer_tol, inner_tol, max_iters, info);
  if (s == MRCG_ERR_CUDA || s == MRCG_ERR_OOM) cudaStreamSynchronize(h->stream);
  if (info) {
    info->solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (s == MRCG_ERR_CUDA || s == MRCG_ERR_OOM) info->status = s;
  }
  return s;
}

mrcg_status mrcg_apply_A(mrcg_handle h, const double* x, double* y) {
  if (!h || !x || !y) return MRCG_ERR_INVALID;
  DeviceGuard g(h->device);
  ST(stage_in(h, x, h->v[0]));
  LK(launch_spmv(h->oargs, h->v[0], h->zraw));
  ST(stage_out(h, h->zraw, y));
  CK(cudaStreamSynchronize(h->stream));
  return MRCG_OK;
}

mrcg_status mrcg_apply_mmr(mrcg_handle h, const double* u, double* out) {
  if (!h || !u || !out) return MRCG_ERR_INVALID;
  DeviceGuard g(h->device);
  ST(stage_in(h, u, h->v[0]));
  reset_state(h, 0.5, 0);
  ST(upload_state(h));
  const void* val = h->fp32 ? (const void*)h->d_val32 : (const void*)h->d_val64;
  const void* V = h->fp32 ? (const void*)h->d_V32 : (const void*)h->d_V64;
  LK(launch_mmr(h->oargs, h->fp32, val, V, h->k, nullptr, h->v[0], h->zraw, h->ir, h->iq));
  ST(stage_out(h, h->zraw, out));
  CK(cudaStreamSynchronize(h->stream));
  return MRCG_OK;
}

mrcg_status mrcg_inner_solve(mrcg_handle h, const double* y, double* z, double inner_tol, int64_t max_iters,
                             int64_t* iters) {
  if (!h || !y || !z) return MRCG_ERR_INVALID;
  if (!(inner_tol > 0.0) || !(inner_tol < 1.0)) return MRCG_ERR_INVALID;
  DeviceGuard g(h->device);
  ST(stage_in(h, y, h->v[0]));
  reset_state(h, inner_tol, max_iters > 0 ? (long long)max_iters : (1LL << 31));
  h->h_init->cg.vin = h->v[0];
  h->h_init->cg.zout = h->zraw;
  ST(upload_state(h));
  ST(run_inner(h));
  ST(stage_out(h, h->zraw, z));
  ST(read_state(h));
  if (iters) *iters = h->h_st->cg.iters;
  switch (h->h_st->cg.done) {
    case kConverged: return MRCG_OK;
    case kNotSpd: return MRCG_ERR_NOT_SPD;
    case kNonFinite: return MRCG_ERR_NONFINITE;
    case kBreakdown: return MRCG_ERR_BREAKDOWN;
    case kStall: return MRCG_ERR_CUDA;
    default: return MRCG_ERR_MAXITER;
  }
}

mrcg_status mrcg_launch_config(mrcg_handle h, int32_t* cfg) {
  if (!h || !cfg) return MRCG_ERR_INVALID;
  cfg[0] = h->spec.var_a;
  cfg[1] = h->spec.grid_spmv;
  cfg[2] = h->spec.grid_stream_b;
  cfg[3] = h->spec.unroll;
  cfg[4] = h->k == 0 ? 0 : h->k <= 8 ? 8 : h->k <= 12 ? 12 : h->k <= 16 ? 16 : h->k <= 24 ? 24 : 32;
  cfg[5] = h->A.col16 ? 2 : 4;
  cfg[6] = is_staged_variant(h->spec.var_a) ? h->spec.stages : 0;
  return MRCG_OK;
}

mrcg_status mrcg_time_inner_kernels(mrcg_handle h, int32_t iters, double* ms) {
  if (!h || !ms || iters < 1 || iters > 4096) return MRCG_ERR_INVALID;
  DeviceGuard g(h->device);
  reset_state(h, 1e-300, (long long)iters + 16);
  h->h_init->cg.vin = h->v[0];
  h->h_init->cg.zout = h->zraw;
  ST(upload_state(h));
  double t4[4] = {0.0, 0.0, 0.0, 0.0};
  LK(time_inner_kernels(h->spec, iters, h->stream, h->v[0], h->n, t4));
  ms[0] = t4[2];
  ms[1] = t4[3];
  ST(read_state(h));
  if (h->h_st->cg.done != kRunning && h->h_st->cg.iters < iters) return MRCG_ERR_BREAKDOWN;
  return MRCG_OK;
}

mrcg_status mrcg_time_inner_graph(mrcg_handle h, int32_t iters, double* ms_per_iter) {
  if (!h || !ms_per_iter || iters < 8 || iters > 65536) return MRCG_ERR_INVALID;
  DeviceGuard g(h->device);
  // a fixed right-hand side (the pattern of the standalone timing) in v[0]
  std::vector<double> pat((size_t)h->n_pad, 0.0);
  for (int64_t i = 0; i < h->n; ++i) pat[i] = 1.0 + 0.125 * (double)(i % 7) - 0.0625 * (double)(i % 3);
  CK(cudaMemcpyAsync(h->v[0], pat.data(), pat.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  // one inner solve of exactly `n_it` iterations (tolerance 1e-300: only the
  // budget stops it), bracketed by events on the handle's stream
  // returns the iterations the solve ran (it stops at the budget unless the
  // recursion itself ends, e.g. a residual that reaches exactly zero)
  auto timed = [&](long long n_it, float* ms, long long* ran) -> mrcg_status {
    reset_state(h, 1e-300, n_it);
    h->h_init->cg.vin = h->v[0];
    h->h_init->cg.zout = h->zraw;
    ST(upload_state(h));
    CK(cudaEventRecord(e0, h->stream));
    ST(run_inner(h));
    CK(cudaEventRecord(e1, h->stream));
    CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(ms, e0, e1));
    ST(read_state(h));
    *ran = h->h_st->cg.iters;
    if (getenv("MRCG_DEBUG"))
      fprintf(stderr, "mrcg time_inner_graph: budget %lld ran %lld done %d in %.3f ms\n", n_it, *ran,
              h->h_st->cg.done, (double)*ms);
    return MRCG_OK;
  };
  const long long base = 2LL * h->unroll;
  float t_short = 0.f, t_long = 0.f, unused = 0.f;
  long long r0 = 0, r1 = 0, r2 = 0;
  // warm-up and probe: with no tolerance to stop it, an FP32 recursion that
  // has reached its rounding floor can end on its own (p^T q <= 0); the long
  // run then keeps to three quarters of the iterations the probe reached
  mrcg_status st = timed(base + iters, &unused, &r0);
  long long n_long = base + iters;
  if (st == MRCG_OK && r0 < n_long) n_long = std::max(base + 8, r0 * 3 / 4);
  // the difference of two solves cancels the per-solve kernels (norm, init, finish)
  if (st == MRCG_OK) st = timed(base, &t_short, &r1);
  if (st == MRCG_OK) st = timed(n_long, &t_long, &r2);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != MRCG_OK) return st;
  if (r2 - r1 < 8) return MRCG_ERR_BREAKDOWN;  // the recursion stops too early: no steady state to time
  *ms_per_iter = (double)(t_long - t_short) / (double)(r2 - r1);
  return MRCG_OK;
}

}  // extern "C"
