// Complex shifted systems of the disk-brake application (Sec. 3): for the
// companion linearisation A = [[0, I], [-K, -D]], B = [[I, 0], [0, Mass]] of a
// quadratic pencil, solve C (x + i y) = f + i g with C = gamma B - A through
// the double-size real system
//     [[Bh, -Ah], [Ah, Bh]] [x; -y] = [g; f],
//     Ah = [[gr I, -I], [K, gr Mass + D]],   Bh = [[gi I, 0], [0, gi Mass]],
// preconditioned by M = [[Bt, -At], [At, Bt]], At = [[gr I, -I], [KE, gr Mass]],
// Bt = Bh (KE the symmetric positive definite stiffness, Mass lumped).  M is
// applied by its block LU: Bt solves (diagonal), the Schur complement
// S = Bt + At Bt^-1 At = S1 S2 with S1 = diag(Mass^-1, I), and S2 solved by a
// Krylov method preconditioned with its block lower triangular part S2t,
// whose two diagonal solves are with -(1/gi)(KE - |gamma|^2 Mass): the
// symmetric indefinite inner-level system, solved by MINRES-CG with the
// library's own single-system solver (its negative eigenpairs computed once,
// by the setup eigensolver unless given; reused for every gamma of the same
// |gamma|).
//
// Krylov methods: flexible GMRES (right preconditioning, restarted) on the
// real-equivalent system, and flexible GMRES (one cycle) on S2, because both
// preconditioners contain inexact inner solves.  Orthogonalisation: classical
// Gram-Schmidt applied twice; Hessenberg least squares by Givens rotations on
// the host.  All vectors are FP64 on the device; the inner MINRES-CG runs in
// its handle's precision.
//
// Vector layout: a real-equivalent vector is [z1; z2] with z1 = [u1; v1],
// z2 = [u2; v2], four blocks of n (u: positions, v: velocities).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <new>
#include <vector>

#include "common.cuh"
#include "mrcg.h"

namespace mrcg {
namespace cplx {

struct Csr {
  int64_t n;
  const int64_t* rowptr;
  const int32_t* col;
  const double* val;
};

__device__ __forceinline__ double row_dot(const Csr& A, int64_t i, const double* __restrict__ x) {
  double acc = 0.0;
  for (int64_t p = A.rowptr[i]; p < A.rowptr[i + 1]; ++p) acc = fma(A.val[p], __ldg(x + A.col[p]), acc);
  return acc;
}

#define CX_ROWS(i, n) \
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < (n); i += (int64_t)gridDim.x * kThreads)

// out = [[Bh, -Ah], [Ah, Bh]] z   (z, out: 4n)
__global__ void __launch_bounds__(kThreads) cx_apply_kernel(Csr K, Csr D, const double* __restrict__ m, double gr,
                                                           double gi, const double* __restrict__ z,
                                                           double* __restrict__ out) {
  const int64_t n = K.n;
  const double* u1 = z;
  const double* v1 = z + n;
  const double* u2 = z + 2 * n;
  const double* v2 = z + 3 * n;
  CX_ROWS(i, n) {
    const double ku1 = row_dot(K, i, u1), ku2 = row_dot(K, i, u2);
    const double dv1 = row_dot(D, i, v1), dv2 = row_dot(D, i, v2);
    const double mi = m[i];
    // Bh z1 - Ah z2
    out[i] = gi * u1[i] - (gr * u2[i] - v2[i]);
    out[n + i] = gi * mi * v1[i] - (ku2 + gr * mi * v2[i] + dv2);
    // Ah z1 + Bh z2
    out[2 * n + i] = gr * u1[i] - v1[i] + gi * u2[i];
    out[3 * n + i] = ku1 + gr * mi * v1[i] + dv1 + gi * mi * v2[i];
  }
}

// block LU, forward part: w1 = Bt^-1 r1 and t = S1^-1 (r2 - At w1), the KE w1u
// term left to cx_spmv_axpy (t_v -= KE w1u)
__global__ void __launch_bounds__(kThreads) cx_forward_kernel(int64_t n, const double* __restrict__ m, double gr,
                                                             double gi, const double* __restrict__ r,
                                                             double* __restrict__ w1, double* __restrict__ t) {
  CX_ROWS(i, n) {
    const double mi = m[i];
    const double wu = r[i] / gi, wv = r[n + i] / (gi * mi);
    w1[i] = wu;
    w1[n + i] = wv;
    t[i] = mi * (r[2 * n + i] - (gr * wu - wv));   // S1^-1 = diag(Mass, I)
    t[n + i] = r[3 * n + i] - gr * mi * wv;
  }
}

// y = alpha (A x) + y
__global__ void __launch_bounds__(kThreads) cx_spmv_axpy_kernel(Csr A, double alpha, const double* __restrict__ x,
                                                               double* __restrict__ y) {
  CX_ROWS(i, A.n) y[i] += alpha * row_dot(A, i, x);
}

// block LU, backward part: u2 = w2, u1 = w1 + Bt^-1 At u2  (out: 4n)
__global__ void __launch_bounds__(kThreads) cx_backward_kernel(Csr KE, const double* __restrict__ m, double gr,
                                                              double gi, const double* __restrict__ w1,
                                                              const double* __restrict__ w2, double* __restrict__ out) {
  const int64_t n = KE.n;
  CX_ROWS(i, n) {
    const double mi = m[i];
    const double u2 = w2[i], v2 = w2[n + i];
    out[i] = w1[i] + (gr * u2 - v2) / gi;
    out[n + i] = w1[n + i] + (row_dot(KE, i, w2) + gr * mi * v2) / (gi * mi);
    out[2 * n + i] = u2;
    out[3 * n + i] = v2;
  }
}

// S2 [x; y] = [Di x - c2 Mass y; c2 KE x + Di y],  Di w = c Mass w - KE w / gi
__global__ void __launch_bounds__(kThreads) cx_s2_kernel(Csr KE, const double* __restrict__ m, double c, double c2,
                                                        double gi, const double* __restrict__ xy,
                                                        double* __restrict__ out) {
  const int64_t n = KE.n;
  const double* x = xy;
  const double* y = xy + n;
  CX_ROWS(i, n) {
    const double kx = row_dot(KE, i, x), ky = row_dot(KE, i, y);
    const double mi = m[i];
    out[i] = c * mi * x[i] - kx / gi - c2 * mi * y[i];
    out[n + i] = c2 * kx + c * mi * y[i] - ky / gi;
  }
}

// y = alpha x
__global__ void __launch_bounds__(kThreads) cx_scale_kernel(int64_t N, double alpha, const double* __restrict__ x,
                                                           double* __restrict__ y) {
  CX_ROWS(i, N) y[i] = alpha * x[i];
}

// y = x - w  (residual)
__global__ void __launch_bounds__(kThreads) cx_sub_kernel(int64_t N, const double* __restrict__ x,
                                                         const double* __restrict__ w, double* __restrict__ y) {
  CX_ROWS(i, N) y[i] = x[i] - w[i];
}

// partials[c * gridDim.x + b] = block b's share of <V_c, w>, c < ncol (V_c at V + c * ld)
__global__ void __launch_bounds__(kThreads) cx_mdot_kernel(int64_t N, const double* __restrict__ V, int64_t ld,
                                                          int ncol, const double* __restrict__ w,
                                                          double* __restrict__ partials) {
  __shared__ double sm[kThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c = 0; c < ncol; ++c) {
    const double* v = V + (size_t)c * ld;
    double s = 0.0;
    CX_ROWS(i, N) s = fma(v[i], w[i], s);
    s = warp_sum(s);
    if (lane == 0) sm[warp] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int q = 0; q < kThreads / 32; ++q) t += sm[q];
      partials[(size_t)c * gridDim.x + blockIdx.x] = t;
    }
    __syncthreads();
  }
}

// out[c] = sum over blocks (fixed order), one warp per value
__global__ void __launch_bounds__(kThreads) cx_reduce_kernel(const double* __restrict__ partials, int nblk, int nval,
                                                            double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int e = blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
  if (e >= nval) return;
  double s = lane_sum8(partials + (size_t)e * nblk, nblk, lane);
  s = warp_sum(s);
  if (lane == 0) out[e] = s;
}

// w -= sum_c h[c] V_c   (h in device memory, ncol <= 128)
__global__ void __launch_bounds__(kThreads) cx_maxpy_kernel(int64_t N, const double* __restrict__ V, int64_t ld,
                                                           int ncol, const double* __restrict__ h,
                                                           double* __restrict__ w) {
  __shared__ double hs[128];
  for (int c = threadIdx.x; c < ncol; c += kThreads) hs[c] = h[c];
  __syncthreads();
  CX_ROWS(i, N) {
    double acc = w[i];
    for (int c = 0; c < ncol; ++c) acc -= hs[c] * V[(size_t)c * ld + i];
    w[i] = acc;
  }
}

// x += sum_c y[c] Z_c
__global__ void __launch_bounds__(kThreads) cx_update_kernel(int64_t N, const double* __restrict__ Z, int64_t ld,
                                                            int ncol, const double* __restrict__ y,
                                                            double* __restrict__ x) {
  __shared__ double ys[128];
  for (int c = threadIdx.x; c < ncol; c += kThreads) ys[c] = y[c];
  __syncthreads();
  CX_ROWS(i, N) {
    double acc = x[i];
    for (int c = 0; c < ncol; ++c) acc += ys[c] * Z[(size_t)c * ld + i];
    x[i] = acc;
  }
}

}  // namespace cplx
}  // namespace mrcg

using namespace mrcg;
using namespace mrcg::cplx;

struct mrcg_complex {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int64_t n = 0;
  double gamma_abs = 0.0;
  Csr KE{}, K{}, D{};
  double* mass = nullptr;
  mrcg_handle inner = nullptr;
  int k = 0;
  int grid = 1;
  double* partials = nullptr;
  double* small = nullptr;  // reduced dot products (device)
  std::vector<void*> allocs;
  // counters of the running solve
  long long inner_solves = 0, inner_cg = 0, s2_iters = 0;
  mrcg_status inner_status = MRCG_OK;
};

namespace {

#define XCK(call)                                                                                  \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) {                                                                       \
      if (getenv("MRCG_DEBUG")) fprintf(stderr, "mrcg complex: %s failed: %s (%s:%d)\n", #call,     \
                                        cudaGetErrorString(e_), __FILE__, __LINE__);               \
      return e_ == cudaErrorMemoryAllocation ? MRCG_ERR_OOM : MRCG_ERR_CUDA;                       \
    }                                                                                              \
  } while (0)
#define XST(call)                 \
  do {                            \
    mrcg_status s_ = (call);      \
    if (s_ != MRCG_OK) return s_; \
  } while (0)

constexpr int kDotBlocks = 304;
constexpr int kMaxRestart = 120;

bool x_is_device(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

template <typename T>
mrcg_status xalloc(mrcg_complex* h, T** p, size_t count) {
  void* q = nullptr;
  if (cudaMalloc(&q, std::max<size_t>(count * sizeof(T), 256)) != cudaSuccess) {
    cudaGetLastError();
    return MRCG_ERR_OOM;
  }
  h->allocs.push_back(q);
  *p = reinterpret_cast<T*>(q);
  return MRCG_OK;
}

template <typename T>
mrcg_status xfetch(const T* src, size_t count, std::vector<T>& dst) {
  dst.resize(count);
  if (!count) return MRCG_OK;
  if (!src) return MRCG_ERR_INVALID;
  if (x_is_device(src)) XCK(cudaMemcpy(dst.data(), src, count * sizeof(T), cudaMemcpyDeviceToHost));
  else std::memcpy(dst.data(), src, count * sizeof(T));
  return MRCG_OK;
}

// host copy of one CSR input, validated
mrcg_status fetch_csr(int64_t n, const int64_t* rp_in, const int32_t* ci_in, const double* va_in,
                      std::vector<int64_t>& rp, std::vector<int32_t>& ci, std::vector<double>& va) {
  XST(xfetch(rp_in, (size_t)n + 1, rp));
  if (rp[0] != 0) return MRCG_ERR_INVALID;
  for (int64_t i = 0; i < n; ++i)
    if (rp[i + 1] < rp[i]) return MRCG_ERR_INVALID;
  XST(xfetch(ci_in, (size_t)rp[n], ci));
  XST(xfetch(va_in, (size_t)rp[n], va));
  for (int64_t p = 0; p < rp[n]; ++p) {
    if (ci[p] < 0 || ci[p] >= n) return MRCG_ERR_INVALID;
    if (!std::isfinite(va[p])) return MRCG_ERR_NONFINITE;
  }
  return MRCG_OK;
}

mrcg_status upload_csr(mrcg_complex* h, const std::vector<int64_t>& rp, const std::vector<int32_t>& ci,
                       const std::vector<double>& va, Csr* out) {
  int64_t* d_rp = nullptr;
  int32_t* d_ci = nullptr;
  double* d_va = nullptr;
  XST(xalloc(h, &d_rp, rp.size()));
  XST(xalloc(h, &d_ci, ci.size()));
  XST(xalloc(h, &d_va, va.size()));
  XCK(cudaMemcpyAsync(d_rp, rp.data(), rp.size() * sizeof(int64_t), cudaMemcpyHostToDevice, h->stream));
  if (!ci.empty()) {
    XCK(cudaMemcpyAsync(d_ci, ci.data(), ci.size() * sizeof(int32_t), cudaMemcpyHostToDevice, h->stream));
    XCK(cudaMemcpyAsync(d_va, va.data(), va.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  }
  XCK(cudaStreamSynchronize(h->stream));
  *out = {(int64_t)rp.size() - 1, d_rp, d_ci, d_va};
  return MRCG_OK;
}

// dots[c] = <V_c, w>, c < ncol (host result)
mrcg_status mdot(mrcg_complex* h, int64_t N, const double* V, int64_t ld, int ncol, const double* w, double* dots) {
  cx_mdot_kernel<<<kDotBlocks, kThreads, 0, h->stream>>>(N, V, ld, ncol, w, h->partials);
  cx_reduce_kernel<<<(ncol + kThreads / 32 - 1) / (kThreads / 32), kThreads, 0, h->stream>>>(h->partials, kDotBlocks,
                                                                                            ncol, h->small);
  XCK(cudaGetLastError());
  XCK(cudaMemcpyAsync(dots, h->small, ncol * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  XCK(cudaStreamSynchronize(h->stream));
  return MRCG_OK;
}

using Op = std::function<mrcg_status(const double*, double*)>;

struct FgmresWork {
  double* V = nullptr;  // (m + 1) x N
  double* Z = nullptr;  // m x N
  double* w = nullptr;  // N
  double* hd = nullptr; // coefficients on the device (m + 1)
};

// Flexible GMRES (restarted, right preconditioning): A x = b from the x given.
// Stops when the residual estimate falls to tol ||b|| (the true residual is
// recomputed at each restart and at the end).  Returns iterations in *its and
// the final true relative residual in *relres.
mrcg_status fgmres(mrcg_complex* h, int64_t N, const Op& A, const Op& P, const double* b, double* x, double tol,
                   int m, int max_iters, FgmresWork& wk, int* its, double* relres) {
  *its = 0;
  double bn = 0.0;
  XST(mdot(h, N, b, N, 1, b, &bn));
  bn = std::sqrt(bn);
  if (bn == 0.0) {
    XCK(cudaMemsetAsync(x, 0, N * sizeof(double), h->stream));
    *relres = 0.0;
    return MRCG_OK;
  }
  std::vector<double> H((size_t)(m + 1) * m, 0.0), cs(m), sn(m), g(m + 1), hcol(m + 1), h2(m + 1);
  for (;;) {
    // r = b - A x  into V_0
    XST(A(x, wk.w));
    cx_sub_kernel<<<kDotBlocks, kThreads, 0, h->stream>>>(N, b, wk.w, wk.V);
    double beta = 0.0;
    XST(mdot(h, N, wk.V, N, 1, wk.V, &beta));
    beta = std::sqrt(beta);
    *relres = beta / bn;
    if (!std::isfinite(beta)) return MRCG_ERR_NONFINITE;
    if (*relres <= tol || *its >= max_iters) return *relres <= tol ? MRCG_OK : MRCG_ERR_MAXITER;
    cx_scale_kernel<<<kDotBlocks, kThreads, 0, h->stream>>>(N, 1.0 / beta, wk.V, wk.V);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int j = 0;
    for (; j < m && *its < max_iters; ++j) {
      double* vj = wk.V + (size_t)j * N;
      double* zj = wk.Z + (size_t)j * N;
      XST(P(vj, zj));
      XST(A(zj, wk.w));
      // classical Gram-Schmidt, twice
      std::fill(hcol.begin(), hcol.end(), 0.0);
      for (int pass = 0; pass < 2; ++pass) {
        XST(mdot(h, N, wk.V, N, j + 1, wk.w, h2.data()));
        XCK(cudaMemcpyAsync(wk.hd, h2.data(), (j + 1) * sizeof(double), cudaMemcpyHostToDevice, h->stream));
        cx_maxpy_kernel<<<kDotBlocks, kThreads, 0, h->stream>>>(N, wk.V, N, j + 1, wk.hd, wk.w);
        XCK(cudaStreamSynchronize(h->stream));  // h2 is reused by the next pass
        for (int i = 0; i <= j; ++i) hcol[i] += h2[i];
      }
      double hn = 0.0;
      XST(mdot(h, N, wk.w, N, 1, wk.w, &hn));
      hn = std::sqrt(hn);
      hcol[j + 1] = hn;
      if (hn > 0.0) cx_scale_kernel<<<kDotBlocks, kThreads, 0, h->stream>>>(N, 1.0 / hn, wk.w, wk.V + (size_t)(j + 1) * N);
      // Givens rotations of the new column
      for (int i = 0; i < j; ++i) {
        const double t = cs[i] * hcol[i] + sn[i] * hcol[i + 1];
        hcol[i + 1] = -sn[i] * hcol[i] + cs[i] * hcol[i + 1];
        hcol[i] = t;
      }
      const double r = std::hypot(hcol[j], hcol[j + 1]);
      cs[j] = r > 0.0 ? hcol[j] / r : 1.0;
      sn[j] = r > 0.0 ? hcol[j + 1] / r : 0.0;
      hcol[j] = r;
      hcol[j + 1] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hcol[i];
      ++*its;
      if (std::fabs(g[j + 1]) <= tol * bn || hn == 0.0) {
        ++j;
        break;
      }
    }
    // y = R^-1 g, x += Z y
    std::vector<double> y(j, 0.0);
    for (int i = j - 1; i >= 0; --i) {
      double s = g[i];
      for (int l = i + 1; l < j; ++l) s -= H[(size_t)i * m + l] * y[l];
      y[i] = s / H[(size_t)i * m + i];
    }
    XCK(cudaMemcpyAsync(wk.hd, y.data(), j * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    cx_update_kernel<<<kDotBlocks, kThreads, 0, h->stream>>>(N, wk.Z, N, j, wk.hd, x);
    XCK(cudaStreamSynchronize(h->stream));
  }
}

}  // namespace

extern "C" {

mrcg_status mrcg_complex_create(const mrcg_complex_args* a, mrcg_complex_handle* out) {
  if (!a || !out) return MRCG_ERR_INVALID;
  *out = nullptr;
  if (a->n < 1 || a->n > (int64_t)0x1fffff00 || !(a->gamma_abs > 0.0) || !a->mass) return MRCG_ERR_INVALID;
  if (a->k > kMaxK || (a->k > 0 && (!a->V || !a->lambda)) || a->eig_block > 64) return MRCG_ERR_INVALID;
  mrcg_complex* h = new (std::nothrow) mrcg_complex();
  if (!h) return MRCG_ERR_OOM;
  auto fail = [&](mrcg_status s) {
    mrcg_complex_destroy(h);
    cudaGetLastError();
    return s;
  };
  if (cudaGetDevice(&h->device) != cudaSuccess) return fail(MRCG_ERR_CUDA);
  const int64_t n = a->n;
  h->n = n;
  h->gamma_abs = a->gamma_abs;
  if (a->stream) {
    h->stream = (cudaStream_t)a->stream;
  } else {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) return fail(MRCG_ERR_CUDA);
    h->own_stream = true;
  }
  std::vector<int64_t> rpE, rpK, rpD;
  std::vector<int32_t> ciE, ciK, ciD;
  std::vector<double> vaE, vaK, vaD, mass;
  mrcg_status st;
  if ((st = fetch_csr(n, a->ke_rowptr, a->ke_colind, a->ke_val, rpE, ciE, vaE)) != MRCG_OK) return fail(st);
  if ((st = fetch_csr(n, a->k_rowptr, a->k_colind, a->k_val, rpK, ciK, vaK)) != MRCG_OK) return fail(st);
  if ((st = fetch_csr(n, a->d_rowptr, a->d_colind, a->d_val, rpD, ciD, vaD)) != MRCG_OK) return fail(st);
  if ((st = xfetch(a->mass, (size_t)n, mass)) != MRCG_OK) return fail(st);
  for (double mi : mass)
    if (!(mi > 0.0) || !std::isfinite(mi)) return fail(MRCG_ERR_INVALID);
  // the inner-level matrix KE - |gamma|^2 Mass: KE's pattern with its diagonal shifted
  std::vector<double> vaIn = vaE;
  const double mod2 = a->gamma_abs * a->gamma_abs;
  for (int64_t i = 0; i < n; ++i) {
    bool diag = false;
    for (int64_t p = rpE[i]; p < rpE[i + 1]; ++p)
      if (ciE[p] == i) {
        vaIn[p] -= mod2 * mass[i];
        diag = true;
      }
    if (!diag) return fail(MRCG_ERR_INVALID);  // a stiffness matrix has its diagonal
  }
  // its negative eigenpairs: given, or from the setup eigensolver
  std::vector<double> V, lam;
  int k = a->k;
  if (k < 0) {
    const int block = a->eig_block > 0 ? a->eig_block : 32;
    V.assign((size_t)n * block, 0.0);
    lam.assign(block, 0.0);
    int32_t kk = 0;
    if ((st = mrcg_negative_eigenpairs(n, rpE.data(), ciE.data(), vaIn.data(), block, 1e-11, 400000, 1, &kk,
                                       V.data(), lam.data(), nullptr)) != MRCG_OK)
      return fail(st);
    k = kk;
    V.resize((size_t)n * k);
    lam.resize(k);
  } else if (k > 0) {
    if ((st = xfetch(a->V, (size_t)n * k, V)) != MRCG_OK) return fail(st);
    if ((st = xfetch(a->lambda, (size_t)k, lam)) != MRCG_OK) return fail(st);
  }
  if (k > kMaxK) return fail(MRCG_ERR_INVALID);
  h->k = k;
  mrcg_create_args ia = {};
  ia.n = n;
  ia.nnz = rpE[n];
  ia.rowptr = rpE.data();
  ia.colind = ciE.data();
  ia.val = vaIn.data();
  ia.k = k;
  ia.V = k > 0 ? V.data() : nullptr;
  ia.lambda = k > 0 ? lam.data() : nullptr;
  ia.precision = a->precision;
  ia.inner_prec = a->inner_prec;
  ia.validate = 1;
  ia.stream = h->stream;
  if ((st = mrcg_solver_create(&ia, &h->inner)) != MRCG_OK) return fail(st);
  if ((st = upload_csr(h, rpE, ciE, vaE, &h->KE)) != MRCG_OK) return fail(st);
  if ((st = upload_csr(h, rpK, ciK, vaK, &h->K)) != MRCG_OK) return fail(st);
  if ((st = upload_csr(h, rpD, ciD, vaD, &h->D)) != MRCG_OK) return fail(st);
  if ((st = xalloc(h, &h->mass, (size_t)n)) != MRCG_OK) return fail(st);
  if (cudaMemcpy(h->mass, mass.data(), n * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(MRCG_ERR_CUDA);
  if ((st = xalloc(h, &h->partials, (size_t)(kMaxRestart + 1) * kDotBlocks)) != MRCG_OK) return fail(st);
  if ((st = xalloc(h, &h->small, (size_t)kMaxRestart + 1)) != MRCG_OK) return fail(st);
  int nsm = 1;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device);
  h->grid = nsm * 4;
  *out = h;
  return MRCG_OK;
}

int32_t mrcg_complex_negative_count(mrcg_complex_handle h) { return h ? h->k : -1; }

mrcg_status mrcg_complex_solve(mrcg_complex_handle h, double gamma_re, double gamma_im, const double* f,
                               const double* g, double* x, double* y, double tol, int32_t restart,
                               int32_t max_iters, double s2_tol, int32_t s2_max, double inner_tol,
                               double cg_tol, mrcg_complex_info* info) {
  if (!h || !f || !g || !x || !y) return MRCG_ERR_INVALID;
  if (!(gamma_im > 0.0) || !(tol > 0.0) || restart < 1 || restart > kMaxRestart || max_iters < 1 ||
      !(s2_tol > 0.0) || s2_max < 1 || s2_max > kMaxRestart || !(inner_tol > 0.0) || !(cg_tol > 0.0) ||
      !(cg_tol < 1.0))
    return MRCG_ERR_INVALID;
  const double gabs = std::hypot(gamma_re, gamma_im);
  if (std::fabs(gabs - h->gamma_abs) > 1e-10 * h->gamma_abs) return MRCG_ERR_INVALID;  // the inner level is per |gamma|
  const auto t0 = std::chrono::steady_clock::now();
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != h->device) cudaSetDevice(h->device);
  const int64_t n = h->n, N4 = 4 * n, N2 = 2 * n;
  const double gr = gamma_re, gi = gamma_im;
  const double c = gi + gr * gr / gi, c2 = 2.0 * gr / gi;
  h->inner_solves = h->inner_cg = h->s2_iters = 0;
  h->inner_status = MRCG_OK;
  mrcg_status st = MRCG_OK;
  // work space of this call (freed at the end)
  std::vector<void*> mine;
  auto alloc = [&](double** p, size_t cnt) -> mrcg_status {
    void* q = nullptr;
    if (cudaMalloc(&q, std::max<size_t>(cnt * sizeof(double), 256)) != cudaSuccess) {
      cudaGetLastError();
      return MRCG_ERR_OOM;
    }
    mine.push_back(q);
    *p = reinterpret_cast<double*>(q);
    return MRCG_OK;
  };
  double *rhs = nullptr, *sol = nullptr, *w1 = nullptr, *t = nullptr, *w2 = nullptr, *a1 = nullptr, *a2 = nullptr;
  FgmresWork wo, ws;
  auto alloc_fw = [&](int64_t N, int m, FgmresWork& wk) -> mrcg_status {
    XST(alloc(&wk.V, (size_t)(m + 1) * N));
    XST(alloc(&wk.Z, (size_t)m * N));
    XST(alloc(&wk.w, (size_t)N));
    XST(alloc(&wk.hd, (size_t)(m + 1)));
    return MRCG_OK;
  };
  auto run = [&]() -> mrcg_status {
    XST(alloc(&rhs, N4));
    XST(alloc(&sol, N4));
    XST(alloc(&w1, N2));
    XST(alloc(&t, N2));
    XST(alloc(&w2, N2));
    XST(alloc(&a1, n));
    XST(alloc(&a2, n));
    XST(alloc_fw(N4, restart, wo));
    XST(alloc_fw(N2, s2_max, ws));
    // right-hand side [g; f] and start [x; -y] = 0
    const bool dev_in = x_is_device(f);
    XCK(cudaMemcpyAsync(rhs, g, N2 * sizeof(double), dev_in ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                        h->stream));
    XCK(cudaMemcpyAsync(rhs + N2, f, N2 * sizeof(double),
                        x_is_device(f) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->stream));
    XCK(cudaMemsetAsync(sol, 0, N4 * sizeof(double), h->stream));
    // Di^-1 v = -gi (KE - |gamma|^2 Mass)^-1 v by MINRES-CG (out may not alias v)
    auto di_solve = [&](const double* v, double* out) -> mrcg_status {
      XCK(cudaMemsetAsync(out, 0, n * sizeof(double), h->stream));
      mrcg_info inf = {};
      const mrcg_status s = mrcg_solve(h->inner, v, out, inner_tol, cg_tol, 0, &inf);
      ++h->inner_solves;
      h->inner_cg += inf.inner_iters_total;
      if (s != MRCG_OK && s != MRCG_ERR_MAXITER) return s;
      if (s == MRCG_ERR_MAXITER) h->inner_status = s;
      cx_scale_kernel<<<h->grid, kThreads, 0, h->stream>>>(n, -gi, out, out);
      XCK(cudaGetLastError());
      return MRCG_OK;
    };
    // S2t^-1 [a; b]: t1 = Di^-1 a, t2 = Di^-1 (b - c2 KE t1)
    Op s2t = [&](const double* ab, double* out) -> mrcg_status {
      XST(di_solve(ab, out));
      XCK(cudaMemcpyAsync(a2, ab + n, n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
      cx_spmv_axpy_kernel<<<h->grid, kThreads, 0, h->stream>>>(h->KE, -c2, out, a2);
      XST(di_solve(a2, out + n));
      return MRCG_OK;
    };
    Op s2 = [&](const double* xy, double* out) -> mrcg_status {
      cx_s2_kernel<<<h->grid, kThreads, 0, h->stream>>>(h->KE, h->mass, c, c2, gi, xy, out);
      XCK(cudaGetLastError());
      return MRCG_OK;
    };
    // M^-1 r by the block LU (Sec. 3), S2 by flexible GMRES with S2t
    Op prec = [&](const double* r, double* out) -> mrcg_status {
      cx_forward_kernel<<<h->grid, kThreads, 0, h->stream>>>(n, h->mass, gr, gi, r, w1, t);
      cx_spmv_axpy_kernel<<<h->grid, kThreads, 0, h->stream>>>(h->KE, -1.0, w1, t + n);  // t_v -= KE w1_u
      XCK(cudaGetLastError());
      XCK(cudaMemsetAsync(w2, 0, N2 * sizeof(double), h->stream));
      int its = 0;
      double rr = 0.0;
      const mrcg_status s = fgmres(h, N2, s2, s2t, t, w2, s2_tol, s2_max, s2_max, ws, &its, &rr);
      h->s2_iters += its;
      if (s != MRCG_OK && s != MRCG_ERR_MAXITER) return s;  // a partial S2 solve still preconditions
      cx_backward_kernel<<<h->grid, kThreads, 0, h->stream>>>(h->KE, h->mass, gr, gi, w1, w2, out);
      XCK(cudaGetLastError());
      return MRCG_OK;
    };
    Op op = [&](const double* z, double* out) -> mrcg_status {
      cx_apply_kernel<<<h->grid, kThreads, 0, h->stream>>>(h->K, h->D, h->mass, gr, gi, z, out);
      XCK(cudaGetLastError());
      return MRCG_OK;
    };
    int its = 0;
    double rr = 0.0;
    const mrcg_status s = fgmres(h, N4, op, prec, rhs, sol, tol, restart, max_iters, wo, &its, &rr);
    if (info) {
      info->outer_iters = its;
      info->s2_iters_total = (int32_t)h->s2_iters;
      info->inner_solves = h->inner_solves;
      info->inner_cg_iters = h->inner_cg;
      info->true_relres = rr;
    }
    // x = sol[0:2n], y = -sol[2n:4n]
    cx_scale_kernel<<<h->grid, kThreads, 0, h->stream>>>(N2, -1.0, sol + N2, sol + N2);
    const bool dev_out = x_is_device(x);
    XCK(cudaMemcpyAsync(x, sol, N2 * sizeof(double), dev_out ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                        h->stream));
    XCK(cudaMemcpyAsync(y, sol + N2, N2 * sizeof(double),
                        x_is_device(y) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->stream));
    XCK(cudaStreamSynchronize(h->stream));
    return s;
  };
  st = run();
  cudaStreamSynchronize(h->stream);
  for (void* p : mine) cudaFree(p);
  cudaGetLastError();
  if (cur != h->device) cudaSetDevice(cur);
  if (info) {
    info->solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    info->status = st;
  }
  return st;
}

void mrcg_complex_destroy(mrcg_complex_handle h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->inner) mrcg_solver_destroy(h->inner);
  for (void* p : h->allocs) cudaFree(p);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  cudaGetLastError();
  delete h;
}

}  // extern "C"
