// Setup stage 2 of the method (Sec. 2, the three-stage summary): the negative
// eigenpairs (V_hat, Lambda_hat) of the sparse symmetric A that define
// M_mr = A + 2 V_hat |Lambda_hat| V_hat^T.  The paper computes them with a
// Krylov eigensolver (MATLAB eigs) and amortises that cost over many solves.
//
// Here: Chebyshev-filtered subspace iteration on a block of m vectors.  Every
// filter step is a block SpMV with the same CSR A (HBM / FP64-pipe bound);
// between filters a Rayleigh-Ritz step on the block gives the Ritz pairs:
//   1. Gershgorin bounds [lo, hi] of the spectrum;
//   2. X (n x m) from a counter-based hash of (seed, row, column),
//      orthonormalised;
//   3. repeat: Rayleigh-Ritz (H = X^T A X, H = Q Theta Q^T, X <- X Q),
//      residual norms ||A x_i - theta_i x_i||; stop when every Ritz value
//      below zero has converged and the block's largest Ritz value is
//      positive (then no negative eigenvalue is missing from the block);
//      else filter X <- p_d(A) X with the degree-d Chebyshev polynomial that
//      damps [theta_m, hi] and grows below it (scaled at theta_1 so nothing
//      overflows), and orthonormalise X again (Cholesky QR, twice).
// The filter runs in FP32 (A's values and the blocks rounded) while the
// lowest Ritz pairs are far from converged, then in FP64 to the end
// (MRCG_EIG_FP32=0: FP64 throughout); Rayleigh-Ritz, the orthonormalisation
// and the residuals are always FP64, on FP64 blocks.  The m x m
// eigenproblems and Cholesky factorisations run on the host (m <= 64).
//
// Layout: blocks are row-major n x MP (MP = 32 or 64 >= m, padding columns
// zero), so one warp owns a row and lane j (+ 32 g) owns column j (+ 32 g).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "mrcg.h"

namespace mrcg {
namespace eig {

constexpr int kGramBlocks = 608;
// relative Ritz residual below which an FP32 filter step cannot help: its rounding
// noise, about the FP32 epsilon per step over up to 64 steps, is of that size
constexpr double kF32Floor = 1e-5;
// natural log of the largest growth an FP32 filter may apply (FP32 overflows near 3.4e38)
constexpr double kF32Growth = 60.0;

template <typename T>
struct CsrT {
  int64_t n;
  const int64_t* rowptr;
  const int32_t* col;
  const T* val;
};
using Csr = CsrT<double>;

// Y = ca * (A X) + cx * X + cp * P   (P may be null when cp == 0): one warp
// per row (the FP64 step is bound by the FP64 pipe, not by its gathers)
template <typename T, int NM>
__global__ void __launch_bounds__(kThreads) eig_cheb_kernel(CsrT<T> A, const T* __restrict__ X,
                                                           const T* __restrict__ P, T* __restrict__ Y, T ca, T cx,
                                                           T cp) {
  constexpr int MP = 32 * NM;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
  for (int64_t row = (int64_t)blockIdx.x * (kThreads / 32) + warp; row < A.n; row += nwarps) {
    const int64_t e0 = A.rowptr[row];
    const int nnz = (int)(A.rowptr[row + 1] - e0);
    T acc[NM];
#pragma unroll
    for (int g = 0; g < NM; ++g) acc[g] = 0;
    for (int base = 0; base < nnz; base += 32) {
      const bool has = lane + base < nnz;
      const T my_val = has ? A.val[e0 + base + lane] : (T)0;
      const int my_col = has ? A.col[e0 + base + lane] : 0;
      const int cnt = min(32, nnz - base);
      for (int j = 0; j < cnt; ++j) {
        const T av = __shfl_sync(0xffffffffu, my_val, j);
        const int64_t cj = (int64_t)__shfl_sync(0xffffffffu, my_col, j) * MP + lane;
#pragma unroll
        for (int g = 0; g < NM; ++g) acc[g] = fma(av, __ldg(X + cj + 32 * g), acc[g]);
      }
    }
#pragma unroll
    for (int g = 0; g < NM; ++g) {
      const int64_t idx = row * MP + lane + 32 * g;
      T y = ca * acc[g] + cx * X[idx];
      if (cp != (T)0) y += cp * P[idx];
      Y[idx] = y;
    }
  }
}

// The FP32 filter step.  Its arithmetic is light, so it is bound by the
// latency of its gathers: a warp takes 4 consecutive rows per trip; when they
// hold at most 32 entries and none more than 8 (stencil rows), one coalesced
// load brings all their values and columns and the gathers of two rows (one
// row of a 64-wide block) are in flight together; other groups take each
// row's entries 32 at a time.  Each row sums its entries in CSR order.
template <int NM>
__global__ void __launch_bounds__(kThreads) eig_cheb32_kernel(CsrT<float> A, const float* __restrict__ X,
                                                             const float* __restrict__ P, float* __restrict__ Y,
                                                             float ca, float cx, float cp) {
  constexpr int MP = 32 * NM;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
  for (int64_t r0 = ((int64_t)blockIdx.x * (kThreads / 32) + warp) * 4; r0 < A.n; r0 += nwarps * 4) {
    const int nr = (int)min((int64_t)4, A.n - r0);
    const int64_t rp = lane <= nr ? A.rowptr[r0 + lane] : 0;
    const int64_t nxt = __shfl_sync(0xffffffffu, rp, min(lane + 1, 31));
    const int len_l = lane < nr ? (int)(nxt - rp) : 0;
    const int64_t g0 = __shfl_sync(0xffffffffu, rp, 0);
    const int tot = (int)(__shfl_sync(0xffffffffu, rp, nr) - g0);
    const bool fast = tot <= 32 && __all_sync(0xffffffffu, len_l <= 8);
    // own rows of X (and P) for the 4 rows: independent of the entries
    float xo[4][NM], po[4][NM];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int g = 0; g < NM; ++g) {
        const int64_t idx = (r0 + q) * MP + 32 * g + lane;
        xo[q][g] = q < nr ? X[idx] : 0.0f;
        po[q][g] = (q < nr && cp != 0.0f) ? P[idx] : 0.0f;
      }
    float acc[4][NM];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int g = 0; g < NM; ++g) acc[q][g] = 0.0f;
    if (fast) {
      const float my_val = lane < tot ? A.val[g0 + lane] : 0.0f;
      const int my_col = lane < tot ? A.col[g0 + lane] : 0;
      constexpr int U = NM == 1 ? 2 : 1;  // rows whose gathers are in flight together
#pragma unroll
      for (int h = 0; h < 4; h += U) {
        float gx[U][8][NM];
        int len[U], st[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int q = h + u;
          st[u] = (int)(__shfl_sync(0xffffffffu, rp, q) - g0);
          len[u] = __shfl_sync(0xffffffffu, len_l, q);
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int64_t cj = (int64_t)__shfl_sync(0xffffffffu, my_col, (st[u] + j) & 31) * MP + lane;
#pragma unroll
            for (int g = 0; g < NM; ++g) gx[u][j][g] = j < len[u] ? __ldg(X + cj + 32 * g) : 0.0f;
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const float av = __shfl_sync(0xffffffffu, my_val, (st[u] + j) & 31);
            if (j < len[u])
#pragma unroll
              for (int g = 0; g < NM; ++g) acc[h + u][g] = fma(av, gx[u][j][g], acc[h + u][g]);
          }
      }
    } else {
      for (int q = 0; q < nr; ++q) {
        const int64_t e0 = __shfl_sync(0xffffffffu, rp, q);
        const int nnz = __shfl_sync(0xffffffffu, len_l, q);
        float a[NM];
#pragma unroll
        for (int g = 0; g < NM; ++g) a[g] = 0.0f;
        for (int base = 0; base < nnz; base += 32) {
          const bool has = lane + base < nnz;
          const float my_val = has ? A.val[e0 + base + lane] : 0.0f;
          const int my_col = has ? A.col[e0 + base + lane] : 0;
          const int cnt = min(32, nnz - base);
          for (int j = 0; j < cnt; ++j) {
            const float av = __shfl_sync(0xffffffffu, my_val, j);
            const int64_t cj = (int64_t)__shfl_sync(0xffffffffu, my_col, j) * MP + lane;
#pragma unroll
            for (int g = 0; g < NM; ++g) a[g] = fma(av, __ldg(X + cj + 32 * g), a[g]);
          }
        }
        // q is warp-uniform: select the accumulator row without dynamic indexing
#pragma unroll
        for (int qq = 0; qq < 4; ++qq)
          if (qq == q)
#pragma unroll
            for (int g = 0; g < NM; ++g) acc[qq][g] = a[g];
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      if (q >= nr) break;
#pragma unroll
      for (int g = 0; g < NM; ++g) {
        float y = ca * acc[q][g] + cx * xo[q][g];
        if (cp != 0.0f) y += cp * po[q][g];
        Y[(r0 + q) * MP + 32 * g + lane] = y;
      }
    }
  }
}

// y = x rounded to FP32 / widened to FP64, count elements
__global__ void __launch_bounds__(kThreads) eig_to_f32_kernel(const double* __restrict__ x, float* __restrict__ y,
                                                             int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < count; i += (int64_t)gridDim.x * kThreads)
    y[i] = (float)x[i];
}
__global__ void __launch_bounds__(kThreads) eig_to_f64_kernel(const float* __restrict__ x, double* __restrict__ y,
                                                             int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < count; i += (int64_t)gridDim.x * kThreads)
    y[i] = (double)x[i];
}

// block partials of G[jg*32 + j][lg*32 + l] = sum_rows X[row][jg*32 + j] * Y[row][lg*32 + l]
// stored as partials[(j * 32 + l) * gridDim.x + blockIdx.x]
template <int NM>
__global__ void __launch_bounds__(kThreads) eig_gram_kernel(int64_t n, const double* __restrict__ X,
                                                           const double* __restrict__ Y, int jg, int lg,
                                                           double* __restrict__ partials) {
  constexpr int MP = 32 * NM;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
  double acc[32];
#pragma unroll
  for (int l = 0; l < 32; ++l) acc[l] = 0.0;
  for (int64_t row = (int64_t)blockIdx.x * (kThreads / 32) + warp; row < n; row += nwarps) {
    const double x = X[row * MP + 32 * jg + lane];
    const double y = Y[row * MP + 32 * lg + lane];
#pragma unroll
    for (int l = 0; l < 32; ++l) acc[l] = fma(x, __shfl_sync(0xffffffffu, y, l), acc[l]);
  }
  // the warps add their 32 x 32 tiles into one shared tile in turn (fixed order)
  __shared__ double sm[32][33];
  for (int w = 0; w < kThreads / 32; ++w) {
    if (warp == w) {
#pragma unroll
      for (int l = 0; l < 32; ++l) sm[lane][l] = (w == 0 ? 0.0 : sm[lane][l]) + acc[l];
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < 32 * 32; e += kThreads) partials[(size_t)e * gridDim.x + blockIdx.x] = sm[e >> 5][e & 31];
}

// out[e] = sum over blocks of partials (fixed order), one warp per entry
__global__ void __launch_bounds__(kThreads) eig_reduce_kernel(const double* __restrict__ partials, int nblk,
                                                             int nval, double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int e = blockIdx.x * (kThreads / 32) + (threadIdx.x >> 5);
  if (e >= nval) return;
  double s = lane_sum8(partials + (size_t)e * nblk, nblk, lane);
  s = warp_sum(s);
  if (lane == 0) out[e] = s;
}

// Y[row][j] = sum_l X[row][l] * Q[l][j]  (Q: MP x MP row-major, zero outside m x m)
template <int NM>
__global__ void __launch_bounds__(kThreads) eig_rotate_kernel(int64_t n, const double* __restrict__ X,
                                                             const double* __restrict__ Q, double* __restrict__ Y) {
  constexpr int MP = 32 * NM;
  __shared__ double qs[MP * MP];
  for (int i = threadIdx.x; i < MP * MP; i += kThreads) qs[i] = Q[i];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
  for (int64_t row = (int64_t)blockIdx.x * (kThreads / 32) + warp; row < n; row += nwarps) {
    double x[NM], y[NM];
#pragma unroll
    for (int g = 0; g < NM; ++g) {
      x[g] = X[row * MP + 32 * g + lane];
      y[g] = 0.0;
    }
#pragma unroll
    for (int gl = 0; gl < NM; ++gl)
#pragma unroll 8
      for (int l = 0; l < 32; ++l) {
        const double xl = __shfl_sync(0xffffffffu, x[gl], l);
#pragma unroll
        for (int g = 0; g < NM; ++g) y[g] = fma(xl, qs[(32 * gl + l) * MP + 32 * g + lane], y[g]);
      }
#pragma unroll
    for (int g = 0; g < NM; ++g) Y[row * MP + 32 * g + lane] = y[g];
  }
}

// block partials of ||W[:, j] - theta_j X[:, j]||^2, partials[j * gridDim.x + blockIdx.x]
template <int NM>
__global__ void __launch_bounds__(kThreads) eig_resid_kernel(int64_t n, const double* __restrict__ W,
                                                            const double* __restrict__ X,
                                                            const double* __restrict__ theta,
                                                            double* __restrict__ partials) {
  constexpr int MP = 32 * NM;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kThreads) >> 5;
  double th[NM], acc[NM];
#pragma unroll
  for (int g = 0; g < NM; ++g) {
    th[g] = theta[32 * g + lane];
    acc[g] = 0.0;
  }
  for (int64_t row = (int64_t)blockIdx.x * (kThreads / 32) + warp; row < n; row += nwarps) {
#pragma unroll
    for (int g = 0; g < NM; ++g) {
      const int64_t idx = row * MP + 32 * g + lane;
      const double r = W[idx] - th[g] * X[idx];
      acc[g] = fma(r, r, acc[g]);
    }
  }
  __shared__ double sm[kThreads / 32][MP];
#pragma unroll
  for (int g = 0; g < NM; ++g) sm[warp][32 * g + lane] = acc[g];
  __syncthreads();
  for (int j = threadIdx.x; j < MP; j += kThreads) {
    double s = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) s += sm[w][j];
    partials[(size_t)j * gridDim.x + blockIdx.x] = s;
  }
}

// counter-based start block: splitmix64 of (seed, row, column) mapped to [-1, 1);
// columns m .. MP-1 are zero
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

template <int NM>
__global__ void __launch_bounds__(kThreads) eig_random_kernel(int64_t n, int m, uint64_t seed,
                                                             double* __restrict__ X) {
  constexpr int MP = 32 * NM;
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n * MP; i += (int64_t)gridDim.x * kThreads) {
    const int j = (int)(i % MP);
    const uint64_t h = splitmix64(seed ^ splitmix64((uint64_t)i));
    X[i] = j < m ? (double)(h >> 11) * (2.0 / 9007199254740992.0) - 1.0 : 0.0;
  }
}

// column-major n x k output from columns 0..k-1 of the row-major block
template <int NM>
__global__ void __launch_bounds__(kThreads) eig_extract_kernel(int64_t n, int k, const double* __restrict__ X,
                                                              double* __restrict__ V) {
  constexpr int MP = 32 * NM;
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n * k; i += (int64_t)gridDim.x * kThreads) {
    const int64_t j = i / n, row = i % n;
    V[i] = X[row * MP + j];
  }
}

// ------------------------------------------------------------------ host linear algebra (m <= 64)

// Jacobi eigenvalue iteration (cyclic, with the classical rotation angle) on
// a symmetric m x m matrix H (row-major, overwritten); eigenvalues ascending
// in w, eigenvectors as the columns of Q (row-major m x m).
void sym_eig(int m, std::vector<double>& H, std::vector<double>& w, std::vector<double>& Q) {
  Q.assign((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i) Q[(size_t)i * m + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) {
        const double h = H[(size_t)i * m + j];
        tot += h * h;
        if (i != j) off += h * h;
      }
    if (off <= 1e-32 * tot || off == 0.0) break;
    for (int p = 0; p < m - 1; ++p)
      for (int q = p + 1; q < m; ++q) {
        const double apq = H[(size_t)p * m + q];
        if (apq == 0.0) continue;
        const double app = H[(size_t)p * m + p], aqq = H[(size_t)q * m + q];
        const double theta = (aqq - app) / (2.0 * apq);
        const double t = (theta >= 0.0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < m; ++k) {  // columns p, q of H
          const double hkp = H[(size_t)k * m + p], hkq = H[(size_t)k * m + q];
          H[(size_t)k * m + p] = c * hkp - s * hkq;
          H[(size_t)k * m + q] = s * hkp + c * hkq;
        }
        for (int k = 0; k < m; ++k) {  // rows p, q
          const double hpk = H[(size_t)p * m + k], hqk = H[(size_t)q * m + k];
          H[(size_t)p * m + k] = c * hpk - s * hqk;
          H[(size_t)q * m + k] = s * hpk + c * hqk;
        }
        for (int k = 0; k < m; ++k) {
          const double qkp = Q[(size_t)k * m + p], qkq = Q[(size_t)k * m + q];
          Q[(size_t)k * m + p] = c * qkp - s * qkq;
          Q[(size_t)k * m + q] = s * qkp + c * qkq;
        }
      }
  }
  // sort ascending
  std::vector<int> idx(m);
  for (int i = 0; i < m; ++i) idx[i] = i;
  std::sort(idx.begin(), idx.end(), [&](int a, int b) { return H[(size_t)a * m + a] < H[(size_t)b * m + b]; });
  std::vector<double> Qs((size_t)m * m);
  w.resize(m);
  for (int j = 0; j < m; ++j) {
    w[j] = H[(size_t)idx[j] * m + idx[j]];
    for (int i = 0; i < m; ++i) Qs[(size_t)i * m + j] = Q[(size_t)i * m + idx[j]];
  }
  Q.swap(Qs);
}

// upper-triangular R with G = R^T R (G symmetric positive definite, m x m
// row-major); false when a pivot is not positive
bool cholesky_upper(int m, const std::vector<double>& G, std::vector<double>& R) {
  R.assign((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i) {
    double d = G[(size_t)i * m + i];
    for (int k = 0; k < i; ++k) d -= R[(size_t)k * m + i] * R[(size_t)k * m + i];
    if (!(d > 0.0)) return false;
    const double rii = std::sqrt(d);
    R[(size_t)i * m + i] = rii;
    for (int j = i + 1; j < m; ++j) {
      double s = G[(size_t)i * m + j];
      for (int k = 0; k < i; ++k) s -= R[(size_t)k * m + i] * R[(size_t)k * m + j];
      R[(size_t)i * m + j] = s / rii;
    }
  }
  return true;
}

// inverse of an upper-triangular m x m matrix (row-major)
void upper_inverse(int m, const std::vector<double>& R, std::vector<double>& Ri) {
  Ri.assign((size_t)m * m, 0.0);
  for (int j = 0; j < m; ++j) {
    Ri[(size_t)j * m + j] = 1.0 / R[(size_t)j * m + j];
    for (int i = j - 1; i >= 0; --i) {
      double s = 0.0;
      for (int k = i + 1; k <= j; ++k) s += R[(size_t)i * m + k] * Ri[(size_t)k * m + j];
      Ri[(size_t)i * m + j] = -s / R[(size_t)i * m + i];
    }
  }
}

struct Ctx {
  cudaStream_t s = nullptr;
  int64_t n = 0;
  int m = 0, mp = 0, nm = 1, grid = 1, nblk_gram = kGramBlocks;
  Csr A{};
  double *X = nullptr, *Y = nullptr, *Z = nullptr, *W = nullptr, *Qd = nullptr, *partials = nullptr, *small = nullptr,
         *theta = nullptr;
  // FP32 filter steps (the early ones): A's values and three blocks in FP32
  bool mixed = false;
  CsrT<float> Af{};
  float *Xf = nullptr, *Yf = nullptr, *Zf = nullptr;
  std::vector<void*> allocs;
  long long spmv_blocks = 0;
};

#define ECK(call)                                                                            \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) {                                                                 \
      if (getenv("MRCG_DEBUG")) fprintf(stderr, "mrcg eig: %s failed: %s (%s:%d)\n", #call, \
                                        cudaGetErrorString(e_), __FILE__, __LINE__);        \
      return e_ == cudaErrorMemoryAllocation ? MRCG_ERR_OOM : MRCG_ERR_CUDA;                \
    }                                                                                        \
  } while (0)

template <typename T>
mrcg_status ealloc(Ctx& c, T** p, size_t count) {
  void* q = nullptr;
  if (cudaMalloc(&q, std::max<size_t>(count * sizeof(T), 256)) != cudaSuccess) {
    cudaGetLastError();
    return MRCG_ERR_OOM;
  }
  c.allocs.push_back(q);
  *p = reinterpret_cast<T*>(q);
  return MRCG_OK;
}

// Y = ca A X + cx X + cp P
mrcg_status cheb(Ctx& c, const double* X, const double* P, double* Y, double ca, double cx, double cp) {
  if (c.nm == 1) eig_cheb_kernel<double, 1><<<c.grid, kThreads, 0, c.s>>>(c.A, X, P, Y, ca, cx, cp);
  else eig_cheb_kernel<double, 2><<<c.grid, kThreads, 0, c.s>>>(c.A, X, P, Y, ca, cx, cp);
  ECK(cudaGetLastError());
  ++c.spmv_blocks;
  return MRCG_OK;
}

// the same step in FP32 (coefficients rounded to FP32)
mrcg_status cheb32(Ctx& c, const float* X, const float* P, float* Y, double ca, double cx, double cp) {
  if (c.nm == 1)
    eig_cheb32_kernel<1><<<c.grid, kThreads, 0, c.s>>>(c.Af, X, P, Y, (float)ca, (float)cx, (float)cp);
  else
    eig_cheb32_kernel<2><<<c.grid, kThreads, 0, c.s>>>(c.Af, X, P, Y, (float)ca, (float)cx, (float)cp);
  ECK(cudaGetLastError());
  ++c.spmv_blocks;
  return MRCG_OK;
}

// G (m x m, host, row-major) = X^T Y
mrcg_status gram(Ctx& c, const double* X, const double* Y, std::vector<double>& G) {
  std::vector<double> tile(32 * 32);
  G.assign((size_t)c.m * c.m, 0.0);
  for (int jg = 0; jg < c.nm; ++jg)
    for (int lg = 0; lg < c.nm; ++lg) {
      if (32 * jg >= c.m || 32 * lg >= c.m) continue;
      if (c.nm == 1) eig_gram_kernel<1><<<c.nblk_gram, kThreads, 0, c.s>>>(c.n, X, Y, jg, lg, c.partials);
      else eig_gram_kernel<2><<<c.nblk_gram, kThreads, 0, c.s>>>(c.n, X, Y, jg, lg, c.partials);
      eig_reduce_kernel<<<(32 * 32 + kThreads / 32 - 1) / (kThreads / 32), kThreads, 0, c.s>>>(c.partials,
                                                                                               c.nblk_gram, 32 * 32,
                                                                                               c.small);
      ECK(cudaGetLastError());
      ECK(cudaMemcpyAsync(tile.data(), c.small, 32 * 32 * sizeof(double), cudaMemcpyDeviceToHost, c.s));
      ECK(cudaStreamSynchronize(c.s));
      for (int j = 0; j < 32; ++j)
        for (int l = 0; l < 32; ++l) {
          const int gj = 32 * jg + j, gl = 32 * lg + l;
          if (gj < c.m && gl < c.m) G[(size_t)gj * c.m + gl] = tile[(size_t)j * 32 + l];
        }
    }
  return MRCG_OK;
}

// Y = X Q with Q (m x m host, row-major) padded to MP x MP
mrcg_status rotate(Ctx& c, const double* X, const std::vector<double>& Q, double* Y) {
  std::vector<double> qp((size_t)c.mp * c.mp, 0.0);
  for (int i = 0; i < c.m; ++i)
    for (int j = 0; j < c.m; ++j) qp[(size_t)i * c.mp + j] = Q[(size_t)i * c.m + j];
  ECK(cudaMemcpyAsync(c.Qd, qp.data(), qp.size() * sizeof(double), cudaMemcpyHostToDevice, c.s));
  if (c.nm == 1) eig_rotate_kernel<1><<<c.grid, kThreads, 0, c.s>>>(c.n, X, c.Qd, Y);
  else eig_rotate_kernel<2><<<c.grid, kThreads, 0, c.s>>>(c.n, X, c.Qd, Y);
  ECK(cudaGetLastError());
  ECK(cudaStreamSynchronize(c.s));  // qp is reused by the next call
  return MRCG_OK;
}

// X <- X R^{-1} with X^T X = R^T R, twice (Cholesky QR 2); uses Y as scratch
mrcg_status orthonormalise(Ctx& c) {
  for (int pass = 0; pass < 2; ++pass) {
    std::vector<double> G, R, Ri;
    mrcg_status st = gram(c, c.X, c.X, G);
    if (st != MRCG_OK) return st;
    if (!cholesky_upper(c.m, G, R)) return MRCG_ERR_BREAKDOWN;  // the block lost rank
    upper_inverse(c.m, R, Ri);
    if ((st = rotate(c, c.X, Ri, c.Y)) != MRCG_OK) return st;
    std::swap(c.X, c.Y);
  }
  return MRCG_OK;
}

// Rayleigh-Ritz on the orthonormal block X: theta (ascending), X <- X Q,
// W <- A X, res[j] = ||A x_j - theta_j x_j||
mrcg_status rayleigh_ritz(Ctx& c, std::vector<double>& theta, std::vector<double>& res) {
  mrcg_status st = cheb(c, c.X, nullptr, c.W, 1.0, 0.0, 0.0);
  if (st != MRCG_OK) return st;
  std::vector<double> H, Q;
  if ((st = gram(c, c.X, c.W, H)) != MRCG_OK) return st;
  for (int i = 0; i < c.m; ++i)  // symmetrise the rounding
    for (int j = i + 1; j < c.m; ++j) {
      const double h = 0.5 * (H[(size_t)i * c.m + j] + H[(size_t)j * c.m + i]);
      H[(size_t)i * c.m + j] = H[(size_t)j * c.m + i] = h;
    }
  sym_eig(c.m, H, theta, Q);
  if ((st = rotate(c, c.X, Q, c.Y)) != MRCG_OK) return st;
  std::swap(c.X, c.Y);
  if ((st = rotate(c, c.W, Q, c.Y)) != MRCG_OK) return st;
  std::swap(c.W, c.Y);
  std::vector<double> th((size_t)c.mp, 0.0);
  for (int j = 0; j < c.m; ++j) th[j] = theta[j];
  ECK(cudaMemcpyAsync(c.theta, th.data(), th.size() * sizeof(double), cudaMemcpyHostToDevice, c.s));
  if (c.nm == 1) eig_resid_kernel<1><<<c.nblk_gram, kThreads, 0, c.s>>>(c.n, c.W, c.X, c.theta, c.partials);
  else eig_resid_kernel<2><<<c.nblk_gram, kThreads, 0, c.s>>>(c.n, c.W, c.X, c.theta, c.partials);
  eig_reduce_kernel<<<(c.mp + kThreads / 32 - 1) / (kThreads / 32), kThreads, 0, c.s>>>(c.partials, c.nblk_gram,
                                                                                       c.mp, c.small);
  ECK(cudaGetLastError());
  res.assign((size_t)c.mp, 0.0);
  ECK(cudaMemcpyAsync(res.data(), c.small, c.mp * sizeof(double), cudaMemcpyDeviceToHost, c.s));
  ECK(cudaStreamSynchronize(c.s));
  res.resize(c.m);
  for (double& r : res) r = std::sqrt(std::max(r, 0.0));
  return MRCG_OK;
}

// X <- p_d(A) X: the Chebyshev polynomial of degree d on [a, b] (|p| <= 1 there
// after scaling), scaled so that p_d(a0) = 1 (a0 < a, the lowest Ritz value)
mrcg_status filter(Ctx& c, int d, double a, double b, double a0, bool f32) {
  const double e = 0.5 * (b - a), ctr = 0.5 * (b + a);
  double sigma = e / (ctr - a0);
  const double tau = 2.0 / sigma;
  if (f32) {
    // the same recurrence on FP32 copies; the result is widened back into X
    const int64_t cnt = c.n * c.mp;
    float *x = c.Xf, *y = c.Yf, *z = c.Zf;
    eig_to_f32_kernel<<<c.grid, kThreads, 0, c.s>>>(c.X, x, cnt);
    ECK(cudaGetLastError());
    mrcg_status st = cheb32(c, x, nullptr, y, sigma / e, -ctr * sigma / e, 0.0);
    if (st != MRCG_OK) return st;
    for (int i = 2; i <= d; ++i) {
      const double sn = 1.0 / (tau - sigma);
      if ((st = cheb32(c, y, x, z, 2.0 * sn / e, -2.0 * ctr * sn / e, -sigma * sn)) != MRCG_OK) return st;
      float* t = x;
      x = y;
      y = z;
      z = t;
      sigma = sn;
    }
    eig_to_f64_kernel<<<c.grid, kThreads, 0, c.s>>>(y, c.X, cnt);
    ECK(cudaGetLastError());
    return MRCG_OK;
  }
  // Y = (A X - ctr X) sigma / e
  mrcg_status st = cheb(c, c.X, nullptr, c.Y, sigma / e, -ctr * sigma / e, 0.0);
  if (st != MRCG_OK) return st;
  for (int i = 2; i <= d; ++i) {
    const double sn = 1.0 / (tau - sigma);
    // Z = (A Y - ctr Y) 2 sn / e - sigma sn X
    if ((st = cheb(c, c.Y, c.X, c.Z, 2.0 * sn / e, -2.0 * ctr * sn / e, -sigma * sn)) != MRCG_OK) return st;
    double* t = c.X;
    c.X = c.Y;
    c.Y = c.Z;
    c.Z = t;
    sigma = sn;
  }
  std::swap(c.X, c.Y);
  return MRCG_OK;
}

}  // namespace eig
}  // namespace mrcg

using namespace mrcg;
using namespace mrcg::eig;

namespace {

bool e_is_device(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

template <typename T>
mrcg_status e_fetch(const T* src, size_t count, std::vector<T>& dst) {
  dst.resize(count);
  if (!count) return MRCG_OK;
  if (e_is_device(src)) ECK(cudaMemcpy(dst.data(), src, count * sizeof(T), cudaMemcpyDeviceToHost));
  else std::memcpy(dst.data(), src, count * sizeof(T));
  return MRCG_OK;
}

mrcg_status run(Ctx& c, const std::vector<int64_t>& rp, const std::vector<int32_t>& ci, const std::vector<double>& va,
                double tol, int64_t max_spmv, uint64_t seed, int32_t* k_out, double* V_out, double* lam_out,
                mrcg_eig_info* info) {
  const int64_t n = c.n;
  // Gershgorin bounds of the spectrum
  double lo = 1e300, hi = -1e300;
  for (int64_t i = 0; i < n; ++i) {
    double d = 0.0, off = 0.0;
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      if (ci[p] == i) d += va[p];
      else off += std::fabs(va[p]);
    }
    lo = std::min(lo, d - off);
    hi = std::max(hi, d + off);
  }
  const double anorm = std::max(std::fabs(lo), std::fabs(hi));
  int64_t* d_rp = nullptr;
  int32_t* d_ci = nullptr;
  double* d_va = nullptr;
  mrcg_status st;
  if ((st = ealloc(c, &d_rp, rp.size())) != MRCG_OK) return st;
  if ((st = ealloc(c, &d_ci, ci.size())) != MRCG_OK) return st;
  if ((st = ealloc(c, &d_va, va.size())) != MRCG_OK) return st;
  ECK(cudaMemcpyAsync(d_rp, rp.data(), rp.size() * sizeof(int64_t), cudaMemcpyHostToDevice, c.s));
  if (!ci.empty()) {
    ECK(cudaMemcpyAsync(d_ci, ci.data(), ci.size() * sizeof(int32_t), cudaMemcpyHostToDevice, c.s));
    ECK(cudaMemcpyAsync(d_va, va.data(), va.size() * sizeof(double), cudaMemcpyHostToDevice, c.s));
  }
  c.A = {n, d_rp, d_ci, d_va};
  const size_t blk = (size_t)n * c.mp;
  for (double** p : {&c.X, &c.Y, &c.Z, &c.W})
    if ((st = ealloc(c, p, blk)) != MRCG_OK) return st;
  if ((st = ealloc(c, &c.Qd, (size_t)c.mp * c.mp)) != MRCG_OK) return st;
  if ((st = ealloc(c, &c.partials, (size_t)32 * 32 * c.nblk_gram)) != MRCG_OK) return st;
  if ((st = ealloc(c, &c.small, (size_t)32 * 32)) != MRCG_OK) return st;
  if ((st = ealloc(c, &c.theta, (size_t)c.mp)) != MRCG_OK) return st;
  {
    const char* e = getenv("MRCG_EIG_FP32");
    c.mixed = !(e && atoi(e) == 0);
  }
  if (c.mixed) {
    float* d_vaf = nullptr;
    if ((st = ealloc(c, &d_vaf, va.size())) != MRCG_OK) return st;
    for (float** p : {&c.Xf, &c.Yf, &c.Zf})
      if ((st = ealloc(c, p, blk)) != MRCG_OK) return st;
    if (!va.empty()) eig_to_f32_kernel<<<c.grid, kThreads, 0, c.s>>>(d_va, d_vaf, (int64_t)va.size());
    ECK(cudaGetLastError());
    c.Af = {n, d_rp, d_ci, d_vaf};
  }
  if (c.nm == 1) eig_random_kernel<1><<<c.grid, kThreads, 0, c.s>>>(n, c.m, seed, c.X);
  else eig_random_kernel<2><<<c.grid, kThreads, 0, c.s>>>(n, c.m, seed, c.X);
  ECK(cudaGetLastError());
  if ((st = orthonormalise(c)) != MRCG_OK) return st;

  std::vector<double> theta, res;
  int degree = 8;
  int rr_steps = 0;
  bool f32 = c.mixed;  // FP32 filters until the leading Ritz pairs reach FP32's floor, then FP64 to the end
  bool converged = false;
  int kneg = 0;
  double maxres = 0.0;
  for (;;) {
    if ((st = rayleigh_ritz(c, theta, res)) != MRCG_OK) return st;
    ++rr_steps;
    kneg = 0;
    while (kneg < c.m && theta[kneg] < 0.0) ++kneg;
    maxres = 0.0;
    bool all = true;
    for (int j = 0; j < kneg; ++j) {
      maxres = std::max(maxres, res[j]);
      if (!(res[j] <= tol * anorm)) all = false;
    }
    // the block must hold a nonnegative Ritz value, and the first of them must
    // have settled too (to sqrt(tol)): the Ritz values bound the eigenvalues
    // from above, so a negative eigenvalue missing from the block would keep
    // that pair from converging
    if (all && kneg < c.m && std::isfinite(maxres) && res[kneg] <= std::sqrt(tol) * anorm) {
      converged = true;
      break;
    }
    if (c.spmv_blocks >= max_spmv) break;
    for (double t : theta)
      if (!std::isfinite(t)) return MRCG_ERR_NONFINITE;
    // damp [theta_m, hi], grow everything below theta_m; scale at theta_1
    const double b = hi + 1e-12 * anorm;
    const double a = std::min(theta[c.m - 1], b - 1e-6 * anorm);
    const double a0 = std::min(theta[0], a - 1e-9 * anorm);
    if (f32) {
      double lead = 0.0;  // the residuals of the negative Ritz pairs (at least the lowest pair)
      for (int j = 0; j < std::max(kneg, 1); ++j) lead = std::max(lead, res[j]);
      if (!(lead > kF32Floor * anorm)) {
        // the FP64 steps start again from a low degree: a degree-64 filter on
        // a block whose wanted pairs are already this close makes the block
        // too ill-conditioned for the Cholesky QR that follows
        f32 = false;
        degree = 8;
      }
    }
    // an FP32 filter must not overflow: below a0 the scaled polynomial grows
    // like exp(d (acosh t(lambda) - acosh t(a0))), largest at the Gershgorin
    // bound lo; beyond about 1e26 this filter runs in FP64
    bool use32 = f32;
    if (use32) {
      const double e = 0.5 * (b - a), ctr = 0.5 * (b + a);
      auto ach = [](double t) { return t <= 1.0 ? 0.0 : std::log(t + std::sqrt(t * t - 1.0)); };
      const double growth = degree * (ach((ctr - std::min(lo, a0)) / e) - ach((ctr - a0) / e));
      use32 = std::isfinite(growth) && growth < kF32Growth;
    }
    if ((st = filter(c, degree, a, b, a0, use32)) != MRCG_OK) return st;
    if ((st = orthonormalise(c)) != MRCG_OK) return st;
    degree = std::min(degree * 2, 64);
  }
  if (info) {
    info->rayleigh_ritz_steps = rr_steps;
    info->block_spmvs = c.spmv_blocks;
    info->max_residual = maxres;
    info->spectrum_lo = lo;
    info->spectrum_hi = hi;
    info->negative_found = kneg;
  }
  if (!converged) return MRCG_ERR_MAXITER;
  *k_out = kneg;
  if (kneg > 0) {
    double* Vd = nullptr;
    const bool vdev = e_is_device(V_out);
    if (vdev) {
      Vd = V_out;
    } else if ((st = ealloc(c, &Vd, (size_t)n * kneg)) != MRCG_OK) {
      return st;
    }
    if (c.nm == 1) eig_extract_kernel<1><<<c.grid, kThreads, 0, c.s>>>(n, kneg, c.X, Vd);
    else eig_extract_kernel<2><<<c.grid, kThreads, 0, c.s>>>(n, kneg, c.X, Vd);
    ECK(cudaGetLastError());
    if (!vdev) ECK(cudaMemcpyAsync(V_out, Vd, (size_t)n * kneg * sizeof(double), cudaMemcpyDeviceToHost, c.s));
    ECK(cudaStreamSynchronize(c.s));
    if (e_is_device(lam_out)) ECK(cudaMemcpy(lam_out, theta.data(), kneg * sizeof(double), cudaMemcpyHostToDevice));
    else std::memcpy(lam_out, theta.data(), kneg * sizeof(double));
  }
  return MRCG_OK;
}

}  // namespace

extern "C" mrcg_status mrcg_negative_eigenpairs(int64_t n, const int64_t* rowptr, const int32_t* colind,
                                                const double* val, int32_t block, double tol, int64_t max_spmv,
                                                uint64_t seed, int32_t* k, double* V, double* lambda,
                                                mrcg_eig_info* info) {
  if (info) std::memset(info, 0, sizeof(*info));
  if (n < 1 || n > (int64_t)0x7fffff00 || !rowptr || !k || !V || !lambda) return MRCG_ERR_INVALID;
  if (block < 2 || block > 64 || block > n || !(tol > 0.0) || max_spmv < 1) return MRCG_ERR_INVALID;
  const auto t0 = std::chrono::steady_clock::now();
  std::vector<int64_t> rp;
  std::vector<int32_t> ci;
  std::vector<double> va;
  mrcg_status st = e_fetch(rowptr, (size_t)n + 1, rp);
  if (st != MRCG_OK) return st;
  if (rp[0] != 0) return MRCG_ERR_INVALID;
  for (int64_t i = 0; i < n; ++i)
    if (rp[i + 1] < rp[i]) return MRCG_ERR_INVALID;
  const int64_t nnz = rp[n];
  if (nnz > 0 && (!colind || !val)) return MRCG_ERR_INVALID;
  if ((st = e_fetch(colind, (size_t)nnz, ci)) != MRCG_OK) return st;
  if ((st = e_fetch(val, (size_t)nnz, va)) != MRCG_OK) return st;
  for (int64_t p = 0; p < nnz; ++p) {
    if (ci[p] < 0 || ci[p] >= n) return MRCG_ERR_INVALID;
    if (!std::isfinite(va[p])) return MRCG_ERR_NONFINITE;
  }
  Ctx c;
  c.n = n;
  c.m = block;
  c.mp = block <= 32 ? 32 : 64;
  c.nm = c.mp / 32;
  int dev = 0, nsm = 1;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return MRCG_ERR_CUDA;
  c.grid = nsm * 4;
  if (cudaStreamCreateWithFlags(&c.s, cudaStreamNonBlocking) != cudaSuccess) return MRCG_ERR_CUDA;
  st = run(c, rp, ci, va, tol, max_spmv, seed, k, V, lambda, info);
  cudaStreamSynchronize(c.s);
  for (void* p : c.allocs) cudaFree(p);
  cudaStreamDestroy(c.s);
  cudaGetLastError();
  if (info) {
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    info->status = st;
  }
  return st;
}
