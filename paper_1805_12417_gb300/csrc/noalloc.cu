// Allocation-free M_mr product for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code that runs inside another
// framework's memory pool with a fixed budget, plugins whose host forbids
// allocations after start-up, or paths that must not take the allocator's
// locks or synchronisation.  For them mrcg_mmr_apply_noalloc computes
//     out = A u + 2 V (|Lambda| (V^T u))
// straight from the caller's device CSR arrays, using as its only scratch the
// fixed array below (no handle, no cudaMalloc/cudaFree, no library routine
// that allocates).
//
// Scratch: kNaBlocks block partials of up to kMaxK values, the k reduced
// coefficients and one ticket counter -- 262,656 bytes, held by every GPU that
// loads this library until the process exits.  The grid is fixed at
// kNaBlocks blocks and rows are covered by grid-stride loops, so n is not
// limited by the scratch; k is (k <= 32).
#include <mutex>

#include "common.cuh"
#include "mrcg.h"

namespace mrcg {
namespace {

constexpr int kNaBlocks = 1024;

struct NaScratch {
  double partials[kMaxK * kNaBlocks];  // value-major: [value][block]
  double c[kMaxK];                     // 2 |lambda_j| (V^T u)_j
  unsigned int ticket;                 // must be 0 when a call starts
  unsigned int pad[63];
};

static __device__ __align__(256) NaScratch g_na_scratch;

// Device address of g_na_scratch, looked up once per CUDA context.  The
// address belongs to the module instance loaded in one context: after a
// cudaDeviceReset, or in another context on the same device, the module is
// loaded again and the array may sit elsewhere.  So the cache is keyed by the
// context's process-unique id (cuCtxGetId), not by the device ordinal, and a
// new context gets its own lookup.  The two driver calls are reached through
// the runtime's entry-point query, so the library does not link libcuda.
constexpr int kNaMaxContexts = 64;
struct NaEntry {
  unsigned long long ctx_id;
  NaScratch* ptr;
};
NaEntry g_na_cache[kNaMaxContexts] = {};
int g_na_count = 0;
std::mutex g_na_mutex;

typedef int (*CtxGetCurrentFn)(void** ctx);
typedef int (*CtxGetIdFn)(void* ctx, unsigned long long* id);

// id of the calling thread's current context; false when there is none (yet)
bool current_context_id(unsigned long long* id) {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool tried = false;
  if (!tried) {  // under g_na_mutex
    tried = true;
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
        q2 == cudaDriverEntryPointSuccess) {
      get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
      get_id = reinterpret_cast<CtxGetIdFn>(f2);
    }
    cudaGetLastError();
  }
  if (!get_current || !get_id) return false;
  void* ctx = nullptr;
  if (get_current(&ctx) != 0 || !ctx) return false;
  return get_id(ctx, id) == 0;
}

// set-up of the current context: the symbol's device address, cached per context
mrcg_status scratch_address(NaScratch** out) {
  std::lock_guard<std::mutex> lock(g_na_mutex);
  unsigned long long id = 0;
  if (current_context_id(&id)) {
    for (int i = 0; i < g_na_count; ++i)
      if (g_na_cache[i].ctx_id == id) {
        *out = g_na_cache[i].ptr;
        return MRCG_OK;
      }
  }
  // first call in this context (this also creates the device's primary
  // context when none is current yet)
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_na_scratch) != cudaSuccess || !p) {
    cudaGetLastError();
    return MRCG_ERR_CUDA;
  }
  *out = reinterpret_cast<NaScratch*>(p);
  if (current_context_id(&id)) {
    if (g_na_count < kNaMaxContexts) {
      g_na_cache[g_na_count++] = {id, *out};
    } else {  // many contexts over the process lifetime: recycle the oldest slot
      for (int i = 1; i < kNaMaxContexts; ++i) g_na_cache[i - 1] = g_na_cache[i];
      g_na_cache[kNaMaxContexts - 1] = {id, *out};
    }
  }
  // without a context id nothing is cached: the lookup then runs on every call
  return MRCG_OK;
}

__global__ void __launch_bounds__(kThreads) na_vtu_kernel(NaScratch* sc, int64_t n, int k,
                                                            const double* __restrict__ V,
                                                            const double* __restrict__ lambda,
                                                            const double* __restrict__ u) {
  double acc[kMaxK];
#pragma unroll
  for (int l = 0; l < kMaxK; ++l) acc[l] = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
    const double ui = u[i];
#pragma unroll
    for (int l = 0; l < kMaxK; ++l)
      if (l < k) acc[l] += V[(size_t)l * n + i] * ui;
  }
  block_partials<kMaxK>(acc, k, sc->partials);
  if (last_block(&sc->ticket)) {
    __shared__ double tot[kMaxK];
    final_sums(sc->partials, k, tot);
    if (threadIdx.x < k) sc->c[threadIdx.x] = 2.0 * fabs(lambda[threadIdx.x]) * tot[threadIdx.x];
  }
}

// one thread per row: entries in stored order, then the low-rank term
__global__ void __launch_bounds__(kThreads) na_csr_mmr_kernel(const NaScratch* sc, int64_t n, int k,
                                                                const int64_t* __restrict__ rowptr,
                                                                const int32_t* __restrict__ colind,
                                                                const double* __restrict__ val,
                                                                const double* __restrict__ V,
                                                                const double* __restrict__ u,
                                                                double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads) {
    double acc = 0.0;
    for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) acc += val[p] * __ldg(u + colind[p]);
    for (int l = 0; l < k; ++l) acc += V[(size_t)l * n + i] * sc->c[l];
    out[i] = acc;
  }
}

}  // namespace
}  // namespace mrcg

using namespace mrcg;

extern "C" mrcg_status mrcg_mmr_apply_noalloc(int64_t n, const int64_t* rowptr, const int32_t* colind,
                                              const double* val, int32_t k, const double* V,
                                              const double* lambda, const double* u, double* out, void* stream) {
  if (n < 1 || n > (int64_t)0x7fffffff || k < 0 || k > kMaxK) return MRCG_ERR_INVALID;
  if (!rowptr || !val || !colind || !u || !out || (k > 0 && (!V || !lambda))) return MRCG_ERR_INVALID;
  NaScratch* sc = nullptr;
  if (const mrcg_status st = scratch_address(&sc); st != MRCG_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  // the ticket must start at zero; the partials and c are overwritten in full
  if (cudaMemsetAsync(&sc->ticket, 0, sizeof(unsigned int), s) != cudaSuccess) return MRCG_ERR_CUDA;
  if (k > 0) na_vtu_kernel<<<kNaBlocks, kThreads, 0, s>>>(sc, n, k, V, lambda, u);
  na_csr_mmr_kernel<<<kNaBlocks, kThreads, 0, s>>>(sc, n, k, rowptr, colind, val, V, u, out);
  if (cudaGetLastError() != cudaSuccess) return MRCG_ERR_CUDA;
  return MRCG_OK;
}
