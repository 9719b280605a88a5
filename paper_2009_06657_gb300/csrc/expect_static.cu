#include <mutex>

#include "common.cuh"
#include "kernels.h"
#include "lret.h"

// ---------------------------------------------------------------------------
// Allocation-free variant of the Pauli-sum expectation (lr_expect_static).
//
// Some callers cannot allocate device memory at the time they need a readout:
// a serving loop that has reserved all device memory up front for its own pool,
// or a host thread that must not take the implicit device synchronisation that
// cudaMalloc / cudaFree imply. This entry point reads a caller-owned device
// state and keeps its scratch (term masks and per-block partial sums) in a
// fixed array below, which every GPU that loads this library holds until the
// process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr int kStaticMaxTerms = LR_STATIC_MAX_TERMS;
constexpr int kStaticMaxBlocks = lret::kReadoutMaxBlocks;  // launch_pauli_expect never uses more
// layout (doubles): [xmask T][zmask T][out T][partials T * blocks]
constexpr size_t kStaticDoubles = (size_t)kStaticMaxTerms * (3 + kStaticMaxBlocks);

static __device__ __align__(256) double g_expect_scratch[kStaticDoubles];

std::mutex g_static_mu;
double* g_static_ptr[64] = {nullptr};  // device address of g_expect_scratch, per device

// Device address of the scratch array on the current device (looked up once
// per device; host code cannot use the symbol itself as a device pointer).
int static_scratch(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return LR_ECUDA;
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_expect_scratch) != cudaSuccess || !p) return LR_ECUDA;
    g_static_ptr[dev] = (double*)p;
  }
  *out = g_static_ptr[dev];
  return LR_OK;
}

}  // namespace

extern "C" int lr_expect_static(const void* V_dev, int n, int c, int ld, int dtype, int T,
                                const uint64_t* xmask, const uint64_t* zmask, const double* coeff,
                                double* out_host, void* stream) {
  if (!V_dev || !out_host || n < 1 || n > 30 || c < 1 || ld < c || T < 0 ||
      (dtype != LR_C64 && dtype != LR_C128) || (T > 0 && (!xmask || !zmask || !coeff)))
    return LR_EINVAL;
  if (T > kStaticMaxTerms) return LR_ECAPACITY;  // more terms than the fixed scratch holds
  if (T == 0) {
    *out_host = 0.0;
    return LR_OK;
  }
  const uint64_t lim = (1ull << n) - 1ull;
  for (int t = 0; t < T; ++t)
    if ((xmask[t] & ~lim) || (zmask[t] & ~lim)) return LR_EINVAL;
  double* base = nullptr;
  int rc = static_scratch(&base);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  uint64_t* dxm = (uint64_t*)base;
  uint64_t* dzm = dxm + T;
  double* dout = base + 2 * (size_t)T;
  double* part = base + 3 * (size_t)T;  // every block writes its own slot: nothing to clear
  const int64_t N = 1ll << n;
  if (cudaMemcpyAsync(dxm, xmask, sizeof(uint64_t) * T, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(dzm, zmask, sizeof(uint64_t) * T, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return LR_ECUDA;
  cudaError_t e = dtype == LR_C64
                      ? lret::launch_pauli_expect<float>(V_dev, N, c, ld, T, dxm, dzm, part, dout, s)
                      : lret::launch_pauli_expect<double>(V_dev, N, c, ld, T, dxm, dzm, part, dout, s);
  if (e != cudaSuccess) return LR_ECUDA;
  double vals[kStaticMaxTerms];
  if (cudaMemcpyAsync(vals, dout, sizeof(double) * T, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return LR_ECUDA;
  double acc = 0.0;
  for (int t = 0; t < T; ++t) acc += coeff[t] * vals[t];
  *out_host = acc;
  return LR_OK;
}
