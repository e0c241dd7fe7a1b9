// Mirror-descent update that allocates no device memory.
//
// Some callers cannot call cudaMalloc: code that runs while a CUDA graph is being captured
// (an allocation there would break or serialise the capture), inference servers and
// embedded runtimes that hand every byte of device memory to their own pool at start-up,
// and plug-in hosts that forbid a library from growing the device footprint behind their
// back.  For them, firal_md_step_static() performs the same update as firal_md_step()
// (z <- z exp(-beta g), z <- budget z / sum(z), beta = beta0 / ||g||_inf) using only the
// caller's z and g plus a fixed scratch array that lives in this file for the life of the
// process.
//
// Scratch: kStaticSlots doubles per partial (block maxima and block sums), 2 * 4096 doubles =
// 64 KiB in total, resident on every GPU that loads this library.  One block reduces
// kStaticChunk = 4096 elements, so n is limited to 4096 * 4096 = 16,777,216.  Every slot a
// call reads is written earlier in the same call, so nothing needs clearing between calls;
// the array keeps the last call's values.  Calls whose kernels overlap on the GPU (for
// example on two streams at once) share the array and race.
#include <mutex>

#include "firal_internal.cuh"

namespace firal {
namespace {

constexpr int kStaticChunk = 4096;   // elements per block
constexpr int kStaticSlots = 4096;   // partial slots per reduction
constexpr int kThreads = 256;

__device__ __align__(256) double g_md_scratch[2 * kStaticSlots];

std::mutex g_scratch_mu;
void* g_scratch_addr[128] = {};

// Device address of g_md_scratch on the current device (looked up once per device).
int32_t scratch_address(double** out) {
  int dev = 0;
  FIRAL_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 128) return fail(FIRAL_ERR_UNSUPPORTED, "device ordinal >= 128");
  std::lock_guard<std::mutex> g(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    FIRAL_CUDA_TRY(cudaGetSymbolAddress(&p, g_md_scratch));
    g_scratch_addr[dev] = p;
  }
  *out = static_cast<double*>(g_scratch_addr[dev]);
  return FIRAL_OK;
}

__device__ __forceinline__ double nan_max(double a, double b) {
  return (b > a || b != b) ? b : a;
}

template <class T>
__global__ void k_static_absmax(const T* __restrict__ g, int64_t n, double* part) {
  __shared__ double sh[kThreads / 32];
  const int64_t base = (int64_t)blockIdx.x * kStaticChunk;
  double mx = 0.0;
  for (int t = threadIdx.x; t < kStaticChunk; t += kThreads) {
    const int64_t i = base + t;
    if (i < n) mx = nan_max(mx, fabs((double)g[i]));
  }
  for (int o = 16; o > 0; o >>= 1) mx = nan_max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) r = nan_max(r, sh[w]);
    part[blockIdx.x] = r;
  }
}

template <class T>
__global__ void k_static_exp(T* __restrict__ z, const T* __restrict__ g, int64_t n, double beta0,
                             const double* maxpart, int nb, double* sumpart) {
  __shared__ double sh[kThreads / 32];
  __shared__ double s_beta;
  if (threadIdx.x == 0) {
    double mx = 0.0;
    for (int b = 0; b < nb; ++b) mx = nan_max(mx, maxpart[b]);
    s_beta = mx > 0.0 ? beta0 / mx : 0.0;
  }
  __syncthreads();
  const double beta = s_beta;
  const int64_t base = (int64_t)blockIdx.x * kStaticChunk;
  double acc = 0.0;
  for (int t = threadIdx.x; t < kStaticChunk; t += kThreads) {
    const int64_t i = base + t;
    if (i < n) {
      const T v = (T)((double)z[i] * exp(-beta * (double)g[i]));
      z[i] = v;
      acc += (double)v;
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) r += sh[w];
    sumpart[blockIdx.x] = r;
  }
}

template <class T>
__global__ void k_static_scale(T* __restrict__ z, int64_t n, double budget, const double* sumpart,
                               int nb) {
  __shared__ double s_scale;
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int b = 0; b < nb; ++b) tot += sumpart[b];
    s_scale = budget / tot;
  }
  __syncthreads();
  const double sc = s_scale;
  const int64_t base = (int64_t)blockIdx.x * kStaticChunk;
  for (int t = threadIdx.x; t < kStaticChunk; t += kThreads) {
    const int64_t i = base + t;
    if (i < n) z[i] = (T)((double)z[i] * sc);
  }
}

template <class T>
int32_t md_static(T* z, const T* g, int64_t n, double budget, double beta0, cudaStream_t st) {
  double* scratch = nullptr;
  FIRAL_TRY(scratch_address(&scratch));
  const int nb = (int)((n + kStaticChunk - 1) / kStaticChunk);
  double* maxpart = scratch;
  double* sumpart = scratch + kStaticSlots;
  k_static_absmax<T><<<nb, kThreads, 0, st>>>(g, n, maxpart);
  k_static_exp<T><<<nb, kThreads, 0, st>>>(z, g, n, beta0, maxpart, nb, sumpart);
  k_static_scale<T><<<nb, kThreads, 0, st>>>(z, n, budget, sumpart, nb);
  count_launch(3);
  FIRAL_CUDA_TRY(cudaGetLastError());
  return FIRAL_OK;
}

}  // namespace
}  // namespace firal

extern "C" int32_t firal_md_step_static(void* z, const void* g, int64_t n, int32_t dtype,
                                        double budget, double beta0, void* stream) {
  using namespace firal;
  if (!z || !g) return fail(FIRAL_ERR_ARG, "z and g must be non-null");
  if (n < 1) return fail(FIRAL_ERR_ARG, "n must be >= 1");
  if (n > (int64_t)kStaticChunk * kStaticSlots)
    return fail(FIRAL_ERR_ARG, "n = " + std::to_string(n) + " exceeds the static scratch limit of " +
                                   std::to_string((int64_t)kStaticChunk * kStaticSlots) +
                                   " points; use firal_md_step");
  if (!(budget > 0)) return fail(FIRAL_ERR_ARG, "budget must be > 0");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (dtype == FIRAL_DT_F32)
    return md_static<float>(static_cast<float*>(z), static_cast<const float*>(g), n, budget, beta0,
                            st);
  if (dtype == FIRAL_DT_F64)
    return md_static<double>(static_cast<double*>(z), static_cast<const double*>(g), n, budget,
                             beta0, st);
  return fail(FIRAL_ERR_ARG, "dtype must be FIRAL_DT_F32 or FIRAL_DT_F64");
}
