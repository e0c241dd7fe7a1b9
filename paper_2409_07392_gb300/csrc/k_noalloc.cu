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
// Scratch: kStaticSlots doubles for the block maxima, as many for the block sums, and a few
// control slots (beta, the normalising scale, a non-finite flag): 64 KiB + 64 bytes,
// resident on every GPU that loads this library.  One block reduces kStaticChunk = 4096
// elements, so n is limited to 4096 * 4096 = 16,777,216.  Each partial is reduced once, by
// a one-block kernel, which writes the step's scalar into a control slot for the next
// kernel.  Every slot a call reads is written earlier in the same call, so nothing needs
// clearing between calls; the array keeps the last call's values.  Calls whose kernels
// overlap on the GPU (for example on two streams at once) share the array and race.
//
// Non-finite input: if ||g||_inf is NaN or infinite, or the updated z does not have a
// positive finite sum, the last kernel leaves z unchanged (the flag slot records why).  The
// call returns once its kernels are enqueued, so its status cannot report this.
#include "firal_internal.cuh"

namespace firal {
namespace {

constexpr int kStaticChunk = 4096;   // elements per block
constexpr int kStaticSlots = 4096;   // partial slots per reduction
constexpr int kThreads = 256;
// control slots after the two partial arrays
constexpr int kBeta = 2 * kStaticSlots, kScale = kBeta + 1, kFlag = kBeta + 2;
constexpr int kCtlSlots = 8;

__device__ __align__(256) double g_md_scratch[2 * kStaticSlots + kCtlSlots];

// Device address of g_md_scratch on the current device.  Looked up on every call (no
// allocation), so the address stays right if the device's context is torn down and made
// again; the first lookup on a device may load this library's device code there.
int32_t scratch_address(double** out) {
  void* p = nullptr;
  FIRAL_CUDA_TRY(cudaGetSymbolAddress(&p, g_md_scratch));
  *out = static_cast<double*>(p);
  return FIRAL_OK;
}

__device__ __forceinline__ double nan_max(double a, double b) {
  return (b > a || b != b) ? b : a;
}

__device__ __forceinline__ bool is_finite_d(double v) {
  return v == v && fabs(v) <= 1.7976931348623157e308;
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

// One block: ||g||_inf from the nb block maxima (fixed order), beta = beta0 / ||g||_inf into
// the beta slot; flag 1 when ||g||_inf is not finite.
__global__ void k_static_beta(double* scratch, int nb, double beta0) {
  __shared__ double sh[kThreads / 32];
  double mx = 0.0;
  for (int b = threadIdx.x; b < nb; b += kThreads) mx = nan_max(mx, scratch[b]);
  for (int o = 16; o > 0; o >>= 1) mx = nan_max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) r = nan_max(r, sh[w]);
    const bool ok = is_finite_d(r);
    scratch[kBeta] = (ok && r > 0.0) ? beta0 / r : 0.0;
    scratch[kFlag] = ok ? 0.0 : 1.0;
  }
}

// the updated value before normalisation, rounded to T as firal_md_step stores it
template <class T>
__device__ __forceinline__ T md_update(T zi, T gi, double beta) {
  return (T)((double)zi * exp(-beta * (double)gi));
}

// Block sums of the updated z (z itself is not written yet).
template <class T>
__global__ void k_static_expsum(const T* __restrict__ z, const T* __restrict__ g, int64_t n,
                                double* scratch) {
  __shared__ double sh[kThreads / 32];
  const double beta = scratch[kBeta];
  const int64_t base = (int64_t)blockIdx.x * kStaticChunk;
  double acc = 0.0;
  for (int t = threadIdx.x; t < kStaticChunk; t += kThreads) {
    const int64_t i = base + t;
    if (i < n) acc += (double)md_update(z[i], g[i], beta);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) r += sh[w];
    scratch[kStaticSlots + blockIdx.x] = r;
  }
}

// One block: the sum of the updated z from the nb block sums (fixed order) and the scale
// budget / sum into the scale slot; flag 2 when the sum is not positive and finite.
__global__ void k_static_total(double* scratch, int nb, double budget) {
  __shared__ double sh[kThreads / 32];
  double acc = 0.0;
  for (int b = threadIdx.x; b < nb; b += kThreads) acc += scratch[kStaticSlots + b];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) tot += sh[w];
    const bool ok = is_finite_d(tot) && tot > 0.0;
    scratch[kScale] = ok ? budget / tot : 0.0;
    if (!ok && scratch[kFlag] == 0.0) scratch[kFlag] = 2.0;
  }
}

// z <- budget z exp(-beta g) / sum, unless a flag is set (then z is left as it was).
template <class T>
__global__ void k_static_scale(T* __restrict__ z, const T* __restrict__ g, int64_t n,
                               const double* scratch) {
  if (scratch[kFlag] != 0.0) return;
  const double beta = scratch[kBeta], sc = scratch[kScale];
  const int64_t base = (int64_t)blockIdx.x * kStaticChunk;
  for (int t = threadIdx.x; t < kStaticChunk; t += kThreads) {
    const int64_t i = base + t;
    if (i < n) z[i] = (T)((double)md_update(z[i], g[i], beta) * sc);
  }
}

template <class T>
int32_t md_static(T* z, const T* g, int64_t n, double budget, double beta0, cudaStream_t st) {
  double* scratch = nullptr;
  FIRAL_TRY(scratch_address(&scratch));
  const int nb = (int)((n + kStaticChunk - 1) / kStaticChunk);
  k_static_absmax<T><<<nb, kThreads, 0, st>>>(g, n, scratch);
  k_static_beta<<<1, kThreads, 0, st>>>(scratch, nb, beta0);
  k_static_expsum<T><<<nb, kThreads, 0, st>>>(z, g, n, scratch);
  k_static_total<<<1, kThreads, 0, st>>>(scratch, nb, budget);
  k_static_scale<T><<<nb, kThreads, 0, st>>>(z, g, n, scratch);
  count_launch(5);
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
