// SIMT (CUDA-core) kernels of the Approx-FIRAL hot path, templated on the vector type
// (float for FIRAL_FP32, double for FIRAL_FP64).
//
// Hessian apply (Lemma 1, Section 3.1).  For weights w over all rows (labelled rows first),
//   sum_i w_i H_i v = blockdiag_k(S_k) v  -  K^T diag(w) K v,
//   S_k = sum_i w_i h_ik x_i x_i^T,   K = rows (h_i (x) x_i),
// because [diag(h_i) - h_i h_i^T] (x) x_i x_i^T = diag(h_i) (x) x_i x_i^T - (h_i (x) x_i)(h_i (x) x_i)^T.
// The low-rank part is alpha_ij = (h_i (x) x_i) . v_j = sum_k h_ik (x_i . V_j[:,k]) (the
// alpha of Lemma 1), followed by out_j[k] -= sum_i w_i alpha_ij h_ik x_i.  The diagonal part
// costs 2 c d^2 s flops per apply once S_k is formed (once per weight vector).
#include <cuda_bf16.h>

#include <type_traits>

#include "firal_internal.cuh"


namespace firal {

// ------------------------------------------------------------------------------------------
// small helpers
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ double to_double(float v) { return (double)v; }
__device__ __forceinline__ double to_double(double v) { return v; }
__device__ __forceinline__ double to_double(__nv_bfloat16 v) { return (double)__bfloat162float(v); }

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide deterministic sum (fixed tree); result valid in every thread.
template <class T>
__device__ T block_sum(T v, T* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  T r = 0;
  for (int i = 0; i < nw; ++i) r += red[i];
  __syncthreads();
  return r;
}

// Sums over groups of `gsz` consecutive threads (gsz a multiple of 32): every thread gets its
// group's total, added in the same fixed order as block_sum over a gsz-thread block.
// red must hold blockDim.x / 32 entries.
template <class T>
__device__ T group_sum(T v, T* red, int gsz) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, gw = gsz >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  const int g0 = (wid / gw) * gw;
  T r = 0;
  for (int i = 0; i < gw; ++i) r += red[g0 + i];
  __syncthreads();
  return r;
}

static inline int grid_for(int64_t total, int threads, int cap = 65535 * 8) {
  int64_t g = (total + threads - 1) / threads;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return (int)g;
}

// ------------------------------------------------------------------------------------------
// input preparation
// ------------------------------------------------------------------------------------------
template <class T, class Tin>
__global__ void k_copy_rows(T* dst, const Tin* a, int64_t ma, const Tin* b, int64_t nb, int cols) {
  const int64_t total = (ma + nb) * cols;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = idx / cols;
    const int col = (int)(idx - r * cols);
    const double v = r < ma ? to_double(a[r * cols + col]) : to_double(b[(r - ma) * cols + col]);
    dst[idx] = (T)v;
  }
}

template <class T>
__global__ void k_transpose(T* dst, const T* src, int64_t rows, int cols) {
  __shared__ T tile[32][33];
  const int64_t rb = (int64_t)blockIdx.x * 32;
  const int cb = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t r = rb + i;
    const int col = cb + threadIdx.x;
    if (r < rows && col < cols) tile[i][threadIdx.x] = src[r * cols + col];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int col = cb + i;
    const int64_t r = rb + threadIdx.x;
    if (r < rows && col < cols) dst[(int64_t)col * rows + r] = tile[threadIdx.x][i];
  }
}

template <class T, class Tin>
static int32_t copy_rows_t(void* dst, const void* a, int64_t ma, const void* b, int64_t nb,
                           int cols, cudaStream_t st) {
  const int64_t total = (ma + nb) * cols;
  ProfScope ps(st, PF_PREP);
  if (std::is_same<T, Tin>::value) {
    // the same type: two contiguous device-to-device copies at copy bandwidth
    const size_t ba = (size_t)ma * cols * sizeof(T), bb = (size_t)nb * cols * sizeof(T);
    if (ba) FIRAL_CUDA_TRY(cudaMemcpyAsync(dst, a, ba, cudaMemcpyDeviceToDevice, st));
    if (bb)
      FIRAL_CUDA_TRY(cudaMemcpyAsync((char*)dst + ba, b, bb, cudaMemcpyDeviceToDevice, st));
    return FIRAL_OK;
  }
  count_launch();
  k_copy_rows<T, Tin><<<grid_for(total, 256), 256, 0, st>>>(
      (T*)dst, (const Tin*)a, ma, (const Tin*)b, nb, cols);
  FIRAL_CUDA_TRY(cudaGetLastError());
  return FIRAL_OK;
}

int32_t copy_rows(bool dbl, void* dst, const void* a, int64_t ma, const void* b, int64_t nb,
                  int cols, int32_t src_dtype, cudaStream_t st) {
  if (dbl) {
    if (src_dtype == FIRAL_DT_F64) return copy_rows_t<double, double>(dst, a, ma, b, nb, cols, st);
    if (src_dtype == FIRAL_DT_F32) return copy_rows_t<double, float>(dst, a, ma, b, nb, cols, st);
    return copy_rows_t<double, __nv_bfloat16>(dst, a, ma, b, nb, cols, st);
  }
  if (src_dtype == FIRAL_DT_F64) return copy_rows_t<float, double>(dst, a, ma, b, nb, cols, st);
  if (src_dtype == FIRAL_DT_F32) return copy_rows_t<float, float>(dst, a, ma, b, nb, cols, st);
  return copy_rows_t<float, __nv_bfloat16>(dst, a, ma, b, nb, cols, st);
}

int32_t transpose(bool dbl, void* dst, const void* src, int64_t rows, int cols, cudaStream_t st) {
  dim3 grid((unsigned)((rows + 31) / 32), (unsigned)((cols + 31) / 32));
  dim3 blk(32, 8);
  ProfScope ps(st, PF_PREP);
  count_launch();
  if (dbl)
    k_transpose<double><<<grid, blk, 0, st>>>((double*)dst, (const double*)src, rows, cols);
  else
    k_transpose<float><<<grid, blk, 0, st>>>((float*)dst, (const float*)src, rows, cols);
  FIRAL_CUDA_TRY(cudaGetLastError());
  return FIRAL_OK;
}

// Class-major copy h^T (c x N) read by the CUDA-core kernels.  FP32 / FP64 problems make it
// when they are created; a mixed-precision problem needs it only for the FP64-accumulated
// block sums of Round and makes it on first use (never inside a stream capture: Round and the
// block-sum entry points are not captured).
int32_t class_major_h(firal_problem* P) {
  if (P->HaT.p) return FIRAL_OK;
  const size_t vs = P->dbl ? sizeof(double) : sizeof(float);
  FIRAL_TRY(P->HaT.ensure((size_t)P->N * P->c * vs));
  return transpose(P->dbl, P->HaT.p, P->Ha.p, P->N, P->c, P->H->stream);
}

// weights over all rows: [lab_val] * m, then z (or zconst) on the pool rows
template <class T>
__global__ void k_fill_w(T* w, int64_t m, T lab_val, const T* z, T zconst, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m + n;
       i += (int64_t)gridDim.x * blockDim.x)
    w[i] = i < m ? lab_val : (z ? z[i - m] : zconst);
}

int32_t fill_weights(bool dbl, void* w, int64_t m, double lab_val, const void* z, double zconst,
                     int64_t n, cudaStream_t st) {
  const int g = grid_for(m + n, 256);
  ProfScope ps(st, PF_PREP);
  count_launch();
  if (dbl)
    k_fill_w<double><<<g, 256, 0, st>>>((double*)w, m, lab_val, (const double*)z, zconst, n);
  else
    k_fill_w<float><<<g, 256, 0, st>>>((float*)w, m, (float)lab_val, (const float*)z,
                                       (float)zconst, n);
  FIRAL_CUDA_TRY(cudaGetLastError());
  return FIRAL_OK;
}

// ------------------------------------------------------------------------------------------
// Rademacher probes (Algorithm 2 line 4), SplitMix64 counter rule
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

template <class T>
// Pooled problems: the entries of pool p are those of its own probe vector (dimension
// d_p c_p, counters local to the pool) and 0 on the padded features e >= d_p.
__global__ void k_probes(T* V, uint64_t seed, uint64_t t_host, const int64_t* t_dev, int s,
                         int64_t D, PoolTab pt, int d) {
  const uint64_t t = t_dev ? (uint64_t)*t_dev : t_host;
  const int64_t total = (int64_t)s * D;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t j = (uint64_t)(idx / D);
    uint64_t q = (uint64_t)(idx % D), Dq = (uint64_t)D;
    if (pt.Q) {
      const int k = (int)(q / (uint64_t)d), e = (int)(q % (uint64_t)d);
      const int p = pt.cpool[k], dq = pt.pdim[p];
      if (e >= dq) {
        V[idx] = T(0);
        continue;
      }
      q = (uint64_t)(k - pt.coff[p]) * (uint64_t)dq + (uint64_t)e;
      Dq = (uint64_t)(pt.coff[p + 1] - pt.coff[p]) * (uint64_t)dq;
    }
    const uint64_t ctr = (t * (uint64_t)s + j) * Dq + q;
    const uint64_t bits = splitmix64(seed ^ splitmix64(ctr));
    V[idx] = (bits >> 63) ? T(-1) : T(1);
  }
}

int32_t probes(bool dbl, void* V, uint64_t seed, int64_t t, int s, int64_t D, cudaStream_t st,
               const int64_t* t_dev, const PoolTab* pt, int d) {
  const int g = grid_for((int64_t)s * D, 256);
  const PoolTab tab = pt ? *pt : PoolTab{};
  ProfScope ps(st, PF_PROBES);
  count_launch();
  if (dbl) k_probes<double><<<g, 256, 0, st>>>((double*)V, seed, (uint64_t)t, t_dev, s, D, tab, d);
  else k_probes<float><<<g, 256, 0, st>>>((float*)V, seed, (uint64_t)t, t_dev, s, D, tab, d);
  FIRAL_CUDA_TRY(cudaGetLastError());
  return FIRAL_OK;
}

__global__ void k_tick(int64_t* t_dev) { *t_dev += 1; }
__global__ void k_set(int64_t* t_dev, int64_t v) { *t_dev = v; }

int32_t tick(int64_t* t_dev, cudaStream_t st) {
  count_launch();
  k_tick<<<1, 1, 0, st>>>(t_dev);
  FIRAL_CUDA_TRY(cudaGetLastError());
  return FIRAL_OK;
}

int32_t set_step(int64_t* t_dev, int64_t v, cudaStream_t st) {
  count_launch();
  k_set<<<1, 1, 0, st>>>(t_dev, v);
  FIRAL_CUDA_TRY(cudaGetLastError());
  return FIRAL_OK;
}

// ------------------------------------------------------------------------------------------
// Weighted block sums (eq. 13 and the diagonal part of the apply), partial over row splits:
//   partS[split][k][e][f] = sum_{i in split} w_i h_ik x_ie x_if
//   partP[split][k][e][f] = sum_{i in split} w_i h_ik (1 - h_ik) x_ie x_if
// 256 threads as 16 x 16, each owning a TE x TE tile of the (16 TE)^2 output; G classes per CTA.
// ------------------------------------------------------------------------------------------
template <class T, int TE, int G>
__global__ __launch_bounds__(256) void k_syrk(const T* __restrict__ Xa, const T* __restrict__ HaT,
                                              const T* __restrict__ w, int64_t N, int d, int c,
                                              int64_t rows_per_split, T* partS, T* partP) {
  constexpr int DP = 16 * TE;
  constexpr int PC = 32;
  __shared__ __align__(16) T xs[PC][DP];
  __shared__ T wsS[G][PC];
  __shared__ T wsP[G][PC];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int k0 = blockIdx.x * G;
  const int split = blockIdx.y;
  const int64_t i0 = (int64_t)split * rows_per_split;
  const int64_t i1 = min(N, i0 + rows_per_split);
  T accS[G][TE][TE], accP[G][TE][TE];
#pragma unroll
  for (int g = 0; g < G; ++g)
#pragma unroll
    for (int r = 0; r < TE; ++r)
#pragma unroll
      for (int q = 0; q < TE; ++q) accS[g][r][q] = accP[g][r][q] = T(0);

  for (int64_t ib = i0; ib < i1; ib += PC) {
    for (int idx = threadIdx.x; idx < PC * DP; idx += 256) {
      const int p = idx / DP, e = idx - p * DP;
      const int64_t i = ib + p;
      xs[p][e] = (i < i1 && e < d) ? Xa[i * d + e] : T(0);
    }
    for (int idx = threadIdx.x; idx < G * PC; idx += 256) {
      const int g = idx / PC, p = idx - g * PC;
      const int64_t i = ib + p;
      const int k = k0 + g;
      const T hv = (i < i1 && k < c) ? HaT[(int64_t)k * N + i] : T(0);
      const T wv = (i < i1) ? w[i] : T(0);
      wsS[g][p] = wv * hv;
      wsP[g][p] = wv * hv * (T(1) - hv);
    }
    __syncthreads();
#pragma unroll 4
    for (int p = 0; p < PC; ++p) {
      T a[TE], b[TE];
#pragma unroll
      for (int r = 0; r < TE; ++r) {
        a[r] = xs[p][ty * TE + r];
        b[r] = xs[p][tx * TE + r];
      }
#pragma unroll
      for (int g = 0; g < G; ++g) {
        const T sS = wsS[g][p], sP = wsP[g][p];
#pragma unroll
        for (int r = 0; r < TE; ++r) {
          const T as = sS * a[r], ap = sP * a[r];
#pragma unroll
          for (int q = 0; q < TE; ++q) {
            accS[g][r][q] = fma(as, b[q], accS[g][r][q]);
            accP[g][r][q] = fma(ap, b[q], accP[g][r][q]);
          }
        }
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const int k = k0 + g;
    if (k >= c) continue;
#pragma unroll
    for (int r = 0; r < TE; ++r) {
      const int e = ty * TE + r;
      if (e >= d) continue;
#pragma unroll
      for (int q = 0; q < TE; ++q) {
        const int f = tx * TE + q;
        if (f >= d) continue;
        const int64_t o = (((int64_t)split * c + k) * d + e) * d + f;
        if (partS) partS[o] = accS[g][r][q];
        if (partP) partP[o] = accP[g][r][q];
      }
    }
  }
}

// out[k][e][f] = sum_split part[split][k][e][f] (+ lam on the diagonal), as double and/or T
template <class T>
__global__ void k_syrk_reduce(const T* part, int splits, int64_t per, int d, double lam,
                              double* out_d, T* out_t, const T* add = nullptr) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < per;
       idx += (int64_t)gridDim.x * blockDim.x) {
    double acc = add ? (double)add[idx] : 0.0;
#pragma unroll 8
    for (int sp = 0; sp < splits; ++sp) acc += (double)part[(int64_t)sp * per + idx];
    const int64_t ef = idx % ((int64_t)d * d);
    const int e = (int)(ef / d), f = (int)(ef % d);
    if (e == f) acc += lam;
    if (out_d) out_d[idx] = acc;
    if (out_t) out_t[idx] = (T)acc;
  }
}

static int syrk_splits(int64_t N, int cgroups, int sms) {
  int64_t want = (4LL * sms + cgroups - 1) / cgroups;
  int64_t by_rows = (N + 65535) / 65536;
  int64_t s = want > by_rows ? want : by_rows;
  int64_t max_by_size = (N + 255) / 256;
  if (s > max_by_size) s = max_by_size;
  if (s < 1) s = 1;
  if (s > 4096) s = 4096;
  return (int)s;
}

template <class T>
static int32_t syrk_t(firal_problem* P, const T* w, double lamS, T* outS, double lamP,
                      double* outP) {
  cudaStream_t st = P->H->stream;
  const int d = P->d, c = P->c;
  const int TE = d <= 32 ? 2 : (d <= 64 ? 4 : 8);
  const int G = (sizeof(T) == 8 || TE == 8) ? 1 : 4;
  const int cgroups = (c + G - 1) / G;
  const int splits = syrk_splits(P->N, cgroups, P->sms);
  const int64_t rps = (P->N + splits - 1) / splits;
  const int64_t per = (int64_t)c * d * d;
  FIRAL_TRY(P->syrk_part.ensure((size_t)per * splits * 2 * sizeof(T)));
  T* partS = outS ? P->syrk_part.as<T>() : nullptr;
  T* partP = outP ? P->syrk_part.as<T>() + per * splits : nullptr;
  dim3 grid(cgroups, splits);
  ProfScope ps(st, PF_SYRK);
  count_launch(1 + (outS ? 1 : 0) + (outP ? 1 : 0));
  const T* Xa = P->Xa.as<T>();
  const T* HaT = P->HaT.as<T>();
#define FIRAL_SYRK(TE_, G_) \
  k_syrk<T, TE_, G_><<<grid, 256, 0, st>>>(Xa, HaT, w, P->N, d, c, rps, partS, partP)
  if (TE == 2) { if (G == 4) FIRAL_SYRK(2, 4); else FIRAL_SYRK(2, 1); }
  else if (TE == 4) { if (G == 4) FIRAL_SYRK(4, 4); else FIRAL_SYRK(4, 1); }
  else FIRAL_SYRK(8, 1);
#undef FIRAL_SYRK
  FIRAL_CUDA_TRY(cudaGetLastError());
  const int g = grid_for(per, 256, 4096);
  if (outS) k_syrk_reduce<T><<<g, 256, 0, st>>>(partS, splits, per, d, lamS, nullptr, outS);
  if (outP) k_syrk_reduce<T><<<g, 256, 0, st>>>(partP, splits, per, d, lamP, outP, nullptr);
  FIRAL_CUDA_TRY(cudaGetLastError());
  return FIRAL_OK;
}

int32_t syrk_reduce_f32(firal_problem* P, const float* partS, const float* partP, int splits,
                        double lamS, float* outS, double lamP, double* outP, const float* addS) {
  cudaStream_t st = P->H->stream;
  const int64_t per = (int64_t)P->c * P->d * P->d;
  const int g = grid_for(per, 256, 4096);
  ProfScope ps(st, PF_SYRK);
  count_launch((outS ? 1 : 0) + (outP ? 1 : 0));
  if (outS)
    k_syrk_reduce<float><<<g, 256, 0, st>>>(partS, splits, per, P->d, lamS, nullptr, outS, addS);
  if (outP) k_syrk_reduce<float><<<g, 256, 0, st>>>(partP, splits, per, P->d, lamP, outP, nullptr);
  FIRAL_CUDA_TRY(cudaGetLastError());
  return FIRAL_OK;
}

int32_t syrk_blocks(firal_problem* P, const void* w, double lamS, void* outS, double lamP,
                    double* outP) {
  FIRAL_TRY(class_major_h(P));
  if (P->dbl) return syrk_t<double>(P, (const double*)w, lamS, (double*)outS, lamP, outP);
  return syrk_t<float>(P, (const float*)w, lamS, (float*)outS, lamP, outP);
}

// ------------------------------------------------------------------------------------------
// Low-rank part of the apply, step 1:  walpha[i][j] = w_i sum_k h_ik (x_i . V_j[:,k]).
// One thread per row; x_i staged (transposed) in shared memory; probe block in chunks.
// ------------------------------------------------------------------------------------------
template <class T, int KC>
__global__ __launch_bounds__(128) void k_alpha(const T* __restrict__ Xa, const T* __restrict__ HaT,
                                               const T* __restrict__ w, const T* __restrict__ V,
                                               int64_t N, int d, int c, int s, int64_t D,
                                               T* __restrict__ walpha) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* xs = (T*)smem_raw;              // [d][128]
  T* Vs = xs + (size_t)d * 128;      // [d][KC]
  T* hs = Vs + (size_t)d * KC;       // [KC][128]
  const int tid = threadIdx.x;
  const int64_t i0 = (int64_t)blockIdx.x * 128;
  const int64_t i = i0 + tid;
  for (int idx = tid; idx < d * 128; idx += 128) {
    const int r = idx / d, e = idx - r * d;     // coalesced read of row-major X
    const int64_t ii = i0 + r;
    xs[e * 128 + r] = ii < N ? Xa[ii * d + e] : T(0);
  }
  const T wi = i < N ? w[i] : T(0);
  for (int j = 0; j < s; ++j) {
    T acc = T(0);
    for (int k0 = 0; k0 < c; k0 += KC) {
      __syncthreads();
      for (int idx = tid; idx < KC * d; idx += 128) {
        const int kk = idx / d, e = idx - kk * d;
        const int k = k0 + kk;
        Vs[e * KC + kk] = k < c ? V[(int64_t)j * D + (int64_t)k * d + e] : T(0);
      }
      for (int idx = tid; idx < KC * 128; idx += 128) {
        const int kk = idx / 128, r = idx - kk * 128;
        const int k = k0 + kk;
        const int64_t ii = i0 + r;
        hs[kk * 128 + r] = (k < c && ii < N) ? HaT[(int64_t)k * N + ii] : T(0);
      }
      __syncthreads();
      T gam[KC];
#pragma unroll
      for (int kk = 0; kk < KC; ++kk) gam[kk] = T(0);
      for (int e = 0; e < d; ++e) {
        const T xe = xs[e * 128 + tid];
#pragma unroll
        for (int kk = 0; kk < KC; ++kk) gam[kk] = fma(xe, Vs[e * KC + kk], gam[kk]);
      }
#pragma unroll
      for (int kk = 0; kk < KC; ++kk) acc = fma(hs[kk * 128 + tid], gam[kk], acc);
    }
    if (i < N) walpha[i * s + j] = wi * acc;
  }
}

// Low-rank part, step 2:  Dpart[split][k][j d + e] = sum_{i in split} h_ik walpha[i][j] x_ie.
// 64 (j,e) x 64 k tile per CTA; 256 threads, 4 x 4 register tiles; rows in chunks of 32.
template <class T>
__global__ __launch_bounds__(256) void k_dterm(const T* __restrict__ Xa, const T* __restrict__ Ha,
                                               const T* __restrict__ walpha, int64_t N, int d,
                                               int c, int s, int64_t rows_per_split,
                                               T* __restrict__ Dpart) {
  constexpr int PC = 32;
  __shared__ __align__(16) T Ys[PC][64];
  __shared__ __align__(16) T Hs[PC][64];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int r0 = blockIdx.x * 64, k0 = blockIdx.y * 64;
  const int split = blockIdx.z;
  const int sd = s * d;
  const int64_t i0 = (int64_t)split * rows_per_split;
  const int64_t i1 = min(N, i0 + rows_per_split);
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
  for (int64_t ib = i0; ib < i1; ib += PC) {
    for (int idx = threadIdx.x; idx < PC * 64; idx += 256) {
      const int p = idx >> 6, col = idx & 63;
      const int64_t i = ib + p;
      const int r = r0 + col;
      T y = T(0);
      if (i < i1 && r < sd) {
        const int j = r / d, e = r - j * d;
        y = walpha[i * s + j] * Xa[i * d + e];
      }
      Ys[p][col] = y;
      const int k = k0 + col;
      Hs[p][col] = (i < i1 && k < c) ? Ha[i * c + k] : T(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int p = 0; p < PC; ++p) {
      T a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        a[q] = Ys[p][ty * 4 + q];
        b[q] = Hs[p][tx * 4 + q];
      }
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) acc[x][y] = fma(a[x], b[y], acc[x][y]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int y = 0; y < 4; ++y) {
    const int k = k0 + tx * 4 + y;
    if (k >= c) continue;
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      const int r = r0 + ty * 4 + x;
      if (r < sd) Dpart[((int64_t)split * c + k) * sd + r] = acc[x][y];
    }
  }
}

// out_j[k] = S_k V_j[k] - sum_split Dpart[split][k][j d + .]; optional pq[j c + k] = V_j[k].out_j[k]
// Block = class k x JB probes; thread (jj, e) with e < dpad = d rounded up to 32.
template <class T, int JB>
__global__ void k_combine(const T* __restrict__ S, const T* __restrict__ V,
                          const T* __restrict__ Dpart, int splits, int d, int c, int s, int64_t D,
                          T* __restrict__ out, double* pq, const T* __restrict__ vmean,
                          PoolTab pt) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Ss = (T*)smem_raw;            // d*d
  T* vs = Ss + (size_t)d * d;      // JB*d
  __shared__ double red[32];
  const int k = blockIdx.x;
  const int j0 = blockIdx.y * JB;
  const int dpad = (d + 31) & ~31;
  const int jj = threadIdx.x / dpad, e = threadIdx.x - jj * dpad;
  for (int idx = threadIdx.x; idx < d * d; idx += blockDim.x) Ss[idx] = S[(int64_t)k * d * d + idx];
  for (int idx = threadIdx.x; idx < JB * d; idx += blockDim.x) {
    const int q = idx / d, f = idx - q * d;
    const int vm = ((j0 + q) * pool_count(pt) + pool_of(pt, k)) * d + f;
    vs[idx] = (j0 + q < s) ? V[(int64_t)(j0 + q) * D + (int64_t)k * d + f] -
                                 (vmean ? vmean[vm] : T(0))
                           : T(0);
  }
  __syncthreads();
  const int sd = s * d;
  const int j = j0 + jj;
  T q = T(0);
  if (j < s && e < d) {
    T acc = T(0);
    for (int f = 0; f < d; ++f) acc = fma(Ss[f * d + e], vs[jj * d + f], acc);   // S symmetric
    T dsum = T(0);
    const T* dp = Dpart + (int64_t)k * sd + j * d + e;
    const int64_t stride = (int64_t)c * sd;
#pragma unroll 4
    for (int sp = 0; sp < splits; ++sp) dsum += dp[sp * stride];
    q = acc - dsum;
    out[(int64_t)j * D + (int64_t)k * d + e] = q;
  }
  if (pq) {
    const double contrib = (j < s && e < d) ? (double)vs[jj * d + e] * (double)q : 0.0;
    const double tot = group_sum(contrib, red, dpad);
    if (e == 0 && j < s) pq[(int64_t)j * c + k] = tot;
  }
}

// The same combination for the f32 tensor-core path, four features per thread with 16-byte
// loads: one CTA per class block covers JB probes (all 16 of the usual probe block), so the
// d x d block is staged once per class, and each thread keeps 8 split-partial loads in flight.
// Per output the additions run in the same order as in k_combine (features f ascending, then
// splits ascending), so both give identical results.  Needs d % 4 == 0 and 16-byte aligned
// S, Dpart and out; blockDim = JB * d / 4.
template <int JB>
__global__ void k_combine4(const float* __restrict__ S, const float* __restrict__ V,
                           const float* __restrict__ Dpart, int splits, int d, int c, int s,
                           int64_t D, float* __restrict__ out, const float* __restrict__ vmean,
                           PoolTab pt) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* Ss = (float*)smem_raw;      // d*d
  float* vs = Ss + (size_t)d * d;    // JB*d
  const int k = blockIdx.x;
  const int j0 = blockIdx.y * JB;
  const int d4 = d >> 2;
  const int jj = threadIdx.x / d4, e4 = threadIdx.x - jj * d4;
  const float4* S4 = reinterpret_cast<const float4*>(S + (int64_t)k * d * d);
  for (int idx = threadIdx.x; idx < d * d4; idx += blockDim.x)
    reinterpret_cast<float4*>(Ss)[idx] = S4[idx];
  for (int idx = threadIdx.x; idx < JB * d; idx += blockDim.x) {
    const int q = idx / d, f = idx - q * d;
    const int vm = ((j0 + q) * pool_count(pt) + pool_of(pt, k)) * d + f;
    vs[idx] = (j0 + q < s) ? V[(int64_t)(j0 + q) * D + (int64_t)k * d + f] -
                                 (vmean ? vmean[vm] : 0.0f)
                           : 0.0f;
  }
  __syncthreads();
  const int j = j0 + jj;
  if (jj >= JB || j >= s) return;
  float4 acc = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  for (int f = 0; f < d; ++f) {   // S symmetric: row f of the block
    const float4 sv = reinterpret_cast<const float4*>(Ss + f * d)[e4];
    const float v = vs[jj * d + f];
    acc.x = fmaf(sv.x, v, acc.x);
    acc.y = fmaf(sv.y, v, acc.y);
    acc.z = fmaf(sv.z, v, acc.z);
    acc.w = fmaf(sv.w, v, acc.w);
  }
  const int64_t sd = (int64_t)s * d;
  const float4* dp = reinterpret_cast<const float4*>(Dpart + (int64_t)k * sd + (int64_t)j * d) + e4;
  const int64_t stride4 = ((int64_t)c * sd) >> 2;
  float4 dsum = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll 8
  for (int sp = 0; sp < splits; ++sp) {
    const float4 t = dp[sp * stride4];
    dsum.x += t.x;
    dsum.y += t.y;
    dsum.z += t.z;
    dsum.w += t.w;
  }
  reinterpret_cast<float4*>(out + (int64_t)j * D + (int64_t)k * d)[e4] =
      make_float4(acc.x - dsum.x, acc.y - dsum.y, acc.z - dsum.z, acc.w - dsum.w);
}

static int dterm_splits(int tiles, int64_t N, int sms) {
  int64_t want = (3LL * sms + tiles - 1) / tiles;
  int64_t max_by_rows = (N + 1023) / 1024;
  if (want > max_by_rows) want = max_by_rows;
  if (want < 1) want = 1;
  if (want > 256) want = 256;
  return (int)want;
}

template <class T>
static int32_t apply_t(firal_problem* P, const T* w, const T* Sblk, const T* V, int s, T* out,
                       double* pq) {
  cudaStream_t st = P->H->stream;
  const int d = P->d, c = P->c;
  const int64_t N = P->N, D = P->D;
  FIRAL_TRY(P->walpha.ensure((size_t)N * s * sizeof(T)));
  constexpr int KC = 16;
  const size_t smem_a = ((size_t)d * 128 + (size_t)d * KC + (size_t)KC * 128) * sizeof(T);
  static bool attr_set[2] = {false, false};
  if (!attr_set[sizeof(T) == 8]) {
    FIRAL_CUDA_TRY(cudaFuncSetAttribute(k_alpha<T, KC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        200 * 1024));
    FIRAL_CUDA_TRY(cudaFuncSetAttribute(k_combine<T, 4>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr_set[sizeof(T) == 8] = true;
  }
  {
  ProfScope ps(st, PF_ALPHA);
  count_launch();
  k_alpha<T, KC><<<(unsigned)((N + 127) / 128), 128, smem_a, st>>>(
      P->Xa.as<T>(), P->HaT.as<T>(), w, V, N, d, c, s, D, P->walpha.as<T>());
  }
  FIRAL_CUDA_TRY(cudaGetLastError());
  const int sd = s * d;
  const int tr = (sd + 63) / 64, tk = (c + 63) / 64;
  const int splits = forced_splits() > 0 ? (int)std::min<int64_t>(forced_splits(), (N + 31) / 32)
                                         : dterm_splits(tr * tk, N, P->sms);
  const int64_t rps = (N + splits - 1) / splits;
  FIRAL_TRY(P->Dpart.ensure((size_t)splits * c * sd * sizeof(T)));
  {
  ProfScope ps(st, PF_DTERM);
  count_launch();
  k_dterm<T><<<dim3(tr, tk, splits), 256, 0, st>>>(P->Xa.as<T>(), P->Ha.as<T>(),
                                                   P->walpha.as<T>(), N, d, c, s, rps,
                                                   P->Dpart.as<T>());
  }
  FIRAL_CUDA_TRY(cudaGetLastError());
  const int threads = ((d + 31) / 32) * 32 * 4;   // 4 probes in parallel
  const size_t smem_c = ((size_t)d * d + 4 * (size_t)d) * sizeof(T);
  ProfScope ps(st, PF_COMBINE);
  count_launch();
  k_combine<T, 4><<<dim3(c, (s + 3) / 4), threads, smem_c, st>>>(Sblk, V, P->Dpart.as<T>(),
                                                                  splits, d, c, s, D, out, pq,
                                                                  nullptr, P->pt);
  FIRAL_CUDA_TRY(cudaGetLastError());
  return FIRAL_OK;
}

int32_t combine_f32(firal_problem* P, const float* Sblk, const float* V, int splits, int s,
                    float* out, double* pq, const float* vmean) {
  const int d = P->d, c = P->c;
  const auto a16 = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; };
  if (!pq && d % 4 == 0 && a16(Sblk) && a16(P->Dpart.p) && a16(out)) {
    // 16 probes per CTA (d / 4 threads each, at most 512 threads at d = 128)
    constexpr int JB = 16;
    const int threads = JB * (d / 4);
    const size_t smem4 = ((size_t)d * d + (size_t)JB * d) * sizeof(float);
    static bool attr4 = false;
    if (!attr4) {
      FIRAL_CUDA_TRY(cudaFuncSetAttribute(k_combine4<JB>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
      attr4 = true;
    }
    ProfScope ps(P->H->stream, PF_COMBINE);
    count_launch();
    k_combine4<JB><<<dim3(c, (s + JB - 1) / JB), threads, smem4, P->H->stream>>>(
        Sblk, V, P->Dpart.as<float>(), splits, d, c, s, P->D, out, vmean, P->pt);
    FIRAL_CUDA_TRY(cudaGetLastError());
    return FIRAL_OK;
  }
  const int threads = ((d + 31) / 32) * 32 * 4;   // 4 probes in parallel
  const size_t smem_c = ((size_t)d * d + 4 * (size_t)d) * sizeof(float);
  FIRAL_CUDA_TRY(cudaFuncSetAttribute(k_combine<float, 4>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  ProfScope ps(P->H->stream, PF_COMBINE);
  count_launch();
  k_combine<float, 4><<<dim3(c, (s + 3) / 4), threads, smem_c, P->H->stream>>>(
      Sblk, V, P->Dpart.as<float>(), splits, d, c, s, P->D, out, pq, vmean, P->pt);
  FIRAL_CUDA_TRY(cudaGetLastError());
  return FIRAL_OK;
}

int32_t hessian_apply_simt(firal_problem* P, const void* w, const void* Sblk, const void* V,
                           int s, void* out, double* pq) {
  FIRAL_TRY(class_major_h(P));
  if (P->dbl)
    return apply_t<double>(P, (const double*)w, (const double*)Sblk, (const double*)V, s,
                           (double*)out, pq);
  return apply_t<float>(P, (const float*)w, (const float*)Sblk, (const float*)V, s, (float*)out,
                        pq);
}

// ------------------------------------------------------------------------------------------
// Preconditioned CG (Algorithm 2 lines 5-8), per-column recurrences with FP64 scalars.
// Partial sums are per (column j, class block k) and reduced in a fixed order.
// ------------------------------------------------------------------------------------------
template <class T, int JB>
__global__ void k_cg_init(const T* __restrict__ Minv, const T* __restrict__ B, int d, int c,
                          int s, int64_t D, T* X, T* R, T* Z, T* Pd, double* p_rz, double* p_bb) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Ms = (T*)smem_raw;           // d*d
  T* rs = Ms + (size_t)d * d;     // JB*d
  __shared__ double red[32];
  const int k = blockIdx.x;
  const int dpad = (d + 31) & ~31;
  const int jj = threadIdx.x / dpad, e = threadIdx.x - jj * dpad;
  const int j = blockIdx.y * JB + jj;
  for (int idx = threadIdx.x; idx < d * d; idx += blockDim.x) Ms[idx] = Minv[(int64_t)k * d * d + idx];
  const int64_t base = (int64_t)j * D + (int64_t)k * d;
  T r = T(0);
  if (j < s && e < d) {
    r = B[base + e];
    rs[jj * d + e] = r;
  }
  __syncthreads();
  T z = T(0);
  if (j < s && e < d) {
    for (int f = 0; f < d; ++f) z = fma(Ms[f * d + e], rs[jj * d + f], z);
    X[base + e] = T(0);
    R[base + e] = r;
    Z[base + e] = z;
    Pd[base + e] = z;
  }
  const double rz = group_sum(e < d ? (double)r * (double)z : 0.0, red, dpad);
  const double bb = group_sum(e < d ? (double)r * (double)r : 0.0, red, dpad);
  if (e == 0 && j < s) {
    p_rz[(int64_t)j * c + k] = rz;
    p_bb[(int64_t)j * c + k] = bb;
  }
}

// one warp per column: deterministic reduction of c partials
__device__ __forceinline__ double warp_reduce_partials(const double* p, int c) {
  const int lane = threadIdx.x & 31;
  double acc = 0.0;
  for (int k = lane; k < c; k += 32) acc += p[k];
  return warp_sum(acc);
}

// CG scalars live per (column j, pool p) at cols[j * Qe + p]: the partials of the pool's
// classes [k0, k1) are reduced (all classes for an ordinary problem).
__device__ __forceinline__ bool cg_slot(const PoolTab& pt, int c, int s, int& j, int& k0,
                                        int& k1) {
  const int Qe = pool_count(pt);
  const int slot = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (slot >= s * Qe) return false;
  j = slot / Qe;
  const int p = slot - j * Qe;
  k0 = pt.Q ? pt.coff[p] : 0;
  k1 = pt.Q ? pt.coff[p + 1] : c;
  return true;
}

__global__ void k_cg_init_cols(const double* p_rz, const double* p_bb, int c, int s, double tol,
                               int fixed, CGCol* cols, PoolTab pt) {
  int j, k0, k1;
  if (!cg_slot(pt, c, s, j, k0, k1)) return;
  const int slot = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const double rz = warp_reduce_partials(p_rz + (int64_t)j * c + k0, k1 - k0);
  const double bb = warp_reduce_partials(p_bb + (int64_t)j * c + k0, k1 - k0);
  if ((threadIdx.x & 31) == 0) {
    CGCol cc;
    cc.rho = rz;
    cc.bnorm2 = bb;
    cc.alpha = 0.0;
    cc.beta = 0.0;
    cc.relres = bb > 0 ? 1.0 : 0.0;
    cc.iters = 0;
    cc.active = (bb > 0.0) && (fixed || !(1.0 <= tol)) ? 1 : 0;
    cols[slot] = cc;
  }
}

__global__ void k_cg_alpha(const double* p_pq, int c, int s, CGCol* cols, PoolTab pt) {
  int j, k0, k1;
  if (!cg_slot(pt, c, s, j, k0, k1)) return;
  const int slot = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const double pq = warp_reduce_partials(p_pq + (int64_t)j * c + k0, k1 - k0);
  if ((threadIdx.x & 31) == 0) {
    CGCol cc = cols[slot];
    if (cc.active && pq > 0.0 && isfinite(pq)) {
      cc.alpha = cc.rho / pq;
    } else {
      cc.active = 0;
      cc.alpha = 0.0;
    }
    cols[slot] = cc;
  }
}

template <class T, int JB>
__global__ void k_cg_update(const T* __restrict__ Minv, int d, int c, int s, int64_t D,
                            const CGCol* __restrict__ cols, T* X, T* R, const T* Pd,
                            const T* Q, T* Z, double* p_rr, double* p_rz, PoolTab pt) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Ms = (T*)smem_raw;
  T* rs = Ms + (size_t)d * d;     // JB*d
  __shared__ double red[32];
  const int k = blockIdx.x;
  const int dpad = (d + 31) & ~31;
  const int jj = threadIdx.x / dpad, e = threadIdx.x - jj * dpad;
  const int j = blockIdx.y * JB + jj;
  for (int idx = threadIdx.x; idx < d * d; idx += blockDim.x) Ms[idx] = Minv[(int64_t)k * d * d + idx];
  const int slot = j * pool_count(pt) + pool_of(pt, k);
  const bool live = j < s && cols[slot].active;   // uniform over the probe's thread group
  const int64_t base = (int64_t)j * D + (int64_t)k * d;
  T r = T(0);
  if (live && e < d) {
    const T a = (T)cols[slot].alpha;
    X[base + e] = fma(a, Pd[base + e], X[base + e]);
    r = fma(-a, Q[base + e], R[base + e]);
    R[base + e] = r;
    rs[jj * d + e] = r;
  }
  __syncthreads();
  T z = T(0);
  if (live && e < d) {
    for (int f = 0; f < d; ++f) z = fma(Ms[f * d + e], rs[jj * d + f], z);
    Z[base + e] = z;
  }
  const double rr = group_sum(e < d ? (double)r * (double)r : 0.0, red, dpad);
  const double rz = group_sum(e < d ? (double)r * (double)z : 0.0, red, dpad);
  if (live && e == 0) {
    p_rr[(int64_t)j * c + k] = rr;
    p_rz[(int64_t)j * c + k] = rz;
  }
}

__global__ void k_cg_beta(const double* p_rr, const double* p_rz, int c, int s, double tol,
                          int fixed, CGCol* cols, PoolTab pt) {
  int j, k0, k1;
  if (!cg_slot(pt, c, s, j, k0, k1)) return;
  const int slot = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const double rr = warp_reduce_partials(p_rr + (int64_t)j * c + k0, k1 - k0);
  const double rz = warp_reduce_partials(p_rz + (int64_t)j * c + k0, k1 - k0);
  if ((threadIdx.x & 31) == 0) {
    CGCol cc = cols[slot];
    if (cc.active) {
      cc.iters += 1;
      cc.relres = sqrt(rr / cc.bnorm2);
      if (!fixed && cc.relres <= tol) {
        cc.active = 0;
      } else {
        cc.beta = rz / cc.rho;
        cc.rho = rz;
      }
    }
    cols[slot] = cc;
  }
}

template <class T>
__global__ void k_cg_pupdate(const CGCol* __restrict__ cols, int s, int64_t D, const T* Z, T* Pd,
                             PoolTab pt, int d) {
  const int64_t total = (int64_t)s * D;
  const int Qe = pool_count(pt);
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(idx / D);
    const int p = pt.Q ? pt.cpool[(int)((idx - (int64_t)j * D) / d)] : 0;
    const CGCol cc = cols[j * Qe + p];
    if (cc.active) Pd[idx] = fma((T)cc.beta, Pd[idx], Z[idx]);
  }
}

template <class T>
static int32_t cg_setup_attrs() {
  static bool done[2] = {false, false};
  if (!done[sizeof(T) == 8]) {
    FIRAL_CUDA_TRY(cudaFuncSetAttribute(k_cg_init<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        200 * 1024));
    FIRAL_CUDA_TRY(cudaFuncSetAttribute(k_cg_update<T, 4>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    done[sizeof(T) == 8] = true;
  }
  return FIRAL_OK;
}

int32_t cg_init(firal_problem* P, const void* B, int s, double tol, int fixed) {
  cudaStream_t st = P->H->stream;
  const int d = P->d, c = P->c;
  const int threads = ((d + 31) / 32) * 32 * 4;   // 4 probes in parallel
  double* p1 = P->cgpart1.as<double>();
  double* p2 = P->cgpart2.as<double>();
  CGCol* cols = P->cgcols.as<CGCol>();
  ProfScope ps(st, PF_CG);
  count_launch(2);
  if (P->dbl) {
    FIRAL_TRY(cg_setup_attrs<double>());
    const size_t sm = ((size_t)d * d + 4 * (size_t)d) * sizeof(double);
    k_cg_init<double, 4><<<dim3(c, (s + 3) / 4), threads, sm, st>>>(
        P->Minv.as<double>(), (const double*)B, d, c, s, P->D, P->cgX.as<double>(),
        P->cgR.as<double>(), P->cgZ.as<double>(), P->cgP.as<double>(), p1, p2);
  } else {
    FIRAL_TRY(cg_setup_attrs<float>());
    const size_t sm = ((size_t)d * d + 4 * (size_t)d) * sizeof(float);
    k_cg_init<float, 4><<<dim3(c, (s + 3) / 4), threads, sm, st>>>(
        P->Minv.as<float>(), (const float*)B, d, c, s, P->D, P->cgX.as<float>(),
        P->cgR.as<float>(), P->cgZ.as<float>(), P->cgP.as<float>(), p1, p2);
  }
  FIRAL_CUDA_TRY(cudaGetLastError());
  const int slots = s * pool_count(P->pt);
  k_cg_init_cols<<<(slots + 3) / 4, 128, 0, st>>>(p1, p2, c, s, tol, fixed, cols, P->pt);
  FIRAL_CUDA_TRY(cudaGetLastError());
  return FIRAL_OK;
}

// one CG iteration after Q = A P with pq partials already in cgpart1
int32_t cg_iterate_tail(firal_problem* P, int s, double tol, int fixed) {
  cudaStream_t st = P->H->stream;
  const int d = P->d, c = P->c;
  const int threads = ((d + 31) / 32) * 32 * 4;   // 4 probes in parallel
  double* p1 = P->cgpart1.as<double>();
  double* p2 = P->cgpart2.as<double>();
  CGCol* cols = P->cgcols.as<CGCol>();
  ProfScope ps(st, PF_CG);
  count_launch(4);
  const int slots = s * pool_count(P->pt);
  k_cg_alpha<<<(slots + 3) / 4, 128, 0, st>>>(p1, c, s, cols, P->pt);
  FIRAL_CUDA_TRY(cudaGetLastError());
  const int64_t total = (int64_t)s * P->D;
  if (P->dbl) {
    const size_t sm = ((size_t)d * d + 4 * (size_t)d) * sizeof(double);
    k_cg_update<double, 4><<<dim3(c, (s + 3) / 4), threads, sm, st>>>(
        P->Minv.as<double>(), d, c, s, P->D, cols, P->cgX.as<double>(), P->cgR.as<double>(),
        P->cgP.as<double>(), P->cgQ.as<double>(), P->cgZ.as<double>(), p1, p2, P->pt);
    FIRAL_CUDA_TRY(cudaGetLastError());
    k_cg_beta<<<(slots + 3) / 4, 128, 0, st>>>(p1, p2, c, s, tol, fixed, cols, P->pt);
    k_cg_pupdate<double><<<grid_for(total, 256), 256, 0, st>>>(cols, s, P->D, P->cgZ.as<double>(),
                                                              P->cgP.as<double>(), P->pt, d);
  } else {
    const size_t sm = ((size_t)d * d + 4 * (size_t)d) * sizeof(float);
    k_cg_update<float, 4><<<dim3(c, (s + 3) / 4), threads, sm, st>>>(
        P->Minv.as<float>(), d, c, s, P->D, cols, P->cgX.as<float>(), P->cgR.as<float>(),
        P->cgP.as<float>(), P->cgQ.as<float>(), P->cgZ.as<float>(), p1, p2, P->pt);
    FIRAL_CUDA_TRY(cudaGetLastError());
    k_cg_beta<<<(slots + 3) / 4, 128, 0, st>>>(p1, p2, c, s, tol, fixed, cols, P->pt);
    k_cg_pupdate<float><<<grid_for(total, 256), 256, 0, st>>>(cols, s, P->D, P->cgZ.as<float>(),
                                                             P->cgP.as<float>(), P->pt, d);
  }
  FIRAL_CUDA_TRY(cudaGetLastError());
  return FIRAL_OK;
}

// ------------------------------------------------------------------------------------------
// Per-point quadratic forms (eq. 11):  g_i = -(scale/s) sum_j a_j^T H_i b_j for pool rows,
//   a_j^T H_i b_j = sum_k h_ik (x_i.A_j[k]) (x_i.B_j[k]) - (sum_k h_ik x_i.A_j[k])(sum_k h_ik x_i.B_j[k]).
// ------------------------------------------------------------------------------------------
template <class T, int KC>
__global__ __launch_bounds__(128) void k_quad(const T* __restrict__ Xa, const T* __restrict__ HaT,
                                              const T* __restrict__ A, const T* __restrict__ B,
                                              int64_t m, int64_t N, int d, int c, int s, int64_t D,
                                              double scale, T* __restrict__ g) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* xs = (T*)smem_raw;               // [d][128]
  T* As = xs + (size_t)d * 128;       // [d][KC]
  T* Bs = As + (size_t)d * KC;        // [d][KC]
  T* hs = Bs + (size_t)d * KC;        // [KC][128]
  const int tid = threadIdx.x;
  const int64_t i0 = m + (int64_t)blockIdx.x * 128;
  const int64_t i = i0 + tid;
  for (int idx = tid; idx < d * 128; idx += 128) {
    const int r = idx / d, e = idx - r * d;
    const int64_t ii = i0 + r;
    xs[e * 128 + r] = ii < N ? Xa[ii * d + e] : T(0);
  }
  double q = 0.0;
  for (int j = 0; j < s; ++j) {
    T s1 = T(0), sa = T(0), sb = T(0);
    for (int k0 = 0; k0 < c; k0 += KC) {
      __syncthreads();
      for (int idx = tid; idx < KC * d; idx += 128) {
        const int kk = idx / d, e = idx - kk * d;
        const int k = k0 + kk;
        const int64_t src = (int64_t)j * D + (int64_t)k * d + e;
        As[e * KC + kk] = k < c ? A[src] : T(0);
        Bs[e * KC + kk] = k < c ? B[src] : T(0);
      }
      for (int idx = tid; idx < KC * 128; idx += 128) {
        const int kk = idx / 128, r = idx - kk * 128;
        const int k = k0 + kk;
        const int64_t ii = i0 + r;
        hs[kk * 128 + r] = (k < c && ii < N) ? HaT[(int64_t)k * N + ii] : T(0);
      }
      __syncthreads();
      T ga[KC], gb[KC];
#pragma unroll
      for (int kk = 0; kk < KC; ++kk) ga[kk] = gb[kk] = T(0);
      for (int e = 0; e < d; ++e) {
        const T xe = xs[e * 128 + tid];
#pragma unroll
        for (int kk = 0; kk < KC; ++kk) {
          ga[kk] = fma(xe, As[e * KC + kk], ga[kk]);
          gb[kk] = fma(xe, Bs[e * KC + kk], gb[kk]);
        }
      }
#pragma unroll
      for (int kk = 0; kk < KC; ++kk) {
        const T hv = hs[kk * 128 + tid];
        const T ha = hv * ga[kk];
        s1 = fma(ha, gb[kk], s1);
        sa += ha;
        sb = fma(hv, gb[kk], sb);
      }
    }
    q += (double)s1 - (double)sa * (double)sb;
  }
  if (i < N) g[i - m] = (T)(-scale / s * q);
}

int32_t quad_forms_simt(firal_problem* P, const void* A, const void* B, int s, double scale,
                        void* g) {
  FIRAL_TRY(class_major_h(P));
  cudaStream_t st = P->H->stream;
  const int d = P->d, c = P->c;
  constexpr int KC = 16;
  const unsigned grid = (unsigned)((P->n + 127) / 128);
  ProfScope ps(st, PF_QUAD);
  count_launch();
  if (P->dbl) {
    const size_t sm = ((size_t)d * 128 + 2 * (size_t)d * KC + KC * 128) * sizeof(double);
    FIRAL_CUDA_TRY(cudaFuncSetAttribute(k_quad<double, KC>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    k_quad<double, KC><<<grid, 128, sm, st>>>(P->Xa.as<double>(), P->HaT.as<double>(),
                                              (const double*)A, (const double*)B, P->m, P->N, d,
                                              c, s, P->D, scale, (double*)g);
  } else {
    const size_t sm = ((size_t)d * 128 + 2 * (size_t)d * KC + KC * 128) * sizeof(float);
    FIRAL_CUDA_TRY(cudaFuncSetAttribute(k_quad<float, KC>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    k_quad<float, KC><<<grid, 128, sm, st>>>(P->Xa.as<float>(), P->HaT.as<float>(),
                                             (const float*)A, (const float*)B, P->m, P->N, d, c,
                                             s, P->D, scale, (float*)g);
  }
  FIRAL_CUDA_TRY(cudaGetLastError());
  return FIRAL_OK;
}

// ------------------------------------------------------------------------------------------
// Dot products over probe blocks: out = (1/s) sum over all elements a*b (the f^ estimate)
// ------------------------------------------------------------------------------------------
template <class T>
__global__ void k_dot_partial(const T* a, const T* b, int64_t total, double* part) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x)
    acc += (double)a[idx] * (double)b[idx];
  const double tot = block_sum(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void k_sum_partials(const double* part, int np, double scale, double* out) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) acc += part[i];
  const double tot = block_sum(acc, red);
  if (threadIdx.x == 0) *out = tot * scale;
}

int32_t dot_scaled(bool dbl, const void* a, const void* b, int64_t total, double scale,
                   double* part /* >= 256 */, double* out, cudaStream_t st) {
  const int np = 256;
  ProfScope ps(st, PF_DOT);
  count_launch(2);
  if (dbl) k_dot_partial<double><<<np, 256, 0, st>>>((const double*)a, (const double*)b, total, part);
  else k_dot_partial<float><<<np, 256, 0, st>>>((const float*)a, (const float*)b, total, part);
  FIRAL_CUDA_TRY(cudaGetLastError());
  k_sum_partials<<<1, 256, 0, st>>>(part, np, scale, out);
  FIRAL_CUDA_TRY(cudaGetLastError());
  return FIRAL_OK;
}

// ------------------------------------------------------------------------------------------
// Mirror-descent update (Algorithm 2 lines 10-11) on the budget simplex.
// red layout: [0..255] max partials, [256..511] sum partials, [512] gmax, [513] zmax
// ------------------------------------------------------------------------------------------
template <class T>
__global__ void k_absmax_partial(const T* g, int64_t n, double* part) {
  __shared__ double red[32];
  double mx = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = fabs((double)g[i]);
    mx = (v > mx || v != v) ? v : mx;
  }
  // block max (fixed tree)
  for (int o = 16; o > 0; o >>= 1) {
    const double other = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = (other > mx || other != other) ? other : mx;
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r = (red[i] > r || red[i] != red[i]) ? red[i] : r;
    part[blockIdx.x] = r;
  }
}

template <class T>
__global__ void k_md_exp(T* z, const T* g, int64_t n, double beta0, double* red) {
  __shared__ double sh[32];
  __shared__ double s_beta;
  if (threadIdx.x == 0) {
    double mx = 0.0;
    for (int i = 0; i < 256; ++i) mx = (red[i] > mx || red[i] != red[i]) ? red[i] : mx;
    s_beta = mx > 0.0 ? beta0 / mx : 0.0;
    if (blockIdx.x == 0) red[512] = mx;
  }
  __syncthreads();
  const double beta = s_beta;
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const T zn = (T)((double)z[i] * exp(-beta * (double)g[i]));
    z[i] = zn;
    acc += (double)zn;
  }
  const double tot = block_sum(acc, sh);
  if (threadIdx.x == 0) red[256 + blockIdx.x] = tot;
}

template <class T>
__global__ void k_md_scale(T* z, int64_t n, double budget, double* red) {
  __shared__ double s_scale;
  __shared__ double sh[32];
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int i = 0; i < 256; ++i) tot += red[256 + i];
    s_scale = budget / tot;
  }
  __syncthreads();
  const double sc = s_scale;
  double mx = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const T v = (T)((double)z[i] * sc);
    z[i] = v;
    mx = (double)v > mx ? (double)v : mx;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double other = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = other > mx ? other : mx;
  }
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r = sh[i] > r ? sh[i] : r;
    red[768 + blockIdx.x] = r;
  }
}

__global__ void k_md_zmax(double* red) {
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int i = 0; i < 256; ++i) r = red[768 + i] > r ? red[768 + i] : r;
    red[513] = r;
  }
}

// Pooled problems: the MD update of every pool on its own simplex (Alg. 2 lines 10-11 with
// that pool's ||g||_inf and budget).  Pool p owns z[zoff[p] .. zoff[p+1]); MD_POOL_BLOCKS
// blocks share it (blockIdx.y), in three passes with per-block partials reduced in a fixed
// order: ||g||_inf, then z exp(-beta g) and its sum, then the rescale to the budget.
constexpr int MD_POOL_BLOCKS = 16;

template <class T>
__global__ void k_md_pooled_max(const T* g, const int64_t* zoff, double* part) {
  __shared__ double red[32];
  const int p = blockIdx.x, b = blockIdx.y;
  const int64_t a = zoff[p], e = zoff[p + 1];
  double mx = 0.0;
  for (int64_t i = a + (int64_t)b * blockDim.x + threadIdx.x; i < e;
       i += (int64_t)gridDim.y * blockDim.x) {
    const double v = fabs((double)g[i]);
    mx = (v > mx || v != v) ? v : mx;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double other = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = (other > mx || other != other) ? other : mx;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r = (red[i] > r || red[i] != red[i]) ? red[i] : r;
    part[(int64_t)p * MD_POOL_BLOCKS + b] = r;
  }
}

template <class T>
__global__ void k_md_pooled_exp(T* z, const T* g, const int64_t* zoff, double beta0,
                                double* part) {
  __shared__ double sh[32];
  __shared__ double s_beta;
  const int p = blockIdx.x, b = blockIdx.y;
  const int Q = gridDim.x;
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int i = 0; i < MD_POOL_BLOCKS; ++i) {
      const double v = part[(int64_t)p * MD_POOL_BLOCKS + i];
      r = (v > r || v != v) ? v : r;
    }
    s_beta = r > 0.0 ? beta0 / r : 0.0;
  }
  __syncthreads();
  const double beta = s_beta;
  const int64_t a = zoff[p], e = zoff[p + 1];
  double acc = 0.0;
  for (int64_t i = a + (int64_t)b * blockDim.x + threadIdx.x; i < e;
       i += (int64_t)gridDim.y * blockDim.x) {
    const T zn = (T)((double)z[i] * exp(-beta * (double)g[i]));
    z[i] = zn;
    acc += (double)zn;
  }
  const double tot = block_sum(acc, sh);
  if (threadIdx.x == 0) part[(int64_t)(Q + p) * MD_POOL_BLOCKS + b] = tot;
}

template <class T>
__global__ void k_md_pooled_scale(T* z, const int64_t* zoff, const double* budget,
                                  const double* part) {
  __shared__ double s_sc;
  const int p = blockIdx.x, b = blockIdx.y;
  const int Q = gridDim.x;
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int i = 0; i < MD_POOL_BLOCKS; ++i) tot += part[(int64_t)(Q + p) * MD_POOL_BLOCKS + i];
    s_sc = budget[p] / tot;
  }
  __syncthreads();
  const double sc = s_sc;
  const int64_t a = zoff[p], e = zoff[p + 1];
  for (int64_t i = a + (int64_t)b * blockDim.x + threadIdx.x; i < e;
       i += (int64_t)gridDim.y * blockDim.x)
    z[i] = (T)((double)z[i] * sc);
}

int32_t md_step_pooled(firal_problem* P, void* z, const void* g, double beta0, cudaStream_t st) {
  const int Q = P->pt.Q;
  const double* budget = P->pool_z.as<double>();
  const int64_t* zoff = reinterpret_cast<const int64_t*>(budget + Q);
  FIRAL_TRY(P->md_part.ensure((size_t)2 * Q * MD_POOL_BLOCKS * sizeof(double)));
  double* part = P->md_part.as<double>();
  const dim3 grid((unsigned)Q, MD_POOL_BLOCKS);
  ProfScope ps(st, PF_MD);
  count_launch(3);
  if (P->dbl) {
    k_md_pooled_max<double><<<grid, 256, 0, st>>>((const double*)g, zoff, part);
    k_md_pooled_exp<double><<<grid, 256, 0, st>>>((double*)z, (const double*)g, zoff, beta0, part);
    k_md_pooled_scale<double><<<grid, 256, 0, st>>>((double*)z, zoff, budget, part);
  } else {
    k_md_pooled_max<float><<<grid, 256, 0, st>>>((const float*)g, zoff, part);
    k_md_pooled_exp<float><<<grid, 256, 0, st>>>((float*)z, (const float*)g, zoff, beta0, part);
    k_md_pooled_scale<float><<<grid, 256, 0, st>>>((float*)z, zoff, budget, part);
  }
  FIRAL_CUDA_TRY(cudaGetLastError());
  return FIRAL_OK;
}

// ------------------------------------------------------------------------------------------
// Block PCG (O'Leary 1980): s x s Gram matrices, small FP64 solves and block updates.
// Vector blocks are probe-major: column j of a block is V[j * D .. j * D + D).
// ------------------------------------------------------------------------------------------
// part[k][a][b] = sum over class block k of A_a . B_b (a, b < s); one block per class
template <class T>
__global__ void k_gram_part(const T* __restrict__ A, const T* __restrict__ B, int s, int64_t D,
                            int d, double* part) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* As = (T*)smem_raw;            // s x d
  T* Bs = As + (size_t)s * d;      // s x d
  const int k = blockIdx.x;
  for (int i = threadIdx.x; i < s * d; i += blockDim.x) {
    const int a = i / d, e = i - a * d;
    As[i] = A[(int64_t)a * D + (int64_t)k * d + e];
    Bs[i] = B[(int64_t)a * D + (int64_t)k * d + e];
  }
  __syncthreads();
  for (int ab = threadIdx.x; ab < s * s; ab += blockDim.x) {
    const int a = ab / s, b = ab - a * s;
    double acc = 0.0;
    for (int e = 0; e < d; ++e) acc += (double)As[a * d + e] * (double)Bs[b * d + e];
    part[((int64_t)k * s + a) * s + b] = acc;
  }
}

// G[a][b] = sum_k part[k][a][b] in a fixed order
__global__ void k_gram_sum(const double* part, int c, int s, double* G) {
  for (int ab = threadIdx.x; ab < s * s; ab += blockDim.x) {
    double acc = 0.0;
    for (int k = 0; k < c; ++k) acc += part[(int64_t)k * s * s + ab];
    G[ab] = acc;
  }
}

// X = A^{-1} Y for s x s SPD A (Cholesky, FP64), one thread; flag = 1 when A is not SPD
__global__ void k_small_spd_solve(const double* A, const double* Y, int s, double* X, int* flag) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (*flag) {   // an earlier step lost rank: the block iterate stays where it is
    for (int q = 0; q < s * s; ++q) X[q] = 0.0;
    return;
  }
  double L[32 * 32];
  for (int i = 0; i < s; ++i)
    for (int j = 0; j <= i; ++j) {
      double v = 0.5 * (A[i * s + j] + A[j * s + i]);
      for (int k = 0; k < j; ++k) v -= L[i * s + k] * L[j * s + k];
      if (i == j) {
        if (!(v > 0.0)) {
          *flag = 1;
          for (int q = 0; q < s * s; ++q) X[q] = 0.0;
          return;
        }
        L[i * s + i] = sqrt(v);
      } else {
        L[i * s + j] = v / L[j * s + j];
      }
    }
  for (int col = 0; col < s; ++col) {
    double y[32];
    for (int i = 0; i < s; ++i) {
      double v = Y[i * s + col];
      for (int k = 0; k < i; ++k) v -= L[i * s + k] * y[k];
      y[i] = v / L[i * s + i];
    }
    for (int i = s - 1; i >= 0; --i) {
      double v = y[i];
      for (int k = i + 1; k < s; ++k) v -= L[k * s + i] * X[k * s + col];
      X[i * s + col] = v / L[i * s + i];
    }
  }
}

// Y[j] = Z[j] + sign * sum_l P[l] M[l][j] for every column j (Y may alias Z or P: each
// thread reads all s entries of its element before writing)
template <class T>
__global__ void k_block_axpy(T* Y, const T* Z, const T* P, const double* M, double sign, int s,
                             int64_t D) {
  __shared__ double Ms[32 * 32];
  for (int i = threadIdx.x; i < s * s; i += blockDim.x) Ms[i] = M[i];
  __syncthreads();
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < D;
       q += (int64_t)gridDim.x * blockDim.x) {
    double p[32], z[32];
    for (int l = 0; l < s; ++l) {
      p[l] = (double)P[(int64_t)l * D + q];
      z[l] = (double)Z[(int64_t)l * D + q];
    }
    for (int j = 0; j < s; ++j) {
      double acc = 0.0;
      for (int l = 0; l < s; ++l) acc += p[l] * Ms[l * s + j];
      Y[(int64_t)j * D + q] = (T)(z[j] + sign * acc);
    }
  }
}

// Z[j][k] = Minv_k R[j][k] (block-Jacobi preconditioner), block = class k x 4 probes
template <class T>
__global__ void k_precond_apply(const T* __restrict__ Minv, const T* R, int d, int s, int64_t D,
                                T* Z) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Ms = (T*)smem_raw;
  T* rs = Ms + (size_t)d * d;
  const int k = blockIdx.x;
  const int dpad = (d + 31) & ~31;
  const int jj = threadIdx.x / dpad, e = threadIdx.x - jj * dpad;
  const int j = blockIdx.y * 4 + jj;
  for (int i = threadIdx.x; i < d * d; i += blockDim.x) Ms[i] = Minv[(int64_t)k * d * d + i];
  if (j < s && e < d) rs[jj * d + e] = R[(int64_t)j * D + (int64_t)k * d + e];
  __syncthreads();
  if (j < s && e < d) {
    T z = T(0);
    for (int f = 0; f < d; ++f) z = fma(Ms[f * d + e], rs[jj * d + f], z);
    Z[(int64_t)j * D + (int64_t)k * d + e] = z;
  }
}

int32_t block_gram(firal_problem* P, const void* A, const void* B, int s, double* part,
                   double* G) {
  cudaStream_t st = P->H->stream;
  const int d = P->d, c = P->c;
  const size_t smem = (size_t)2 * s * d * (P->dbl ? 8 : 4);
  if (P->dbl) FIRAL_CUDA_TRY(cudaFuncSetAttribute(k_gram_part<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  else FIRAL_CUDA_TRY(cudaFuncSetAttribute(k_gram_part<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  ProfScope ps(st, PF_CG);
  count_launch(2);
  if (P->dbl) k_gram_part<double><<<c, 256, smem, st>>>((const double*)A, (const double*)B, s, P->D, d, part);
  else k_gram_part<float><<<c, 256, smem, st>>>((const float*)A, (const float*)B, s, P->D, d, part);
  k_gram_sum<<<1, 1024, 0, st>>>(part, c, s, G);
  FIRAL_CUDA_TRY(cudaGetLastError());
  return FIRAL_OK;
}

int32_t small_spd_solve(const double* A, const double* Y, int s, double* X, int* flag,
                        cudaStream_t st) {
  count_launch();
  k_small_spd_solve<<<1, 32, 0, st>>>(A, Y, s, X, flag);
  FIRAL_CUDA_TRY(cudaGetLastError());
  return FIRAL_OK;
}

int32_t block_axpy(firal_problem* P, void* Y, const void* Z, const void* Pm, const double* M,
                   double sign, int s) {
  cudaStream_t st = P->H->stream;
  const int g = grid_for(P->D, 256, 4096);
  ProfScope ps(st, PF_CG);
  count_launch();
  if (P->dbl)
    k_block_axpy<double><<<g, 256, 0, st>>>((double*)Y, (const double*)Z, (const double*)Pm, M, sign, s, P->D);
  else
    k_block_axpy<float><<<g, 256, 0, st>>>((float*)Y, (const float*)Z, (const float*)Pm, M, sign, s, P->D);
  FIRAL_CUDA_TRY(cudaGetLastError());
  return FIRAL_OK;
}

int32_t precond_apply(firal_problem* P, const void* R, int s, void* Z) {
  cudaStream_t st = P->H->stream;
  const int d = P->d, c = P->c;
  const int threads = ((d + 31) / 32) * 32 * 4;
  const size_t smem = ((size_t)d * d + 4 * (size_t)d) * (P->dbl ? 8 : 4);
  ProfScope ps(st, PF_CG);
  count_launch();
  if (P->dbl) {
    FIRAL_CUDA_TRY(cudaFuncSetAttribute(k_precond_apply<double>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    k_precond_apply<double><<<dim3(c, (s + 3) / 4), threads, smem, st>>>(
        P->Minv.as<double>(), (const double*)R, d, s, P->D, (double*)Z);
  } else {
    FIRAL_CUDA_TRY(cudaFuncSetAttribute(k_precond_apply<float>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    k_precond_apply<float><<<dim3(c, (s + 3) / 4), threads, smem, st>>>(
        P->Minv.as<float>(), (const float*)R, d, s, P->D, (float*)Z);
  }
  FIRAL_CUDA_TRY(cudaGetLastError());
  return FIRAL_OK;
}

template <class T>
__global__ void k_selected_weights(T* w, int64_t N, int64_t m, const int32_t* sel, int32_t b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    w[i] = T(0);
  __syncthreads();
  if (blockIdx.x == 0)
    for (int t = threadIdx.x; t < b; t += blockDim.x) w[m + sel[t]] = T(1);
}

int32_t selected_weights(firal_problem* P, const int32_t* sel, int32_t b, cudaStream_t st) {
  count_launch();
  // one block: the zeroing must finish before the ones are written
  if (P->dbl) k_selected_weights<double><<<1, 1024, 0, st>>>(P->zsave.as<double>(), P->N, P->m, sel, b);
  else k_selected_weights<float><<<1, 1024, 0, st>>>(P->zsave.as<float>(), P->N, P->m, sel, b);
  FIRAL_CUDA_TRY(cudaGetLastError());
  return FIRAL_OK;
}

int32_t md_step_simt(bool dbl, void* z, const void* g, int64_t n, double budget, double beta0,
                     double* red, cudaStream_t st) {
  ProfScope ps(st, PF_MD);
  count_launch(4);
  if (dbl) {
    k_absmax_partial<double><<<256, 256, 0, st>>>((const double*)g, n, red);
    k_md_exp<double><<<256, 256, 0, st>>>((double*)z, (const double*)g, n, beta0, red);
    k_md_scale<double><<<256, 256, 0, st>>>((double*)z, n, budget, red);
  } else {
    k_absmax_partial<float><<<256, 256, 0, st>>>((const float*)g, n, red);
    k_md_exp<float><<<256, 256, 0, st>>>((float*)z, (const float*)g, n, beta0, red);
    k_md_scale<float><<<256, 256, 0, st>>>((float*)z, n, budget, red);
  }
  k_md_zmax<<<1, 32, 0, st>>>(red);
  FIRAL_CUDA_TRY(cudaGetLastError());
  return FIRAL_OK;
}

// ------------------------------------------------------------------------------------------
// Row-sharded problems: the MD update with its two scalars added across processes, and the
// per-block dot products of an apply recomputed after its partial was added up.
// ------------------------------------------------------------------------------------------
// red[off] = max (op 1) or sum (op 0) of red[off .. off + count), fixed order; the rest zeroed
__global__ void k_collapse(double* red, int off, int count, int op) {
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int i = 0; i < count; ++i) {
      const double v = red[off + i];
      r = op == 1 ? ((v > r || v != v) ? v : r) : r + v;
      red[off + i] = 0.0;
    }
    red[off] = r;
  }
}

int32_t md_step_sharded(firal_problem* P, void* z, const void* g, double budget, double beta0,
                        double* red, cudaStream_t st) {
  const int64_t n = P->n;
  ProfScope ps(st, PF_MD);
  count_launch(2);
  if (P->dbl) k_absmax_partial<double><<<256, 256, 0, st>>>((const double*)g, n, red);
  else k_absmax_partial<float><<<256, 256, 0, st>>>((const float*)g, n, red);
  k_collapse<<<1, 32, 0, st>>>(red, 0, 256, 1);
  FIRAL_CUDA_TRY(cudaGetLastError());
  FIRAL_TRY(shard_allreduce(P, red, 1, FIRAL_DT_F64, 1));            // ||g||_inf
  count_launch(2);
  if (P->dbl) k_md_exp<double><<<256, 256, 0, st>>>((double*)z, (const double*)g, n, beta0, red);
  else k_md_exp<float><<<256, 256, 0, st>>>((float*)z, (const float*)g, n, beta0, red);
  k_collapse<<<1, 32, 0, st>>>(red, 256, 256, 0);
  FIRAL_CUDA_TRY(cudaGetLastError());
  FIRAL_TRY(shard_allreduce(P, red + 256, 1, FIRAL_DT_F64, 0));      // sum z exp(-beta g)
  count_launch(2);
  if (P->dbl) k_md_scale<double><<<256, 256, 0, st>>>((double*)z, n, budget, red);
  else k_md_scale<float><<<256, 256, 0, st>>>((float*)z, n, budget, red);
  k_md_zmax<<<1, 32, 0, st>>>(red);
  FIRAL_CUDA_TRY(cudaGetLastError());
  return shard_allreduce(P, red + 513, 1, FIRAL_DT_F64, 1);         // max z (stats)
}

// pq[j c + k] = <V_j[k], out_j[k]> (double), one block per (class, probe)
template <class T>
__global__ void k_block_dots(const T* V, const T* out, int c, int d, int64_t D, double* pq) {
  __shared__ double red[32];
  const int k = blockIdx.x, j = blockIdx.y;
  double acc = 0.0;
  for (int e = threadIdx.x; e < d; e += blockDim.x) {
    const int64_t o = (int64_t)j * D + (int64_t)k * d + e;
    acc += (double)V[o] * (double)out[o];
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    pq[(int64_t)j * c + k] = t;
  }
}

int32_t block_dots(firal_problem* P, const void* V, const void* out, int s, double* pq) {
  const int threads = ((P->d + 31) / 32) * 32;
  count_launch();
  if (P->dbl)
    k_block_dots<double><<<dim3(P->c, s), threads, 0, P->H->stream>>>(
        (const double*)V, (const double*)out, P->c, P->d, P->D, pq);
  else
    k_block_dots<float><<<dim3(P->c, s), threads, 0, P->H->stream>>>(
        (const float*)V, (const float*)out, P->c, P->d, P->D, pq);
  FIRAL_CUDA_TRY(cudaGetLastError());
  return FIRAL_OK;
}

}  // namespace firal
