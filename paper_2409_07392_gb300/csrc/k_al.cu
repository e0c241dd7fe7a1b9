// Multinomial logistic regression pieces of the active-learning outer loop (Section 5): class
// probabilities h_i = softmax(W x_i) (eq. 1 with W of shape c x d), the residual
// h_i - e_{y_i} and the ridge loss sum_i -log h_{i, y_i} + (gamma / 2) ||W||_F^2 whose gradient
// and Hessian (sum_i H_i + gamma I, H_i of eq. 2) drive the classifier refit, plus the row
// gathers that move selected points from the pool to the labelled set.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "firal_internal.cuh"

namespace firal {
namespace {

// In-place softmax of each row of L (rows x c), one warp per row, in the vec type.
template <class T>
__global__ void k_row_softmax(T* L, int64_t rows, int c) {
  const int lane = threadIdx.x & 31;
  const int64_t r = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= rows) return;
  T* row = L + r * c;
  T mx = T(-INFINITY);
  for (int k = lane; k < c; k += 32) mx = max(mx, row[k]);
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  T sum = T(0);
  for (int k = lane; k < c; k += 32) sum += exp(row[k] - mx);
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  const T inv = T(1) / sum;
  for (int k = lane; k < c; k += 32) row[k] = exp(row[k] - mx) * inv;
}

// R = h - onehot(y), rows x c
template <class T>
__global__ void k_residual(const T* __restrict__ h, const int32_t* __restrict__ y, int64_t m,
                           int c, T* __restrict__ R) {
  const int64_t tot = m * c;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / c;
    const int k = (int)(idx - i * c);
    R[idx] = h[idx] - (y[i] == k ? T(1) : T(0));
  }
}

// part[block] = sum over its rows of -log h_{i, y_i}
template <class T>
__global__ void k_nll_partial(const T* __restrict__ h, const int32_t* __restrict__ y, int64_t m,
                              int c, double* part) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    acc -= log((double)h[i * c + y[i]]);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    part[blockIdx.x] = s;
  }
}

__global__ void k_sum_part(const double* part, int np, double* out) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) acc += part[i];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    *out = s;
  }
}

// out = a X + b Y (elementwise, n values)
template <class T>
__global__ void k_axpby(T* out, double a, const T* X, double b, const T* Y, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (T)(a * (double)X[i] + (Y ? b * (double)Y[i] : 0.0));
}

template <class T>
__global__ void k_gather_rows(const T* __restrict__ src, const int32_t* __restrict__ idx,
                              int64_t rows, int cols, T* __restrict__ dst) {
  const int64_t tot = rows * cols;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < tot;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = q / cols;
    const int e = (int)(q - r * cols);
    dst[q] = src[(int64_t)idx[r] * cols + e];
  }
}

int grid_for(int64_t n) { return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4096)); }

}  // namespace

int32_t lr_probs(bool dbl, const void* X, const void* W, int64_t rows, int d, int c, void* h,
                 cudaStream_t st) {
  if (rows <= 0) return FIRAL_OK;
  // logits = X W^T (rows x c), then the row softmax in place
  FIRAL_TRY(dense_gemm(dbl, st, false, true, (int)rows, c, d, 1.0, X, d, W, d, 0.0, h, c));
  ProfScope ps(st, PF_LR);
  count_launch();
  const int blocks = (int)((rows + 7) / 8);
  if (dbl) k_row_softmax<double><<<blocks, 256, 0, st>>>((double*)h, rows, c);
  else k_row_softmax<float><<<blocks, 256, 0, st>>>((float*)h, rows, c);
  FIRAL_CUDA_TRY(cudaGetLastError());
  return FIRAL_OK;
}

int32_t lr_grad(bool dbl, const void* X, const int32_t* y, const void* h, const void* W,
                int64_t m, int d, int c, double gamma, void* R, void* g, cudaStream_t st) {
  {
    ProfScope ps(st, PF_LR);
    count_launch(2);
    const int64_t D = (int64_t)c * d;
    if (dbl) {
      k_residual<double><<<grid_for(m * c), 256, 0, st>>>((const double*)h, y, m, c, (double*)R);
      k_axpby<double><<<grid_for(D), 256, 0, st>>>((double*)g, gamma, (const double*)W, 0.0, nullptr, D);
    } else {
      k_residual<float><<<grid_for(m * c), 256, 0, st>>>((const float*)h, y, m, c, (float*)R);
      k_axpby<float><<<grid_for(D), 256, 0, st>>>((float*)g, gamma, (const float*)W, 0.0, nullptr, D);
    }
    FIRAL_CUDA_TRY(cudaGetLastError());
  }
  // g += R^T X  (c x d)
  return dense_gemm(dbl, st, true, false, c, d, (int)m, 1.0, R, c, X, d, 1.0, g, d);
}

int32_t lr_nll(bool dbl, const void* h, const int32_t* y, int64_t m, int c, double* part,
               double* out, cudaStream_t st) {
  ProfScope ps(st, PF_LR);
  count_launch(2);
  const int np = 256;
  if (dbl) k_nll_partial<double><<<np, 256, 0, st>>>((const double*)h, y, m, c, part);
  else k_nll_partial<float><<<np, 256, 0, st>>>((const float*)h, y, m, c, part);
  FIRAL_CUDA_TRY(cudaGetLastError());
  k_sum_part<<<1, 256, 0, st>>>(part, np, out);
  FIRAL_CUDA_TRY(cudaGetLastError());
  return FIRAL_OK;
}

int32_t axpby(bool dbl, void* out, double a, const void* X, double b, const void* Y, int64_t n,
              cudaStream_t st) {
  ProfScope ps(st, PF_LR);
  count_launch();
  if (dbl) k_axpby<double><<<grid_for(n), 256, 0, st>>>((double*)out, a, (const double*)X, b, (const double*)Y, n);
  else k_axpby<float><<<grid_for(n), 256, 0, st>>>((float*)out, a, (const float*)X, b, (const float*)Y, n);
  FIRAL_CUDA_TRY(cudaGetLastError());
  return FIRAL_OK;
}

// dst[r] = src[idx[r]] for rows of `cols` elements: vec-type rows (dbl selects double / float)
// or int32 labels (labels = true, cols = 1).
int32_t gather_rows(bool dbl, bool labels, const void* src, const int32_t* idx, int64_t rows,
                    int cols, void* dst, cudaStream_t st) {
  if (rows <= 0) return FIRAL_OK;
  ProfScope ps(st, PF_LR);
  count_launch();
  const int g = grid_for(rows * cols);
  if (labels) k_gather_rows<int32_t><<<g, 256, 0, st>>>((const int32_t*)src, idx, rows, cols, (int32_t*)dst);
  else if (dbl) k_gather_rows<double><<<g, 256, 0, st>>>((const double*)src, idx, rows, cols, (double*)dst);
  else k_gather_rows<float><<<g, 256, 0, st>>>((const float*)src, idx, rows, cols, (float*)dst);
  FIRAL_CUDA_TRY(cudaGetLastError());
  return FIRAL_OK;
}

}  // namespace firal
