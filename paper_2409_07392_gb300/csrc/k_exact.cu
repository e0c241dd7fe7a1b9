// Exact-FIRAL (Algorithm 1 of the paper) on dense d~ x d~ matrices, d~ = d c: the Relax
// objective f(z) = Tr(Sigma_z^{-1} H_p) (eqs. 4, 5, 7), its exact gradient
// g_i = -Tr(H_i Sigma_z^{-1} H_p Sigma_z^{-1}) (eq. 6), entropic mirror descent on the budget
// simplex, and the FTRL Round on the full Hessians (eqs. 8-10).
//
// Layout: every d~ x d~ matrix is row-major with leading dimension d~; row and column index
// k d + e stand for class k and feature e (the Kronecker order of eq. 2).  Everything runs in
// the problem's vec type (float, or double for FIRAL_FP64); the factorisation and inverse of
// each diagonal tile, the Round's c x c systems and all scalar reductions use double.
//
// Building blocks:
//   * k_pair_syrk + k_pair_reduce: sum_i w_i H_i (+ base matrices) built per class pair
//     (k, l), k <= l, as sum_i w_i q_i^{kl} x_i x_i^T with q^{kl} = delta_kl h_k - h_k h_l
//     (eq. 2 written block by block), mirrored into the lower blocks;
//   * k_gemm: C = alpha op(A) op(B) + beta C, SIMT, 128 x 128 (float) / 64 x 64 (double)
//     tiles, with optional skipping of tiles above the diagonal and of K ranges that a
//     triangular operand makes zero;
//   * k_potrf_diag: Cholesky and inverse of one 64 x 64 diagonal tile; with k_gemm it makes
//     the blocked right-looking Cholesky and the blocked (doubling) triangular inverse;
//   * k_pair_quad: x_i^T M_kl x_i for every class pair -- the exact gradient and the c x c
//     matrices of the Round scores;
//   * k_exact_score: eq. 9's trace for one candidate from its c x c matrices (Woodbury).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "firal_internal.cuh"

namespace firal {
namespace {

constexpr int NB = 64;    // panel width of the blocked Cholesky and triangular inverse
constexpr int GBK = 8;    // K depth of one GEMM stage

// ------------------------------------------------------------------------------ vector loads
template <class T, int W>
__device__ __forceinline__ void ld_vec(const T* p, T* out) {
#pragma unroll
  for (int q = 0; q < W; ++q) out[q] = p[q];
}
template <>
__device__ __forceinline__ void ld_vec<float, 4>(const float* p, float* out) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w;
}
template <>
__device__ __forceinline__ void ld_vec<float, 8>(const float* p, float* out) {
  ld_vec<float, 4>(p, out);
  ld_vec<float, 4>(p + 4, out + 4);
}
template <>
__device__ __forceinline__ void ld_vec<float, 2>(const float* p, float* out) {
  const float2 v = *reinterpret_cast<const float2*>(p);
  out[0] = v.x; out[1] = v.y;
}
template <>
__device__ __forceinline__ void ld_vec<double, 2>(const double* p, double* out) {
  const double2 v = *reinterpret_cast<const double2*>(p);
  out[0] = v.x; out[1] = v.y;
}
template <>
__device__ __forceinline__ void ld_vec<double, 4>(const double* p, double* out) {
  ld_vec<double, 2>(p, out);
  ld_vec<double, 2>(p + 2, out + 2);
}
template <>
__device__ __forceinline__ void ld_vec<double, 8>(const double* p, double* out) {
  ld_vec<double, 4>(p, out);
  ld_vec<double, 4>(p + 4, out + 4);
}

// ------------------------------------------------------------------------------ dense GEMM
template <class T> struct GemmCfg;
template <> struct GemmCfg<float> { static constexpr int BM = 128, PAD = 4; };
template <> struct GemmCfg<double> { static constexpr int BM = 64, PAD = 2; };

// K-range flags for triangular operands (tile-level bounds; every skipped term is zero):
constexpr int K_FROM_N0 = 1;   // op(B) lower triangular: k >= n0
constexpr int K_FROM_M0 = 2;   // op(A) upper triangular (A^T of a lower one): k >= m0
constexpr int K_TO_M1 = 4;     // op(A) lower triangular: k < m0 + BM

// C (M x N) = alpha op(A) op(B) + beta C for every batch z (operands offset by z sA, z sB,
// z sC elements).  op(A) is M x K (A row-major M x K, or K x M when
// TA); op(B) is K x N (B row-major K x N, or N x K when TB).  lower: tiles wholly above the
// diagonal are skipped (the caller uses only the lower triangle).  beta == 0 never reads C.
// A may alias C only when one CTA covers every column of C (N <= BM) and reads only its own
// rows of A: all of a CTA's reads finish before its epilogue writes.
template <class T, bool TA, bool TB>
__global__ __launch_bounds__(256) void k_gemm(int M, int N, int K, T alpha, const T* A,
                                              int64_t lda, const T* B, int64_t ldb, T beta,
                                              T* C, int64_t ldc, int lower, int kflags,
                                              int64_t sA, int64_t sB, int64_t sC) {
  A += blockIdx.z * sA;
  B += blockIdx.z * sB;
  C += blockIdx.z * sC;
  constexpr int BM = GemmCfg<T>::BM, BN = BM, PAD = GemmCfg<T>::PAD;
  constexpr int TM = BM / 16, TN = BN / 16, G = 16 / (int)sizeof(T);
  constexpr int LA = BM * GBK / 256, LB = BN * GBK / 256;
  __shared__ __align__(16) T As[2][GBK][BM + PAD];
  __shared__ __align__(16) T Bs[2][GBK][BN + PAD];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  if (lower && n0 >= m0 + BM) return;
  int kb = 0, ke = K;
  if (kflags & K_FROM_N0) kb = max(kb, n0);
  if (kflags & K_FROM_M0) kb = max(kb, m0);
  if (kflags & K_TO_M1) ke = min(ke, m0 + BM);
  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = T(0);
  T ra[LA], rb[LB];
  auto gload = [&](int k0) {
#pragma unroll
    for (int q = 0; q < LA; ++q) {
      const int idx = tid + q * 256;
      int mm, kk;
      if (TA) { kk = idx / BM; mm = idx - kk * BM; }
      else { mm = idx / GBK; kk = idx - mm * GBK; }
      const int gm = m0 + mm, gk = k0 + kk;
      ra[q] = (gm < M && gk < ke) ? (TA ? A[(int64_t)gk * lda + gm] : A[(int64_t)gm * lda + gk])
                                  : T(0);
    }
#pragma unroll
    for (int q = 0; q < LB; ++q) {
      const int idx = tid + q * 256;
      int nn, kk;
      if (TB) { nn = idx / GBK; kk = idx - nn * GBK; }
      else { kk = idx / BN; nn = idx - kk * BN; }
      const int gn = n0 + nn, gk = k0 + kk;
      rb[q] = (gn < N && gk < ke) ? (TB ? B[(int64_t)gn * ldb + gk] : B[(int64_t)gk * ldb + gn])
                                  : T(0);
    }
  };
  auto sstore = [&](int buf) {
#pragma unroll
    for (int q = 0; q < LA; ++q) {
      const int idx = tid + q * 256;
      int mm, kk;
      if (TA) { kk = idx / BM; mm = idx - kk * BM; }
      else { mm = idx / GBK; kk = idx - mm * GBK; }
      As[buf][kk][mm] = ra[q];
    }
#pragma unroll
    for (int q = 0; q < LB; ++q) {
      const int idx = tid + q * 256;
      int nn, kk;
      if (TB) { nn = idx / GBK; kk = idx - nn * GBK; }
      else { kk = idx / BN; nn = idx - kk * BN; }
      Bs[buf][kk][nn] = rb[q];
    }
  };
  const int nk = ke > kb ? (ke - kb + GBK - 1) / GBK : 0;
  if (nk > 0) {
    gload(kb);
    sstore(0);
    __syncthreads();
    for (int kt = 0; kt < nk; ++kt) {
      const int buf = kt & 1;
      if (kt + 1 < nk) gload(kb + (kt + 1) * GBK);
#pragma unroll
      for (int kk = 0; kk < GBK; ++kk) {
        T a[TM], b[TN];
#pragma unroll
        for (int i = 0; i < TM; i += G) ld_vec<T, G>(&As[buf][kk][(i / G) * 16 * G + ty * G], a + i);
#pragma unroll
        for (int j = 0; j < TN; j += G) ld_vec<T, G>(&Bs[buf][kk][(j / G) * 16 * G + tx * G], b + j);
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
      if (kt + 1 < nk) sstore(buf ^ 1);
      __syncthreads();
    }
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int gm = m0 + (i / G) * 16 * G + ty * G + (i % G);
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int gn = n0 + (j / G) * 16 * G + tx * G + (j % G);
      if (gn >= N) continue;
      T v = alpha * acc[i][j];
      if (beta != T(0)) v = fma(beta, C[(int64_t)gm * ldc + gn], v);
      C[(int64_t)gm * ldc + gn] = v;
    }
  }
}

template <class T>
int32_t gemm(cudaStream_t st, bool ta, bool tb, int M, int N, int K, double alpha, const T* A,
             int64_t lda, const T* B, int64_t ldb, double beta, T* C, int64_t ldc,
             bool lower = false, int kflags = 0, int batch = 1, int64_t sA = 0, int64_t sB = 0,
             int64_t sC = 0) {
  if (M <= 0 || N <= 0 || batch <= 0) return FIRAL_OK;
  constexpr int BM = GemmCfg<T>::BM;
  const dim3 grid((N + BM - 1) / BM, (M + BM - 1) / BM, batch);
  ProfScope ps(st, PF_EXACT_GEMM);
  count_launch();
  const T a = (T)alpha, b = (T)beta;
  const int lw = lower ? 1 : 0;
#define FIRAL_GEMM_ARGS M, N, K, a, A, lda, B, ldb, b, C, ldc, lw, kflags, sA, sB, sC
  if (!ta && !tb) k_gemm<T, false, false><<<grid, 256, 0, st>>>(FIRAL_GEMM_ARGS);
  else if (!ta && tb) k_gemm<T, false, true><<<grid, 256, 0, st>>>(FIRAL_GEMM_ARGS);
  else if (ta && !tb) k_gemm<T, true, false><<<grid, 256, 0, st>>>(FIRAL_GEMM_ARGS);
  else k_gemm<T, true, true><<<grid, 256, 0, st>>>(FIRAL_GEMM_ARGS);
#undef FIRAL_GEMM_ARGS
  FIRAL_CUDA_TRY(cudaGetLastError());
  return FIRAL_OK;
}

// ------------------------------------------------------------------ Cholesky / inverse tiles
// Cholesky of the diagonal tile A[j0 .. j0+jb)^2 (lower) in shared memory, in the vec type
// (like the GEMM updates around it), written back in place (zeros above its diagonal), and the
// tile's inverse written to Winv at the same place (lower, zeros above).  One CTA runs the jb
// sequential steps, so the kernel is latency-bound (about 60 us for a 64 x 64 tile on GB300).
// A pivot that is not positive and finite sets *flag and leaves both tiles unwritten.
template <class T>
__global__ __launch_bounds__(256) void k_potrf_diag(T* A, T* Winv, int64_t ld, int j0, int jb,
                                                    int* flag) {
  extern __shared__ __align__(16) unsigned char potrf_raw[];   // L | Li (NB x NB+1 each) | red
  T(*L)[NB + 1] = reinterpret_cast<T(*)[NB + 1]>(potrf_raw);
  T(*Li)[NB + 1] = L + NB;
  T(*red)[NB] = reinterpret_cast<T(*)[NB]>(&Li[NB][0]);
  __shared__ int bad;
  const int tid = threadIdx.x;
  if (tid == 0) bad = 0;
  for (int idx = tid; idx < jb * jb; idx += blockDim.x) {
    const int i = idx / jb, j = idx - i * jb;
    L[i][j] = j <= i ? A[(int64_t)(j0 + i) * ld + j0 + j] : T(0);
  }
  __syncthreads();
  // column k: every thread takes the pivot from L[k][k] (final after step k-1), scales the
  // column below it, and after one barrier updates its share of the trailing triangle; the
  // pivot itself is stored after that barrier, when no thread reads L[k][k] any more.
  const int tx = tid & 15, ty = tid >> 4;
  for (int k = 0; k < jb; ++k) {
    const T p = L[k][k];
    if (!(p > T(0)) || !(p < T(INFINITY))) {
      if (tid == 0) bad = 1;
      break;
    }
    const T piv = sqrt(p);
    if (tid > k && tid < jb) L[tid][k] /= piv;
    __syncthreads();
    if (tid == 0) L[k][k] = piv;
    for (int i = k + 1 + ty; i < jb; i += 16) {
      const T lik = L[i][k];
      for (int j = k + 1 + tx; j <= i; j += 16) L[i][j] = fma(-lik, L[j][k], L[i][j]);
    }
    __syncthreads();
  }
  __syncthreads();
  if (bad) {
    if (tid == 0) atomicExch(flag, 1);
    return;
  }
  // inverse of the lower-triangular tile: forward substitution on the identity, row by row,
  // all NB right-hand sides at once; row i = (e_i - L[i][0:i] Li[0:i][:]) / L[i][i], each dot
  // product split over four threads (entries above the diagonal come out as exact zeros)
  const int col = tid & (NB - 1), part = tid >> 6;
  for (int i = 0; i < jb; ++i) {
    T acc = T(0);
    for (int k = part; k < i; k += 4) acc = fma(L[i][k], Li[k][col], acc);
    red[part][col] = acc;
    __syncthreads();
    if (part == 0 && col < jb) {
      const T v = (col == i ? T(1) : T(0)) -
                  ((red[0][col] + red[1][col]) + (red[2][col] + red[3][col]));
      Li[i][col] = v / L[i][i];
    }
    __syncthreads();
  }
  for (int idx = tid; idx < jb * jb; idx += blockDim.x) {
    const int i = idx / jb, j = idx - i * jb;
    const int64_t o = (int64_t)(j0 + i) * ld + j0 + j;
    A[o] = L[i][j];
    Winv[o] = Li[i][j];
  }
}

// Blocked right-looking Cholesky A = L L^T in place (lower triangle; the strict upper triangle
// of A is left stale outside the diagonal tiles) and W = L^{-1} (lower, zeros above).  Tmp:
// scratch of D * D / 4 elements.  A non-SPD matrix sets *flag.
template <class T>
int32_t potrf_trtri(cudaStream_t st, T* A, T* W, T* Tmp, int64_t D, int* flag) {
  const size_t psm = (2 * NB * (NB + 1) + 4 * NB) * sizeof(T);
  FIRAL_CUDA_TRY(cudaFuncSetAttribute(k_potrf_diag<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)psm));
  {
    ProfScope ps(st, PF_EXACT_FACTOR);
    FIRAL_CUDA_TRY(cudaMemsetAsync(W, 0, (size_t)D * D * sizeof(T), st));
  }
  for (int64_t j0 = 0; j0 < D; j0 += NB) {
    const int jb = (int)std::min<int64_t>(NB, D - j0);
    {
      ProfScope ps(st, PF_EXACT_FACTOR);
      count_launch();
      k_potrf_diag<T><<<1, 256, psm, st>>>(A, W, D, (int)j0, jb, flag);
      FIRAL_CUDA_TRY(cudaGetLastError());
    }
    const int rest = (int)(D - j0 - jb);
    if (rest > 0) {
      T* A21 = A + (j0 + jb) * D + j0;
      // L21 = A21 L11^{-T} (in place: one CTA column, N = jb <= tile width)
      FIRAL_TRY(gemm<T>(st, false, true, rest, jb, jb, 1.0, A21, D, W + j0 * D + j0, D, 0.0,
                        A21, D));
      // A22 -= L21 L21^T (lower tiles)
      FIRAL_TRY(gemm<T>(st, false, true, rest, rest, jb, -1.0, A21, D, A21, D, 1.0, A21 + jb, D,
                        true));
    }
  }
  // W = L^{-1} by doubling: [[P, 0], [Q, R]]^{-1} = [[P^-1, 0], [-R^-1 Q P^-1, R^-1]].  At
  // level s the pairs (P, R) of s x s blocks sit at o = 2 s q; the full ones (R of size s) are
  // one batched launch per product, the ragged last one (R smaller) a launch of its own.
  for (int64_t s = NB; s < D; s *= 2) {
    const int64_t step = 2 * s * (D + 1);           // element distance between pairs
    const int nfull = (int)(D / (2 * s));            // pairs with o + 2 s <= D
    if (nfull > 0) {
      // Tmp_q (s x s) = Q_q P_q^{-1}; P^{-1} is lower triangular
      FIRAL_TRY(gemm<T>(st, false, false, (int)s, (int)s, (int)s, 1.0, A + s * D, D, W, D, 0.0,
                        Tmp, s, false, K_FROM_N0, nfull, step, step, s * s));
      // W_q[c0.., o..] = -R_q^{-1} Tmp_q; R^{-1} is lower triangular
      FIRAL_TRY(gemm<T>(st, false, false, (int)s, (int)s, (int)s, -1.0, W + s * (D + 1), D, Tmp,
                        s, 0.0, W + s * D, D, false, K_TO_M1, nfull, step, s * s, step));
    }
    const int64_t o = 2 * s * nfull, c0 = o + s;
    if (c0 < D) {
      const int cs = (int)(D - c0);
      FIRAL_TRY(gemm<T>(st, false, false, cs, (int)s, (int)s, 1.0, A + c0 * D + o, D,
                        W + o * D + o, D, 0.0, Tmp, s, false, K_FROM_N0));
      FIRAL_TRY(gemm<T>(st, false, false, cs, (int)s, cs, -1.0, W + c0 * D + c0, D, Tmp, s, 0.0,
                        W + c0 * D + o, D, false, K_TO_M1));
    }
  }
  return FIRAL_OK;
}

// --------------------------------------------------------------------- elementwise / sym
// out = a X + b Y + cz Z + diag I over a D x D matrix (null operands skipped)
template <class T>
__global__ void k_combine(T* out, double a, const T* X, double b, const T* Y, double cz,
                          const T* Z, double diag, int64_t D) {
  const int64_t tot = D * D;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot;
       idx += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    if (X) v += a * (double)X[idx];
    if (Y) v += b * (double)Y[idx];
    if (Z) v += cz * (double)Z[idx];
    if (idx / D == idx % D) v += diag;
    out[idx] = (T)v;
  }
}

// Copy the lower triangle onto the upper one, 32 x 32 tiles through shared memory.
template <class T>
__global__ void k_sym_from_lower(T* A, int64_t D) {
  __shared__ T tile[32][33];
  const int bi = blockIdx.y, bj = blockIdx.x;   // destination tile (bi <= bj)
  if (bi > bj) return;
  const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
  for (int r = ty; r < 32; r += 8) {
    const int64_t gi = (int64_t)bj * 32 + r, gj = (int64_t)bi * 32 + tx;   // source (lower)
    tile[r][tx] = (gi < D && gj < D) ? A[gi * D + gj] : T(0);
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int64_t gi = (int64_t)bi * 32 + r, gj = (int64_t)bj * 32 + tx;   // destination
    if (gi < D && gj < D && gj > gi) A[gi * D + gj] = tile[tx][r];
  }
}

template <class T>
int32_t combine(cudaStream_t st, T* out, double a, const T* X, double b, const T* Y, double cz,
                const T* Z, double diag, int64_t D) {
  ProfScope ps(st, PF_EXACT_BUILD);
  count_launch();
  const int64_t tot = D * D;
  const int blocks = (int)std::min<int64_t>((tot + 255) / 256, 4096);
  k_combine<T><<<blocks, 256, 0, st>>>(out, a, X, b, Y, cz, Z, diag, D);
  FIRAL_CUDA_TRY(cudaGetLastError());
  return FIRAL_OK;
}

template <class T>
int32_t sym_from_lower(cudaStream_t st, T* A, int64_t D) {
  ProfScope ps(st, PF_EXACT_GEMM);
  count_launch();
  const int nt = (int)((D + 31) / 32);
  k_sym_from_lower<T><<<dim3(nt, nt), dim3(32, 8), 0, st>>>(A, D);
  FIRAL_CUDA_TRY(cudaGetLastError());
  return FIRAL_OK;
}

// -------------------------------------------------------------------- class-pair build
// Partial sums P_kl = sum_i w_i q_i^{kl} x_i x_i^T over a share of rows [r0, r0 + rows) of X
// and h, q^{kl} = delta_kl h_k - h_k h_l, for the class pair of blockIdx.x; blockIdx.y is the
// row split.  w: weights of rows r0.. (null = 1), all scaled by wsc.  part: DP x DP per
// (split, pair), features e, f < d meaningful.
template <class T, int DPB>
__global__ __launch_bounds__(256) void k_pair_syrk(const T* __restrict__ X,
                                                   const T* __restrict__ Hh,
                                                   const T* __restrict__ w, double wsc,
                                                   int64_t r0, int64_t rows, int d, int c,
                                                   const int2* __restrict__ pairs, int npairs,
                                                   T* __restrict__ part) {
  constexpr int DP = 16 * DPB, CH = 32;
  __shared__ __align__(16) T xs[CH][DP];
  __shared__ T ws[CH];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int2 kl = pairs[blockIdx.x];
  const int64_t per = (rows + gridDim.y - 1) / gridDim.y;
  const int64_t rb = (int64_t)blockIdx.y * per, re = std::min<int64_t>(rows, rb + per);
  T acc[DPB][DPB];
#pragma unroll
  for (int a = 0; a < DPB; ++a)
#pragma unroll
    for (int b = 0; b < DPB; ++b) acc[a][b] = T(0);
  for (int64_t c0 = rb; c0 < re; c0 += CH) {
    __syncthreads();
    for (int idx = tid; idx < CH * DP; idx += 256) {
      const int p = idx / DP, e = idx - p * DP;
      const int64_t i = c0 + p;
      xs[p][e] = (e < d && i < re) ? X[(r0 + i) * d + e] : T(0);
    }
    if (tid < CH) {
      const int64_t i = c0 + tid;
      T v = T(0);
      if (i < re) {
        const T hk = Hh[(r0 + i) * c + kl.x], hl = Hh[(r0 + i) * c + kl.y];
        const T q = (kl.x == kl.y ? hk : T(0)) - hk * hl;
        v = (T)wsc * (w ? w[i] : T(1)) * q;
      }
      ws[tid] = v;
    }
    __syncthreads();
    const int pend = (int)std::min<int64_t>(CH, re - c0);
    for (int p = 0; p < pend; ++p) {
      T xa[DPB], xb[DPB];
      ld_vec<T, DPB>(&xs[p][ty * DPB], xa);
      ld_vec<T, DPB>(&xs[p][tx * DPB], xb);
      const T wp = ws[p];
#pragma unroll
      for (int a = 0; a < DPB; ++a) xa[a] *= wp;
#pragma unroll
      for (int a = 0; a < DPB; ++a)
#pragma unroll
        for (int b = 0; b < DPB; ++b) acc[a][b] = fma(xa[a], xb[b], acc[a][b]);
    }
  }
  T* out = part + ((int64_t)blockIdx.y * npairs + blockIdx.x) * DP * DP;
#pragma unroll
  for (int a = 0; a < DPB; ++a)
#pragma unroll
    for (int b = 0; b < DPB; ++b) out[(ty * DPB + a) * DP + tx * DPB + b] = acc[a][b];
}

// out = sum_splits part + base + s2 base2 + diag I, on the class-pair blocks (k <= l) and
// mirrored onto (l, k).  base / base2 symmetric (may alias out; null = 0).
template <class T>
__global__ void k_pair_reduce(const T* __restrict__ part, int nsplit, int npairs, int DP, int d,
                              const int2* __restrict__ pairs, const T* base, double s2,
                              const T* base2, double diag, T* out, int64_t D) {
  const int64_t tot = (int64_t)npairs * d * d;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int p = (int)(idx / ((int64_t)d * d));
    const int r = (int)(idx - (int64_t)p * d * d);
    const int e = r / d, f = r - e * d;
    const int2 kl = pairs[p];
    double v = 0.0;
    for (int s = 0; s < nsplit; ++s) v += (double)part[((int64_t)s * npairs + p) * DP * DP + e * DP + f];
    const int64_t pos = ((int64_t)kl.x * d + e) * D + (int64_t)kl.y * d + f;
    if (base) v += (double)base[pos];
    if (base2) v += s2 * (double)base2[pos];
    if (kl.x == kl.y && e == f) v += diag;
    out[pos] = (T)v;
    if (kl.x != kl.y) out[((int64_t)kl.y * d + f) * D + (int64_t)kl.x * d + e] = (T)v;
  }
}

// --------------------------------------------------------------- class-pair quadratic forms
// For the points [r0, r0 + nrows) and the class pairs of pair group blockIdx.y:
//   MODE 0: gpart[y][i] = -sum_pairs (2 - delta_kl) q_i^{kl} x_i^T M1_kl x_i   (eq. 6 with M1 =
//           Sigma^-1 H_p Sigma^-1, symmetric);
//   MODE 1: K1[i][k][l] = K1[i][l][k] = x_i^T M1_kl x_i, the same for M2 into K2.
// Thread (pg, fg) owns points pg*PT .. +PT and features fg*DPB .. +DPB of the CTA's tile.
template <class T, int DPB, int PT, int MODE>
__global__ __launch_bounds__(256, 1) void k_pair_quad(const T* __restrict__ X,
                                                   const T* __restrict__ Hh, int64_t r0,
                                                   int64_t nrows, int d, int c,
                                                   const int2* __restrict__ pairs, int npairs,
                                                   int ppg, const T* __restrict__ M1,
                                                   const T* __restrict__ M2, int64_t ld,
                                                   double* __restrict__ gpart,
                                                   T* __restrict__ K1, T* __restrict__ K2) {
  constexpr int DP = 16 * DPB, PTS = 16 * PT;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* xs = reinterpret_cast<T*>(smraw);   // [DP][PTS]
  T* Ms = xs + DP * PTS;                 // [DP][DP]
  const int tid = threadIdx.x, fg = tid & 15, pg = tid >> 4;
  const int64_t t0 = (int64_t)blockIdx.x * PTS;
  for (int idx = tid; idx < PTS * DP; idx += 256) {
    const int p = idx / DP, e = idx - p * DP;
    const int64_t i = t0 + p;
    xs[e * PTS + p] = (e < d && i < nrows) ? X[(r0 + i) * d + e] : T(0);
  }
  __syncthreads();
  T xr[PT][DPB];
#pragma unroll
  for (int a = 0; a < PT; ++a)
#pragma unroll
    for (int b = 0; b < DPB; ++b) xr[a][b] = xs[(fg * DPB + b) * PTS + pg * PT + a];
  double gacc[PT];
#pragma unroll
  for (int a = 0; a < PT; ++a) gacc[a] = 0.0;
  const int pb = blockIdx.y * ppg, pe = std::min(npairs, pb + ppg);
  for (int pi = pb; pi < pe; ++pi) {
    const int2 kl = pairs[pi];
    for (int which = 0; which < (MODE == 1 ? 2 : 1); ++which) {
      const T* Mg = (which ? M2 : M1) + (int64_t)kl.x * d * ld + (int64_t)kl.y * d;
      __syncthreads();
      for (int idx = tid; idx < DP * DP; idx += 256) {
        const int e = idx / DP, f = idx - e * DP;
        Ms[idx] = (e < d && f < d) ? Mg[(int64_t)e * ld + f] : T(0);
      }
      __syncthreads();
      T acc[PT][DPB];
#pragma unroll
      for (int a = 0; a < PT; ++a)
#pragma unroll
        for (int b = 0; b < DPB; ++b) acc[a][b] = T(0);
      for (int e = 0; e < d; ++e) {
        T xa[PT], mb[DPB];
        ld_vec<T, PT>(&xs[e * PTS + pg * PT], xa);
        ld_vec<T, DPB>(&Ms[e * DP + fg * DPB], mb);
#pragma unroll
        for (int a = 0; a < PT; ++a)
#pragma unroll
          for (int b = 0; b < DPB; ++b) acc[a][b] = fma(xa[a], mb[b], acc[a][b]);
      }
#pragma unroll
      for (int a = 0; a < PT; ++a) {
        T s = T(0);
#pragma unroll
        for (int b = 0; b < DPB; ++b) s = fma(acc[a][b], xr[a][b], s);
#pragma unroll
        for (int o = 1; o < 16; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        const int64_t i = t0 + pg * PT + a;
        if (fg == 0 && i < nrows) {
          if (MODE == 0) {
            const double hk = (double)Hh[(r0 + i) * c + kl.x], hl = (double)Hh[(r0 + i) * c + kl.y];
            const double q = (kl.x == kl.y ? hk : 0.0) - hk * hl;
            gacc[a] -= (kl.x == kl.y ? 1.0 : 2.0) * q * (double)s;
          } else {
            T* Ko = (which ? K2 : K1) + i * c * c;
            Ko[kl.x * c + kl.y] = s;
            Ko[kl.y * c + kl.x] = s;
          }
        }
      }
    }
  }
  if (MODE == 0 && fg == 0) {
#pragma unroll
    for (int a = 0; a < PT; ++a) {
      const int64_t i = t0 + pg * PT + a;
      if (i < nrows) gpart[(int64_t)blockIdx.y * nrows + i] = gacc[a];
    }
  }
}

// g[i] = sum over pair groups of gpart
template <class T>
__global__ void k_sum_groups(const double* __restrict__ gpart, int ng, int64_t n, T* g) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int s = 0; s < ng; ++s) v += gpart[(int64_t)s * n + i];
    g[i] = (T)v;
  }
}

// ---------------------------------------------------------------------- Round scores
// r_i = Tr(Sigma G^-1) - eta Tr[(I + eta Psi K1)^{-1} Psi K2], Psi = diag(h_i) - h_i h_i^T
// (eq. 9 through the Woodbury identity with H_i = (I (x) x_i) Psi (I (x) x_i)^T), for the
// candidates j of a chunk (pool index i0 + j, h row r0 + j).  One CTA per candidate; FP64
// Gaussian elimination with partial pivoting on [E | F] in shared memory, then one thread per
// right-hand side column for the back substitution.  negr[i] = -r_i (-inf when masked).
template <class T>
__global__ __launch_bounds__(128) void k_exact_score(const T* __restrict__ K1,
                                                     const T* __restrict__ K2,
                                                     const T* __restrict__ Hh, int64_t r0,
                                                     int64_t i0, int c, double eta,
                                                     const double* __restrict__ tr1,
                                                     const uint8_t* __restrict__ mask,
                                                     double* __restrict__ negr) {
  extern __shared__ __align__(16) double sm[];
  double* E = sm;               // c x c
  double* F = E + c * c;        // c x c
  double* hs = F + c * c;       // c
  double* u = hs + c;           // c
  double* v = u + c;            // c
  double* fac = v + c;          // c
  __shared__ int piv_row;
  __shared__ double red[4];
  const int tid = threadIdx.x;
  const int64_t j = blockIdx.x, i = i0 + j;
  if (mask && mask[i]) {
    if (tid == 0) negr[i] = -INFINITY;
    return;
  }
  const int cc = c * c;
  for (int q = tid; q < c; q += blockDim.x) hs[q] = (double)Hh[(r0 + j) * c + q];
  for (int q = tid; q < cc; q += blockDim.x) {
    E[q] = (double)K1[j * cc + q];
    F[q] = (double)K2[j * cc + q];
  }
  __syncthreads();
  for (int l = tid; l < c; l += blockDim.x) {
    double su = 0.0, sv = 0.0;
    for (int m = 0; m < c; ++m) {
      su = fma(hs[m], E[m * c + l], su);
      sv = fma(hs[m], F[m * c + l], sv);
    }
    u[l] = su;
    v[l] = sv;
  }
  __syncthreads();
  for (int q = tid; q < cc; q += blockDim.x) {
    const int jj = q / c, l = q - jj * c;
    E[q] = (jj == l ? 1.0 : 0.0) + eta * hs[jj] * (E[q] - u[l]);
    F[q] = hs[jj] * (F[q] - v[l]);
  }
  __syncthreads();
  for (int col = 0; col < c; ++col) {
    if (tid < 32) {
      double best = -1.0;
      int bidx = col;
      for (int r = col + tid; r < c; r += 32) {
        const double a = fabs(E[r * c + col]);
        if (a > best) { best = a; bidx = r; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bidx, o);
        if (ob > best || (ob == best && oi < bidx)) { best = ob; bidx = oi; }
      }
      if (tid == 0) piv_row = bidx;
    }
    __syncthreads();
    const int pr = piv_row;
    if (pr != col) {
      for (int q = tid; q < 2 * c; q += blockDim.x) {
        double* Mx = q < c ? E : F;
        const int k = q < c ? q : q - c;
        const double t = Mx[col * c + k];
        Mx[col * c + k] = Mx[pr * c + k];
        Mx[pr * c + k] = t;
      }
      __syncthreads();
    }
    const double dpiv = E[col * c + col];
    for (int r = col + 1 + tid; r < c; r += blockDim.x) fac[r] = E[r * c + col] / dpiv;
    __syncthreads();
    const int nr = c - col - 1, ne = c - col - 1, ncol = ne + c;
    for (int q = tid; q < nr * ncol; q += blockDim.x) {
      const int r = col + 1 + q / ncol, k = q % ncol;
      if (k < ne) E[r * c + col + 1 + k] -= fac[r] * E[col * c + col + 1 + k];
      else F[r * c + (k - ne)] -= fac[r] * F[col * c + (k - ne)];
    }
    __syncthreads();
  }
  double tr = 0.0;
  for (int l = tid; l < c; l += blockDim.x) {
    for (int jj = c - 1; jj >= 0; --jj) {
      double s = F[jj * c + l];
      for (int k = jj + 1; k < c; ++k) s = fma(-E[jj * c + k], F[k * c + l], s);
      F[jj * c + l] = s / E[jj * c + jj];
    }
    tr += F[l * c + l];
  }
  for (int o = 16; o > 0; o >>= 1) tr += __shfl_xor_sync(0xffffffffu, tr, o);
  if ((tid & 31) == 0) red[tid >> 5] = tr;
  __syncthreads();
  if (tid == 0) {
    const double t = red[0] + red[1] + red[2] + red[3];
    const double r = *tr1 - eta * t;
    negr[i] = (r == r) ? -r : -INFINITY;
  }
}

// Block-wise argmax of v[0..n) (lowest index on ties), one partial per block.
__global__ void k_argmax_partial(const double* __restrict__ v, int64_t n, double* pv,
                                 int64_t* pi) {
  __shared__ double bv[8];
  __shared__ int64_t bi[8];
  const int64_t per = (n + gridDim.x - 1) / gridDim.x;
  const int64_t b0 = (int64_t)blockIdx.x * per, b1 = std::min<int64_t>(n, b0 + per);
  double val = -INFINITY;
  int64_t idx = INT64_MAX;
  for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
    const double x = v[i];
    if (x > val || (x == val && i < idx)) { val = x; idx = i; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, val, o);
    const int64_t oi = __shfl_xor_sync(0xffffffffu, idx, o);
    if (ov > val || (ov == val && oi < idx)) { val = ov; idx = oi; }
  }
  if ((threadIdx.x & 31) == 0) { bv[threadIdx.x >> 5] = val; bi[threadIdx.x >> 5] = idx; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      if (bv[w] > val || (bv[w] == val && bi[w] < idx)) { val = bv[w]; idx = bi[w]; }
    pv[blockIdx.x] = val;
    pi[blockIdx.x] = idx;
  }
}

// Rank-c factors of L^{-1} H_i L^{-T} = Y Psi Y^T for one point: Y[r][k] = sum_e
// Linv[r][k d + e] x_e (thread per (r, k)), then Z = Y Psi (thread per (r, l)).
template <class T>
__global__ void k_exact_y(const T* __restrict__ Linv, int64_t D, const T* __restrict__ x, int d,
                          int c, T* __restrict__ Y) {
  const int64_t tot = D * c;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = idx / c;
    const int k = (int)(idx - r * c);
    const T* row = Linv + r * D + (int64_t)k * d;
    double s = 0.0;
    for (int e = 0; e < d; ++e) s = fma((double)row[e], (double)x[e], s);
    Y[idx] = (T)s;
  }
}
template <class T>
__global__ void k_exact_z(const T* __restrict__ Y, int64_t D, const T* __restrict__ h, int c,
                          T* __restrict__ Z) {
  const int64_t tot = D * c;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < tot;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = idx / c;
    const int l = (int)(idx - r * c);
    double s = 0.0;
    for (int k = 0; k < c; ++k) s = fma((double)Y[r * c + k], (double)h[k], s);
    Z[idx] = (T)((double)h[l] * ((double)Y[idx] - s));
  }
}

// ------------------------------------------------------------------------- host helpers
template <class T>
size_t quad_smem(int dpb) {
  const int DP = 16 * dpb, PTS = 16 * (dpb == 8 ? 4 : 8);
  return (size_t)(DP * PTS + DP * DP) * sizeof(T);
}

int dpb_of(int d) {
  const int dp = ((d + 15) / 16) * 16;
  const int b = dp / 16;
  return b <= 1 ? 1 : b <= 2 ? 2 : b <= 4 ? 4 : 8;
}

template <class T>
T* mat(ExactWs& ex, int i) {
  return ex.m[i].as<T>();
}

int32_t ensure_pairs(firal_problem* P) {
  ExactWs& ex = *P->ex;
  const int c = P->c;
  const int np = c * (c + 1) / 2;
  if (ex.npairs == np) return FIRAL_OK;
  std::vector<int2> tab;
  tab.reserve(np);
  for (int k = 0; k < c; ++k)
    for (int l = k; l < c; ++l) tab.push_back(make_int2(k, l));
  FIRAL_TRY(ex.pairs.ensure(tab.size() * sizeof(int2)));
  FIRAL_CUDA_TRY(cudaMemcpyAsync(ex.pairs.p, tab.data(), tab.size() * sizeof(int2),
                                 cudaMemcpyHostToDevice, P->H->stream));
  FIRAL_CUDA_TRY(cudaStreamSynchronize(P->H->stream));
  ex.npairs = np;
  return FIRAL_OK;
}

// out = base + s2 base2 + diag I + wsc sum_{rows [r0, r0 + rows)} w_i H_i (dense, symmetric)
template <class T>
int32_t pair_build(firal_problem* P, int64_t r0, int64_t rows, const T* w, double wsc,
                   const T* base, double s2, const T* base2, double diag, T* out) {
  ExactWs& ex = *P->ex;
  cudaStream_t st = P->H->stream;
  const int d = P->d, c = P->c, dpb = dpb_of(d), DP = 16 * dpb;
  const int np = ex.npairs;
  int ns = (int)std::max<int64_t>(1, std::min<int64_t>((2LL * P->sms + np - 1) / np, rows / 256));
  ns = std::max(1, std::min(ns, 64));
  FIRAL_TRY(ex.part.ensure((size_t)ns * np * DP * DP * sizeof(T)));
  const dim3 grid(np, ns);
  {
    ProfScope ps(st, PF_EXACT_BUILD);
    count_launch(2);
    T* part = ex.part.as<T>();
    const int2* pr = ex.pairs.as<int2>();
    if (rows > 0) {
      switch (dpb) {
        case 1: k_pair_syrk<T, 1><<<grid, 256, 0, st>>>(P->Xa.as<T>(), P->Ha.as<T>(), w, wsc, r0, rows, d, c, pr, np, part); break;
        case 2: k_pair_syrk<T, 2><<<grid, 256, 0, st>>>(P->Xa.as<T>(), P->Ha.as<T>(), w, wsc, r0, rows, d, c, pr, np, part); break;
        case 4: k_pair_syrk<T, 4><<<grid, 256, 0, st>>>(P->Xa.as<T>(), P->Ha.as<T>(), w, wsc, r0, rows, d, c, pr, np, part); break;
        default: k_pair_syrk<T, 8><<<grid, 256, 0, st>>>(P->Xa.as<T>(), P->Ha.as<T>(), w, wsc, r0, rows, d, c, pr, np, part); break;
      }
      FIRAL_CUDA_TRY(cudaGetLastError());
    } else {
      FIRAL_CUDA_TRY(cudaMemsetAsync(part, 0, (size_t)np * DP * DP * sizeof(T), st));
      ns = 1;
    }
    const int64_t tot = (int64_t)np * d * d;
    const int blocks = (int)std::min<int64_t>((tot + 255) / 256, 8192);
    k_pair_reduce<T><<<blocks, 256, 0, st>>>(part, ns, np, DP, d, pr, base, s2, base2, diag,
                                             out, P->D);
    FIRAL_CUDA_TRY(cudaGetLastError());
  }
  return FIRAL_OK;
}

template <class T, int MODE>
int32_t pair_quad_launch(firal_problem* P, int64_t r0, int64_t nrows, const T* M1, const T* M2,
                         double* gpart, T* K1, T* K2, int* ngroups_out) {
  ExactWs& ex = *P->ex;
  cudaStream_t st = P->H->stream;
  const int d = P->d, c = P->c, dpb = dpb_of(d);
  const int PTS = 16 * (dpb == 8 ? 4 : 8);
  const int np = ex.npairs;
  const int64_t tiles = (nrows + PTS - 1) / PTS;
  // pair groups spread the CTAs over the SMs; every (point, pair) output belongs to one CTA
  int ng = (int)std::min<int64_t>(np, std::max<int64_t>(1, (4LL * P->sms + tiles - 1) / tiles));
  ng = std::min(ng, 64);
  const int ppg = (np + ng - 1) / ng;
  ng = (np + ppg - 1) / ppg;
  if (ngroups_out) *ngroups_out = ng;
  const size_t sm = quad_smem<T>(dpb);
  const dim3 grid((unsigned)tiles, ng);
  const int2* pr = ex.pairs.as<int2>();
  const T* X = P->Xa.as<T>();
  const T* Hh = P->Ha.as<T>();
  ProfScope ps(st, PF_EXACT_QUAD);
  count_launch();
#define FIRAL_QUAD_CASE(B, PTv)                                                               \
  case B: {                                                                                   \
    auto kf = k_pair_quad<T, B, PTv, MODE>;                                                   \
    FIRAL_CUDA_TRY(cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize,      \
                                        (int)sm));                                            \
    kf<<<grid, 256, sm, st>>>(X, Hh, r0, nrows, d, c, pr, np, ppg, M1, M2, P->D, gpart, K1,   \
                              K2);                                                            \
    break;                                                                                    \
  }
  switch (dpb) {
    FIRAL_QUAD_CASE(1, 8)
    FIRAL_QUAD_CASE(2, 8)
    FIRAL_QUAD_CASE(4, 8)
    default: {
      auto kf = k_pair_quad<T, 8, 4, MODE>;
      FIRAL_CUDA_TRY(cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
      kf<<<grid, 256, sm, st>>>(X, Hh, r0, nrows, d, c, pr, np, ppg, M1, M2, P->D, gpart, K1, K2);
      break;
    }
  }
#undef FIRAL_QUAD_CASE
  FIRAL_CUDA_TRY(cudaGetLastError());
  return FIRAL_OK;
}

int32_t read_flag(firal_problem* P, int* val) {
  cudaStream_t st = P->H->stream;
  FIRAL_CUDA_TRY(cudaMemcpyAsync(val, P->ex->flag.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  FIRAL_CUDA_TRY(cudaStreamSynchronize(st));
  return FIRAL_OK;
}

int32_t clear_flag(firal_problem* P) {
  FIRAL_CUDA_TRY(cudaMemsetAsync(P->ex->flag.p, 0, sizeof(int), P->H->stream));
  return FIRAL_OK;
}

int32_t ensure_ws(firal_problem* P) {
  if (!P->ex) P->ex = new ExactWs();
  ExactWs& ex = *P->ex;
  const size_t vs = P->dbl ? 8 : 4;
  const size_t DD = (size_t)P->D * P->D * vs;
  for (int i = 0; i < EX_MATS_RELAX; ++i) FIRAL_TRY(ex.m[i].ensure(DD));
  FIRAL_TRY(ex.flag.ensure(64));
  FIRAL_TRY(ex.scal.ensure(4096 * sizeof(double)));
  FIRAL_TRY(ensure_pairs(P));
  return FIRAL_OK;
}

// H_o (labelled Hessians + lambda I) and H_p (pool average), cached for the problem's life.
template <class T>
int32_t ensure_ho_hp(firal_problem* P) {
  ExactWs& ex = *P->ex;
  if (!ex.ho_ready) {
    FIRAL_TRY(pair_build<T>(P, 0, P->m, nullptr, 1.0, nullptr, 0.0, nullptr, P->lambda,
                            mat<T>(ex, EX_HO)));
    ex.ho_ready = true;
  }
  if (!ex.hp_ready) {
    FIRAL_TRY(pair_build<T>(P, P->m, P->n, nullptr, 1.0 / (double)P->n, nullptr, 0.0, nullptr,
                            0.0, mat<T>(ex, EX_HP)));
    ex.hp_ready = true;
  }
  return FIRAL_OK;
}

template <class T>
int32_t objective_t(firal_problem* P, const T* z, double* f_host, T* g) {
  FIRAL_TRY(ensure_ws(P));
  ExactWs& ex = *P->ex;
  cudaStream_t st = P->H->stream;
  const int64_t D = P->D;
  FIRAL_TRY(ensure_ho_hp<T>(P));
  T* A = mat<T>(ex, EX_A);
  T* W = mat<T>(ex, EX_W);
  T* S = mat<T>(ex, EX_S);
  T* T1 = mat<T>(ex, EX_T);
  T* M = mat<T>(ex, EX_M);
  // Sigma_z = H_o + sum_pool z_i H_i (eq. 7)
  FIRAL_TRY(pair_build<T>(P, P->m, P->n, z, 1.0, mat<T>(ex, EX_HO), 0.0, nullptr, 0.0, A));
  FIRAL_TRY(clear_flag(P));
  FIRAL_TRY(potrf_trtri<T>(st, A, W, T1, D, P->ex->flag.as<int>()));
  // Sigma^{-1} = W^T W
  FIRAL_TRY(gemm<T>(st, true, false, (int)D, (int)D, (int)D, 1.0, W, D, W, D, 0.0, S, D, true,
                    K_FROM_N0 | K_FROM_M0));
  FIRAL_TRY(sym_from_lower<T>(st, S, D));
  double* f_dev = ex.scal.as<double>();
  FIRAL_TRY(dot_scaled(P->dbl, S, mat<T>(ex, EX_HP), D * D, 1.0, f_dev + 64, f_dev, st));
  if (g) {
    // M = Sigma^{-1} H_p Sigma^{-1}, then g_i = -Tr(H_i M) (eq. 6)
    FIRAL_TRY(gemm<T>(st, false, false, (int)D, (int)D, (int)D, 1.0, S, D, mat<T>(ex, EX_HP), D,
                      0.0, T1, D));
    FIRAL_TRY(gemm<T>(st, false, false, (int)D, (int)D, (int)D, 1.0, T1, D, S, D, 0.0, M, D));
    int ng = 1;
    const int PTS = 16 * (dpb_of(P->d) == 8 ? 4 : 8);
    const int64_t tiles = (P->n + PTS - 1) / PTS;
    const int ngmax = (int)std::min<int64_t>(64, std::max<int64_t>(1, (4LL * P->sms + tiles - 1) / tiles));
    FIRAL_TRY(ex.gpart.ensure((size_t)ngmax * P->n * sizeof(double)));
    FIRAL_TRY((pair_quad_launch<T, 0>(P, P->m, P->n, M, nullptr, ex.gpart.as<double>(), nullptr,
                                      nullptr, &ng)));
    ProfScope ps(st, PF_EXACT_QUAD);
    count_launch();
    const int blocks = (int)std::min<int64_t>((P->n + 255) / 256, 4096);
    k_sum_groups<T><<<blocks, 256, 0, st>>>(ex.gpart.as<double>(), ng, P->n, g);
    FIRAL_CUDA_TRY(cudaGetLastError());
  }
  double hv[1];
  FIRAL_CUDA_TRY(cudaMemcpyAsync(hv, f_dev, sizeof(double), cudaMemcpyDeviceToHost, st));
  int bad = 0;
  FIRAL_TRY(read_flag(P, &bad));
  if (bad) return fail(FIRAL_ERR_NOT_SPD, "Sigma_z is not positive definite");
  if (!(hv[0] == hv[0]) || std::isinf(hv[0])) return fail(FIRAL_ERR_NONFINITE, "f(z) not finite");
  if (f_host) *f_host = hv[0];
  return FIRAL_OK;
}

// Tr((nu I + Mhat)^{-2}) and Tr((nu I + Mhat)^{-3}) through the Cholesky factor C of
// nu I + Mhat: S = C^{-T} C^{-1} is the inverse, Tr(S^2) = <S, S>, Tr(S^3) = <S S, S>.  *pd = 0
// when nu I + Mhat is not positive definite.
template <class T>
int32_t trace_inv_pows(firal_problem* P, double nu, double* v2, double* v3, int* pd) {
  ExactWs& ex = *P->ex;
  cudaStream_t st = P->H->stream;
  const int64_t D = P->D;
  T* X = mat<T>(ex, EX_A);
  T* W = mat<T>(ex, EX_W);
  T* S = mat<T>(ex, EX_S);
  T* S2 = mat<T>(ex, EX_M);
  FIRAL_TRY(combine<T>(st, X, 1.0, mat<T>(ex, EX_MHAT), 0.0, nullptr, 0.0, nullptr, nu, D));
  FIRAL_TRY(clear_flag(P));
  FIRAL_TRY(potrf_trtri<T>(st, X, W, mat<T>(ex, EX_T), D, ex.flag.as<int>()));
  FIRAL_TRY(gemm<T>(st, true, false, (int)D, (int)D, (int)D, 1.0, W, D, W, D, 0.0, S, D, true,
                    K_FROM_N0 | K_FROM_M0));
  FIRAL_TRY(sym_from_lower<T>(st, S, D));
  FIRAL_TRY(gemm<T>(st, false, false, (int)D, (int)D, (int)D, 1.0, S, D, S, D, 0.0, S2, D));
  double* sc = ex.scal.as<double>();
  FIRAL_TRY(dot_scaled(P->dbl, S, S, D * D, 1.0, sc + 64, sc + 1, st));
  FIRAL_TRY(dot_scaled(P->dbl, S2, S, D * D, 1.0, sc + 64, sc + 4, st));
  double h[4] = {0, 0, 0, 0};
  FIRAL_CUDA_TRY(cudaMemcpyAsync(h, sc + 1, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
  int bad = 0;
  FIRAL_TRY(read_flag(P, &bad));
  *v2 = h[0];
  *v3 = h[3];
  *pd = (!bad && h[0] == h[0] && h[0] > 0.0 && !std::isinf(h[0]) && h[3] > 0.0 &&
         !std::isinf(h[3])) ? 1 : 0;
  return FIRAL_OK;
}

// nu with Tr((nu I + Mhat)^{-2}) = 1 (eq. 10), starting from hi where Tr(...) <= 1.
// psi(nu) = Tr(...)^{-1/2} - 1 is increasing and concave (a power mean of nu + lambda_j with
// exponent -2), so Newton steps land left of the root at most once and then climb to it
// monotonically; a trial point where nu I + Mhat is not positive definite halves the bracket.
template <class T>
int32_t nu_root(firal_problem* P, double hi, double* nu_out, int* evals) {
  const double tol = P->dbl ? 1e-13 : 2e-6;        // on psi
  const double brk = P->dbl ? 1e-14 : 1e-7;        // relative bracket width
  double lo = -INFINITY, x = hi;
  *evals = 0;
  for (int it = 0; it < 60; ++it) {
    double v2, v3;
    int pd;
    FIRAL_TRY(trace_inv_pows<T>(P, x, &v2, &v3, &pd));
    ++*evals;
    if (!pd) {
      if (it == 0) return fail(FIRAL_ERR_NOT_SPD, "nu root: A_t not positive definite");
      lo = x;
      x = 0.5 * (lo + hi);
      continue;
    }
    const double psi = 1.0 / std::sqrt(v2) - 1.0;
    if (std::fabs(psi) <= tol) { *nu_out = x; return FIRAL_OK; }
    if (psi > 0.0) hi = x; else lo = x;
    if (std::isfinite(lo) && hi - lo <= brk * std::max(1.0, std::fabs(hi))) break;
    const double dpsi = v3 / (v2 * std::sqrt(v2));   // psi'(nu) = Tr(S^3) / Tr(S^2)^{3/2}
    double xn = x - psi / dpsi;
    if (!(dpsi > 0.0) || !std::isfinite(xn) || xn >= hi || (std::isfinite(lo) && xn <= lo))
      xn = std::isfinite(lo) ? 0.5 * (lo + hi) : x - std::fabs(psi) - 1.0;
    x = xn;
  }
  *nu_out = std::isfinite(lo) ? 0.5 * (lo + hi) : hi;
  return FIRAL_OK;
}

template <class T>
int32_t round_t(firal_problem* P, const T* zd, int b, double eta, int exclude, int32_t* sel,
                double* r_host, double* nu_host, int* evals_total) {
  FIRAL_TRY(ensure_ws(P));
  ExactWs& ex = *P->ex;
  const size_t vs = sizeof(T);
  const int64_t D = P->D;
  const int c = P->c, d = P->d;
  const size_t DD = (size_t)D * D * vs;
  for (int i = EX_MATS_RELAX; i < EX_MATS; ++i) FIRAL_TRY(ex.m[i].ensure(DD));
  cudaStream_t st = P->H->stream;
  FIRAL_TRY(ensure_ho_hp<T>(P));
  T* Ho = mat<T>(ex, EX_HO);
  T* Sig = mat<T>(ex, EX_SIG);
  T* Linv = mat<T>(ex, EX_LINV);
  T* Hsum = mat<T>(ex, EX_HSUM);
  T* Hho = mat<T>(ex, EX_HHO);
  T* Mhat = mat<T>(ex, EX_MHAT);
  T* A = mat<T>(ex, EX_A);
  T* W = mat<T>(ex, EX_W);
  T* S = mat<T>(ex, EX_S);
  T* T1 = mat<T>(ex, EX_T);
  T* M2 = mat<T>(ex, EX_M);
  // candidates per chunk: two c x c matrices each, at most ~1 GiB
  const int64_t per = (int64_t)c * c * 2 * vs;
  const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(P->n, (1LL << 30) / per));
  FIRAL_TRY(ex.K.ensure((size_t)chunk * per));
  FIRAL_TRY(ex.YZ.ensure((size_t)D * c * 2 * vs));
  FIRAL_TRY(ex.negr.ensure((size_t)P->n * sizeof(double)));
  FIRAL_TRY(ex.mask.ensure((size_t)P->n));
  const int np = 512;
  FIRAL_TRY(ex.argp.ensure((size_t)np * 16));
  double* pv = ex.argp.as<double>();
  int64_t* pi = reinterpret_cast<int64_t*>(pv + np);
  double* sc = ex.scal.as<double>();   // [0] f, [1] trace, [2] tr1, [3] pick score, [64..] partials
  FIRAL_CUDA_TRY(cudaMemsetAsync(ex.mask.p, 0, (size_t)P->n, st));
  // Sigma_diamond = H_o + H_{z_diamond}; L^{-1}; H^_o = L^{-1} H_o L^{-T}
  FIRAL_TRY(pair_build<T>(P, P->m, P->n, zd, 1.0, Ho, 0.0, nullptr, 0.0, Sig));
  FIRAL_TRY(combine<T>(st, A, 1.0, Sig, 0.0, nullptr, 0.0, nullptr, 0.0, D));
  FIRAL_TRY(clear_flag(P));
  FIRAL_TRY(potrf_trtri<T>(st, A, Linv, T1, D, ex.flag.as<int>()));
  {
    int bad = 0;
    FIRAL_TRY(read_flag(P, &bad));
    if (bad) return fail(FIRAL_ERR_NOT_SPD, "Sigma_diamond is not positive definite");
  }
  FIRAL_TRY(gemm<T>(st, false, false, (int)D, (int)D, (int)D, 1.0, Linv, D, Ho, D, 0.0, T1, D,
                    false, K_TO_M1));
  FIRAL_TRY(gemm<T>(st, false, true, (int)D, (int)D, (int)D, 1.0, T1, D, Linv, D, 0.0, Hho, D,
                    true));
  FIRAL_TRY(sym_from_lower<T>(st, Hho, D));
  FIRAL_CUDA_TRY(cudaMemsetAsync(Hsum, 0, DD, st));
  FIRAL_CUDA_TRY(cudaMemsetAsync(Mhat, 0, DD, st));
  double nu = std::sqrt((double)D);   // A_1 = sqrt(d~) I
  *evals_total = 0;
  T* K1 = ex.K.as<T>();
  T* K2 = K1 + (size_t)chunk * c * c;
  T* Y = ex.YZ.as<T>();
  T* Z = Y + (size_t)D * c;
  const size_t score_smem = (size_t)(2 * c * c + 4 * c) * sizeof(double);
  FIRAL_CUDA_TRY(cudaFuncSetAttribute(k_exact_score<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)score_smem));
  for (int t = 0; t < b; ++t) {
    if (nu_host) nu_host[t] = nu;
    // G_t = nu Sigma + eta H_sum + (eta / b) H_o; Tr[(A_t + eta/b H~_o + eta H~_i)^{-1}] =
    // Tr[Sigma (G_t + eta H_i)^{-1}] (eqs. 8, 9)
    FIRAL_TRY(combine<T>(st, A, nu, Sig, eta, Hsum, eta / b, Ho, 0.0, D));
    FIRAL_TRY(clear_flag(P));
    FIRAL_TRY(potrf_trtri<T>(st, A, W, T1, D, ex.flag.as<int>()));
    FIRAL_TRY(gemm<T>(st, true, false, (int)D, (int)D, (int)D, 1.0, W, D, W, D, 0.0, S, D, true,
                      K_FROM_N0 | K_FROM_M0));
    FIRAL_TRY(sym_from_lower<T>(st, S, D));                              // S = G^{-1}
    FIRAL_TRY(dot_scaled(P->dbl, Sig, S, D * D, 1.0, sc + 64, sc + 2, st));   // Tr(Sigma G^-1)
    FIRAL_TRY(gemm<T>(st, false, false, (int)D, (int)D, (int)D, 1.0, S, D, Sig, D, 0.0, T1, D));
    FIRAL_TRY(gemm<T>(st, false, false, (int)D, (int)D, (int)D, 1.0, T1, D, S, D, 0.0, M2, D));
    for (int64_t c0 = 0; c0 < P->n; c0 += chunk) {
      const int64_t cn = std::min<int64_t>(chunk, P->n - c0);
      FIRAL_TRY((pair_quad_launch<T, 1>(P, P->m + c0, cn, S, M2, nullptr, K1, K2, nullptr)));
      ProfScope ps(st, PF_EXACT_SCORE);
      count_launch();
      k_exact_score<T><<<(unsigned)cn, 128, score_smem, st>>>(
          K1, K2, P->Ha.as<T>(), P->m + c0, c0, c, eta, sc + 2,
          exclude ? ex.mask.as<uint8_t>() : nullptr, ex.negr.as<double>());
      FIRAL_CUDA_TRY(cudaGetLastError());
    }
    {
      ProfScope ps(st, PF_EXACT_SCORE);
      count_launch();
      const int npart = (int)std::min<int64_t>(np, (P->n + 255) / 256);
      k_argmax_partial<<<npart, 256, 0, st>>>(ex.negr.as<double>(), P->n, pv, pi);
      FIRAL_CUDA_TRY(cudaGetLastError());
      FIRAL_TRY(round_pick(pv, pi, npart, ex.mask.as<uint8_t>(), sel, t, sc + 3, st));
    }
    int32_t it = 0;
    double best = 0.0;
    FIRAL_CUDA_TRY(cudaMemcpyAsync(&it, sel + t, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    FIRAL_CUDA_TRY(cudaMemcpyAsync(&best, sc + 3, sizeof(double), cudaMemcpyDeviceToHost, st));
    int bad = 0;
    FIRAL_TRY(read_flag(P, &bad));
    if (bad) return fail(FIRAL_ERR_NOT_SPD, "Round: G_t is not positive definite");
    if (it < 0 || it >= P->n) return fail(FIRAL_ERR_NONFINITE, "Round: no finite score");
    if (r_host) r_host[t] = -best;
    if (t + 1 == b) break;
    // H~ += H~_o / b + H~_{i_t}: dense H_sum and Mhat = eta L^{-1} H_sum L^{-T}
    FIRAL_TRY(pair_build<T>(P, P->m + it, 1, nullptr, 1.0, Hsum, 1.0 / b, Ho, 0.0, Hsum));
    {
      ProfScope ps(st, PF_EXACT_BUILD);
      count_launch(2);
      const T* xi = P->Xa.as<T>() + (P->m + it) * d;
      const T* hi = P->Ha.as<T>() + (P->m + it) * c;
      const int blocks = (int)std::min<int64_t>((D * c + 255) / 256, 4096);
      k_exact_y<T><<<blocks, 256, 0, st>>>(Linv, D, xi, d, c, Y);
      k_exact_z<T><<<blocks, 256, 0, st>>>(Y, D, hi, c, Z);
      FIRAL_CUDA_TRY(cudaGetLastError());
    }
    FIRAL_TRY(combine<T>(st, Mhat, 1.0, Mhat, eta / b, Hho, 0.0, nullptr, 0.0, D));
    FIRAL_TRY(gemm<T>(st, false, true, (int)D, (int)D, c, eta, Z, c, Y, c, 1.0, Mhat, D, true));
    // nu_{t+1}: root of sum_j (nu + lambda_j(eta H~))^{-2} = 1 (eq. 10), bracketed by nu_t
    int ev = 0;
    FIRAL_TRY(nu_root<T>(P, nu, &nu, &ev));
    *evals_total += ev;
  }
  return FIRAL_OK;
}

}  // namespace

int32_t dense_gemm(bool dbl, cudaStream_t st, bool ta, bool tb, int M, int N, int K,
                   double alpha, const void* A, int64_t lda, const void* B, int64_t ldb,
                   double beta, void* C, int64_t ldc) {
  if (dbl)
    return gemm<double>(st, ta, tb, M, N, K, alpha, (const double*)A, lda, (const double*)B, ldb,
                        beta, (double*)C, ldc);
  return gemm<float>(st, ta, tb, M, N, K, alpha, (const float*)A, lda, (const float*)B, ldb,
                     beta, (float*)C, ldc);
}

int32_t exact_objective(firal_problem* P, const void* z, double* f_host, void* g) {
  if (P->dbl) return objective_t<double>(P, (const double*)z, f_host, (double*)g);
  return objective_t<float>(P, (const float*)z, f_host, (float*)g);
}

int32_t exact_relax(firal_problem* P, double budget, int T, double beta0, const void* z0,
                    void* z, double* hist) {
  cudaStream_t st = P->H->stream;
  const size_t vs = P->dbl ? 8 : 4;
  if (z0) {
    if (z0 != z)
      FIRAL_CUDA_TRY(cudaMemcpyAsync(z, z0, (size_t)P->n * vs, cudaMemcpyDeviceToDevice, st));
  } else {
    FIRAL_TRY(fill_weights(P->dbl, z, 0, 0.0, nullptr, budget / (double)P->n, P->n, st));
  }
  for (int t = 0; t < T; ++t) {
    double f = 0.0;
    FIRAL_TRY(exact_objective(P, z, &f, P->g.p));          // Algorithm 1 lines 5-6
    if (hist) hist[t] = f;
    FIRAL_TRY(md_step_simt(P->dbl, z, P->g.p, P->n, budget, beta0, P->red.as<double>(), st));
  }
  return FIRAL_OK;
}

int32_t exact_round(firal_problem* P, const void* zd, int b, double eta, int exclude,
                    int32_t* sel, double* r_host, double* nu_host, int* evals) {
  if (P->dbl)
    return round_t<double>(P, (const double*)zd, b, eta, exclude, sel, r_host, nu_host, evals);
  return round_t<float>(P, (const float*)zd, b, eta, exclude, sel, r_host, nu_host, evals);
}

void exact_release(firal_problem* P) {
  if (!P->ex) return;
  ExactWs& ex = *P->ex;
  for (auto& b : ex.m) b.release();
  for (DBuf* b : {&ex.pairs, &ex.part, &ex.gpart, &ex.K, &ex.YZ, &ex.negr, &ex.mask, &ex.argp,
                  &ex.flag, &ex.scal})
    b->release();
  delete P->ex;
  P->ex = nullptr;
}

}  // namespace firal
