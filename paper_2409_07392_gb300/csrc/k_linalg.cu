// FP64 block linear algebra and the Round-step kernels (Algorithm 3).
//
//  * k_chol_inv   -- Cholesky of c SPD d x d blocks (one CTA per block, shared memory),
//                    explicit inverse A^{-1} = L^{-T} L^{-1}; a non-positive pivot raises a
//                    device flag (FIRAL_ERR_NOT_SPD) instead of trapping.
//  * k_tilde_eig  -- eigenvalues of L^{-1} H L^{-T} (similar to Sigma^{-1/2} H Sigma^{-1/2}):
//                    two in-place triangular solves, Householder tridiagonalisation and
//                    Sturm-sequence bisection (Golub & Van Loan, Sections 8.3 and 8.4).
//  * k_nu         -- the root of sum_j (nu + mu_j)^{-2} = 1 (eq. 10) by bisection.
//  * Round kernels -- eq. 14 scores with a masked argmax, the block update of H, and the
//                    assembly of B_t (Algorithm 3 lines 7-11).
#include <cooperative_groups.h>

#include "firal_internal.cuh"

namespace cg = cooperative_groups;

namespace firal {

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ double block_sum_d(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum_d(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double r = 0;
  for (int i = 0; i < nw; ++i) r += red[i];
  __syncthreads();
  return r;
}

// ------------------------------------------------------------------------------------------
// Cholesky + inverse of c blocks
// ------------------------------------------------------------------------------------------
// Shared-memory layout: the block in rows of ld = d + 1 doubles (an odd stride: the threads of
// a half-warp reading one column each hit distinct banks).  The factor L fills the lower
// triangle; Y = L^{-1} goes to the strict upper triangle transposed (Y[i][c], i > c, at row c,
// column i) with its diagonal in yd.  TPR = blockDim / d threads (at least 1) share each row or
// column, so no index is divided by a run-time size.
template <class T>
__global__ void k_chol_inv(const double* __restrict__ A, int d, T* __restrict__ inv_t,
                           double* __restrict__ inv_d, double* __restrict__ L_out,
                           int32_t* not_spd) {
  extern __shared__ double sh[];
  const int ld = d + 1;
  double* Ls = sh;              // d x ld
  double* yd = sh + d * ld;     // d
  const int k = blockIdx.x, tid = threadIdx.x, bd = blockDim.x;
  const int tpr = bd >= d ? bd / d : 1;
  const int row = tid % d, ph = tid / d;        // this thread's row (or column) and phase
  const bool act = ph < tpr;
  const double* Ak = A + (int64_t)k * d * d;
  for (int i = 0; i < d; ++i)
    for (int e = tid; e < d; e += bd) Ls[i * ld + e] = Ak[(int64_t)i * d + e];
  __syncthreads();
  // right-looking Cholesky: pivot, column below it, trailing lower triangle
  for (int j = 0; j < d; ++j) {
    if (tid == 0) {
      double v = Ls[j * ld + j];
      if (!(v > 0.0)) {
        atomicExch(not_spd, 1);
        v = fabs(v) > 1e-300 ? fabs(v) : 1e-300;
      }
      Ls[j * ld + j] = sqrt(v);
      yd[j] = 1.0 / Ls[j * ld + j];
    }
    __syncthreads();
    const double rjj = yd[j];   // FP64 division is several FMAs: one per pivot
    for (int i = j + 1 + tid; i < d; i += bd) Ls[i * ld + j] *= rjj;
    __syncthreads();
    if (act && row > j) {
      const double lij = Ls[row * ld + j];
      for (int kk = j + 1 + ph; kk <= row; kk += tpr) Ls[row * ld + kk] -= lij * Ls[kk * ld + j];
    }
    __syncthreads();
  }
  if (L_out) {
    for (int i = 0; i < d; ++i)
      for (int e = tid; e < d; e += bd)
        L_out[(int64_t)k * d * d + (int64_t)i * d + e] = e <= i ? Ls[i * ld + e] : 0.0;
  }
  if (!inv_t && !inv_d) return;
  // Y = L^{-1} by rows: Y[i][c] = -(L[i][c] Y[c][c] + sum_{c < p < i} L[i][p] Y[p][c]) Y[i][i],
  // Y[i][i] = 1 / L[i][i] (yd, from the factorisation)
  for (int i = 1; i < d; ++i) {
    for (int c = tid; c < i; c += bd) {
      double acc = Ls[i * ld + c] * yd[c];
      for (int p = c + 1; p < i; ++p) acc += Ls[i * ld + p] * Ls[c * ld + p];
      Ls[c * ld + i] = -acc * yd[i];
    }
    __syncthreads();
  }
  // A^{-1}[a][b] = sum_{i >= max(a,b)} Y[i][a] Y[i][b]: thread (column b, phase) takes
  // a = ph, ph + TPR, ... <= b and writes both (a, b) and (b, a)
  if (act) {
    const int b = row;
    for (int a = ph; a <= b; a += tpr) {
      double acc = (a == b ? yd[a] : Ls[a * ld + b]) * yd[b];
      for (int i = b + 1; i < d; ++i) acc += Ls[a * ld + i] * Ls[b * ld + i];
      const int64_t o1 = (int64_t)k * d * d + (int64_t)a * d + b;
      const int64_t o2 = (int64_t)k * d * d + (int64_t)b * d + a;
      if (inv_t) {
        inv_t[o1] = (T)acc;
        inv_t[o2] = (T)acc;
      }
      if (inv_d) {
        inv_d[o1] = acc;
        inv_d[o2] = acc;
      }
    }
  }
}

static int threads_for(int d) {
  int t = ((d * 2 + 31) / 32) * 32;
  if (t < 64) t = 64;
  if (t > 256) t = 256;
  return t;
}

int32_t chol_inv(bool dbl, const double* A, int c, int d, void* inv_t, double* inv_d,
                 double* L_out, int32_t* not_spd, cudaStream_t st) {
  const size_t smem = ((size_t)d * (d + 1) + d) * sizeof(double);
  const int thr = threads_for(d);
  if (smem > 200 * 1024 || thr < d)
    return fail(FIRAL_ERR_UNSUPPORTED, "block factorisation needs d <= 158");
  ProfScope ps(st, PF_CHOL);
  count_launch();
  if (dbl) {
    FIRAL_CUDA_TRY(cudaFuncSetAttribute(k_chol_inv<double>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    k_chol_inv<double><<<c, thr, smem, st>>>(A, d, (double*)inv_t, inv_d, L_out, not_spd);
  } else {
    FIRAL_CUDA_TRY(cudaFuncSetAttribute(k_chol_inv<float>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    k_chol_inv<float><<<c, thr, smem, st>>>(A, d, (float*)inv_t, inv_d, L_out, not_spd);
  }
  FIRAL_CUDA_TRY(cudaGetLastError());
  return FIRAL_OK;
}

// ------------------------------------------------------------------------------------------
// eigenvalues of L^{-1} H L^{-T}, per block
// ------------------------------------------------------------------------------------------
__device__ int sturm_count(const double* dg, const double* e2, int d, double x) {
  int cnt = 0;
  double q = dg[0] - x;
  if (q < 0) ++cnt;
  for (int i = 1; i < d; ++i) {
    if (q == 0.0) q = 1e-300;
    q = dg[i] - x - e2[i - 1] / q;
    if (q < 0) ++cnt;
  }
  return cnt;
}

// Tridiagonal form of L^{-1} H L^{-T} for one block, in the block's shared memory: the
// similarity (two triangular solves with the reciprocal pivots of L), symmetrisation and
// Householder reduction.  On return dg holds the diagonal and e2 the squared off-diagonal
// (e2[i] couples i and i + 1).  M: d*d doubles; v, p, dg, e2, rl: d doubles each.
__device__ void householder_tridiag(int d, double* M, double* v, double* p, double* dg,
                                    double* e2, double* red);

__device__ void tilde_tridiag(const double* __restrict__ Lk, const double* __restrict__ Hk,
                              int d, double* M, double* v, double* p, double* dg, double* e2,
                              double* rl, double* red) {
  const int tid = threadIdx.x, bd = blockDim.x;
  for (int i = tid; i < d; i += bd) rl[i] = 1.0 / Lk[(int64_t)i * d + i];
  __syncthreads();
  // pass 1: column col of A = L^{-1} H, stored transposed in row col of M
  for (int col = tid; col < d; col += bd) {
    for (int i = 0; i < d; ++i) {
      double acc = Hk[(int64_t)i * d + col];
      for (int q = 0; q < i; ++q) acc -= Lk[(int64_t)i * d + q] * M[col * d + q];
      M[col * d + i] = acc * rl[i];
    }
  }
  __syncthreads();
  // pass 2: column col of M currently holds row col of A; solve L m = that column in place
  for (int col = tid; col < d; col += bd) {
    for (int i = 0; i < d; ++i) {
      double acc = M[i * d + col];
      for (int q = 0; q < i; ++q) acc -= Lk[(int64_t)i * d + q] * M[q * d + col];
      M[i * d + col] = acc * rl[i];
    }
  }
  __syncthreads();
  // symmetrise (rounding)
  for (int t = tid; t < d * d; t += bd) {
    const int i = t / d, j = t % d;
    if (j < i) {
      const double a = 0.5 * (M[i * d + j] + M[j * d + i]);
      M[i * d + j] = a;
      M[j * d + i] = a;
    }
  }
  __syncthreads();
  householder_tridiag(d, M, v, p, dg, e2, red);
}

// Householder reduction of the symmetric d x d matrix M (shared memory, overwritten) to
// tridiagonal form: dg = diagonal, e2 = squared off-diagonal (e2[i] couples i and i + 1).
__device__ void householder_tridiag(int d, double* M, double* v, double* p, double* dg,
                                    double* e2, double* red) {
  const int tid = threadIdx.x, bd = blockDim.x;
  for (int kk = 0; kk + 2 < d; ++kk) {
    double part = 0.0;
    for (int i = kk + 2 + tid; i < d; i += bd) part += M[i * d + kk] * M[i * d + kk];
    const double sigma = block_sum_d(part, red);
    const double x0 = M[(kk + 1) * d + kk];
    if (sigma == 0.0) {
      if (tid == 0) e2[kk] = x0 * x0;
      __syncthreads();
      continue;
    }
    const double mu = sqrt(x0 * x0 + sigma);
    const double alpha = x0 > 0 ? -mu : mu;
    for (int i = kk + 1 + tid; i < d; i += bd) v[i] = i == kk + 1 ? x0 - alpha : M[i * d + kk];
    __syncthreads();
    const double vtv = (x0 - alpha) * (x0 - alpha) + sigma;
    const double tau = 2.0 / vtv;
    for (int i = kk + 1 + tid; i < d; i += bd) {
      double acc = 0.0;
      for (int j = kk + 1; j < d; ++j) acc += M[i * d + j] * v[j];
      p[i] = tau * acc;
    }
    __syncthreads();
    double pv = 0.0;
    for (int i = kk + 1 + tid; i < d; i += bd) pv += p[i] * v[i];
    const double Kc = 0.5 * tau * block_sum_d(pv, red);
    for (int i = kk + 1 + tid; i < d; i += bd) p[i] -= Kc * v[i];   // p becomes w
    __syncthreads();
    const int rem = d - kk - 1;
    for (int t = tid; t < rem * rem; t += bd) {
      const int i = kk + 1 + t / rem, j = kk + 1 + t % rem;
      M[i * d + j] -= v[i] * p[j] + p[i] * v[j];
    }
    if (tid == 0) e2[kk] = alpha * alpha;
    __syncthreads();
  }
  if (tid == 0) {
    if (d >= 2) e2[d - 2] = M[(d - 1) * d + (d - 2)] * M[(d - 1) * d + (d - 2)];
  }
  for (int i = tid; i < d; i += bd) dg[i] = M[i * d + i];
  __syncthreads();
}

__global__ void k_tilde_eig(const double* __restrict__ L, const double* __restrict__ H, int d,
                            double* __restrict__ eig) {
  extern __shared__ double sh[];
  double* M = sh;              // d*d
  double* v = M + d * d;       // d
  double* p = v + d;           // d
  double* dg = p + d;          // d
  double* e2 = dg + d;         // d  (squared off-diagonal)
  double* rl = e2 + d;         // d  (reciprocal pivots of L)
  __shared__ double red[32];
  __shared__ double s_bcast[4];
  const int k = blockIdx.x, tid = threadIdx.x, bd = blockDim.x;
  tilde_tridiag(L + (int64_t)k * d * d, H + (int64_t)k * d * d, d, M, v, p, dg, e2, rl, red);
  // Gershgorin interval (thread 0)
  if (tid == 0) {
    double lo = 1e300, hi = -1e300;
    for (int i = 0; i < d; ++i) {
      const double r = (i > 0 ? sqrt(e2[i - 1]) : 0.0) + (i + 1 < d ? sqrt(e2[i]) : 0.0);
      lo = fmin(lo, dg[i] - r);
      hi = fmax(hi, dg[i] + r);
    }
    const double pad = 1e-12 * fmax(fabs(lo), fabs(hi)) + 1e-300;
    s_bcast[0] = lo - pad;
    s_bcast[1] = hi + pad;
  }
  __syncthreads();
  for (int mth = tid; mth < d; mth += bd) {
    double lo = s_bcast[0], hi = s_bcast[1];
    for (int it = 0; it < 200; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (mid <= lo || mid >= hi) break;
      if (sturm_count(dg, e2, d, mid) > mth) hi = mid;
      else lo = mid;
      if (hi - lo <= 4e-16 * fmax(fabs(lo), fabs(hi))) break;
    }
    eig[(int64_t)k * d + mth] = 0.5 * (lo + hi);
  }
}

// The tridiagonal forms alone (Round's nu needs no individual eigenvalue): tri[k] = dg (d) then
// e2 (d) of block k; gb[k] = its Gershgorin interval (lo, hi).
__global__ void k_tilde_tri(const double* __restrict__ L, const double* __restrict__ H, int d,
                            double* __restrict__ tri, double* __restrict__ gb) {
  extern __shared__ double sh[];
  double* M = sh;
  double* v = M + d * d;
  double* p = v + d;
  double* dg = p + d;
  double* e2 = dg + d;
  double* rl = e2 + d;
  __shared__ double red[32];
  const int k = blockIdx.x, tid = threadIdx.x, bd = blockDim.x;
  tilde_tridiag(L + (int64_t)k * d * d, H + (int64_t)k * d * d, d, M, v, p, dg, e2, rl, red);
  for (int i = tid; i < d; i += bd) {
    tri[(int64_t)k * 2 * d + i] = dg[i];
    tri[(int64_t)k * 2 * d + d + i] = i + 1 < d ? e2[i] : 0.0;
  }
  if (tid == 0) {
    double lo = 1e300, hi = -1e300;
    for (int i = 0; i < d; ++i) {
      const double r = (i > 0 ? sqrt(e2[i - 1]) : 0.0) + (i + 1 < d ? sqrt(e2[i]) : 0.0);
      lo = fmin(lo, dg[i] - r);
      hi = fmax(hi, dg[i] + r);
    }
    gb[2 * k] = lo;
    gb[2 * k + 1] = hi;
  }
}

// Tridiagonal forms (as k_tilde_tri) of blocks that are already L^{-1} H L^{-T} (Ht, kept up
// to date by k_round_hupdate): copy to shared memory, Householder reduction.
__global__ void k_sym_tri(const double* __restrict__ Ht, int d, double* __restrict__ tri,
                          double* __restrict__ gb) {
  extern __shared__ double sh[];
  double* M = sh;
  double* v = M + d * d;
  double* p = v + d;
  double* dg = p + d;
  double* e2 = dg + d;
  __shared__ double red[32];
  const int k = blockIdx.x, tid = threadIdx.x, bd = blockDim.x;
  const double* Hk = Ht + (int64_t)k * d * d;
  for (int t = tid; t < d * d; t += bd) M[t] = Hk[t];
  __syncthreads();
  householder_tridiag(d, M, v, p, dg, e2, red);
  for (int i = tid; i < d; i += bd) {
    tri[(int64_t)k * 2 * d + i] = dg[i];
    tri[(int64_t)k * 2 * d + d + i] = i + 1 < d ? e2[i] : 0.0;
  }
  if (tid == 0) {
    double lo = 1e300, hi = -1e300;
    for (int i = 0; i < d; ++i) {
      const double r = (i > 0 ? sqrt(e2[i - 1]) : 0.0) + (i + 1 < d ? sqrt(e2[i]) : 0.0);
      lo = fmin(lo, dg[i] - r);
      hi = fmax(hi, dg[i] + r);
    }
    gb[2 * k] = lo;
    gb[2 * k + 1] = hi;
  }
}

// out_k = L_k^{-1} H_k L_k^{-T} (symmetrised), one block per k
__global__ void k_similarity(const double* __restrict__ L, const double* __restrict__ H, int d,
                             double* __restrict__ out) {
  extern __shared__ double sh[];
  double* M = sh;
  double* rl = M + d * d;
  const int k = blockIdx.x, tid = threadIdx.x, bd = blockDim.x;
  const double* Lk = L + (int64_t)k * d * d;
  const double* Hk = H + (int64_t)k * d * d;
  for (int i = tid; i < d; i += bd) rl[i] = 1.0 / Lk[(int64_t)i * d + i];
  __syncthreads();
  for (int col = tid; col < d; col += bd) {
    for (int i = 0; i < d; ++i) {
      double acc = Hk[(int64_t)i * d + col];
      for (int q = 0; q < i; ++q) acc -= Lk[(int64_t)i * d + q] * M[col * d + q];
      M[col * d + i] = acc * rl[i];
    }
  }
  __syncthreads();
  for (int col = tid; col < d; col += bd) {
    for (int i = 0; i < d; ++i) {
      double acc = M[i * d + col];
      for (int q = 0; q < i; ++q) acc -= Lk[(int64_t)i * d + q] * M[q * d + col];
      M[i * d + col] = acc * rl[i];
    }
  }
  __syncthreads();
  for (int t = tid; t < d * d; t += bd) {
    const int i = t / d, j = t % d;
    out[(int64_t)k * d * d + t] = i == j ? M[t] : 0.5 * (M[i * d + j] + M[j * d + i]);
  }
}

// For A = nu I + eta T (T tridiagonal: diagonal dg, squared off-diagonal e2), the leading
// principal minors theta_i of A (the continuants theta_i = a_i theta_{i-1} - b_i theta_{i-2},
// a_i = nu + eta dg_i, b_i = eta^2 e2_{i-1}) and their first three nu-derivatives follow the
// same three-term recurrence, with no division (rescaled by 2^-400 or 2^400 as they grow or
// shrink; only ratios are used).  With p = theta'/theta, q = theta''/theta, u = theta'''/theta
// of the last minor (theta_d = det A, so p = Tr A^-1):
//   Tr A^-2 = p^2 - q,   d/dnu Tr A^-2 = -2 Tr A^-3 = 3 p q - 2 p^3 - u.
// Returns false when a minor is not positive (nu at or left of -eta lambda_min).
__device__ bool tri_trace2(const double* dg, const double* e2, int d, double nu, double eta,
                           double* f, double* fp) {
  double u0 = 1.0, u1 = 0.0, u2 = 0.0, u3 = 0.0;                  // theta_{i-2} and derivatives
  double v0 = nu + eta * dg[0], v1 = 1.0, v2 = 0.0, v3 = 0.0;     // theta_{i-1}
  if (!(v0 > 0.0)) return false;
  const double eta2 = eta * eta;
  for (int i = 1; i < d; ++i) {
    const double a = nu + eta * dg[i], b = eta2 * e2[i - 1];
    const double w0 = a * v0 - b * u0;
    const double w1 = fma(a, v1, v0) - b * u1;
    const double w2 = fma(a, v2, 2.0 * v1) - b * u2;
    const double w3 = fma(a, v3, 3.0 * v2) - b * u3;
    if (!(w0 > 0.0)) return false;
    u0 = v0; u1 = v1; u2 = v2; u3 = v3;
    v0 = w0; v1 = w1; v2 = w2; v3 = w3;
    const double sc = v0 > 0x1p400 ? 0x1p-400 : (v0 < 0x1p-400 ? 0x1p400 : 1.0);
    if (sc != 1.0) {
      u0 *= sc; u1 *= sc; u2 *= sc; u3 *= sc;
      v0 *= sc; v1 *= sc; v2 *= sc; v3 *= sc;
    }
  }
  const double r = 1.0 / v0;
  const double p = v1 * r, q = v2 * r, uu = v3 * r;
  *f = p * p - q;
  *fp = 3.0 * p * q - 2.0 * p * p * p - uu;
  return true;
}

// nu of eq. 10 from the c tridiagonal forms: the root of F(nu) = sum_k Tr((nu I + eta T_k)^-2)
// = 1, which is what sum_j (nu + eta lambda_j)^-2 = 1 states, the trace taken without the
// eigenvalues.  Newton runs on psi(nu) = F^(-1/2) - 1: a power mean of the nu + eta lambda_j
// (exponent -2) minus 1, increasing, concave and close to linear right of -eta lambda_min, so
// the iterates reach the root in a few steps; they stay inside the bracket
// [-eta max Gershgorin, sqrt(c d) - eta min Gershgorin], and a step that leaves it, or a trial
// outside the SPD domain, bisects instead.  One block; thread k evaluates block k (and
// k + blockDim, ...).
__global__ void k_nu_tri(const double* __restrict__ tri, const double* __restrict__ gb, int c,
                         int d, double eta, double* nu_out) {
  __shared__ double red[32];
  __shared__ double wmn[32], wmx[32];
  __shared__ double s_lo, s_hi, s_nu;
  __shared__ int s_bad, s_done;
  double mn = 1e300, mx = -1e300;
  for (int k = threadIdx.x; k < c; k += blockDim.x) {
    mn = fmin(mn, gb[2 * k]);
    mx = fmax(mx, gb[2 * k + 1]);
  }
  for (int o = 16; o > 0; o >>= 1) {
    mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  if ((threadIdx.x & 31) == 0) {
    wmn[threadIdx.x >> 5] = mn;
    wmx[threadIdx.x >> 5] = mx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 1e300, b = -1e300;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a = fmin(a, wmn[w]);
      b = fmax(b, wmx[w]);
    }
    s_lo = -eta * b;
    s_hi = sqrt((double)c * d) - eta * a;
    s_nu = s_hi;
    s_done = 0;
  }
  __syncthreads();
  for (int it = 0; it < 300; ++it) {
    const double nu = s_nu;
    double f = 0.0, fp = 0.0;
    int bad = 0;
    for (int k = threadIdx.x; k < c; k += blockDim.x) {
      double fk, fpk;
      if (tri_trace2(tri + (int64_t)k * 2 * d, tri + (int64_t)k * 2 * d + d, d, nu, eta, &fk,
                     &fpk)) {
        f += fk;
        fp += fpk;
      } else {
        bad = 1;
      }
    }
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    if (bad) atomicOr(&s_bad, 1);
    const double F = block_sum_d(f, red);   // (synchronises: s_bad is complete after it)
    const double FP = block_sum_d(fp, red);
    if (threadIdx.x == 0) {
      double lo = s_lo, hi = s_hi;
      const bool left = s_bad || F - 1.0 > 0.0;   // left of the root, or of the domain
      if (left) lo = nu;
      else hi = nu;
      if (!s_bad && F - 1.0 == 0.0) {
        s_done = 1;
      } else {
        // psi = F^-1/2 - 1, psi' = -F^-3/2 F' / 2: nu - psi / psi' = nu + 2 (F - F^3/2) / F'
        const bool newton = !s_bad && FP < 0.0 && F > 0.0;
        const double step = newton ? 2.0 * (F - F * sqrt(F)) / FP : 0.0;
        if (newton && fabs(step) <= 1e-12 * fabs(nu)) {
          s_nu = nu + step;   // converged (as in k_nu_coop)
          s_done = 1;
        } else {
          double nx = newton ? nu + step : 0.5 * (lo + hi);
          if (!(nx > lo && nx < hi)) nx = 0.5 * (lo + hi);
          if (nx == nu || hi - lo <= 4e-16 * fmax(fabs(lo), fabs(hi))) s_done = 1;
          s_nu = nx;
        }
      }
      s_lo = lo;
      s_hi = hi;
    }
    __syncthreads();
    if (s_done) break;
  }
  if (threadIdx.x == 0) *nu_out = s_nu;
}

// The same root on many SMs at once.  GB300 runs FP64 at a small fraction of its FP32 rate per
// SM, and each block's recursion is sequential, so one block evaluating all c blocks spends
// most of its time waiting on one SM's FP64 pipe: here block b evaluates classes b, b + grid,
// ... (its lane 0 runs each recursion), and block 0 combines the partials in a fixed order and
// takes the step.  Cooperative launch (every block resident), two grid barriers per step.
// st: [lo, hi, nu, done]; part: 3 doubles per block (F, F', out-of-domain).
__global__ void k_nu_coop(const double* __restrict__ tri, const double* __restrict__ gb, int c,
                          int d, double eta, double* st, double* part, double* nu_out) {
  cg::grid_group grid = cg::this_grid();
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    double a = 1e300, b = -1e300;
    for (int k = 0; k < c; ++k) {
      a = fmin(a, gb[2 * k]);
      b = fmax(b, gb[2 * k + 1]);
    }
    st[0] = -eta * b;
    st[1] = sqrt((double)c * d) - eta * a;
    st[2] = st[1];
    st[3] = 0.0;
  }
  grid.sync();
  for (int it = 0; it < 300; ++it) {
    const double nu = st[2];
    if (threadIdx.x == 0) {
      double f = 0.0, fp = 0.0, bad = 0.0;
      for (int k = blockIdx.x; k < c; k += gridDim.x) {
        double fk, fpk;
        if (tri_trace2(tri + (int64_t)k * 2 * d, tri + (int64_t)k * 2 * d + d, d, nu, eta, &fk,
                       &fpk)) {
          f += fk;
          fp += fpk;
        } else {
          bad = 1.0;
        }
      }
      part[3 * blockIdx.x] = f;
      part[3 * blockIdx.x + 1] = fp;
      part[3 * blockIdx.x + 2] = bad;
    }
    grid.sync();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      double F = 0.0, FP = 0.0;
      bool bad = false;
      for (int b = 0; b < (int)gridDim.x; ++b) {
        F += part[3 * b];
        FP += part[3 * b + 1];
        bad = bad || part[3 * b + 2] != 0.0;
      }
      double lo = st[0], hi = st[1];
      if (bad || F - 1.0 > 0.0) lo = nu;   // left of the root, or of the domain
      else hi = nu;
      if (!bad && F - 1.0 == 0.0) {
        st[3] = 1.0;
      } else {
        // psi = F^-1/2 - 1, psi' = -F^-3/2 F' / 2: nu - psi / psi' = nu + 2 (F - F^3/2) / F'
        const bool newton = !bad && FP < 0.0 && F > 0.0;
        const double step = newton ? 2.0 * (F - F * sqrt(F)) / FP : 0.0;
        // Newton converges quadratically: a step below 1e-12 nu leaves the next one far below
        // the accuracy of F itself (~1e-13, the continuant ratios), so take it and stop
        if (newton && fabs(step) <= 1e-12 * fabs(nu)) {
          st[2] = nu + step;
          st[3] = 1.0;
        } else {
          double nx = newton ? nu + step : 0.5 * (lo + hi);
          if (!(nx > lo && nx < hi)) nx = 0.5 * (lo + hi);
          if (nx == nu || hi - lo <= 4e-16 * fmax(fabs(lo), fabs(hi))) st[3] = 1.0;
          st[2] = nx;
        }
      }
      st[0] = lo;
      st[1] = hi;
    }
    grid.sync();
    if (st[3] != 0.0) break;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *nu_out = st[2];
}

int32_t sym_tri(const double* Ht, int nblocks, int d, double* tri, double* gb, cudaStream_t st) {
  const size_t smem = ((size_t)d * d + 4 * (size_t)d) * sizeof(double);
  FIRAL_CUDA_TRY(cudaFuncSetAttribute(k_sym_tri, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      200 * 1024));
  ProfScope ps(st, PF_ROUND);
  count_launch();
  k_sym_tri<<<nblocks, threads_for(d), smem, st>>>(Ht, d, tri, gb);
  FIRAL_CUDA_TRY(cudaGetLastError());
  return FIRAL_OK;
}

// nu from c tridiagonal forms (tri: 2 c d doubles, gb: 2 c) on up to one block per SM;
// work: 4 + 3 * SMs doubles of step state and per-block partials.
int32_t nu_of_tri(const double* tri, const double* gb, int c, int d, double eta, double* work,
                  double* nu_out, cudaStream_t st) {
  ProfScope ps(st, PF_ROUND);
  count_launch();
  int dev = 0, sms = 0;
  FIRAL_CUDA_TRY(cudaGetDevice(&dev));
  FIRAL_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  int nb = c < sms ? c : sms;
  double* state = work;
  double* part = state + 4;
  void* args[] = {(void*)&tri, (void*)&gb, (void*)&c, (void*)&d, (void*)&eta, (void*)&state,
                  (void*)&part, (void*)&nu_out};
  FIRAL_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)k_nu_coop, dim3(nb), dim3(32), args, 0,
                                             st));
  return FIRAL_OK;
}

int32_t sym_tri_nu(const double* Ht, int c, int d, double eta, double* tri, double* gb,
                   double* nu_out, cudaStream_t st) {
  FIRAL_TRY(sym_tri(Ht, c, d, tri, gb, st));
  // the step state and the per-block partials live after the bounds in the caller's buffer
  return nu_of_tri(tri, gb, c, d, eta, gb + 2 * (size_t)c, nu_out, st);
}

int32_t similarity_blocks(const double* L, const double* H, int c, int d, double* out,
                          cudaStream_t st) {
  const size_t smem = ((size_t)d * d + (size_t)d) * sizeof(double);
  FIRAL_CUDA_TRY(cudaFuncSetAttribute(k_similarity, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      200 * 1024));
  ProfScope ps(st, PF_ROUND);
  count_launch();
  k_similarity<<<c, threads_for(d), smem, st>>>(L, H, d, out);
  FIRAL_CUDA_TRY(cudaGetLastError());
  return FIRAL_OK;
}

int32_t tilde_nu(const double* L, const double* H, int c, int d, double eta, double* tri,
                 double* gb, double* nu_out, cudaStream_t st) {
  const size_t smem = ((size_t)d * d + 5 * (size_t)d) * sizeof(double);
  FIRAL_CUDA_TRY(cudaFuncSetAttribute(k_tilde_tri, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      200 * 1024));
  ProfScope ps(st, PF_ROUND);
  count_launch(2);
  k_tilde_tri<<<c, threads_for(d), smem, st>>>(L, H, d, tri, gb);
  k_nu_tri<<<1, 256, 0, st>>>(tri, gb, c, d, eta, nu_out);
  FIRAL_CUDA_TRY(cudaGetLastError());
  return FIRAL_OK;
}

int32_t tilde_eigvals(const double* L, const double* H, int c, int d, double* eig,
                      cudaStream_t st) {
  const size_t smem = ((size_t)d * d + 5 * (size_t)d) * sizeof(double);
  FIRAL_CUDA_TRY(cudaFuncSetAttribute(k_tilde_eig, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      200 * 1024));
  ProfScope ps(st, PF_ROUND);
  count_launch();
  k_tilde_eig<<<c, threads_for(d), smem, st>>>(L, H, d, eig);
  FIRAL_CUDA_TRY(cudaGetLastError());
  return FIRAL_OK;
}

__global__ void k_identity_blocks(double* L, int64_t total, int d) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i % ((int64_t)d * d);
    L[i] = (r / d == r % d) ? 1.0 : 0.0;
  }
}

int32_t identity_blocks(double* L, int c, int d, cudaStream_t st) {
  const int64_t total = (int64_t)c * d * d;
  count_launch();
  k_identity_blocks<<<(unsigned)std::min<int64_t>((total + 255) / 256, 4096), 256, 0, st>>>(L, total, d);
  FIRAL_CUDA_TRY(cudaGetLastError());
  return FIRAL_OK;
}

// ------------------------------------------------------------------------------------------
// nu of eq. 10: sum_j (nu + scale*lam_j)^{-2} = 1, one block
// ------------------------------------------------------------------------------------------
__global__ void k_nu(const double* lam, int64_t count, double scale, double* nu_out) {
  __shared__ double red[32];
  __shared__ double s_lo, s_hi;
  double mn = 1e300;
  for (int64_t i = threadIdx.x; i < count; i += blockDim.x) mn = fmin(mn, scale * lam[i]);
  // block min
  for (int o = 16; o > 0; o >>= 1) mn = fmin(mn, __shfl_xor_sync(0xffffffffu, mn, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mn;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 1e300;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) m = fmin(m, red[i]);
    s_lo = -m;
    s_hi = sqrt((double)count) - m;
  }
  __syncthreads();
  double lo = s_lo, hi = s_hi;
  for (int it = 0; it < 400; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    double part = 0.0;
    for (int64_t i = threadIdx.x; i < count; i += blockDim.x) {
      const double a = mid + scale * lam[i];
      part += 1.0 / (a * a);
    }
    const double f = block_sum_d(part, red) - 1.0;
    if (f > 0) lo = mid;
    else hi = mid;
    if (hi - lo <= 1e-15 * fmax(fabs(hi), 1.0)) break;
  }
  if (threadIdx.x == 0) *nu_out = 0.5 * (lo + hi);
}

int32_t nu_bisect_dev(const double* lam, int64_t count, double scale, double* nu_out,
                      cudaStream_t st) {
  ProfScope ps(st, PF_ROUND);
  count_launch();
  k_nu<<<1, 256, 0, st>>>(lam, count, scale, nu_out);
  FIRAL_CUDA_TRY(cudaGetLastError());
  return FIRAL_OK;
}

// ------------------------------------------------------------------------------------------
// Round kernels
// ------------------------------------------------------------------------------------------
// out = a*X + b*Y + c*Z (elementwise over c*d*d doubles); Y, Z may be null
__global__ void k_axpbypcz(double* out, double a, const double* X, double b, const double* Y,
                           double cc, const double* Z, int64_t total) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    double v = a * X[i];
    if (Y) v += b * Y[i];
    if (Z) v += cc * Z[i];
    out[i] = v;
  }
}

__global__ void k_axpbypcz_nu(double* out, const double* nu, const double* X, double b,
                              const double* Y, double cc, const double* Z, int64_t total) {
  const double a = *nu;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = a * X[i] + b * Y[i] + cc * Z[i];
}

// M1_k = Binv_k Sig_k Binv_k (double in, T out); M2_k = Binv_k as T.  Binv_k sits in shared
// memory; Sig_k Binv_k goes through the global scratch Tg (c*d*d doubles).
template <class T>
__global__ void k_round_m(const double* __restrict__ Binv, const double* __restrict__ Sig, int d,
                          T* __restrict__ M1, T* __restrict__ M2, double* __restrict__ Tg,
                          int c_sig) {
  extern __shared__ double sh[];
  double* Bs = sh;           // d*d
  const int k = blockIdx.x, tid = threadIdx.x, bd = blockDim.x;
  const double* Bk = Binv + (int64_t)k * d * d;
  const double* Sk = Sig + (int64_t)(k % c_sig) * d * d;   // Sigma shared by stacked chains
  double* Ts = Tg + (int64_t)k * d * d;
  for (int t = tid; t < d * d; t += bd) Bs[t] = Bk[t];
  __syncthreads();
  for (int t = tid; t < d * d; t += bd) {
    const int i = t / d, j = t % d;
    double acc = 0.0;
    for (int q = 0; q < d; ++q) acc += Sk[(int64_t)i * d + q] * Bs[q * d + j];
    Ts[t] = acc;
  }
  __syncthreads();
  for (int t = tid; t < d * d; t += bd) {
    const int i = t / d, j = t % d;
    double acc = 0.0;
    for (int q = 0; q < d; ++q) acc += Bs[i * d + q] * Ts[q * d + j];
    M1[(int64_t)k * d * d + t] = (T)acc;
    M2[(int64_t)k * d * d + t] = (T)Bs[t];
  }
}

// The same for f32 outputs, in f32 arithmetic.  The consumers keep at most f32 (the SIMT
// scores) or bf16 hi + lo (2^-17 per entry, the tensor-core scores) of M1 and M2, and an f32
// product over d terms carries about sqrt(d) 2^-24 of its row norms, so the FP64 products
// (2 d^3 FMAs per block on a part whose FP64 rate is a small fraction of its FP32 rate) buy
// nothing the picks can use.  Binv_k, Sig_k Binv_k and (when it fits) Sig_k in shared memory.
__global__ void k_round_m_f32(const double* __restrict__ Binv, const double* __restrict__ Sig,
                              int d, float* __restrict__ M1, float* __restrict__ M2, int c_sig,
                              int stage_sig) {
  extern __shared__ float shf[];
  float* Bs = shf;               // d*d
  float* Ts = shf + d * d;       // d*d
  float* Ss = shf + 2 * d * d;   // d*d when stage_sig
  const int k = blockIdx.x, tid = threadIdx.x, bd = blockDim.x;
  const double* Bk = Binv + (int64_t)k * d * d;
  const double* Sk = Sig + (int64_t)(k % c_sig) * d * d;   // Sigma shared by stacked chains
  for (int t = tid; t < d * d; t += bd) {
    const float b = (float)Bk[t];
    Bs[t] = b;
    M2[(int64_t)k * d * d + t] = b;
    if (stage_sig) Ss[t] = (float)Sk[t];
  }
  __syncthreads();
  for (int t = tid; t < d * d; t += bd) {
    const int i = t / d, j = t - i * d;
    float acc = 0.0f;
    if (stage_sig)
      for (int q = 0; q < d; ++q) acc = fmaf(Ss[i * d + q], Bs[q * d + j], acc);
    else
      for (int q = 0; q < d; ++q) acc = fmaf((float)Sk[(int64_t)i * d + q], Bs[q * d + j], acc);
    Ts[t] = acc;
  }
  __syncthreads();
  for (int t = tid; t < d * d; t += bd) {
    const int i = t / d, j = t - i * d;
    float acc = 0.0f;
    for (int q = 0; q < d; ++q) acc = fmaf(Bs[i * d + q], Ts[q * d + j], acc);
    M1[(int64_t)k * d * d + t] = acc;
  }
}

// H_k += H_o,k / b + w_ik x_i x_i^T for the pick i (Algorithm 3 line 8; pool row i read from
// the device, w_ik = h_ik (1 - h_ik)); with L and Ht given,
// the transformed blocks too: Ht_k += Hot_k / b + w_ik y y^T with y = L_k^{-1} x_i
// (Hot = L^{-1} H_o L^{-T}), so that Ht stays L^{-1} H L^{-T} without a similarity per pick.
// Dynamic shared memory: d doubles (with L).
template <class T>
__global__ void k_round_hupdate(double* H, const double* Ho, double invb, const T* Xa,
                                const T* Ha, int64_t m, int d, int c, const int32_t* it_ptr,
                                int32_t t_index, const double* L, double* Ht,
                                const double* Hot) {
  extern __shared__ double ys[];
  const int k = blockIdx.x;
  const int64_t row = m + it_ptr[t_index];
  const double hv = (double)Ha[row * c + k];
  const double wk = hv * (1.0 - hv);
  for (int t = threadIdx.x; t < d * d; t += blockDim.x) {
    const int e = t / d, f = t % d;
    const double xe = (double)Xa[row * d + e], xf = (double)Xa[row * d + f];
    H[(int64_t)k * d * d + t] += Ho[(int64_t)k * d * d + t] * invb + wk * xe * xf;
  }
  if (!L) return;
  // y = L_k^{-1} x: forward substitution, column by column
  const double* Lk = L + (int64_t)k * d * d;
  for (int e = threadIdx.x; e < d; e += blockDim.x) ys[e] = (double)Xa[row * d + e];
  __syncthreads();
  for (int q = 0; q < d; ++q) {
    const double yq = ys[q] / Lk[(int64_t)q * d + q];
    __syncthreads();
    if (threadIdx.x == 0) ys[q] = yq;
    for (int i = q + 1 + threadIdx.x; i < d; i += blockDim.x) ys[i] -= Lk[(int64_t)i * d + q] * yq;
    __syncthreads();
  }
  for (int t = threadIdx.x; t < d * d; t += blockDim.x) {
    const int e = t / d, f = t % d;
    Ht[(int64_t)k * d * d + t] += Hot[(int64_t)k * d * d + t] * invb + wk * ys[e] * ys[f];
  }
}

// eq. 14 scores for pool rows, masked argmax partial per block
template <class T>
__global__ __launch_bounds__(128) void k_round_scores(const T* __restrict__ Xa,
                                                      const T* __restrict__ HaT,
                                                      const T* __restrict__ M1,
                                                      const T* __restrict__ M2,
                                                      const uint8_t* __restrict__ mask,
                                                      int64_t m, int64_t N, int d, int c,
                                                      double eta, double* part_val,
                                                      int64_t* part_idx) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* xs = (T*)smem_raw;           // [d][128]
  T* Ms = xs + (size_t)d * 128;   // d*d
  __shared__ double bv[4];
  __shared__ int64_t bi[4];
  const int tid = threadIdx.x;
  const int64_t r0 = m + (int64_t)blockIdx.x * 128;
  const int64_t row = r0 + tid;
  for (int idx = tid; idx < d * 128; idx += 128) {
    const int r = idx / d, e = idx - r * d;
    const int64_t ii = r0 + r;
    xs[e * 128 + r] = ii < N ? Xa[ii * d + e] : T(0);
  }
  double score = 0.0;
  for (int k = 0; k < c; ++k) {
    double q[2];
    for (int which = 0; which < 2; ++which) {
      const T* Mk = (which == 0 ? M1 : M2) + (int64_t)k * d * d;
      __syncthreads();
      for (int t = tid; t < d * d; t += 128) Ms[t] = Mk[t];
      __syncthreads();
      double acc = 0.0;
      for (int e0 = 0; e0 < d; e0 += 16) {
        T y[16];
#pragma unroll
        for (int ee = 0; ee < 16; ++ee) y[ee] = T(0);
        for (int f = 0; f < d; ++f) {
          const T xf = xs[f * 128 + tid];
#pragma unroll
          for (int ee = 0; ee < 16; ++ee)
            if (e0 + ee < d) y[ee] = fma(Ms[f * d + e0 + ee], xf, y[ee]);   // M symmetric
        }
#pragma unroll
        for (int ee = 0; ee < 16; ++ee)
          if (e0 + ee < d) acc += (double)y[ee] * (double)xs[(e0 + ee) * 128 + tid];
      }
      q[which] = acc;
    }
    if (row < N) {
      const double hv = (double)HaT[(int64_t)k * N + row];
      const double wk = hv * (1.0 - hv);
      score += wk * q[0] / (1.0 + eta * wk * q[1]);
    }
  }
  double val = -INFINITY;
  int64_t idx = INT64_MAX;
  if (row < N && !mask[row - m] && score == score) {
    val = score;
    idx = row - m;
  }
  // block argmax, lowest index on ties
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, val, o);
    const int64_t oi = __shfl_xor_sync(0xffffffffu, idx, o);
    if (ov > val || (ov == val && oi < idx)) {
      val = ov;
      idx = oi;
    }
  }
  if ((tid & 31) == 0) {
    bv[tid >> 5] = val;
    bi[tid >> 5] = idx;
  }
  __syncthreads();
  if (tid == 0) {
    for (int w = 1; w < 4; ++w)
      if (bv[w] > val || (bv[w] == val && bi[w] < idx)) {
        val = bv[w];
        idx = bi[w];
      }
    part_val[blockIdx.x] = val;
    part_idx[blockIdx.x] = idx;
  }
}

__global__ void k_round_pick(const double* part_val, const int64_t* part_idx, int np,
                             uint8_t* mask, int32_t* sel, int32_t t, double* score_out) {
  __shared__ double bv[32];
  __shared__ int64_t bi[32];
  double val = -INFINITY;
  int64_t idx = INT64_MAX;
  for (int i = threadIdx.x; i < np; i += blockDim.x) {
    const double v = part_val[i];
    const int64_t ix = part_idx[i];
    if (v > val || (v == val && ix < idx)) {
      val = v;
      idx = ix;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, val, o);
    const int64_t oi = __shfl_xor_sync(0xffffffffu, idx, o);
    if (ov > val || (ov == val && oi < idx)) {
      val = ov;
      idx = oi;
    }
  }
  if ((threadIdx.x & 31) == 0) {
    bv[threadIdx.x >> 5] = val;
    bi[threadIdx.x >> 5] = idx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      if (bv[w] > val || (bv[w] == val && bi[w] < idx)) {
        val = bv[w];
        idx = bi[w];
      }
    if (idx == INT64_MAX) idx = 0;   // nothing selectable (caller validated budget <= n)
    sel[t] = (int32_t)idx;
    mask[idx] = 1;
    *score_out = val;
  }
}

template <class T>
static int32_t round_scores_t(firal_problem* P, const void* M1, const void* M2,
                              const uint8_t* mask, double eta, double* pv, int64_t* pi, int np) {
  const int d = P->d;
  const size_t smem = ((size_t)d * 128 + (size_t)d * d) * sizeof(T);
  FIRAL_CUDA_TRY(cudaFuncSetAttribute(k_round_scores<T>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  ProfScope ps(P->H->stream, PF_ROUND);
  count_launch();
  k_round_scores<T><<<np, 128, smem, P->H->stream>>>(P->Xa.as<T>(), P->HaT.as<T>(), (const T*)M1,
                                                     (const T*)M2, mask, P->m, P->N, d, P->c, eta,
                                                     pv, pi);
  FIRAL_CUDA_TRY(cudaGetLastError());
  return FIRAL_OK;
}

int32_t round_scores(firal_problem* P, const void* M1, const void* M2, const uint8_t* mask,
                     double eta, double* pv, int64_t* pi, int np) {
  FIRAL_TRY(class_major_h(P));
  if (P->dbl) return round_scores_t<double>(P, M1, M2, mask, eta, pv, pi, np);
  return round_scores_t<float>(P, M1, M2, mask, eta, pv, pi, np);
}

int32_t round_pick(const double* pv, const int64_t* pi, int np, uint8_t* mask, int32_t* sel,
                   int32_t t, double* score_out, cudaStream_t st) {
  ProfScope ps(st, PF_ROUND);
  count_launch();
  k_round_pick<<<1, 256, 0, st>>>(pv, pi, np, mask, sel, t, score_out);
  FIRAL_CUDA_TRY(cudaGetLastError());
  return FIRAL_OK;
}

int32_t round_m(bool dbl, const double* Binv, const double* Sig, int c, int d, void* M1, void* M2,
                double* Tg, cudaStream_t st, int n_chain) {
  const size_t smem = (size_t)d * d * sizeof(double);
  const int nb = c * n_chain;   // chains stacked: block k uses Sigma block k mod c
  ProfScope ps(st, PF_ROUND);
  count_launch();
  if (dbl) {
    FIRAL_CUDA_TRY(cudaFuncSetAttribute(k_round_m<double>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    k_round_m<double><<<nb, threads_for(d), smem, st>>>(Binv, Sig, d, (double*)M1, (double*)M2,
                                                        Tg, c);
  } else {
    const int stage_sig = (size_t)3 * d * d * sizeof(float) <= 200 * 1024 ? 1 : 0;
    const size_t smem_f = (size_t)(2 + stage_sig) * d * d * sizeof(float);
    FIRAL_CUDA_TRY(cudaFuncSetAttribute(k_round_m_f32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        200 * 1024));
    k_round_m_f32<<<nb, 256, smem_f, st>>>(Binv, Sig, d, (float*)M1, (float*)M2, c, stage_sig);
  }
  FIRAL_CUDA_TRY(cudaGetLastError());
  return FIRAL_OK;
}

int32_t round_hupdate(firal_problem* P, double* H, const double* Ho, double invb,
                      const int32_t* sel, int32_t t, const double* L, double* Ht,
                      const double* Hot) {
  cudaStream_t st = P->H->stream;
  ProfScope ps(st, PF_ROUND);
  count_launch();
  const size_t smem = (size_t)P->d * sizeof(double);
  if (P->dbl)
    k_round_hupdate<double><<<P->c, 256, smem, st>>>(H, Ho, invb, P->Xa.as<double>(),
                                                     P->Ha.as<double>(), P->m, P->d, P->c, sel,
                                                     t, L, Ht, Hot);
  else
    k_round_hupdate<float><<<P->c, 256, smem, st>>>(H, Ho, invb, P->Xa.as<float>(),
                                                    P->Ha.as<float>(), P->m, P->d, P->c, sel,
                                                    t, L, Ht, Hot);
  FIRAL_CUDA_TRY(cudaGetLastError());
  return FIRAL_OK;
}

int32_t lincomb(double* out, double a, const double* X, double b, const double* Y, double cc,
                const double* Z, int64_t total, cudaStream_t st) {
  ProfScope ps(st, PF_ROUND);
  count_launch();
  k_axpbypcz<<<(unsigned)((total + 255) / 256 > 4096 ? 4096 : (total + 255) / 256), 256, 0, st>>>(
      out, a, X, b, Y, cc, Z, total);
  FIRAL_CUDA_TRY(cudaGetLastError());
  return FIRAL_OK;
}

int32_t lincomb_nu(double* out, const double* nu, const double* X, double b, const double* Y,
                   double cc, const double* Z, int64_t total, cudaStream_t st) {
  ProfScope ps(st, PF_ROUND);
  count_launch();
  k_axpbypcz_nu<<<(unsigned)((total + 255) / 256 > 4096 ? 4096 : (total + 255) / 256), 256, 0,
                  st>>>(out, nu, X, b, Y, cc, Z, total);
  FIRAL_CUDA_TRY(cudaGetLastError());
  return FIRAL_OK;
}

}  // namespace firal
