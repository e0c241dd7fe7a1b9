// Tensor-core (tcgen05 + TMA) kernels of the FIRAL_MIXED_BF16 path.
//
// The low-rank part of the Hessian apply (Lemma 1 regrouped; see k_simt.cu) is two dense
// contractions over bf16 operands with f32 accumulation in TMEM:
//
//   alpha-GEMM:  T[i, (j,part,e)] = sum_k H[i,k] P~[(j,part,e), k]            (K = classes)
//                epilogue: walpha^T[j][i] = w_i sum_e x_ie (T[i,(j,hi,e)] + T[i,(j,lo,e)])
//   D-GEMM:      D[k, (j,e)]     = sum_i H^T[k,i] Y[(j,e), i],  Y = walpha_ij x_ie   (K = points)
//                Y is built per 64-point K-step in shared memory (128-byte swizzle) by
//                producer warps from TMA-staged x^T and walpha^T tiles.
//
// The probe block P (CG direction, f32) enters the alpha-GEMM as two bf16 operands P_hi and
// P_lo = P - P_hi, so the contraction sees P to ~2^-17 relative (FIRAL_MIXED_BF16), or as
// bf16(P) alone, 2^-9 relative and half the tensor work (FIRAL_MIXED_BF16_FAST).  X is stored in bf16 and h
// is rounded to bf16 (independent per-element rounding, averaged by the sums over points).
//
// Warp roles (256 threads): warp 0 = TMA producer, warp 1 = MMA issuer (+ TMEM owner),
// warps 2..7 = Y builders (D-GEMM), warps 4..7 = epilogue (TMEM lanes 32*(warp%4)..+31).
// Every mbarrier wait is bounded; on timeout the CTA raises a device flag, drains its
// in-flight MMAs, releases TMEM and exits (FIRAL_ERR_TIMEOUT on the host).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <climits>
#include <mutex>
#include <vector>

#include "firal_internal.cuh"
#include "tc_ptx.cuh"

namespace firal {

using bf16 = __nv_bfloat16;
using namespace tc;

// ------------------------------------------------------------------------------------------
// driver entry point for tensor maps (fetched once through the runtime)
// ------------------------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

static int32_t get_encoder() {
  static std::once_flag once;
  static int32_t status = FIRAL_OK;
  std::call_once(once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
      status = fail(FIRAL_ERR_CUDA, "cuTensorMapEncodeTiled entry point unavailable");
    else
      g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  });
  return status;
}

// 2-D bf16 tensor map: rows x cols (cols contiguous), box = box_rows x box_cols.
static int32_t make_map(CUtensorMap* m, const void* base, uint64_t rows, uint64_t cols,
                        uint32_t box_rows, uint32_t box_cols, bool swizzle128) {
  FIRAL_TRY(get_encoder());
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {cols * sizeof(bf16)};
  cuuint32_t box[2] = {box_cols, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    return fail(FIRAL_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return FIRAL_OK;
}

// 2-D f32 tensor map with 128-byte swizzle: box = box_rows x 32 columns (128 B rows).
// cols * 4 must be a multiple of 16.
static int32_t make_map_f32(CUtensorMap* m, const void* base, uint64_t rows, uint64_t cols,
                            uint32_t box_rows) {
  FIRAL_TRY(get_encoder());
  cuuint64_t dims[2] = {cols, rows};
  cuuint64_t strides[1] = {cols * sizeof(float)};
  cuuint32_t box[2] = {32, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    return fail(FIRAL_ERR_CUDA, "cuTensorMapEncodeTiled (f32) failed (" + std::to_string((int)r) + ")");
  return FIRAL_OK;
}

static int32_t* tc_error_word(firal_problem* P) { return &P->H->flags.as<DevFlags>()->pad[0]; }

// ------------------------------------------------------------------------------------------
// preparation: padded bf16 copies (rows x cols -> rows_p x cols_p) and transposes
// ------------------------------------------------------------------------------------------
// Grid of the padded conversions: blocks walk rows (x, strided) and column pairs (y); a thread
// converts one pair of columns per row, so no element index is divided by the row length.
static void bf16_pad_grid(int64_t rows_p, int cols_p, dim3& grid, dim3& block) {
  const int pairs = cols_p / 2;
  const int bt = std::min(256, (pairs + 31) / 32 * 32);
  block = dim3((unsigned)bt);
  grid = dim3((unsigned)std::min<int64_t>(rows_p, 16384), (unsigned)((pairs + bt - 1) / bt));
}

// MODE 0: bf16(src); 1: bf16(src - bf16(src)), the low part; 2: bf16(src - e_m) on rows with
// cen[r] = m >= 0 (h_m - 1 is exact in f32 for h_m >= 1/2), bf16(src) elsewhere.  Zero in the
// padding rows and columns.  cols_p even.
template <int MODE>
__global__ void k_bf16_pad(bf16* dst, const float* src, const int* cen, int64_t rows, int cols,
                           int64_t rows_p, int cols_p) {
  const int cc = (blockIdx.y * blockDim.x + threadIdx.x) * 2;
  if (cc >= cols_p) return;
  for (int64_t r = blockIdx.x; r < rows_p; r += gridDim.x) {
    float v0 = 0.0f, v1 = 0.0f;
    if (r < rows) {
      if (cc < cols) v0 = src[r * cols + cc];
      if (cc + 1 < cols) v1 = src[r * cols + cc + 1];
      if (MODE == 2) {
        const int m = cen[r];
        if (m == cc) v0 -= 1.0f;
        if (m == cc + 1) v1 -= 1.0f;
      }
    }
    __nv_bfloat162 o = __floats2bfloat162_rn(v0, v1);
    if (MODE == 1) {
      const float2 f = __bfloat1622float2(o);
      o = __floats2bfloat162_rn(v0 - f.x, v1 - f.y);
    }
    *reinterpret_cast<__nv_bfloat162*>(dst + r * cols_p + cc) = o;
  }
}

// ------------------------------------------------------------------------------------------
// Confident rows.  With h_i = e_m + u_i (m = the row's most probable class, u_i = h_i - e_m),
// diag(h) - h h^T = diag(u) - e_m u^T - u e_m^T - u u^T exactly, so per point (a = V^T x_i)
//     [(diag(h) - h h^T) a]_k = u_k a_k - u_k alpha - [k = m] (u . a),   alpha = h . a = a_m + u . a.
// Every term is of the size of u (1 - h_m, h_k for k != m), so no two large terms cancel:
// rounding u to bf16 is relative to u, where rounding h_m ~ 1 to bf16 errs by up to 2^-9 in
// the same direction on every confident row and that bias is as large as the Hessian itself.
// Rows with h_m > 1/2 (cen[i] = m, else -1; kCentre below) take this form in the tensor-core
// apply:
//   diagonal part  sum_i w_i u_ik x_i x_i^T V_k          (block sums with u in the class operand)
//   low-rank part  sum_i w_i u_ik alpha_i x_i             (alpha-GEMM on u: u . a; plus a_m)
//   class-m part   sum_{i: m_i = k} w_i (u_i . a_i) x_i   (a per-class sum over its rows)
// ------------------------------------------------------------------------------------------
// Rows whose top probability exceeds kCentre are centred.  On a plain row the bf16 rounding
// of h_m (spacing 2^-9 on [1/2, 1)) errs by up to 2^-10 / (1 - h_m) of the row's Hessian: in
// a random direction from row to row, unless h_m sits within a few spacings of 1, where it
// rounds toward 1 on every row.  A threshold of 0.9 keeps that ratio below 1% per row but,
// measured on a classifier with weights x 20, left 2.6e-3 in H_p V at 60 points per class
// against 1.3e-3 with 1/2; 1/2 is also where h_m - 1 becomes exact in f32.
constexpr float kCentre = 0.5f;

// cen[r] = argmax_k h_rk (lowest index on ties) when that probability exceeds kCentre, else -1;
// *count gains the number of such rows and *share the row's low-rank share: sum_k h_rk^2 on a
// plain row (the size of the low-rank term of its Hessian next to the diagonal term), 1 on a
// centred row (all of its terms are of one size).  One warp per row.
__global__ void __launch_bounds__(256) k_row_top(int* cen, unsigned long long* count,
                                                 double* share, const float* src, int64_t rows,
                                                 int cols) {
  __shared__ double s_sh[8];
  __shared__ unsigned long long s_cnt[8];
  const int lane = threadIdx.x & 31, wb = threadIdx.x >> 5;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  double wshare = 0.0;
  unsigned long long wcnt = 0;
  // one warp per row, rows strided over all warps; one pair of atomics per block
  for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + wb; r < rows; r += nwarps) {
    float best = -1.0f;
    int bi = 0x7fffffff;
    float sq = 0.0f;
    for (int k = lane; k < cols; k += 32) {
      const float v = src[r * cols + k];
      sq = fmaf(v, v, sq);
      if (v > best) {
        best = v;
        bi = k;
      }
    }
    for (int o = 16; o > 0; o >>= 1) sq += __shfl_xor_sync(0xffffffffu, sq, o);
    for (int o = 16; o > 0; o >>= 1) {
      const float ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) {
        best = ob;
        bi = oi;
      }
    }
    if (lane == 0) {
      cen[r] = best > kCentre ? bi : -1;
      wcnt += best > kCentre ? 1ULL : 0ULL;
      wshare += best > kCentre ? 1.0 : (double)sq;
    }
  }
  if (lane == 0) {
    s_sh[wb] = wshare;
    s_cnt[wb] = wcnt;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    unsigned long long cn = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      t += s_sh[i];
      cn += s_cnt[i];
    }
    if (cn) atomicAdd(count, cn);
    atomicAdd(share, t);
  }
}

// dst = bf16(h - e_m) on centred rows (h_m - 1 is exact in f32 for h_m >= 1/2), bf16(h)
// elsewhere; padding as k_to_bf16_pad
__global__ void k_to_bf16_centred_pad(bf16* dst, const float* src, const int* cen, int64_t rows,
                                      int cols, int64_t rows_p, int cols_p) {
  const int64_t total = rows_p * cols_p;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = idx / cols_p;
    const int cc = (int)(idx - r * cols_p);
    float v = 0.0f;
    if (r < rows && cc < cols) {
      v = src[r * cols + cc];
      if (cen[r] == cc) v -= 1.0f;
    }
    dst[idx] = __float2bfloat16_rn(v);
  }
}

// The centred rows grouped by class are cut into work items of at most CEN_ITEM rows
// (int4: class, first row, end row in idx, unused), so one large class does not serialise on
// one block.
constexpr int CEN_ITEM = 512;

// a_m for the centred rows of one work item (block): am[i][j] = x_i . P~_j[:, k], the probe
// block as the alpha-GEMM sees it (its bf16 parts summed).
__global__ void k_centre_am(float* am, const bf16* Pb, const bf16* Xb, const int4* items,
                            const int* idx, int s, int npart, int dp, int cp) {
  extern __shared__ float pv[];   // s x dp
  const int4 it = items[blockIdx.x];
  const int k = it.x, r0 = it.y, r1 = it.z;
  for (int t = threadIdx.x; t < s * dp; t += blockDim.x) {
    const int j = t / dp, e = t - j * dp;
    float v = 0.0f;
    for (int part = 0; part < npart; ++part)
      v += __bfloat162float(Pb[((int64_t)(j * npart + part) * dp + e) * cp + k]);
    pv[t] = v;
  }
  __syncthreads();
  const int items_n = (r1 - r0) * s;
  for (int t = threadIdx.x; t < items_n; t += blockDim.x) {
    const int rr = t / s, j = t - rr * s;
    const int64_t row = idx[r0 + rr];
    const __nv_bfloat162* x2 = reinterpret_cast<const __nv_bfloat162*>(Xb + row * dp);
    const float* pj = pv + j * dp;
    float acc = 0.0f;
    for (int e = 0; e < dp; e += 2) {
      const float2 xf = __bfloat1622float2(x2[e >> 1]);
      acc = fmaf(xf.x, pj[e], acc);
      acc = fmaf(xf.y, pj[e + 1], acc);
    }
    am[row * s + j] = acc;
  }
}

// class-m part of the centred rows, per work item: part[item][j d + e] = sum over the item's
// rows of rho[i][j] x_ie (rho = w (u . a) from the alpha epilogue), in row order.  The rows are
// staged 64 at a time in shared memory (their rho and x rows loaded together), so the sums run
// from shared memory; dynamic shared memory 64 (s + dp) floats.  Block (item, y) of 256
// threads covers outputs [2048 y, 2048 y + 2048).
__global__ void k_centre_termc(float* part, const float* rho, const bf16* Xb, const int4* items,
                               const int* idx, int s, int d, int dp) {
  extern __shared__ float stg[];   // rho chunk [64][s] | x chunk [64][dp]
  float* rs = stg;
  float* xs = stg + 64 * s;
  const int4 it = items[blockIdx.x];
  const int r0 = it.y, r1 = it.z;
  const int sd = s * d;
  constexpr int MAXO = 8;   // outputs per thread
  const int o0 = blockIdx.y * MAXO * blockDim.x;
  float acc[MAXO];
#pragma unroll
  for (int q = 0; q < MAXO; ++q) acc[q] = 0.0f;
  for (int c0 = r0; c0 < r1; c0 += 64) {
    const int nr = r1 - c0 < 64 ? r1 - c0 : 64;
    __syncthreads();
    for (int t = threadIdx.x; t < nr * s; t += blockDim.x) {
      const int rr = t / s, j = t - rr * s;
      rs[t] = rho[(int64_t)idx[c0 + rr] * s + j];
    }
    for (int t = threadIdx.x; t < nr * dp; t += blockDim.x) {
      const int rr = t / dp, e = t - rr * dp;
      xs[t] = __bfloat162float(Xb[(int64_t)idx[c0 + rr] * dp + e]);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < MAXO; ++q) {
      const int t = o0 + threadIdx.x + q * blockDim.x;
      if (t < sd) {
        const int j = t / d, e = t - j * d;
        float a = acc[q];
        for (int rr = 0; rr < nr; ++rr) a = fmaf(rs[rr * s + j], xs[rr * dp + e], a);
        acc[q] = a;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < MAXO; ++q) {
    const int t = o0 + threadIdx.x + q * blockDim.x;
    if (t < sd) part[(int64_t)blockIdx.x * sd + t] = acc[q];
  }
}

// out[k][o] = sum of the class's item partials in item order (zero for a class without centred
// rows); it is added to the split-K partials of the D-GEMM.  Block (k, y) as above.
__global__ void k_centre_reduce(float* out, const float* part, const int* ioff, int sd) {
  const int k = blockIdx.x;
  const int i0 = ioff[k], i1 = ioff[k + 1];
  for (int q = 0; q < 8; ++q) {
    const int t = blockIdx.y * 8 * blockDim.x + threadIdx.x + q * blockDim.x;
    if (t >= sd) break;
    float a = 0.0f;
    for (int i = i0; i < i1; ++i) a += part[(int64_t)i * sd + t];
    out[(int64_t)k * sd + t] = a;
  }
}

// Labelled rows of a problem with confident rows.  They are few and carry weight 1 each (a
// large share of Sigma_z), so their bf16 roundings do not average out over many points: their
// Hessians are applied here on CUDA cores in f32 by Lemma 1, per point, and the tensor-core
// part skips them.  G[i][j][k] = w_i ((a_k - alpha) h_ik) with a_k = x_i . V~_j[:, k],
// alpha = h_i . a, V~ = V minus its class mean (the direction the rest of the apply uses).
// Block (i, j); dynamic shared memory c floats.
__global__ void k_lab_gamma(float* G, const float* V, const float* vmean, const float* Xa,
                            const float* Ha, const float* w, int s, int c, int d, int64_t D) {
  extern __shared__ float a_s[];   // c
  __shared__ float red[32];
  const int64_t i = blockIdx.x;
  const int j = blockIdx.y;
  const float* x = Xa + i * d;
  const float* h = Ha + i * c;
  float part = 0.0f;
  for (int k = threadIdx.x; k < c; k += blockDim.x) {
    const float* v = V + (int64_t)j * D + (int64_t)k * d;
    const float* vm = vmean + (int64_t)j * d;
    float acc = 0.0f;
    for (int e = 0; e < d; ++e) acc = fmaf(x[e], v[e] - vm[e], acc);
    a_s[k] = acc;
    part = fmaf(h[k], acc, part);
  }
  for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  float alpha = 0.0f;
  for (int q = 0; q < (int)(blockDim.x >> 5); ++q) alpha += red[q];
  const float wi = w[i];
  for (int k = threadIdx.x; k < c; k += blockDim.x)
    G[(i * s + j) * c + k] = wi * ((a_s[k] - alpha) * h[k]);
}

// out[k][j d + e] = -sum_{i < m} G[i][j][k] x_ie (negated: the combine subtracts its partials)
__global__ void k_lab_scatter(float* out, const float* G, const float* Xa, int64_t m, int s,
                              int c, int d) {
  const int k = blockIdx.x;
  const int sd = s * d;
  for (int t = threadIdx.x; t < sd; t += blockDim.x) {
    const int j = t / d, e = t - j * d;
    float acc = 0.0f;
    for (int64_t i = 0; i < m; ++i) acc = fmaf(G[(i * s + j) * c + k], Xa[i * d + e], acc);
    out[(int64_t)k * sd + t] = -acc;
  }
}

// dst[cols_p x rows_p] = transpose of a padded bf16 matrix src[rows_p x cols_p]
// src (rows_p x cols_p, row-major) -> dst in the K-block-major layout [r / 64][col][r % 64] with
// colsb >= cols_p rows per block (rows cols_p..colsb-1 zero): every 64-point tile of a block of
// rows is one contiguous run, so TMA tiles touch few DRAM pages.  rows_p % 64 == 0.
__global__ void k_block_transpose_bf16(bf16* dst, const bf16* src, int64_t rows_p, int cols_p,
                                       int colsb) {
  __shared__ bf16 tile[32][34];
  const int64_t rb = (int64_t)blockIdx.x * 32;
  const int cb = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t r = rb + i;
    const int col = cb + threadIdx.x;
    tile[i][threadIdx.x] = (r < rows_p && col < cols_p) ? src[r * cols_p + col] : __float2bfloat16(0.0f);
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int col = cb + i;
    const int64_t r = rb + threadIdx.x;
    if (r < rows_p && col < colsb) dst[((r >> 6) * colsb + col) * 64 + (r & 63)] = tile[threadIdx.x][i];
  }
}

// P (s x [c][d], f32) -> P~ rows (j, part, e), columns k (bf16, K-major), part 0 = hi, 1 = lo
// (NPART = 2) or rows (j, e) holding bf16(P) alone (NPART = 1)
template <int NPART>
__global__ void k_split_probes(bf16* Pt, const float* P, const float* vmean, int s, int c, int d,
                               int dp, int cp, int64_t D, PoolTab pt) {
  __shared__ float tile[32][33];
  const int j = blockIdx.z;
  const int k0 = blockIdx.x * 32, e0 = blockIdx.y * 32;
  const int Qe = pool_count(pt);
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int k = k0 + i, e = e0 + threadIdx.x;
    tile[i][threadIdx.x] =
        (k < c && e < d)
            ? P[(int64_t)j * D + (int64_t)k * d + e] - vmean[(j * Qe + pool_of(pt, k)) * d + e]
            : 0.0f;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int e = e0 + i, k = k0 + threadIdx.x;
    if (e >= dp || k >= cp) continue;
    const float v = tile[threadIdx.x][i];
    const bf16 hi = __float2bfloat16_rn(v);
    Pt[((int64_t)(j * NPART + 0) * dp + e) * cp + k] = hi;
    if (NPART == 2)
      Pt[((int64_t)(j * NPART + 1) * dp + e) * cp + k] = __float2bfloat16_rn(v - __bfloat162float(hi));
  }
}

// ------------------------------------------------------------------------------------------
// Null-space handling.  Every H_i vanishes on N = {1_c (x) u} when the rows of h sum to one,
// so Sigma_z = lambda I on N and Sigma_z maps N^perp into itself.  The bf16 low-rank term and
// the f32 diagonal term cancel on N only to 2^-9, which Sigma_z^{-1} would amplify by
// 1/lambda; the mixed apply therefore evaluates
//     Sigma V = P_perp (Sigma~ (P_perp V)) + lambda_N P_N V,
// with P_N V = the class mean of V replicated over classes (exact in real arithmetic).
// ------------------------------------------------------------------------------------------
// mean[j][p][e] = mean over the classes k of pool p of V[j][k][e] (all classes for an ordinary
// problem).  Block (probe j and pool p, split g of G): 1024 threads = (class group, e) over its
// share of the classes, the groups combined in a fixed order.  With G > 1 each split writes a
// partial (part), and the last split of (j, p) to finish (a ticket in cnt, reset by it) adds
// the partials in split order: deterministic, and no other launch.
__global__ void k_class_mean(const float* V, int s, int c, int d, int64_t D, float* mean,
                             PoolTab pt, double* part, unsigned* cnt) {
  __shared__ double red[1024];
  __shared__ bool last;
  const int Qe = pool_count(pt);
  const int jp = blockIdx.x, j = jp / Qe, p = jp - j * Qe;
  const int g = blockIdx.y, G = gridDim.y;
  const int k0 = pt.Q ? pt.coff[p] : 0, k1 = pt.Q ? pt.coff[p + 1] : c;
  const int len = (k1 - k0 + G - 1) / G;
  const int kb = k0 + g * len, ke = kb + len < k1 ? kb + len : k1;
  const int dpad = (d + 31) / 32 * 32;
  const int groups = 1024 / dpad;
  const int e = threadIdx.x % dpad, gr = threadIdx.x / dpad;
  double acc = 0.0;
  if (e < d && gr < groups)
    for (int k = kb + gr; k < ke; k += groups) acc += (double)V[(int64_t)j * D + (int64_t)k * d + e];
  red[threadIdx.x] = acc;
  __syncthreads();
  double tot = 0.0;
  if (threadIdx.x < d)
    for (int q = 0; q < groups; ++q) tot += red[q * dpad + threadIdx.x];
  if (G == 1) {
    if (threadIdx.x < d) mean[jp * d + threadIdx.x] = (float)(tot / (k1 - k0));
    return;
  }
  if (threadIdx.x < d) part[((int64_t)jp * G + g) * d + threadIdx.x] = tot;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(&cnt[jp], 1u) == (unsigned)(G - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (threadIdx.x < d) {
    double t = 0.0;
    for (int q = 0; q < G; ++q) t += __ldcg(&part[((int64_t)jp * G + q) * d + threadIdx.x]);
    mean[jp * d + threadIdx.x] = (float)(t / (k1 - k0));
  }
  if (threadIdx.x == 0) cnt[jp] = 0u;
}

// Class means of the s probes of V into mean (s x pools x d): ordinary problems with many
// classes split each probe's classes over CM_SPLIT blocks.
constexpr int CM_SPLIT = 8;
static int32_t class_mean(firal_problem* P, const float* V, int s, float* mean, cudaStream_t st) {
  const int Qe = pool_count(P->pt);
  const int G = (P->pt.Q == 0 && P->c >= 256) ? CM_SPLIT : 1;
  double* part = nullptr;
  unsigned* cnt = nullptr;
  if (G > 1) {
    // partials then tickets for cm_np probes (at least 512); the tickets are zeroed when the
    // buffer is (re)allocated, and every launch leaves them zero
    if (P->cm_np < s) {
      const int np = s > 512 ? s : 512;
      const size_t bytes = (size_t)np * (CM_SPLIT * P->d * sizeof(double) + sizeof(unsigned));
      FIRAL_TRY(P->cm_scr.ensure(bytes));
      FIRAL_CUDA_TRY(cudaMemsetAsync(P->cm_scr.p, 0, bytes, st));
      P->cm_np = np;
    }
    part = P->cm_scr.as<double>();
    cnt = reinterpret_cast<unsigned*>(part + (size_t)P->cm_np * CM_SPLIT * P->d);
  }
  k_class_mean<<<dim3((unsigned)(s * Qe), (unsigned)G), 1024, 0, st>>>(V, s, P->c, P->d, P->D,
                                                                      mean, P->pt, part, cnt);
  return FIRAL_OK;
}

// out = out - qmean + lam_null * vmean (per class block); pq[j c + k] = <V_j[k], out_j[k]>
__global__ void k_project(float* out, const float* qmean, const float* vmean, const float* V,
                          double lam_null, int s, int c, int d, int64_t D, double* pq,
                          PoolTab pt) {
  __shared__ double red[32];
  const int k = blockIdx.x, e = threadIdx.x;
  const int Qe = pool_count(pt), pk = pool_of(pt, k);
  for (int jj = 0; jj < 4; ++jj) {
    const int j = blockIdx.y * 4 + jj;
    if (j >= s) break;
    double contrib = 0.0;
    if (e < d) {
      const int64_t o = (int64_t)j * D + (int64_t)k * d + e;
      const int m = (j * Qe + pk) * d + e;
      const float q = out[o] - qmean[m] + (float)(lam_null * (double)vmean[m]);
      out[o] = q;
      contrib = (double)V[o] * (double)q;
    }
    if (pq) {
      double v = contrib;
      for (int o2 = 16; o2 > 0; o2 >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o2);
      __syncthreads();
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
      __syncthreads();
      if (threadIdx.x == 0) {
        double tot = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
        pq[(int64_t)j * c + k] = tot;
      }
    }
  }
}

// (e, e') of pair index p in the row-major triangle e <= e' < d
__device__ __forceinline__ void pair_of(int p, int d, int& e, int& e2) {
  int ee = 0, start = 0;
  while (ee < d && start + (d - ee) <= p) {
    start += d - ee;
    ++ee;
  }
  e = ee;
  e2 = ee + (p - start);
}

// ------------------------------------------------------------------------------------------
// alpha-GEMM
// ------------------------------------------------------------------------------------------
namespace alpha_cfg {
constexpr int BM = 128, BN = 256, BK = 64, STAGES = 4;
constexpr int A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2;
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int SMEM = STAGES * STAGE_BYTES + 1024 + 256;
constexpr int SMEM_QUAD(int dp) { return SMEM + dp * BM * 2; }
// with the low part of h as a second A operand (gradient modes): 3 stages of A_hi|A_lo|B
constexpr int STAGES_H = 3;
constexpr int SMEM_H = STAGES_H * (2 * A_BYTES + B_BYTES) + 1024 + 256;
constexpr int SMEM_QUAD_H(int dp) { return SMEM_H + dp * BM * 2; }
// feature-contracted quadratic forms: 2 stages of x | coefficients hi | lo (128 rows each),
// then 2 buffers of the f32 h tile (128 points x 64 classes, two 128-byte-swizzled boxes)
constexpr int C3_BYTES = 128 * BK * 2;
constexpr int H3_BYTES = 128 * 64 * 4;
// MODE 3: the x tile of a point tile stays resident (double buffer of dp/64 K-blocks) and the
// ring stages hold only the coefficient tiles (hi + lo, 32 KB): 4 stages at dp = 64, 3 at 128
constexpr int NST3(int dp) { return dp <= 64 ? 4 : 3; }
constexpr int XB3(int dp) { return (dp / 64) * A_BYTES; }
constexpr int SMEM3(int dp) {
  return NST3(dp) * 2 * C3_BYTES + 2 * XB3(dp) + 2 * H3_BYTES + 1024 + 256;
}
// MODE 4 = MODE 3 in class-chunk-major order: the 16 probes of one 64-class chunk run back to
// back on the same h tile (loaded once per chunk instead of once per probe); the per-probe
// running sums sum h a b, sum h a, sum h b of each row live in shared memory (s <= 16), paid
// for with one coefficient stage less
constexpr int S4MAX = 16;
constexpr int NST4(int dp) { return dp <= 64 ? 3 : 2; }
constexpr int PSUM4 = 3 * S4MAX * 128 * 4;
constexpr int SMEM4(int dp) {
  return NST4(dp) * 2 * C3_BYTES + 2 * XB3(dp) + 2 * H3_BYTES + 1024 + 256 + PSUM4;
}
}  // namespace alpha_cfg

struct TcCtl {   // < 256 bytes
  uint64_t full[4], empty[4], yfull[4], tfull[4], tempty[4], drain, pempty, hfull[2], hempty[2],
      xfull[2], xempty[2];
  uint32_t tmem_base;
  int abort_w;
};
static_assert(sizeof(TcCtl) <= 256, "control block must fit in 256 bytes");

__device__ __forceinline__ void raise_abort(TcCtl* ctl, int32_t* err, int code) {
  ctl->abort_w = 1;
  atomicExch(err, code);
}

// HLO = 1: h enters as bf16 hi + lo.  Every k-step adds H_lo times the hi columns of B
// (MODE 2: the first 128 rows of the tile; MODE 1: the DP hi rows of each probe) into the
// same accumulator columns, so the epilogue sees (H_hi + H_lo) B_hi + H_hi B_lo.
template <int DP, int MODE, int NPART, int HLO = 0>
__global__ void __launch_bounds__(MODE == 4 ? 384 : 256, 1)
    k_tc_alpha(const __grid_constant__ CUtensorMap mapH, const __grid_constant__ CUtensorMap mapP,
               const __grid_constant__ CUtensorMap mapHL, const bf16* __restrict__ Xb,
               const float* __restrict__ w, bf16* __restrict__ aT, float* __restrict__ out32,
               int64_t N, int64_t Np, int s, int kblocks, int n_mt, int n_nt, int npairs, int d,
               int32_t* err, const int2* __restrict__ krange,
               const float* __restrict__ hrow = nullptr, int c = 0, int64_t m = 0,
               float gscale = 0.0f, const int* __restrict__ cen = nullptr,
               const float* __restrict__ cen_am = nullptr, float* __restrict__ cen_rho = nullptr,
               int64_t wskip = 0) {
  using namespace alpha_cfg;
  // MODE 3 stages hold the x tile and two 128-row coefficient tiles (hi and lo), followed by
  // a double buffer of f32 h tiles
  constexpr bool Q3 = MODE == 3 || MODE == 4;   // feature-contracted quadratic forms
  constexpr bool KCM = MODE == 4;                // ... in class-chunk-major tile order
  constexpr int NST = KCM ? NST4(DP) : MODE == 3 ? NST3(DP) : HLO ? STAGES_H : STAGES;
  constexpr int SB = Q3 ? 2 * C3_BYTES : STAGE_BYTES + (HLO ? A_BYTES : 0);
  constexpr int OFF_B = (HLO ? 2 : 1) * A_BYTES;
  constexpr int HBUF = NST * SB;                        // MODE 3 h buffers
  constexpr int XBUF = HBUF + (Q3 ? 2 * H3_BYTES : 0);   // MODE 3/4 resident x tiles
  constexpr int CTL_OFF = XBUF + (Q3 ? 2 * XB3(DP) : 0);
  // TMEM accumulators: four of 128 columns for the quadratic forms (the MMAs run up to three
  // tiles ahead of the epilogue), two of 256 columns otherwise
  constexpr int NACC = Q3 ? 4 : 2;
  constexpr uint32_t ACC_COLS = Q3 ? 128 : BN;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  TcCtl* ctl = (TcCtl*)(sm + CTL_OFF);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int PPN = BN / (NPART * DP);   // probes per N tile
  // MODE 4 tiles carry only 8 MMAs (K = 64, hi and lo), little next to the serial barrier,
  // fence and commit latency of issuing them; two issuer threads (warps 1 and 3) take
  // alternate tiles so that one's hand-offs overlap the other's MMAs.  The operand stages are
  // shared by both, and a parity wait cannot tell a stage's next phase from the one after, so
  // a token passes between the issuers (turn[i]: issuer i may wait for its next tile's stages)
  // and every stage wait happens after the previous use of that stage was seen complete.
  constexpr int NMMA = KCM ? 2 : 1;
  static_assert(MODE != 2 || NPART == 2, "the quadratic mode reads hi and lo halves");
  static_assert(!HLO || (MODE != 0 && NPART == 2), "h_lo is used by the gradient modes");
  // MODE 2: the thread's x row, transposed (column = thread) so reads are conflict-free
  bf16* xsT = (bf16*)(sm + CTL_OFF + 256);   // after the control block
  if (threadIdx.x == 0) {
    for (int i = 0; i < NST; ++i) {
      mbar_init(&ctl->full[i], 1);
      mbar_init(&ctl->empty[i], 1);
    }
    for (int i = 0; i < 4; ++i) {
      mbar_init(&ctl->tfull[i], 1);
      mbar_init(&ctl->tempty[i], 4);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&ctl->hfull[i], 1);
      mbar_init(&ctl->hempty[i], KCM ? 8 : 4);   // MODE 4: both epilogue groups release it
      mbar_init(&ctl->xfull[i], 1);
      mbar_init(&ctl->xempty[i], NMMA);          // MODE 4: both MMA issuers release it
    }
    mbar_init(&ctl->drain, NMMA);
    if (NMMA == 2)
      for (int i = 0; i < 2; ++i) mbar_init(&ctl->yfull[i], 1);   // issuer tokens (turn)
    ctl->abort_w = 0;
    mbar_fence_init();
  }
  if (warp == 1) {
    tmem_alloc(&ctl->tmem_base, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = ctl->tmem_base;
  volatile int* abort_w = &ctl->abort_w;
  const int ntiles = n_mt * n_nt;
  // tile sequence of this CTA: MODE 3 takes every N tile of one point tile in a row (its
  // epilogue accumulates a row over all of them); the other modes stride over all tiles
  // MODE 4: the chunk and probe order of each CTA is rotated by its index, so the CTAs (which
  // run through their point tiles in step) read different coefficient tiles at any moment
  // instead of all hitting the same lines; returns the chunk and probe that iteration nt of a
  // point tile addresses
  const int nkcq = Q3 ? n_nt / s : 1;   // 64-class chunks per probe
  const int rot_k = KCM ? (int)(blockIdx.x % nkcq) : 0;
  const int rot_j = KCM ? (int)((blockIdx.x / nkcq) % s) : 0;
  // Tile cursor.  The quadratic-form modes keep the chunk, probe and h-buffer indices of the
  // current tile incrementally: the producer and MMA roles are single threads whose per-tile
  // work is a handful of instructions, and integer divisions by run-time values on every tile
  // would dominate it.
  //   MODE 4: nt = kr s + jr; chunk (kr + rot_k) mod nkc, probe (jr + rot_j) mod s, hi = it / s
  //   MODE 3: nt = probe nkc + kr; chunk = kr, hi = it
  struct Cur {
    int it, mt, nt, jr, kr, chunk, probe, hi;
  };
  auto cur_set = [&](Cur& q) -> bool {   // other modes: (mt, nt) of q.it
    if (Q3) return q.mt < n_mt;
    const int tile = blockIdx.x + q.it * gridDim.x;
    q.mt = tile / n_nt;
    q.nt = tile % n_nt;
    return tile < ntiles;
  };
  auto cur_first = [&]() -> Cur {
    Cur q{0, (int)blockIdx.x, 0, 0, 0, KCM ? rot_k : 0, KCM ? rot_j : 0, 0};
    cur_set(q);
    return q;
  };
  auto cur_next = [&](Cur& q) -> bool {
    ++q.it;
    if (!Q3) return cur_set(q);
    ++q.nt;
    if (KCM) {
      if (++q.probe == s) q.probe = 0;
      if (++q.jr == s) {
        q.jr = 0;
        q.probe = rot_j;
        ++q.kr;
        ++q.hi;
        if (++q.chunk == nkcq) q.chunk = 0;
      }
    } else {
      ++q.hi;
      if (++q.kr == nkcq) {
        q.kr = 0;
        ++q.probe;
      }
      q.chunk = q.kr;
    }
    if (q.nt == n_nt) {
      q.nt = q.jr = q.kr = 0;
      q.chunk = KCM ? rot_k : 0;
      q.probe = KCM ? rot_j : 0;
      q.mt += gridDim.x;
    }
    return q.mt < n_mt;
  };

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer
    tma_prefetch(&mapH);
    tma_prefetch(&mapP);
    if (HLO || Q3) tma_prefetch(&mapHL);
    int stage = 0;
    uint32_t phase = 0;
    int xcount = 0;   // MODE 3: point tiles whose x rows were loaded
    Cur cu = cur_first();
    for (bool more = Q3 ? cu.mt < n_mt : cur_set(cu); more && !*abort_w; more = cur_next(cu)) {
      const int mt = cu.mt, nt = cu.nt;
      // pooled problems: only the class blocks of the pools in this point tile are non-zero
      const int kb_lo = krange ? krange[mt].x : 0, kb_hi = krange ? krange[mt].y : kblocks;
      if (Q3 && nt == 0) {
        // the point tile's x rows, resident for all its N tiles
        const int xb = xcount & 1;
        if (!mbar_wait(&ctl->xempty[xb], ((xcount >> 1) & 1) ^ 1, abort_w)) {
          raise_abort(ctl, err, 6);
          break;
        }
        unsigned char* xbuf = sm + XBUF + xb * XB3(DP);
        mbar_expect_tx(&ctl->xfull[xb], XB3(DP));
        for (int kb = 0; kb < kblocks; ++kb)
          tma_load_2d(xbuf + kb * A_BYTES, &mapH, &ctl->xfull[xb], kb * BK, mt * BM);
        ++xcount;
      }
      if (MODE == 3 || (KCM && cu.jr == 0)) {
        // the f32 h tile of (point tile, 64-class chunk) for the epilogue (MODE 4: once per
        // chunk, shared by its s probes)
        const int hi = cu.hi;
        const int hb = hi & 1;
        if (!mbar_wait(&ctl->hempty[hb], ((hi >> 1) & 1) ^ 1, abort_w)) {
          raise_abort(ctl, err, 5);
          break;
        }
        const int kc = cu.chunk;
        unsigned char* hbuf = sm + HBUF + hb * H3_BYTES;
        mbar_expect_tx(&ctl->hfull[hb], H3_BYTES);
        tma_load_2d(hbuf, &mapHL, &ctl->hfull[hb], kc * 64, mt * BM);
        tma_load_2d(hbuf + H3_BYTES / 2, &mapHL, &ctl->hfull[hb], kc * 64 + 32, mt * BM);
      }
      for (int kb = kb_lo; kb < kb_hi; ++kb) {
        if (!mbar_wait(&ctl->empty[stage], phase ^ 1, abort_w)) {
          raise_abort(ctl, err, 1);
          break;
        }
        unsigned char* st = sm + stage * SB;
        mbar_expect_tx(&ctl->full[stage], SB);
        if (Q3) {
          // coefficient tiles of (probe j, chunk kc) sit at row block (j nkc + kc) 2 + hl
          const int ntc = KCM ? cu.probe * nkcq + cu.chunk : nt;
          tma_load_2d(st, &mapP, &ctl->full[stage], kb * BK, (2 * ntc) * 128);
          tma_load_2d(st + C3_BYTES, &mapP, &ctl->full[stage], kb * BK, (2 * ntc + 1) * 128);
        } else {
          tma_load_2d(st, &mapH, &ctl->full[stage], kb * BK, mt * BM);
          if (HLO) tma_load_2d(st + A_BYTES, &mapHL, &ctl->full[stage], kb * BK, mt * BM);
          tma_load_2d(st + OFF_B, &mapP, &ctl->full[stage], kb * BK, nt * BN);
        }
        if (++stage == NST) {
          stage = 0;
          phase ^= 1;
        }
      }
    }
    // let every issued load land before the CTA can exit
    for (int i = 0; i < NST; ++i) {
      if (!mbar_wait(&ctl->empty[stage], phase ^ 1, abort_w)) break;
      if (++stage == NST) {
        stage = 0;
        phase ^= 1;
      }
    }
  } else if ((warp == 1 || (NMMA == 2 && warp == 3)) && lane == 0) {
    // ---------------- MMA issuer(s)
    const int mi = warp == 3 ? 1 : 0;
    uint64_t* turn = ctl->yfull;   // MODE 4 issuer tokens (the D-GEMM's y barriers, unused here)
    int nturn = 0;                 // token waits done by this issuer
    bool first_tile = true;
    constexpr uint32_t idesc = idesc_bf16_f32(BM, Q3 ? 128 : BN);
    int stage = 0;
    uint32_t phase = 0;
    int acc = 0;
    uint32_t acc_phase = 0;
    int xcount = 0;
    Cur cu = cur_first();
    for (bool more = Q3 ? cu.mt < n_mt : cur_set(cu); more && !*abort_w; more = cur_next(cu)) {
      const int mt = cu.mt, nt = cu.nt;
      if (Q3 && nt == 0) {
        if (!mbar_wait(&ctl->xfull[xcount & 1], (xcount >> 1) & 1, abort_w)) {
          raise_abort(ctl, err, 7);
          break;
        }
        ++xcount;
      }
      const int kb_lo = krange ? krange[mt].x : 0, kb_hi = krange ? krange[mt].y : kblocks;
      if (NMMA == 2 && (cu.it & 1) != mi) {
        // the other issuer's tile: step over its ring stages and accumulator
        for (int kb = kb_lo; kb < kb_hi; ++kb)
          if (++stage == NST) {
            stage = 0;
            phase ^= 1;
          }
        if (Q3 && nt == n_nt - 1) umma_commit(&ctl->xempty[(xcount - 1) & 1]);
        if (++acc == NACC) {
          acc = 0;
          acc_phase ^= 1;
        }
        continue;
      }
      if (!mbar_wait(&ctl->tempty[acc], acc_phase ^ 1, abort_w)) {
        raise_abort(ctl, err, 2);
        break;
      }
      // issuer 0 holds the token for the CTA's first tile; every other tile waits for it
      if (NMMA == 2 && !(mi == 0 && first_tile)) {
        if (!mbar_wait(&turn[mi], nturn & 1, abort_w)) {
          raise_abort(ctl, err, 8);
          break;
        }
        ++nturn;
      }
      first_tile = false;
      tc_fence_after();
      const uint32_t d = tmem + acc * ACC_COLS;
      bool ok = true;
      for (int kb = kb_lo; kb < kb_hi; ++kb) {
        if (!mbar_wait(&ctl->full[stage], phase, abort_w)) {
          raise_abort(ctl, err, 3);
          ok = false;
          break;
        }
        if (NMMA == 2 && kb == kb_hi - 1) mbar_arrive(&turn[mi ^ 1]);   // pass the token
        tc_fence_after();
        const uint32_t a0 = Q3
                                ? smem_u32(sm + XBUF + ((xcount - 1) & 1) * XB3(DP) + kb * A_BYTES)
                                : smem_u32(sm + stage * SB);
        const uint32_t b0 = Q3 ? smem_u32(sm + stage * SB) : a0 + OFF_B;
#pragma unroll
        for (int k = 0; k < BK / 16; ++k) {
          umma_bf16(d, sdesc_sw128(a0 + k * 32), sdesc_sw128(b0 + k * 32), idesc,
                    (kb != kb_lo || k != 0) ? 1u : 0u);
          if (Q3)   // x (A_lo; B_lo) into the same columns: a and b to ~2^-16
            umma_bf16(d, sdesc_sw128(a0 + k * 32), sdesc_sw128(b0 + C3_BYTES + k * 32), idesc, 1u);
          if (HLO) {
            const uint64_t al = sdesc_sw128(a0 + A_BYTES + k * 32);
            if (MODE == 2) {
              constexpr uint32_t idesc_h = idesc_bf16_f32(BM, BN / 2);
              umma_bf16(d, al, sdesc_sw128(b0 + k * 32), idesc_h, 1u);
            } else {
              constexpr uint32_t idesc_p = idesc_bf16_f32(BM, DP);
#pragma unroll
              for (int jj = 0; jj < PPN; ++jj)
                umma_bf16(d + jj * NPART * DP, al,
                          sdesc_sw128(b0 + jj * NPART * DP * 128 + k * 32), idesc_p, 1u);
            }
          }
        }
        umma_commit(&ctl->empty[stage]);
        if (++stage == NST) {
          stage = 0;
          phase ^= 1;
        }
      }
      if (!ok) break;
      umma_commit(&ctl->tfull[acc]);
      // MODE 3/4: the resident x tile is free once the point tile's last MMAs complete (each
      // issuer commits for its own)
      if (Q3 && nt == n_nt - 1) umma_commit(&ctl->xempty[(xcount - 1) & 1]);
      if (++acc == NACC) {
        acc = 0;
        acc_phase ^= 1;
      }
    }
    // drain: the barrier completes once every MMA issued above (by each issuer) has completed
    umma_commit(&ctl->drain);
    mbar_wait_drain(&ctl->drain, 0);
  } else if (warp >= 4) {
    // ---------------- epilogue: one pool row per thread
    // MODE 4 runs two groups of four warps (384 threads): group g takes the tiles of the probes
    // of parity g, so each SM sub-partition has two epilogue warps to interleave, and the
    // per-probe shared-memory sums of a probe are only ever touched by one group
    const int q = warp & 3;
    const int grp = KCM ? (warp - 4) >> 2 : 0;
    int acc = 0;
    uint32_t acc_phase = 0;
    // MODE 3 running sums of the thread's row: over the classes of the current probe
    // (sum h a b, sum h a, sum h b) and over the probes (q)
    float sab = 0.0f, sa = 0.0f, sb = 0.0f, qacc = 0.0f;
    const int nkc = nkcq;
    float* psum = (float*)(sm + CTL_OFF + 256);   // MODE 4: [3][S4MAX][128] per-probe sums
    Cur cu = cur_first();
    for (bool more = Q3 ? cu.mt < n_mt : cur_set(cu); more && !*abort_w; more = cur_next(cu)) {
      const int mt = cu.mt, nt = cu.nt;
      const int64_t row = (int64_t)mt * BM + q * 32 + lane;
      if (Q3) {
        // per-point quadratic forms (eq. 11) from a = x.A_j[:,k], b = x.B_j[:,k] (K = d), the
        // hi and lo coefficient products summed in TMEM; 64 classes per tile, columns
        // [a (64) | b (64)]; term 1 = sum_k h a b, term 2 = (sum_k h a)(sum_k h b) with the
        // exact f32 h, staged by TMA in 128-byte-swizzled boxes of 32 classes
        const int kc = cu.kr;   // position of the tile's chunk in this point tile's order
        const int hi = cu.hi;
        const int hb = hi & 1;
        const bool own = !KCM || (cu.probe & 1) == grp;
        // every group waits for the h tile (even on tiles it does not own) so that its release
        // below can never count toward a later load of the same buffer
        if (!mbar_wait(&ctl->hfull[hb], (hi >> 1) & 1, abort_w) ||
            (own && !mbar_wait(&ctl->tfull[acc], acc_phase, abort_w))) {
          raise_abort(ctl, err, 4);
          break;
        }
        tc_fence_after();
        const uint32_t tb = tmem + ((uint32_t)(q * 32) << 16) + acc * ACC_COLS;
        const unsigned char* hbuf = sm + HBUF + hb * H3_BYTES;
        const int r = q * 32 + lane;
#pragma unroll 1
        for (int box = 0; box < (own ? 2 : 0); ++box) {
          uint32_t ra[32], rb[32];
          tmem_ld32_async(tb + box * 32, ra);
          tmem_ld32_async(tb + 64 + box * 32, rb);
          // h of classes (2u, 2u + 1) as one packed pair
          uint64_t hv[16];
          const unsigned char* hrow_s = hbuf + box * (H3_BYTES / 2) + r * 128;
#pragma unroll
          for (int ch = 0; ch < 8; ++ch) {
            const ulonglong2 h4 =
                *reinterpret_cast<const ulonglong2*>(hrow_s + ((ch ^ (r & 7)) << 4));
            hv[2 * ch] = h4.x;
            hv[2 * ch + 1] = h4.y;
          }
          tmem_wait_ld();
          // four partial sums per quantity (classes t mod 4), two per packed pair: short
          // dependency chains, half the f32 instructions of the scalar form
          uint64_t pab[2] = {0, 0}, pa[2] = {0, 0}, pb[2] = {0, 0};
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            const uint64_t h2 = hv[u], a2 = f2_pack_u(ra[2 * u], ra[2 * u + 1]),
                           b2 = f2_pack_u(rb[2 * u], rb[2 * u + 1]);
            const uint64_t ha2 = f2_mul(h2, a2);
            pab[u & 1] = f2_fma(ha2, b2, pab[u & 1]);
            pa[u & 1] = f2_add(pa[u & 1], ha2);
            pb[u & 1] = f2_fma(h2, b2, pb[u & 1]);
          }
          float x0, x1, y0, y1;
          f2_unpack(pab[0], x0, x1);
          f2_unpack(pab[1], y0, y1);
          sab += (x0 + x1) + (y0 + y1);
          f2_unpack(pa[0], x0, x1);
          f2_unpack(pa[1], y0, y1);
          sa += (x0 + x1) + (y0 + y1);
          f2_unpack(pb[0], x0, x1);
          f2_unpack(pb[1], y0, y1);
          sb += (x0 + x1) + (y0 + y1);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          if (own) mbar_arrive(&ctl->tempty[acc]);
          if (!KCM || cu.jr == s - 1) mbar_arrive(&ctl->hempty[hb]);
        }
        if (++acc == NACC) {
          acc = 0;
          acc_phase ^= 1;
        }
        if (KCM && own) {
          // probe j's sums over the chunks so far: kept per row in shared memory
          const int j = cu.probe;
          float* ps = psum + j * 128 + r;
          if (kc > 0) {
            sab += ps[0];
            sa += ps[S4MAX * 128];
            sb += ps[2 * S4MAX * 128];
          }
          if (kc == nkc - 1) {
            qacc += sab - sa * sb;
          } else {
            ps[0] = sab;
            ps[S4MAX * 128] = sa;
            ps[2 * S4MAX * 128] = sb;
          }
          sab = sa = sb = 0.0f;
        } else if (kc == nkc - 1) {
          qacc += sab - sa * sb;
          sab = sa = sb = 0.0f;
        }
        if (nt == n_nt - 1) {
          // MODE 4: the two groups' shares land on a zeroed output; with two addends the
          // rounded sum does not depend on their order
          if (row >= m && row < N) {
            if (KCM) atomicAdd(out32 + (row - m), -gscale * qacc);
            else out32[row - m] = -gscale * qacc;
          }
          qacc = 0.0f;
        }
        continue;
      }
      // the thread's x row (packed bf16 pairs) and weight, fetched before the accumulator
      // wait so the global-load latency overlaps the tile's MMAs; reused by every probe/part
      uint32_t xp[DP / 2];
      {
        const uint4* src = reinterpret_cast<const uint4*>(Xb + (row < Np ? row : 0) * DP);
#pragma unroll
        for (int t = 0; t < DP / 8; ++t) {
          const uint4 u = src[t];
          xp[4 * t] = u.x;
          xp[4 * t + 1] = u.y;
          xp[4 * t + 2] = u.z;
          xp[4 * t + 3] = u.w;
        }
      }
      // rows below wskip (labelled rows applied on CUDA cores) take no part here
      const float wi = (MODE == 0) ? (row < N && row >= wskip ? w[row] : 0.0f) : 1.0f;
      // MODE 0 on a centred row: the accumulator holds u . a; alpha = a_m + u . a
      const bool crow = MODE == 0 && cen != nullptr && row < N && cen[row] >= 0;
      if (!mbar_wait(&ctl->tfull[acc], acc_phase, abort_w)) {
        raise_abort(ctl, err, 4);
        break;
      }
      tc_fence_after();
      const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + acc * BN;
      if (MODE == 2) {
        // term1 partial: sum over the 128 pairs of this tile of x_e x_e' (T_hi + T_lo)
        const int tcol = q * 32 + lane;
#pragma unroll
        for (int t = 0; t < DP / 2; ++t) {
          const __nv_bfloat162 pr = *reinterpret_cast<const __nv_bfloat162*>(&xp[t]);
          xsT[(2 * t) * BM + tcol] = pr.x;
          xsT[(2 * t + 1) * BM + tcol] = pr.y;
        }
        float acc1 = 0.0f;
        int e = 0, e2 = 0;
        const int p0 = nt * (BN / 2);
        if (p0 < npairs) pair_of(p0, d, e, e2);
        float xe = __bfloat162float(xsT[e * BM + tcol]);
#pragma unroll 1
        for (int cc = 0; cc < BN / 2; cc += 32) {
          float vh[32], vl[32];
          tmem_ld32(tbase + cc, vh);
          tmem_ld32(tbase + BN / 2 + cc, vl);
#pragma unroll
          for (int t = 0; t < 32; ++t) {
            if (p0 + cc + t < npairs) {
              acc1 = fmaf(xe * __bfloat162float(xsT[e2 * BM + tcol]), vh[t] + vl[t], acc1);
              if (++e2 == d) {
                ++e;
                e2 = e;
                xe = e < DP ? __bfloat162float(xsT[(e < DP ? e : 0) * BM + tcol]) : 0.0f;
              }
            }
          }
        }
        if (row < N) out32[(int64_t)nt * Np + row] = acc1;
      }
#pragma unroll 1
      for (int jj = 0; jj < (MODE == 2 ? 0 : PPN); ++jj) {
        const int j = nt * PPN + jj;
        float sum = 0.0f;
#pragma unroll 1
        for (int part = 0; part < NPART; ++part) {
          constexpr int CW = DP < 32 ? DP : 32;
#pragma unroll
          for (int ec = 0; ec < DP; ec += CW) {
            float v[32];
            const uint32_t col = (uint32_t)((jj * NPART + part) * DP + ec);
            if (CW == 32) tmem_ld32(tbase + col, v);
            else tmem_ld16(tbase + col, v);
#pragma unroll
            for (int t = 0; t < CW; t += 2) {
              const float2 f =
                  __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&xp[(ec + t) / 2]));
              sum = fmaf(f.x, v[t], sum);
              sum = fmaf(f.y, v[t + 1], sum);
            }
          }
        }
        // MODE 0 also zeroes the padding rows N..Np-1: the D-GEMM multiplies them by zero x
        // and h, and a stale non-finite value there would turn the whole probe into NaN
        if (j < s) {
          if (MODE == 0) {
            // walpha^T in the K-block-major layout [row / 64][j][row % 64], sp16 rows per block
            const int sp16 = (s + 15) / 16 * 16;
            float al = sum;
            if (crow) {
              cen_rho[row * s + j] = wi * sum;
              al = cen_am[row * s + j] + sum;
            }
            if (row < Np)
              aT[((row >> 6) * sp16 + j) * 64 + (row & 63)] =
                  __float2bfloat16_rn(row < N ? wi * al : 0.0f);
          } else if (row < N) {
            out32[(int64_t)j * Np + row] = sum;
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&ctl->tempty[acc]);
      acc ^= 1;
      if (acc == 0) acc_phase ^= 1;
    }
  }
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// ------------------------------------------------------------------------------------------
// D-GEMM (split over the point range)
// ------------------------------------------------------------------------------------------
namespace d_cfg {
constexpr int BM = 128, BN = 256, BK = 64;
constexpr int MT = 2;                     // class tiles per CTA sharing one built Y tile
constexpr int A_BYTES = BM * BK * 2;      // one H^T tile
constexpr int Y_BYTES = BN * BK * 2;      // built operand
constexpr int AT_MAX = 16 * BK * 2;       // walpha^T tile (<= 16 probes)
constexpr int NBUILD = 6;                 // builder warps (2..7)
constexpr int64_t D_CHAIN = 512;          // K-steps accumulated in TMEM per split at most
template <int DP> struct Stage {
  static constexpr int XT_BYTES = DP * BK * 2;
  static constexpr int RAW = MT * A_BYTES + Y_BYTES + XT_BYTES + AT_MAX;
  static constexpr int BYTES = (RAW + 1023) / 1024 * 1024;
  static constexpr int STAGES = (3 * BYTES + 2048 <= 227 * 1024) ? 3 : 2;
  static constexpr int SMEM = STAGES * BYTES + 1024 + 256;
};
}  // namespace d_cfg

template <int DP>
__global__ void __launch_bounds__(256, 1)
    k_tc_dterm(const __grid_constant__ CUtensorMap mapHT, const __grid_constant__ CUtensorMap mapXT,
               const __grid_constant__ CUtensorMap mapAT, float* __restrict__ Dpart, int64_t N,
               int c, int d, int s, int n_mt, int n_nt, int splits, int64_t kb_per_split,
               int64_t kb_total, int sp16, int32_t* err, const int4* __restrict__ klist,
               int kbL) {
  using namespace d_cfg;
  using St = Stage<DP>;
  constexpr int STAGES = St::STAGES;
  constexpr int STAGE_BYTES = St::BYTES;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  TcCtl* ctl = (TcCtl*)(sm + STAGES * STAGE_BYTES);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int PPN = BN / DP;                 // probes per N tile
  constexpr int XT_BYTES = St::XT_BYTES;
  constexpr int AT_BYTES = PPN * BK * 2;
  constexpr uint32_t TX = MT * A_BYTES + XT_BYTES + AT_BYTES;
  // stage layout: A (MT class tiles) | Y | x^T | walpha^T
  constexpr int OFF_Y = MT * A_BYTES, OFF_XT = OFF_Y + Y_BYTES, OFF_AT = OFF_XT + XT_BYTES;
  if (threadIdx.x == 0) {
    for (int i = 0; i < STAGES; ++i) {
      mbar_init(&ctl->full[i], 1);
      mbar_init(&ctl->empty[i], 1);
      mbar_init(&ctl->yfull[i], NBUILD);
    }
    mbar_init(&ctl->tfull[0], 1);
    mbar_init(&ctl->tempty[0], 4);
    mbar_init(&ctl->drain, 1);
    ctl->abort_w = 0;
    mbar_fence_init();
  }
  if (warp == 1) {
    tmem_alloc(&ctl->tmem_base, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = ctl->tmem_base;
  volatile int* abort_w = &ctl->abort_w;
  const int nunits = n_mt * n_nt * splits;

  auto unit_range = [&](int u, int& mt, int& nt, int64_t& kb0, int64_t& kb1) {
    // consecutive units share the point range of a split and the class tile: the n tiles
    // of one (split, class tile) run side by side and reuse H^T through L2
    nt = u % n_nt;
    const int rest = u / n_nt;
    mt = rest % n_mt;
    const int sp = rest / n_mt;
    if (klist) {
      // pooled: the tile's K list (virtual K-steps 0..L-1) is split evenly; a unit past its
      // end is empty
      const int64_t L = klist[mt].z, per = (L + splits - 1) / splits;
      kb0 = (int64_t)sp * per;
      kb1 = kb0 + per < L ? kb0 + per : L;
      if (kb0 > kb1) kb0 = kb1;
    } else {
      kb0 = (int64_t)sp * kb_per_split;
      kb1 = kb0 + kb_per_split < kb_total ? kb0 + kb_per_split : kb_total;
    }
  };
  // virtual K-step of tile mt -> K-step of the points (labelled blocks, then the pools' rows)
  auto real_kb = [&](int mt, int64_t v) -> int64_t {
    return (!klist || v < kbL) ? v : klist[mt].x + (v - kbL);
  };

  if (warp == 0 && lane == 0) {
    tma_prefetch(&mapHT);
    tma_prefetch(&mapXT);
    tma_prefetch(&mapAT);
    int stage = 0;
    uint32_t phase = 0;
    bool ok = true;
    for (int u = blockIdx.x; u < nunits && ok && !*abort_w; u += gridDim.x) {
      int mt, nt;
      int64_t kb0, kb1;
      unit_range(u, mt, nt, kb0, kb1);
      for (int64_t kb = kb0; kb < kb1; ++kb) {
        if (!mbar_wait(&ctl->empty[stage], phase ^ 1, abort_w)) {
          raise_abort(ctl, err, 11);
          ok = false;
          break;
        }
        unsigned char* st = sm + stage * STAGE_BYTES;
        mbar_expect_tx(&ctl->full[stage], TX);
        // K-block-major operands: block kb holds n_mt * MT class tiles, DP rows of x^T and
        // sp16 rows of walpha^T, each row 64 points
        const int64_t kr = real_kb(mt, kb);
#pragma unroll
        for (int a = 0; a < MT; ++a)
          tma_load_2d(st + a * A_BYTES, &mapHT, &ctl->full[stage], 0,
                      (int)((kr * n_mt + mt) * MT + a) * BM);
        tma_load_2d(st + OFF_XT, &mapXT, &ctl->full[stage], 0, (int)(kr * DP));
        tma_load_2d(st + OFF_AT, &mapAT, &ctl->full[stage], 0, (int)(kr * sp16 + nt * PPN));
        if (++stage == STAGES) {
          stage = 0;
          phase ^= 1;
        }
      }
    }
    for (int i = 0; i < STAGES; ++i) {
      if (!mbar_wait(&ctl->empty[stage], phase ^ 1, abort_w)) break;
      if (++stage == STAGES) {
        stage = 0;
        phase ^= 1;
      }
    }
  } else if (warp == 1 && lane == 0) {
    constexpr uint32_t idesc = idesc_bf16_f32(BM, BN);
    int stage = 0;
    uint32_t phase = 0;
    uint32_t acc_phase = 0;
    bool ok = true;
    for (int u = blockIdx.x; u < nunits && ok && !*abort_w; u += gridDim.x) {
      int mt, nt;
      int64_t kb0, kb1;
      unit_range(u, mt, nt, kb0, kb1);
      if (kb0 >= kb1) continue;   // empty unit: the epilogue writes zeros without the MMA
      if (!mbar_wait(&ctl->tempty[0], acc_phase ^ 1, abort_w)) {
        raise_abort(ctl, err, 12);
        break;
      }
      tc_fence_after();
      for (int64_t kb = kb0; kb < kb1; ++kb) {
        if (!mbar_wait(&ctl->yfull[stage], phase, abort_w)) {
          raise_abort(ctl, err, 13);
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t a0 = smem_u32(sm + stage * STAGE_BYTES);
        const uint32_t y0 = a0 + OFF_Y;
#pragma unroll
        for (int k = 0; k < BK / 16; ++k) {
          const uint64_t dy = sdesc_sw128(y0 + k * 32);
#pragma unroll
          for (int a = 0; a < MT; ++a)
            umma_bf16(tmem + a * BN, sdesc_sw128(a0 + a * A_BYTES + k * 32), dy, idesc,
                      (kb != kb0) || k != 0);
        }
        umma_commit(&ctl->empty[stage]);
        if (++stage == STAGES) {
          stage = 0;
          phase ^= 1;
        }
      }
      if (!ok) break;
      umma_commit(&ctl->tfull[0]);
      acc_phase ^= 1;
    }
    umma_commit(&ctl->drain);
    mbar_wait_drain(&ctl->drain, 0);
  } else if (warp >= 2) {
    // ---------------- Y builders (warps 2..7), then epilogue (warps 4..7)
    const int bw = warp - 2;
    int stage = 0;
    uint32_t phase = 0;
    uint32_t acc_phase = 0;
    bool ok = true;
    for (int u = blockIdx.x; u < nunits && ok && !*abort_w; u += gridDim.x) {
      int mt, nt;
      int64_t kb0, kb1;
      unit_range(u, mt, nt, kb0, kb1);
      for (int64_t kb = kb0; kb < kb1; ++kb) {
        if (!mbar_wait(&ctl->full[stage], phase, abort_w)) {
          raise_abort(ctl, err, 14);
          ok = false;
          break;
        }
        unsigned char* st = sm + stage * STAGE_BYTES;
        unsigned char* Y = st + OFF_Y;
        const unsigned char* XT = st + OFF_XT;
        const unsigned char* AT = st + OFF_AT;
        // item = (feature e, 8 consecutive points c8).  A thread keeps one c8 (NBUILD*32 is a
        // multiple of 8), holds walpha of its 8 points for every probe of the tile in registers,
        // reads each x chunk once and writes one Y chunk per probe: rows r = jl*DP + e.  The 8
        // threads of a quarter-warp share e, so loads and (swizzled) stores cover one 128-byte
        // row each and are conflict-free.
        {
          const int tid_b = bw * 32 + lane;
          const int c8 = tid_b & 7;
          uint4 av[PPN];
#pragma unroll
          for (int jl = 0; jl < PPN; ++jl)
            av[jl] = *reinterpret_cast<const uint4*>(AT + jl * (BK * 2) + c8 * 16);
          for (int it = tid_b; it < DP * 8; it += NBUILD * 32) {
            const int e = it >> 3;
            const uint4 xv = *reinterpret_cast<const uint4*>(XT + e * (BK * 2) + c8 * 16);
            const __nv_bfloat162* x2 = reinterpret_cast<const __nv_bfloat162*>(&xv);
#pragma unroll
            for (int jl = 0; jl < PPN; ++jl) {
              uint4 yv;
              const __nv_bfloat162* a2 = reinterpret_cast<const __nv_bfloat162*>(&av[jl]);
              __nv_bfloat162* y2 = reinterpret_cast<__nv_bfloat162*>(&yv);
#pragma unroll
              for (int h = 0; h < 4; ++h) y2[h] = __hmul2(x2[h], a2[h]);
              const int r = jl * DP + e;
              *reinterpret_cast<uint4*>(Y + r * 128 + ((c8 ^ (r & 7)) << 4)) = yv;
            }
          }
        }
        fence_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&ctl->yfull[stage]);
        if (++stage == STAGES) {
          stage = 0;
          phase ^= 1;
        }
      }
      if (!ok) break;
      if (kb0 >= kb1) {
        // empty unit: its partial block is zero
        if (warp >= 4) {
          const int q = warp & 3;
          const int sp = (u / n_nt) / n_mt;
          const int sd = s * d;
          for (int a = 0; a < MT; ++a) {
            const int k = (mt * MT + a) * BM + q * 32 + lane;
            if (k >= c) continue;
            float* out = Dpart + ((int64_t)sp * c + k) * sd;
            for (int cc = 0; cc < BN; ++cc) {
              const int col = nt * BN + cc;
              const int j = col / DP, e = col - j * DP;
              if (j < s && e < d) out[j * d + e] = 0.0f;
            }
          }
        }
        continue;
      }
      if (warp >= 4) {
        const int q = warp & 3;
        if (!mbar_wait(&ctl->tfull[0], acc_phase, abort_w)) {
          raise_abort(ctl, err, 15);
          break;
        }
        tc_fence_after();
        const int sp = (u / n_nt) / n_mt;
        const int sd = s * d;
#pragma unroll 1
        for (int a = 0; a < MT; ++a) {
          const int k = (mt * MT + a) * BM + q * 32 + lane;   // class row of this thread
          float* out = Dpart + ((int64_t)sp * c + k) * sd;
          for (int cc = 0; cc < BN; cc += 32) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + a * BN + cc, v);
            if (k < c) {
#pragma unroll
              for (int t = 0; t < 32; ++t) {
                const int col = nt * BN + cc + t;
                const int j = col / DP, e = col - j * DP;
                if (j < s && e < d) out[j * d + e] = v[t];
              }
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&ctl->tempty[0]);
      }
      acc_phase ^= 1;
    }
  }
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// ------------------------------------------------------------------------------------------
// Block sums on tensor cores (eq. 13 and the diagonal-part operator), split over points:
//   S[k,(e,e')] = sum_i (w_i h_ik) x_ie x_ie',   P[k,(e,e')] = sum_i (w_i h_ik (1 - h_ik)) x_ie x_ie'
// for the symmetric pairs e <= e' < d (row-major triangle).  The weight goes into the class
// operand, rebuilt once per call by a streaming kernel,
//   A = (w o h)^T as bf16 hi + lo,   A_P = bf16((w o h (1 - h))^T)        (c x points),
// so that the pair operand Z[(e,e'), i] = x_ie x_ie' depends on the problem only: it is built
// once and stored as bf16 hi + lo, which is exact (a product of two bf16 values has at most 16
// significant bits).  Both block sums are then plain TMA-fed GEMMs over the points:
//   MODE 0:  S ~ A_hi Z_hi + A_lo Z_hi + A_hi Z_lo      (relative error ~2^-16)
//   MODE 1:  one product A Z_hi: P ~ A_P Z_hi (preconditioner), and in the fast mode also
//            S ~ A_hi Z_hi over the pool rows (the bf16 roundings of w h and of x_ie x_ie' are
//            unbiased and independent from point to point, so they average over each class's
//            points)
// Unit = (128 classes, 256 pairs, point range).
//
// Shared-memory bandwidth.  A tcgen05 product reads its A and B operands from shared memory:
// an N = 128, K = 16 product moves 8 KB in 64 tensor cycles, the whole per-SM budget, and the
// TMA writes of the next stages come on top.  N = 256 reads the A tile once for twice the work
// (12 KB in 128 cycles), so the wide tiles take the products further from that bound.
//
// Accumulation length.  The tensor core adds each product block into its f32 accumulator with
// a rounding that is biased (the sum loses magnitude on every add), so a chain of m adds into
// one accumulator carries a relative bias of roughly m * 2^-25; a split of 200k points is
// 37,500 adds, a 1e-3 bias that no averaging removes.  Both sums therefore accumulate in TMEM
// for at most SUBK K-steps (96 adds for MODE 0, 128 for MODE 1) at a time in a short
// buffer, and the epilogue warps fold each finished short buffer into a long TMEM accumulator
// with round-to-nearest f32 adds.  (A biased P would not move the CG solution, but with a
// fixed number of CG iterations it moves the iterates, and with them z.)
// TMEM columns: [0,256) short | [256,512) long (the MMA waits for each fold, once per SUBK
// K-steps).
// ------------------------------------------------------------------------------------------
namespace b_cfg {
constexpr int BM = 128, BK = 64;
constexpr int64_t UNIT_KB = 1024;   // K-steps per unit at most
constexpr int BN = 256;             // pairs per unit
constexpr int NPP_ALIGN = BN;       // pair rows of the pair operand
constexpr int ATILE = BM * BK * 2, ZTILE = BN * BK * 2;
constexpr uint32_t COL_LONG = BN;   // TMEM: short accumulator, then long
template <int MODE> struct Cfg {
  // A_hi A_lo Z_hi Z_lo | A Z_hi
  static constexpr int NT2 = MODE == 0 ? 2 : 1;            // class tiles = pair tiles
  static constexpr int STAGE = NT2 * (ATILE + ZTILE);
  static constexpr int STAGES = (227 * 1024 - 2048) / STAGE < 6 ? (227 * 1024 - 2048) / STAGE : 6;
  static constexpr int64_t SUBK = MODE == 0 ? 8 : 32;
  static constexpr int SMEM = STAGES * STAGE + 1024 + 256;
};
}  // namespace b_cfg

struct BsCtl {   // < 256 bytes
  uint64_t full[8], empty[8], tfull[2], tempty[2], drain;
  uint32_t tmem_base;
  int abort_w;
};
static_assert(sizeof(BsCtl) <= 256, "control block must fit in 256 bytes");

template <int MODE>
__global__ void __launch_bounds__(256, 1)
    k_tc_bsum(const __grid_constant__ CUtensorMap mapA0, const __grid_constant__ CUtensorMap mapA1,
              const __grid_constant__ CUtensorMap mapZ0, const __grid_constant__ CUtensorMap mapZ1,
              float* __restrict__ part, int c, int d, int npairs, int n_mt, int n_nt,
              int splits, int64_t kb_per_split, int64_t kb_total, int32_t* err,
              const int4* __restrict__ klist, int kbL) {
  using namespace b_cfg;
  using C = Cfg<MODE>;
  constexpr int STAGES = C::STAGES;
  constexpr int64_t SUBK = C::SUBK;
  // stage layout: class tile(s), then pair tile(s)
  constexpr int OZ = C::NT2 * ATILE;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  BsCtl* ctl = (BsCtl*)(sm + STAGES * C::STAGE);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < STAGES; ++i) {
      mbar_init(&ctl->full[i], 1);
      mbar_init(&ctl->empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&ctl->tfull[i], 1);
      mbar_init(&ctl->tempty[i], 4);
    }
    mbar_init(&ctl->drain, 1);
    ctl->abort_w = 0;
    mbar_fence_init();
  }
  if (warp == 1) {
    tmem_alloc(&ctl->tmem_base, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = ctl->tmem_base;
  volatile int* abort_w = &ctl->abort_w;
  auto give_up = [&](int code) {
    ctl->abort_w = 1;
    atomicExch(err, code);
  };
  const int nunits = n_mt * n_nt * splits;
  // consecutive units share the point range of a split; the class tiles of one pair tile run
  // side by side (Z tile reused through L2), and so do the pair tiles of one class tile
  auto unit_range = [&](int u, int& mt, int& nt, int& sp, int64_t& kb0, int64_t& kb1) {
    mt = u % n_mt;
    const int rest = u / n_mt;
    nt = rest % n_nt;
    sp = rest / n_nt;
    if (klist) {
      // pooled: the class tile's K list (virtual K-steps 0..L-1) split evenly; a unit past
      // its end is empty and its partial block is written as zeros
      const int64_t L = klist[mt].z, per = (L + splits - 1) / splits;
      kb0 = (int64_t)sp * per;
      kb1 = kb0 + per < L ? kb0 + per : L;
      if (kb0 > kb1) kb0 = kb1;
    } else {
      kb0 = (int64_t)sp * kb_per_split;
      kb1 = kb0 + kb_per_split < kb_total ? kb0 + kb_per_split : kb_total;
    }
  };
  auto real_kb = [&](int mt, int64_t v) -> int64_t {
    return (!klist || v < kbL) ? v : klist[mt].x + (v - kbL);
  };

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer
    tma_prefetch(&mapA0);
    tma_prefetch(&mapZ0);
    if (MODE == 0) {
      tma_prefetch(&mapA1);
      tma_prefetch(&mapZ1);
    }
    int stage = 0;
    uint32_t phase = 0;
    bool ok = true;
    for (int u = blockIdx.x; u < nunits && ok && !*abort_w; u += gridDim.x) {
      int mt, nt, sp;
      int64_t kb0, kb1;
      unit_range(u, mt, nt, sp, kb0, kb1);
      for (int64_t kb = kb0; kb < kb1; ++kb) {
        if (!mbar_wait(&ctl->empty[stage], phase ^ 1, abort_w)) {
          give_up(31);
          ok = false;
          break;
        }
        unsigned char* st = sm + stage * C::STAGE;
        mbar_expect_tx(&ctl->full[stage], C::STAGE);
        const int64_t kr = real_kb(mt, kb);
        const int ya = (int)(kr * n_mt + mt) * BM, yz = (int)(kr * n_nt + nt) * BN;
        tma_load_2d(st, &mapA0, &ctl->full[stage], 0, ya);
        if (MODE == 0) tma_load_2d(st + ATILE, &mapA1, &ctl->full[stage], 0, ya);
        tma_load_2d(st + OZ, &mapZ0, &ctl->full[stage], 0, yz);
        if (MODE == 0) tma_load_2d(st + OZ + ZTILE, &mapZ1, &ctl->full[stage], 0, yz);
        if (++stage == STAGES) {
          stage = 0;
          phase ^= 1;
        }
      }
    }
    // let every issued load land before the CTA can exit
    for (int i = 0; i < STAGES; ++i) {
      if (!mbar_wait(&ctl->empty[stage], phase ^ 1, abort_w)) break;
      if (++stage == STAGES) {
        stage = 0;
        phase ^= 1;
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    constexpr uint32_t idesc = idesc_bf16_f32(BM, BN);
    int stage = 0;
    uint32_t phase = 0;
    uint32_t gsub = 0;   // accumulations issued by this CTA
    bool ok = true;
    for (int u = blockIdx.x; u < nunits && ok && !*abort_w; u += gridDim.x) {
      int mt, nt, sp;
      int64_t kb0, kb1;
      unit_range(u, mt, nt, sp, kb0, kb1);
      for (int64_t c0 = kb0; c0 < kb1 && ok; c0 += SUBK, ++gsub) {
        const int64_t c1 = c0 + SUBK < kb1 ? c0 + SUBK : kb1;
        const uint32_t b = 0, par = gsub & 1;
        if (!mbar_wait(&ctl->tempty[b], par ^ 1, abort_w)) {
          give_up(32);
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t tS = tmem;
        for (int64_t kb = c0; kb < c1; ++kb) {
          if (!mbar_wait(&ctl->full[stage], phase, abort_w)) {
            give_up(33);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a0 = smem_u32(sm + stage * C::STAGE);
#pragma unroll
          for (int k = 0; k < BK / 16; ++k) {
            const uint32_t acc = (kb != c0) || k != 0;
            const uint64_t ah = sdesc_sw128(a0 + k * 32), zh = sdesc_sw128(a0 + OZ + k * 32);
            umma_bf16(tS, ah, zh, idesc, acc);
            if (MODE == 0) {
              umma_bf16(tS, sdesc_sw128(a0 + ATILE + k * 32), zh, idesc, 1u);
              umma_bf16(tS, ah, sdesc_sw128(a0 + OZ + ZTILE + k * 32), idesc, 1u);
            }
          }
          umma_commit(&ctl->empty[stage]);
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1;
          }
        }
        if (!ok) break;
        umma_commit(&ctl->tfull[b]);
      }
    }
    umma_commit(&ctl->drain);
    mbar_wait_drain(&ctl->drain, 0);
  } else if (warp >= 4) {
    // ---------------- epilogue: thread = class row k of the unit (TMEM lane 32 q + lane)
    const int q = warp & 3;
    const uint32_t lanes = (uint32_t)(q * 32) << 16;
    uint32_t gsub = 0;
    bool ok = true;
    for (int u = blockIdx.x; u < nunits && ok && !*abort_w; u += gridDim.x) {
      int mt, nt, sp;
      int64_t kb0, kb1;
      unit_range(u, mt, nt, sp, kb0, kb1);
      const int k = mt * BM + q * 32 + lane;
      if (kb0 >= kb1) {
        // empty unit (pooled problems): zero partial block
        if (k < c) {
          float* out = part + ((int64_t)sp * c + k) * d * d;
          for (int t = 0; t < BN; ++t) {
            const int p = nt * BN + t;
            if (p >= npairs) break;
            int e, e2;
            pair_of(p, d, e, e2);
            out[e * d + e2] = 0.0f;
            out[e2 * d + e] = 0.0f;
          }
        }
        continue;
      }
      for (int64_t c0 = kb0; c0 < kb1; c0 += SUBK, ++gsub) {
        const bool first = c0 == kb0, last = c0 + SUBK >= kb1;
        const uint32_t b = 0, par = gsub & 1;
        if (!mbar_wait(&ctl->tfull[b], par, abort_w)) {
          give_up(34);
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t tS = tmem + lanes, tL = tmem + lanes + COL_LONG;
        float* out = part + ((int64_t)sp * c + k) * d * d;
        for (int cc = 0; cc < BN; cc += 32) {
          float v[32];
          tmem_ld32(tS + cc, v);
          if (!first) {
            float l[32];
            tmem_ld32(tL + cc, l);
#pragma unroll
            for (int t = 0; t < 32; ++t) v[t] += l[t];
          }
          if (!last) {
            tmem_st32(tL + cc, v);
          } else if (k < c) {
            int e = 0, e2 = 0;
            const int p0 = nt * BN + cc;
            if (p0 < npairs) pair_of(p0, d, e, e2);
#pragma unroll
            for (int t = 0; t < 32; ++t) {
              if (p0 + t < npairs) {
                out[e * d + e2] = v[t];
                out[e2 * d + e] = v[t];
                if (++e2 == d) {
                  ++e;
                  e2 = e;
                }
              }
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&ctl->tempty[b]);
      }
    }
  }
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// Z[p][i] = x_ie x_ie' for pair p = (e, e') of the row-major triangle, as bf16 hi and lo (exact);
// rows p >= npairs and columns of padding points are zero.  K-block-major layout
// [i / 64][p][i % 64] (npp rows per block): every 128 x 64 TMA tile is one contiguous 16 KB
// run.  Block = 64 points (staged point-major in shared memory) x every pair; a thread takes
// pairs p, p + 256, ... (consecutive threads read consecutive e' of the staged rows) and
// writes each pair's 64 points as four 32-byte pieces.
__global__ void __launch_bounds__(256) k_build_z(bf16* Zhi, bf16* Zlo, const bf16* Xb, int d,
                                                 int dp, int npairs, int64_t npp) {
  __shared__ __align__(16) bf16 xs[64 * 128];
  const int64_t i0 = (int64_t)blockIdx.x * 64;
  {
    const uint4* src = reinterpret_cast<const uint4*>(Xb + i0 * dp);
    uint4* dst = reinterpret_cast<uint4*>(xs);
    for (int t = threadIdx.x; t < 64 * dp / 8; t += blockDim.x) dst[t] = src[t];
  }
  __syncthreads();
  const int d2 = 2 * d + 1;
  for (int p = threadIdx.x; p < npp; p += blockDim.x) {
    // row e of the triangle: the largest e with e d - e (e - 1) / 2 <= p
    int e = 0, e2 = 0;
    const bool real = p < npairs;
    if (real) {
      e = (int)((d2 - sqrtf((float)(d2 * d2 - 8 * p))) * 0.5f);
      e = e < 0 ? 0 : (e >= d ? d - 1 : e);
      while (e > 0 && e * d - e * (e - 1) / 2 > p) --e;
      while (e + 1 < d && (e + 1) * d - (e + 1) * e / 2 <= p) ++e;
      e2 = e + (p - (e * d - e * (e - 1) / 2));
    }
    bf16* zh = Zhi + ((int64_t)blockIdx.x * npp + p) * 64;
    bf16* zl = Zlo + ((int64_t)blockIdx.x * npp + p) * 64;
#pragma unroll 1
    for (int c16 = 0; c16 < 4; ++c16) {
      uint4 hv[2], lv[2];
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        hv[hh] = make_uint4(0, 0, 0, 0);
        lv[hh] = make_uint4(0, 0, 0, 0);
        if (real) {
          bf16* h = reinterpret_cast<bf16*>(&hv[hh]);
          bf16* l = reinterpret_cast<bf16*>(&lv[hh]);
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            const int i = c16 * 16 + hh * 8 + q;
            const float z = __bfloat162float(xs[i * dp + e]) * __bfloat162float(xs[i * dp + e2]);
            h[q] = __float2bfloat16_rn(z);
            l[q] = __float2bfloat16_rn(z - __bfloat162float(h[q]));
          }
        }
      }
      uint4* oh = reinterpret_cast<uint4*>(zh + c16 * 16);
      uint4* ol = reinterpret_cast<uint4*>(zl + c16 * 16);
      oh[0] = hv[0];
      oh[1] = hv[1];
      ol[0] = lv[0];
      ol[1] = lv[1];
    }
  }
}

// Class operands of the block sums, zero-padded, in the K-block-major layout
// [i / 64][k][i % 64] with cpb rows per block:
//   A_hi = bf16(w u), A_lo = bf16(w u - A_hi), A_P = bf16(w h (1 - h))
// (A_hi only if Ahi, A_lo only if Ahi and Alo, A_P only if AP)
// with u = h, or u = h - e_m on centred rows (cen, may be NULL); rows below wskip take weight
// 0 in A_hi and A_lo (their part of the Hessian apply runs on CUDA cores).
// Block = one 64-point block x 32 classes; each warp store writes one 128-byte row run.
__global__ void k_weighted_hT(bf16* Ahi, bf16* Alo, bf16* AP, const float* Ha, const float* w,
                              int64_t N, int c, int64_t Np, int cpb, const int* cen,
                              int64_t wskip, const int4* klist = nullptr, int kbL = 0) {
  __shared__ float tile[64][33];
  __shared__ float ws[64], wS[64];
  __shared__ int cs[64];
  const int64_t rb = (int64_t)blockIdx.x * 64;
  const int cb = blockIdx.y * 32;
  // pooled: the block sums read, for each 128-class tile, the labelled rows' K-steps and its
  // pools' K-steps only (K list {first, end, ...}); the other blocks stay unwritten
  if (klist) {
    const int64_t kb = blockIdx.x;
    const int4 kl = klist[cb / 128];
    if (kb >= kbL && (kb < kl.x || kb >= kl.y)) return;
  }
  for (int i = threadIdx.y; i < 64; i += blockDim.y) {
    const int64_t r = rb + i;
    const int col = cb + threadIdx.x;
    tile[i][threadIdx.x] = (r < N && col < c) ? Ha[r * c + col] : 0.0f;
  }
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  if (tid < 64) {
    ws[tid] = rb + tid < N ? w[rb + tid] : 0.0f;
    wS[tid] = rb + tid >= wskip ? ws[tid] : 0.0f;
    cs[tid] = (cen != nullptr && rb + tid < N) ? cen[rb + tid] : -1;
  }
  __syncthreads();
  const int t2 = 2 * threadIdx.x;   // points rb + t2, rb + t2 + 1
  const float w0 = ws[t2], w1 = ws[t2 + 1];
  const float ws0 = wS[t2], ws1 = wS[t2 + 1];
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int col = cb + i;
    if (col >= cpb) continue;
    const float h0 = tile[t2][i], h1 = tile[t2 + 1][i];
    // the diagonal-part operator takes u = h - e_m on centred rows
    const float v0 = ws0 * (cs[t2] == col ? h0 - 1.0f : h0);
    const float v1 = ws1 * (cs[t2 + 1] == col ? h1 - 1.0f : h1);
    const int64_t o = ((int64_t)blockIdx.x * cpb + col) * 64 + t2;
    if (Ahi) {
      const __nv_bfloat162 hi = __floats2bfloat162_rn(v0, v1);
      *reinterpret_cast<__nv_bfloat162*>(Ahi + o) = hi;
      if (Alo) {
        const float2 fh = __bfloat1622float2(hi);
        *reinterpret_cast<__nv_bfloat162*>(Alo + o) = __floats2bfloat162_rn(v0 - fh.x, v1 - fh.y);
      }
    }
    if (AP)
      *reinterpret_cast<__nv_bfloat162*>(AP + o) =
          __floats2bfloat162_rn(w0 * h0 * (1.0f - h0), w1 * h1 * (1.0f - h1));
  }
}

// ------------------------------------------------------------------------------------------
// Round scores on tensor cores (eq. 14, Proposition 1):
//   q1_ik = x_i^T M1_k x_i,  q2_ik = x_i^T M2_k x_i,  score_i = sum_k w_ik q1_ik / (1 + eta w_ik q2_ik)
// with w_ik = h_ik (1 - h_ik).  The quadratic forms are a GEMM over feature pairs:
//   q_ik = sum_pairs Z_i(e,e') M~_k(e,e'),  Z_i(e,e') = x_ie x_ie',
// pairs ordered by e with e' running over [8 floor(e/8), d8) so every 8-pair chunk is one
// aligned 16-byte run of x (pairs with e' < e carry weight 0 in M~).  M~ = symmetric weights
// (M_ee on the diagonal, M_ee' + M_e'e above it), fed as bf16 hi + lo.  One unit = one
// 128-point tile; it loops over chunks of 128 classes (N = 256: M1 rows then M2 rows) and keeps
// a running masked argmax per thread (ties to the lowest index).
// ------------------------------------------------------------------------------------------
namespace r_cfg {
constexpr int BM = 128, BN = 256, BK = 64, STAGES = 2, NBUILD = 6;
constexpr int Z_BYTES = BM * BK * 2;
constexpr int M_BYTES = BN * BK * 2;
constexpr int STAGE_BYTES = Z_BYTES + 2 * M_BYTES;       // 80 KB
template <int DP> struct L {
  static constexpr int X_BYTES = BM * DP * 2;
  static constexpr int SMEM = STAGES * STAGE_BYTES + X_BYTES + 1024 + 1024;
};
}  // namespace r_cfg

// Round chains scored in one launch (an eta sweep runs its chains side by side): chain e uses
// eta[e], its own mask (mask + e * mask_stride) and its own M~ rows; its per-CTA winners land
// at part[e * gridDim.x + cta].
constexpr int RC_MAX = 8;
struct RoundChains {
  int n;
  int64_t mask_stride;
  double eta[RC_MAX];
};

struct RoundCtl {
  uint64_t full[2], empty[2], zfull[2], xfull, xempty, tfull, tempty, drain;
  uint32_t tmem_base;
  int abort_w;
  double bval[4 * RC_MAX];
  long long bidx[4 * RC_MAX];
};

template <int DP>
__global__ void __launch_bounds__(256, 1)
    k_tc_round(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapMh,
               const __grid_constant__ CUtensorMap mapMl, const short2* __restrict__ tab,
               const float* __restrict__ Ha, const uint8_t* __restrict__ mask, int64_t m,
               int64_t n, int c, int n_kc, int kblocks, const RoundChains rc,
               double* part_val, int64_t* part_idx, int32_t* err) {
  using namespace r_cfg;
  using LL = L<DP>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* xs = sm + STAGES * STAGE_BYTES;                 // x tile, row i = 2*DP bytes
  RoundCtl* ctl = (RoundCtl*)(xs + LL::X_BYTES);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < STAGES; ++i) {
      mbar_init(&ctl->full[i], 1);
      mbar_init(&ctl->empty[i], 1);
      mbar_init(&ctl->zfull[i], NBUILD);
    }
    mbar_init(&ctl->xfull, 1);
    mbar_init(&ctl->xempty, NBUILD);
    mbar_init(&ctl->tfull, 1);
    mbar_init(&ctl->tempty, 4);
    mbar_init(&ctl->drain, 1);
    ctl->abort_w = 0;
    mbar_fence_init();
  }
  if (warp == 1) {
    tmem_alloc(&ctl->tmem_base, 256);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = ctl->tmem_base;
  volatile int* abort_w = &ctl->abort_w;
  const int n_mt = (int)((n + BM - 1) / BM);
  const int n_ch = rc.n * n_kc;   // (chain, class chunk) pairs, chain-major
  constexpr uint32_t TX = 2 * M_BYTES;

  if (warp == 0 && lane == 0) {
    tma_prefetch(&mapX);
    tma_prefetch(&mapMh);
    tma_prefetch(&mapMl);
    int stage = 0;
    uint32_t phase = 0, xphase = 0;
    bool ok = true;
    for (int mt = blockIdx.x; mt < n_mt && ok && !*abort_w; mt += gridDim.x) {
      if (!mbar_wait(&ctl->xempty, xphase ^ 1, abort_w)) {
        atomicExch(err, 31);
        ctl->abort_w = 1;
        break;
      }
      mbar_expect_tx(&ctl->xfull, LL::X_BYTES);
      tma_load_2d(xs, &mapX, &ctl->xfull, 0, (int)(m + (int64_t)mt * BM));
      xphase ^= 1;
      for (int kc = 0; kc < n_ch && ok; ++kc) {
        for (int kb = 0; kb < kblocks; ++kb) {
          if (!mbar_wait(&ctl->empty[stage], phase ^ 1, abort_w)) {
            atomicExch(err, 32);
            ctl->abort_w = 1;
            ok = false;
            break;
          }
          unsigned char* st = sm + stage * STAGE_BYTES;
          mbar_expect_tx(&ctl->full[stage], TX);
          tma_load_2d(st + Z_BYTES, &mapMh, &ctl->full[stage], kb * BK, kc * BN);
          tma_load_2d(st + Z_BYTES + M_BYTES, &mapMl, &ctl->full[stage], kb * BK, kc * BN);
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1;
          }
        }
      }
    }
    for (int i = 0; i < STAGES; ++i) {
      if (!mbar_wait(&ctl->empty[stage], phase ^ 1, abort_w)) break;
      if (++stage == STAGES) {
        stage = 0;
        phase ^= 1;
      }
    }
  } else if (warp == 1 && lane == 0) {
    constexpr uint32_t idesc = idesc_bf16_f32(BM, BN);
    int stage = 0;
    uint32_t phase = 0, acc_phase = 0;
    bool ok = true;
    for (int mt = blockIdx.x; mt < n_mt && ok && !*abort_w; mt += gridDim.x) {
      for (int kc = 0; kc < n_ch && ok; ++kc) {
        if (!mbar_wait(&ctl->tempty, acc_phase ^ 1, abort_w)) {
          atomicExch(err, 33);
          ctl->abort_w = 1;
          ok = false;
          break;
        }
        tc_fence_after();
        for (int kb = 0; kb < kblocks; ++kb) {
          if (!mbar_wait(&ctl->zfull[stage], phase, abort_w) ||
              !mbar_wait(&ctl->full[stage], phase, abort_w)) {
            atomicExch(err, 34);
            ctl->abort_w = 1;
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t z0 = smem_u32(sm + stage * STAGE_BYTES);
          const uint32_t mh = z0 + Z_BYTES, ml = mh + M_BYTES;
#pragma unroll
          for (int k = 0; k < BK / 16; ++k) {
            const uint64_t dz = sdesc_sw128(z0 + k * 32);
            umma_bf16(tmem, dz, sdesc_sw128(mh + k * 32), idesc, (kb | k) != 0);
            umma_bf16(tmem, dz, sdesc_sw128(ml + k * 32), idesc, 1u);
          }
          umma_commit(&ctl->empty[stage]);
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1;
          }
        }
        if (!ok) break;
        umma_commit(&ctl->tfull);
        acc_phase ^= 1;
      }
    }
    umma_commit(&ctl->drain);
    mbar_wait_drain(&ctl->drain, 0);
  } else if (warp >= 2) {
    const int bw = warp - 2;
    const int tid_b = bw * 32 + lane;
    int stage = 0;
    uint32_t phase = 0, xphase = 0, acc_phase = 0;
    bool ok = true;
    double best[RC_MAX];
    long long besti[RC_MAX];
#pragma unroll
    for (int e = 0; e < RC_MAX; ++e) {
      best[e] = -INFINITY;
      besti[e] = LLONG_MAX;
    }
    for (int mt = blockIdx.x; mt < n_mt && ok && !*abort_w; mt += gridDim.x) {
      if (!mbar_wait(&ctl->xfull, xphase, abort_w)) {
        atomicExch(err, 35);
        ctl->abort_w = 1;
        break;
      }
      xphase ^= 1;
      double score = 0.0;   // epilogue threads: this point's eq. 14 sum over class chunks
      for (int ch = 0; ch < n_ch && ok; ++ch) {
        const int ce = ch / n_kc, kc = ch - ce * n_kc;   // chain, class chunk
        const double eta = rc.eta[ce];
        if (kc == 0) score = 0.0;
        for (int kb = 0; kb < kblocks; ++kb) {
          // the MMA warp must have released this stage (previous round) before Z is rewritten
          if (!mbar_wait(&ctl->empty[stage], phase ^ 1, abort_w)) {
            atomicExch(err, 36);
            ctl->abort_w = 1;
            ok = false;
            break;
          }
          // Z chunks: (row i, 8-pair chunk c8); 8 consecutive threads share row i
          for (int ch = tid_b; ch < BM * 8; ch += NBUILD * 32) {
            const int i = ch >> 3, c8 = ch & 7;
            const short2 ee = tab[kb * 8 + c8];
            uint4 zv = make_uint4(0, 0, 0, 0);
            if (ee.x >= 0) {
              const __nv_bfloat16 xe = *reinterpret_cast<const __nv_bfloat16*>(
                  xs + i * (2 * DP) + ee.x * 2);
              const uint4 xv = *reinterpret_cast<const uint4*>(xs + i * (2 * DP) + ee.y * 2);
              const __nv_bfloat162 x2e = __halves2bfloat162(xe, xe);
              const __nv_bfloat162* a2 = reinterpret_cast<const __nv_bfloat162*>(&xv);
              __nv_bfloat162* z2 = reinterpret_cast<__nv_bfloat162*>(&zv);
#pragma unroll
              for (int h = 0; h < 4; ++h) z2[h] = __hmul2(x2e, a2[h]);
            }
            *reinterpret_cast<uint4*>(sm + stage * STAGE_BYTES + i * 128 + ((c8 ^ (i & 7)) << 4)) = zv;
          }
          fence_async_smem();
          __syncwarp();
          if (lane == 0) mbar_arrive(&ctl->zfull[stage]);
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1;
          }
        }
        if (!ok) break;
        if (warp >= 4) {
          const int q = warp & 3;
          if (!mbar_wait(&ctl->tfull, acc_phase, abort_w)) {
            atomicExch(err, 37);
            ctl->abort_w = 1;
            ok = false;
            break;
          }
          tc_fence_after();
          const int64_t row = (int64_t)mt * BM + q * 32 + lane;    // pool index
          const float* hrow = Ha + (m + (row < n ? row : 0)) * c;
          for (int cc = 0; cc < 128; cc += 32) {
            float q1[32], q2[32];
            tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + cc, q1);
            tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + 128 + cc, q2);
            if (row < n) {
#pragma unroll
              for (int t = 0; t < 32; ++t) {
                const int k = kc * 128 + cc + t;
                if (k < c) {
                  const double hv = (double)hrow[k];
                  const double wk = hv * (1.0 - hv);
                  score += wk * (double)q1[t] / (1.0 + eta * wk * (double)q2[t]);
                }
              }
            }
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&ctl->tempty);
          if (kc == n_kc - 1) {   // the chain's score is complete: masked running argmax
            const int64_t row = (int64_t)mt * BM + q * 32 + lane;
            if (row < n && !mask[ce * rc.mask_stride + row] && score == score &&
                (score > best[ce] || (score == best[ce] && row < besti[ce]))) {
              best[ce] = score;
              besti[ce] = row;
            }
          }
        }
        acc_phase ^= 1;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&ctl->xempty);
    }
    if (warp >= 4) {
      for (int e = 0; e < rc.n; ++e) {
        double bv = best[e];
        long long bix = besti[e];
        for (int o = 16; o > 0; o >>= 1) {
          const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
          const long long oi = __shfl_xor_sync(0xffffffffu, bix, o);
          if (ov > bv || (ov == bv && oi < bix)) {
            bv = ov;
            bix = oi;
          }
        }
        if (lane == 0) {
          ctl->bval[e * 4 + warp - 4] = bv;
          ctl->bidx[e * 4 + warp - 4] = bix;
        }
      }
    }
  }
  __syncthreads();
  if (threadIdx.x < rc.n) {
    const int e = threadIdx.x;
    double b = ctl->bval[e * 4];
    long long bi = ctl->bidx[e * 4];
    for (int w = 1; w < 4; ++w)
      if (ctl->bval[e * 4 + w] > b || (ctl->bval[e * 4 + w] == b && ctl->bidx[e * 4 + w] < bi)) {
        b = ctl->bval[e * 4 + w];
        bi = ctl->bidx[e * 4 + w];
      }
    part_val[e * gridDim.x + blockIdx.x] = b;
    part_idx[e * gridDim.x + blockIdx.x] = bi;
  }
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem, 256);
  }
}

// M~ rows for one Round iteration: row (kc, which, kk) = M_{which, k} symmetric pair weights
// at pair p of the 8-aligned table (0 where e' < e or beyond d), bf16 hi and lo
template <class T>
__global__ void k_round_mpairs(bf16* Mh, bf16* Ml, const T* M1, const T* M2, const short2* tab,
                               int c, int d, int kpad, int n_kc) {
  const int row = blockIdx.x;                 // (chain * n_kc + kc)*256 + which*128 + kk
  const int ce = row / (n_kc * 256), kc = (row / 256) % n_kc, which = (row / 128) & 1,
            kk = row & 127;
  const int k = kc * 128 + kk;
  const T* M = (which == 0 ? M1 : M2) + ((int64_t)ce * c + k) * d * d;
  for (int p = threadIdx.x; p < kpad; p += blockDim.x) {
    float v = 0.0f;
    const short2 ee = tab[p >> 3];
    const int e = ee.x, e2 = ee.y + (p & 7);
    if (k < c && e >= 0 && e2 < d && e2 >= e)
      v = e == e2 ? (float)M[e * d + e] : (float)(M[e * d + e2] + M[e2 * d + e]);
    const bf16 hi = __float2bfloat16_rn(v);
    Mh[(int64_t)row * kpad + p] = hi;
    Ml[(int64_t)row * kpad + p] = __float2bfloat16_rn(v - __bfloat162float(hi));
  }
}

// ------------------------------------------------------------------------------------------
// host side
// ------------------------------------------------------------------------------------------
bool tc_available() { return true; }

static int pow2_dim(int d) {
  int p = 16;
  while (p < d) p <<= 1;
  return p;
}

// Confident rows of a mixed problem (h_m > kCentre): their class m (cen), the rows grouped by class
// in row order (cen_off, cen_idx: a counting sort on the host, so every later per-class sum runs
// in a fixed order) and the centred bf16 copies of h that the Hessian apply's two GEMMs take
// instead of h (Ub row-major, UbT K-block-major).  A problem without confident rows keeps none
// of this and runs exactly as before.
// Labelled rows whose Hessian apply runs on CUDA cores (problems with confident rows; not
// pooled ones): rows [0, lab_rows) take weight 0 in the tensor-core terms.
static int64_t lab_rows(const firal_problem* P) {
  return (P->n_cen > 0 && P->pt.Q == 0) ? P->m : 0;
}

static int32_t tc_prepare_centred(firal_problem* P, int cpb2) {
  cudaStream_t st = P->H->stream;
  const int64_t N = P->N, Np = P->Np;
  const int c = P->c;
  P->n_cen = 0;
  // N class indices, then (8-byte aligned) the count of confident rows and the summed
  // low-rank share of the rows
  const int64_t cnt_off = (N + 1) / 2 * 2;
  FIRAL_TRY(P->cen.ensure((size_t)(cnt_off + 4) * sizeof(int)));
  unsigned long long* cnt = reinterpret_cast<unsigned long long*>(P->cen.as<int>() + cnt_off);
  double* shr = reinterpret_cast<double*>(P->cen.as<int>() + cnt_off + 2);
  FIRAL_CUDA_TRY(cudaMemsetAsync(cnt, 0, 2 * sizeof(unsigned long long), st));
  {
    ProfScope ps(st, PF_PREP);
    count_launch();
    k_row_top<<<(unsigned)std::min<int64_t>((N + 7) / 8, 4LL * P->sms), 256, 0, st>>>(
        P->cen.as<int>(), cnt, shr, P->Ha.as<float>(), N, c);
  }
  FIRAL_CUDA_TRY(cudaGetLastError());
  unsigned long long nconf = 0;
  double share = 0.0;
  FIRAL_CUDA_TRY(cudaMemcpyAsync(&nconf, cnt, sizeof(nconf), cudaMemcpyDeviceToHost, st));
  FIRAL_CUDA_TRY(cudaMemcpyAsync(&share, shr, sizeof(share), cudaMemcpyDeviceToHost, st));
  FIRAL_CUDA_TRY(cudaStreamSynchronize(st));
  P->lowrank_share = share / (double)N;
  if (nconf == 0) {
    P->cen.release();
    return FIRAL_OK;
  }
  std::vector<int> cen(N);
  FIRAL_CUDA_TRY(cudaMemcpyAsync(cen.data(), P->cen.p, (size_t)N * sizeof(int),
                                 cudaMemcpyDeviceToHost, st));
  FIRAL_CUDA_TRY(cudaStreamSynchronize(st));
  std::vector<int> off(c + 1, 0);
  int64_t nc = 0;
  for (int64_t i = 0; i < N; ++i)
    if (cen[i] >= 0) {
      ++off[cen[i] + 1];
      ++nc;
    }
  if (nc == 0) {
    P->cen.release();
    return FIRAL_OK;
  }
  if (nc > INT_MAX) return fail(FIRAL_ERR_UNSUPPORTED, "too many confident rows");
  for (int k = 0; k < c; ++k) off[k + 1] += off[k];
  std::vector<int> idx(nc), pos(off.begin(), off.end() - 1);
  for (int64_t i = 0; i < N; ++i)
    if (cen[i] >= 0) idx[pos[cen[i]]++] = (int)i;
  // work items of at most CEN_ITEM rows of one class; ioff[k] = the class's first item
  std::vector<int4> items;
  std::vector<int> ioff(c + 1, 0);
  for (int k = 0; k < c; ++k) {
    ioff[k] = (int)items.size();
    for (int r = off[k]; r < off[k + 1]; r += CEN_ITEM)
      items.push_back(make_int4(k, r, std::min(r + CEN_ITEM, off[k + 1]), 0));
  }
  ioff[c] = (int)items.size();
  P->n_cen_items = (int)items.size();
  FIRAL_TRY(P->cen_off.ensure((size_t)(c + 1) * sizeof(int)));
  FIRAL_TRY(P->cen_idx.ensure((size_t)nc * sizeof(int)));
  FIRAL_TRY(P->cen_items.ensure(items.size() * sizeof(int4)));
  FIRAL_CUDA_TRY(cudaMemcpyAsync(P->cen_items.p, items.data(), items.size() * sizeof(int4),
                                 cudaMemcpyHostToDevice, st));
  FIRAL_CUDA_TRY(cudaMemcpyAsync(P->cen_off.p, ioff.data(), (size_t)(c + 1) * sizeof(int),
                                 cudaMemcpyHostToDevice, st));
  FIRAL_CUDA_TRY(cudaMemcpyAsync(P->cen_idx.p, idx.data(), (size_t)nc * sizeof(int),
                                 cudaMemcpyHostToDevice, st));
  FIRAL_TRY(P->Ub.ensure((size_t)Np * P->cp * 2));
  FIRAL_TRY(P->UbT.ensure((size_t)Np * cpb2 * 2));
  {
    ProfScope ps(st, PF_PREP);
    count_launch(2);
    dim3 g, b;
    bf16_pad_grid(Np, P->cp, g, b);
    k_bf16_pad<2><<<g, b, 0, st>>>(P->Ub.as<bf16>(), P->Ha.as<float>(), P->cen.as<int>(), N, c,
                                   Np, P->cp);
    k_block_transpose_bf16<<<dim3((unsigned)(Np / 32), (unsigned)(cpb2 / 32)), dim3(32, 8), 0, st>>>(
        P->UbT.as<bf16>(), P->Ub.as<bf16>(), Np, P->cp, cpb2);
  }
  FIRAL_CUDA_TRY(cudaGetLastError());
  // the host vectors are read by the copies: wait before they go out of scope
  FIRAL_CUDA_TRY(cudaStreamSynchronize(st));
  P->n_cen = nc;
  return FIRAL_OK;
}

int32_t tc_prepare(firal_problem* P) {
  cudaStream_t st = P->H->stream;
  if (P->d > 128) return fail(FIRAL_ERR_UNSUPPORTED, "mixed path supports d <= 128");
  P->dp = pow2_dim(P->d);
  P->cp = (int32_t)((P->c + 63) / 64 * 64);
  P->Np = (P->N + 127) / 128 * 128;
  const int64_t Np = P->Np;
  FIRAL_TRY(P->Hb.ensure((size_t)Np * P->cp * 2));
  const int cpb2 = (P->cp + d_cfg::MT * d_cfg::BM - 1) / (d_cfg::MT * d_cfg::BM) * (d_cfg::MT * d_cfg::BM);
  FIRAL_TRY(P->HbT.ensure((size_t)Np * cpb2 * 2));
  FIRAL_TRY(P->Xb.ensure((size_t)Np * P->dp * 2 * 2));   // X (Np x dp) then X^T (dp x Np)
  const int64_t tot_x = Np * P->dp;
  ProfScope ps(st, PF_PREP);
  count_launch(3);
  {
    dim3 g, b;
    bf16_pad_grid(Np, P->cp, g, b);
    k_bf16_pad<0><<<g, b, 0, st>>>(P->Hb.as<bf16>(), P->Ha.as<float>(), nullptr, P->N, P->c, Np,
                                   P->cp);
    bf16_pad_grid(Np, P->dp, g, b);
    k_bf16_pad<0><<<g, b, 0, st>>>(P->Xb.as<bf16>(), P->Xa.as<float>(), nullptr, P->N, P->d, Np,
                                   P->dp);
  }
  FIRAL_CUDA_TRY(cudaGetLastError());
  // h^T and x^T of the D-GEMM, K-block-major
  k_block_transpose_bf16<<<dim3((unsigned)(Np / 32), (unsigned)(cpb2 / 32)), dim3(32, 8), 0, st>>>(
      P->HbT.as<bf16>(), P->Hb.as<bf16>(), Np, P->cp, cpb2);
  k_block_transpose_bf16<<<dim3((unsigned)(Np / 32), (unsigned)((P->dp + 31) / 32)), dim3(32, 8),
                           0, st>>>(P->Xb.as<bf16>() + tot_x, P->Xb.as<bf16>(), Np, P->dp, P->dp);
  FIRAL_CUDA_TRY(cudaGetLastError());
  FIRAL_TRY(tc_prepare_centred(P, cpb2));
  // pair operand of the block sums (problem constant): Z = x (x) x on the pair triangle
  const int npairs = P->d * (P->d + 1) / 2;
  const int64_t npp = (npairs + b_cfg::NPP_ALIGN - 1) / b_cfg::NPP_ALIGN * b_cfg::NPP_ALIGN;
  FIRAL_TRY(P->Zp.ensure((size_t)2 * npp * Np * 2));
  k_build_z<<<(unsigned)(Np / 64), 256, 0, st>>>(
      P->Zp.as<bf16>(), P->Zp.as<bf16>() + npp * Np, P->Xb.as<bf16>(), P->d, P->dp, npairs, npp);
  count_launch();
  FIRAL_CUDA_TRY(cudaGetLastError());
  return FIRAL_OK;
}

template <int DP, int NPART>
static int32_t tc_apply_t(firal_problem* P, const float* w, const float* Sblk, const float* V,
                          int s, float* out, double* pq, double lam_null) {
  using namespace alpha_cfg;
  cudaStream_t st = P->H->stream;
  const int64_t Np = P->Np;
  const int cp = P->cp;
  const int sp16 = (s + 15) / 16 * 16;
  // P~ (hi/lo, or bf16 alone) and walpha^T buffers
  const int64_t prow = (int64_t)s * NPART * DP;
  const int64_t prow_p = (prow + BN - 1) / BN * BN;
  FIRAL_TRY(P->Pb.ensure((size_t)prow_p * cp * 2));
  // probe rows s..sp16-1 of walpha^T feed only D columns that are discarded; keep them finite
  // (zeroed when the buffer is allocated; later calls leave finite values there)
  const size_t wa_before = P->walpha.bytes;
  FIRAL_TRY(P->walpha.ensure((size_t)sp16 * Np * 2));
  if (P->walpha.bytes != wa_before)
    FIRAL_CUDA_TRY(cudaMemsetAsync(P->walpha.p, 0, P->walpha.bytes, st));
  if (prow_p > prow)
    FIRAL_CUDA_TRY(cudaMemsetAsync(P->Pb.as<bf16>() + prow * cp, 0, (prow_p - prow) * cp * 2, st));
  const int Qe = pool_count(P->pt);
  FIRAL_TRY(P->vmean.ensure((size_t)s * Qe * P->d * sizeof(float)));
  FIRAL_TRY(P->qmean.ensure((size_t)s * Qe * P->d * sizeof(float)));
  const int mthreads = (P->d + 31) / 32 * 32;
  {
  ProfScope ps(st, PF_SPLIT);
  count_launch(2);
  FIRAL_TRY(class_mean(P, V, s, P->vmean.as<float>(), st));
  k_split_probes<NPART><<<dim3((unsigned)(cp + 31) / 32, DP / 32 > 0 ? DP / 32 : 1, s), dim3(32, 8), 0,
                   st>>>(P->Pb.as<bf16>(), V, P->vmean.as<float>(), s, P->c, P->d, DP, cp,
                           P->D, P->pt);
  }
  FIRAL_CUDA_TRY(cudaGetLastError());
  // confident rows: a_m = x . P~[:, m] for each, before the alpha-GEMM's epilogue needs it
  const bool centred = P->n_cen > 0;
  // with confident rows the labelled rows (weights 1 in Sigma_z) are applied on CUDA cores
  const int64_t wskip = lab_rows(P);
  const bool lab = wskip > 0 && w == (const float*)P->w_sig.p;
  if (centred) {
    FIRAL_TRY(P->cen_am.ensure((size_t)P->N * s * sizeof(float)));
    FIRAL_TRY(P->cen_rho.ensure((size_t)P->N * s * sizeof(float)));
    const size_t smem_am = (size_t)s * DP * sizeof(float);
    if (smem_am > 48 * 1024)
      FIRAL_CUDA_TRY(cudaFuncSetAttribute(k_centre_am, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem_am));
    ProfScope ps(st, PF_SPLIT);
    count_launch();
    k_centre_am<<<P->n_cen_items, 256, smem_am, st>>>(P->cen_am.as<float>(), P->Pb.as<bf16>(),
                                                      P->Xb.as<bf16>(), P->cen_items.as<int4>(),
                                                      P->cen_idx.as<int>(), s, NPART, DP, cp);
    FIRAL_CUDA_TRY(cudaGetLastError());
  }
  CUtensorMap mH, mP;
  FIRAL_TRY(make_map(&mH, centred ? P->Ub.p : P->Hb.p, Np, cp, BM, BK, true));
  FIRAL_TRY(make_map(&mP, P->Pb.p, prow_p, cp, BN, BK, true));
  const int n_mt = (int)(Np / BM), n_nt = (int)(prow_p / BN);
  const int sms = P->sms;
  const int grid = std::min(n_mt * n_nt, sms);
  static bool attr[4] = {false, false, false, false};
  const int ai = DP == 16 ? 0 : DP == 32 ? 1 : DP == 64 ? 2 : 3;
  if (!attr[ai]) {
    FIRAL_CUDA_TRY(cudaFuncSetAttribute(k_tc_alpha<DP, 0, NPART>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM));
    FIRAL_CUDA_TRY(cudaFuncSetAttribute(k_tc_dterm<DP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        d_cfg::Stage<DP>::SMEM));
    attr[ai] = true;
  }
  {
  ProfScope ps(st, PF_ALPHA);
  count_launch();
  k_tc_alpha<DP, 0, NPART><<<grid, 256, SMEM, st>>>(mH, mP, mH, P->Xb.as<bf16>(), w, P->walpha.as<bf16>(),
                                             nullptr, P->N, Np, s, cp / BK, n_mt, n_nt, 0, P->d,
                                             tc_error_word(P), P->kr_alpha.as<int2>(), nullptr,
                                             0, 0, 0.0f, centred ? P->cen.as<int>() : nullptr,
                                             centred ? P->cen_am.as<float>() : nullptr,
                                             centred ? P->cen_rho.as<float>() : nullptr, wskip);
  }
  FIRAL_CUDA_TRY(cudaGetLastError());
  // D-GEMM
  {
    constexpr int PPN = d_cfg::BN / DP;
    const int sd = s * P->d;
    const int n_mt2 = (cp + d_cfg::MT * d_cfg::BM - 1) / (d_cfg::MT * d_cfg::BM);
    const int n_nt2 = (s * DP + d_cfg::BN - 1) / d_cfg::BN;
    const int64_t kb_total = Np / d_cfg::BK;
    // K-steps a class tile runs over: all points, or (pooled) its longest K list
    const int64_t kL = P->pt.Q ? P->kr_dterm_Lmax : kb_total;
    const int tiles = n_mt2 * n_nt2;
    // at least 16 K-steps per split: short units spend their time in the pipeline ramp and
    // the epilogue, and every split adds one partial block to the combine
    int splits = (int)std::max<int64_t>(1, std::min<int64_t>((4LL * sms + tiles - 1) / tiles,
                                                            kL / 16 > 0 ? kL / 16 : 1));
    // at most D_CHAIN K-steps (4 adds each) per accumulator: the tensor core's f32 accumulation
    // loses about 2^-25 of the running sum per add, so the chain length bounds the bias.  When
    // that raises the split count, round it up to whole waves of units where that costs < 2x.
    const int64_t need = (kL + d_cfg::D_CHAIN - 1) / d_cfg::D_CHAIN;
    if (need > splits) {
      int64_t g = tiles, r = sms;
      while (r) { const int64_t t = g % r; g = r; r = t; }
      const int64_t m = sms / g;                      // splits per whole wave
      const int64_t up = (need + m - 1) / m * m;
      splits = (int)(up < 2 * need ? up : need);
    }
    // a tuned split count (autotuner) may replace the rule, but never below the chain bound
    if (P->tune.dterm_splits > 0)
      splits = (int)std::min<int64_t>(std::max<int64_t>(P->tune.dterm_splits, need), kL);
    if (forced_splits() > 0) splits = (int)std::min<int64_t>(forced_splits(), kL);
    const int64_t kbps = (kL + splits - 1) / splits;
    splits = (int)((kL + kbps - 1) / kbps);
    P->tune_used.dterm_splits = splits;
    // more partial blocks: the class-m part of the centred rows, the labelled rows
    const int extra = (centred ? 1 : 0) + (lab ? 1 : 0);
    FIRAL_TRY(P->Dpart.ensure((size_t)(splits + extra) * P->c * sd * sizeof(float)));
    CUtensorMap mHT, mXT, mAT;
    const uint64_t cpb2 = (uint64_t)n_mt2 * d_cfg::MT * d_cfg::BM;
    FIRAL_TRY(make_map(&mHT, centred ? P->UbT.p : P->HbT.p, (uint64_t)kb_total * cpb2, d_cfg::BK,
                       d_cfg::BM, d_cfg::BK, true));
    FIRAL_TRY(make_map(&mXT, P->Xb.as<bf16>() + Np * DP, (uint64_t)kb_total * DP, d_cfg::BK, DP,
                       d_cfg::BK, false));
    FIRAL_TRY(make_map(&mAT, P->walpha.p, (uint64_t)kb_total * sp16, d_cfg::BK, PPN, d_cfg::BK,
                       false));
    const int units = tiles * splits;
    const int grid2 = std::min(units, sms);
    {
    ProfScope ps(st, PF_DTERM);
    count_launch();
    k_tc_dterm<DP><<<grid2, 256, d_cfg::Stage<DP>::SMEM, st>>>(mHT, mXT, mAT, P->Dpart.as<float>(), P->N, P->c,
                                             P->d, s, n_mt2, n_nt2, splits, kbps, kb_total,
                                             sp16, tc_error_word(P), P->kr_dterm.as<int4>(),
                                             P->kbL);
    }
    FIRAL_CUDA_TRY(cudaGetLastError());
    if (centred) {
      ProfScope ps(st, PF_COMBINE);
      count_launch();
      const size_t smem_c = (size_t)64 * (s + DP) * sizeof(float);
      if (smem_c > 48 * 1024)
        FIRAL_CUDA_TRY(cudaFuncSetAttribute(k_centre_termc,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)smem_c));
      FIRAL_TRY(P->cen_part.ensure((size_t)P->n_cen_items * sd * sizeof(float)));
      count_launch();
      k_centre_termc<<<dim3(P->n_cen_items, (sd + 2047) / 2048), 256, smem_c, st>>>(
          P->cen_part.as<float>(), P->cen_rho.as<float>(), P->Xb.as<bf16>(),
          P->cen_items.as<int4>(), P->cen_idx.as<int>(), s, P->d, DP);
      k_centre_reduce<<<dim3(P->c, (sd + 2047) / 2048), 256, 0, st>>>(
          P->Dpart.as<float>() + (size_t)splits * P->c * sd, P->cen_part.as<float>(),
          P->cen_off.as<int>(), sd);
      FIRAL_CUDA_TRY(cudaGetLastError());
    }
    if (lab) {
      FIRAL_TRY(P->cen_lab.ensure((size_t)P->m * s * P->c * sizeof(float)));
      const size_t smem_g = (size_t)P->c * sizeof(float);
      if (smem_g > 48 * 1024)
        FIRAL_CUDA_TRY(cudaFuncSetAttribute(k_lab_gamma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)smem_g));
      ProfScope ps(st, PF_COMBINE);
      count_launch(2);
      k_lab_gamma<<<dim3((unsigned)P->m, s), 256, smem_g, st>>>(
          P->cen_lab.as<float>(), V, P->vmean.as<float>(), P->Xa.as<float>(), P->Ha.as<float>(),
          w, s, P->c, P->d, P->D);
      k_lab_scatter<<<P->c, 256, 0, st>>>(
          P->Dpart.as<float>() + (size_t)(splits + (centred ? 1 : 0)) * P->c * sd,
          P->cen_lab.as<float>(), P->Xa.as<float>(), P->m, s, P->c, P->d);
      FIRAL_CUDA_TRY(cudaGetLastError());
    }
    FIRAL_TRY(combine_f32(P, Sblk, V, splits + extra, s, out, nullptr, P->vmean.as<float>()));
    // a row-sharded group adds its partials here: the projection below and its dot products
    // act on the whole sum
    FIRAL_TRY(shard_allreduce(P, out, (int64_t)s * P->D, FIRAL_DT_F32, 0));
    ProfScope ps(st, PF_COMBINE);
    count_launch(2);
    FIRAL_TRY(class_mean(P, out, s, P->qmean.as<float>(), st));
    k_project<<<dim3(P->c, (s + 3) / 4), mthreads, 0, st>>>(
        out, P->qmean.as<float>(), P->vmean.as<float>(), V, lam_null, s, P->c, P->d, P->D, pq,
        P->pt);
    FIRAL_CUDA_TRY(cudaGetLastError());
    return FIRAL_OK;
  }
}

static int32_t tc_bsum_launch_attrs() {
  static bool done = false;
  if (!done) {
    FIRAL_CUDA_TRY(cudaFuncSetAttribute(k_tc_bsum<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        b_cfg::Cfg<0>::SMEM));
    FIRAL_CUDA_TRY(cudaFuncSetAttribute(k_tc_bsum<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        b_cfg::Cfg<1>::SMEM));
    done = true;
  }
  return FIRAL_OK;
}

// S (and P if outP) = weighted block sums of the problem's rows with weights w (f32, N).
// The fast mode's bf16 rounding (2^-9 per entry) of the CG direction in the low-rank term and
// of the diagonal-part block sums: kept only while the rows' mean low-rank share (sum_k h_ik^2
// on plain rows, 1 on centred ones: about e / c for flat softmax rows) is at most 0.1;
// otherwise the problem takes the hi + lo forms of the mixed mode.
static bool fast_rounding(const firal_problem* P) {
  return P->prec == FIRAL_MIXED_BF16_FAST && P->lowrank_share <= 0.1;
}

// The labelled rows' diagonal-part block sums S_lab[k] = sum_{i < m} h_ik x_i x_i^T (their
// weight is 1 in every Sigma_z): three products over their K-steps only, once per problem.
// The fast mode's one-product sums leave these rows out: a few rows of weight 1 carry as much
// of S as the whole pool, and their bf16 roundings would not average out.
static int32_t tc_labelled_blocks(firal_problem* P) {
  using namespace b_cfg;
  cudaStream_t st = P->H->stream;
  const int64_t Np = P->Np, m = P->m;
  const int cp = P->cp, c = P->c, d = P->d;
  const int npairs = d * (d + 1) / 2;
  const int64_t npp = (npairs + NPP_ALIGN - 1) / NPP_ALIGN * NPP_ALIGN;
  const int n_mt = (cp + BM - 1) / BM, n_nt = (int)(npp / BN);
  const int cpb = n_mt * BM;
  const int64_t asz = (int64_t)cpb * Np, kb_total = Np / BK, kbm = (m + BK - 1) / BK;
  const int64_t per = (int64_t)c * d * d;
  FIRAL_TRY(P->S_lab.ensure((size_t)per * sizeof(float)));
  FIRAL_TRY(P->w_lab.ensure((size_t)P->N * sizeof(float)));
  FIRAL_TRY(fill_weights(false, P->w_lab.p, m, 1.0, nullptr, 0.0, P->n, st));
  FIRAL_TRY(P->syrk_part.ensure((size_t)per * sizeof(float)));
  FIRAL_TRY(P->Aw.ensure((size_t)3 * asz * 2));
  bf16* Ahi = P->Aw.as<bf16>();
  bf16* Alo = Ahi + asz;
  FIRAL_TRY(tc_bsum_launch_attrs());
  ProfScope ps(st, PF_SYRK);
  count_launch(2);
  k_weighted_hT<<<dim3((unsigned)kbm, (unsigned)(cpb / 32)), dim3(32, 8), 0, st>>>(
      Ahi, Alo, nullptr, P->Ha.as<float>(), P->w_lab.as<float>(), P->N, c, Np, cpb, nullptr, 0);
  FIRAL_CUDA_TRY(cudaGetLastError());
  CUtensorMap mA0, mA1, mZ0, mZ1;
  const uint64_t arows = (uint64_t)kb_total * cpb, zrows = (uint64_t)kb_total * npp;
  FIRAL_TRY(make_map(&mA0, Ahi, arows, BK, BM, BK, true));
  FIRAL_TRY(make_map(&mA1, Alo, arows, BK, BM, BK, true));
  FIRAL_TRY(make_map(&mZ0, P->Zp.p, zrows, BK, BN, BK, true));
  FIRAL_TRY(make_map(&mZ1, P->Zp.as<bf16>() + npp * Np, zrows, BK, BN, BK, true));
  const int tiles = n_mt * n_nt;
  k_tc_bsum<0><<<std::min(tiles, P->sms), 256, Cfg<0>::SMEM, st>>>(
      mA0, mA1, mZ0, mZ1, P->syrk_part.as<float>(), c, d, npairs, n_mt, n_nt, 1, kbm, kbm,
      tc_error_word(P), nullptr, 0);
  FIRAL_CUDA_TRY(cudaGetLastError());
  FIRAL_TRY(syrk_reduce_f32(P, P->syrk_part.as<float>(), nullptr, 1, 0.0, P->S_lab.as<float>(),
                            0.0, nullptr));
  P->slab_ready = true;
  return FIRAL_OK;
}

int32_t tc_syrk_blocks(firal_problem* P, const void* wv, double lamS, void* outS, double lamP,
                       double* outP) {
  using namespace b_cfg;
  const float* w = (const float*)wv;
  cudaStream_t st = P->H->stream;
  const int64_t Np = P->Np;
  const int cp = P->cp, c = P->c, d = P->d;
  const int sms = P->sms;
  // the fused per-point apply of pooled problems has no diagonal-part operator: only the
  // preconditioner blocks are summed
  const bool wantS = !P->pw;
  if (!wantS) outS = nullptr;
  if (!outS && !outP) return FIRAL_OK;
  const int npairs = d * (d + 1) / 2;
  const int64_t npp = (npairs + NPP_ALIGN - 1) / NPP_ALIGN * NPP_ALIGN;
  const int n_mt = (cp + BM - 1) / BM;
  const int n_nt = (int)(npp / BN);
  const int64_t kb_total = Np / BK;
  const int64_t kL = P->pt.Q ? P->kr_bsum_Lmax : kb_total;   // longest class-tile K list
  const int tiles = n_mt * n_nt;
  int splits = (int)std::max<int64_t>(1, std::min<int64_t>((4LL * sms + tiles - 1) / tiles,
                                                          kL / 8 > 0 ? kL / 8 : 1));
  // Units of at most UNIT_KB K-steps: the CTAs that share an A or Z tile stream start each
  // unit together, which keeps them within L2 reach of one another (over long units they
  // drift apart and the shared tiles are fetched from DRAM again).  Whole waves of units.
  const int64_t need = (kL + UNIT_KB - 1) / UNIT_KB;
  if (need > splits) {
    int64_t g = tiles, r = sms;
    while (r) { const int64_t t = g % r; g = r; r = t; }
    const int64_t m = sms / g;
    const int64_t up = (need + m - 1) / m * m;
    splits = (int)(up < 2 * need ? up : need);
  }
  if (P->tune.bsum_splits > 0) splits = (int)std::min<int64_t>(P->tune.bsum_splits, kL);
  if (forced_splits() > 0) splits = (int)std::min<int64_t>(forced_splits(), kL);
  const int64_t kbps = (kL + splits - 1) / splits;
  splits = (int)((kL + kbps - 1) / kbps);
  P->tune_used.bsum_splits = splits;
  const int64_t per = (int64_t)c * d * d;
  FIRAL_TRY(P->syrk_part.ensure((size_t)per * splits * 2 * sizeof(float)));
  float* pS = P->syrk_part.as<float>();
  float* pP = pS + per * splits;
  // class operands for this weight vector: (w h)^T hi | lo | (w h (1 - h))^T, K-block-major
  const int cpb = n_mt * BM;
  const int64_t asz = (int64_t)cpb * Np;
  FIRAL_TRY(P->Aw.ensure((size_t)3 * asz * 2));
  bf16* Ahi = P->Aw.as<bf16>();
  bf16* Alo = Ahi + asz;
  bf16* AP = Ahi + 2 * asz;
  FIRAL_TRY(tc_bsum_launch_attrs());
  const int units = tiles * splits;
  {
    ProfScope ps(st, PF_SYRK);
    // S as one product (A_hi against the pairs' bf16 part Z_hi) in the fast mode, for the
    // Relax operators' weights: the pool rows' bf16 roundings of w h and of x_ie x_ie' (2^-9
    // each) average over each class's points like those of the fast CG direction.  The
    // labelled rows (weight 1 in Sigma_z, 0 in H_p) enter Sigma_z's S through S_lab (three
    // products, once per problem) unless the apply already runs them on CUDA cores
    // (lab_rows).
    const bool sig = w == P->w_sig.as<float>();
    const bool s1 = fast_rounding(P) && !P->pt.Q && (sig || w == P->w_p.as<float>());
    const bool lab_sep = s1 && outS && sig && P->m > 0 && lab_rows(P) == 0;
    if (lab_sep && !P->slab_ready) FIRAL_TRY(tc_labelled_blocks(P));
    count_launch(1 + (outS ? 1 : 0) + (outP ? 1 : 0));
    k_weighted_hT<<<dim3((unsigned)(Np / 64), (unsigned)(cpb / 32)), dim3(32, 8), 0, st>>>(
        outS ? Ahi : nullptr, s1 ? nullptr : Alo, outP ? AP : nullptr, P->Ha.as<float>(), w,
        P->N, c, Np, cpb,
        P->n_cen > 0 ? P->cen.as<int>() : nullptr, lab_sep ? P->m : lab_rows(P),
        P->pt.Q ? P->kr_bsum.as<int4>() : nullptr, P->kbL);
    FIRAL_CUDA_TRY(cudaGetLastError());
    // blocked operands as 2-D tensors of 64-point rows: tile (kb, row block) = 16 KB run
    CUtensorMap mA0, mA1, mA2, mZ0, mZ1;
    const uint64_t arows = (uint64_t)kb_total * cpb, zrows = (uint64_t)kb_total * npp;
    FIRAL_TRY(make_map(&mA0, Ahi, arows, BK, BM, BK, true));
    FIRAL_TRY(make_map(&mA1, Alo, arows, BK, BM, BK, true));
    FIRAL_TRY(make_map(&mA2, AP, arows, BK, BM, BK, true));
    FIRAL_TRY(make_map(&mZ0, P->Zp.p, zrows, BK, BN, BK, true));
    FIRAL_TRY(make_map(&mZ1, P->Zp.as<bf16>() + npp * Np, zrows, BK, BN, BK, true));
    const int grid = std::min(units, sms);
    if (outS && s1) {
      // one product: A_hi against the pair operand's bf16 part
      k_tc_bsum<1><<<grid, 256, Cfg<1>::SMEM, st>>>(mA0, mA0, mZ0, mZ0, pS, c, d, npairs, n_mt,
                                                    n_nt, splits, kbps, kb_total,
                                                    tc_error_word(P), P->kr_bsum.as<int4>(),
                                                    P->kbL);
      FIRAL_CUDA_TRY(cudaGetLastError());
    } else if (outS) {
      k_tc_bsum<0><<<grid, 256, Cfg<0>::SMEM, st>>>(mA0, mA1, mZ0, mZ1, pS, c, d, npairs, n_mt,
                                                    n_nt, splits, kbps, kb_total,
                                                    tc_error_word(P), P->kr_bsum.as<int4>(),
                                                    P->kbL);
      FIRAL_CUDA_TRY(cudaGetLastError());
    }
    if (outP) {
      k_tc_bsum<1><<<grid, 256, Cfg<1>::SMEM, st>>>(mA2, mA2, mZ0, mZ0, pP, c, d, npairs, n_mt,
                                                    n_nt, splits, kbps, kb_total,
                                                    tc_error_word(P), P->kr_bsum.as<int4>(),
                                                    P->kbL);
      FIRAL_CUDA_TRY(cudaGetLastError());
    }
    return syrk_reduce_f32(P, outS ? pS : nullptr, outP ? pP : nullptr, splits, lamS,
                           (float*)outS, lamP, outP, lab_sep ? P->S_lab.as<float>() : nullptr);
  }
}

// ------------------------------------------------------------------------------------------
// Per-point quadratic forms on tensor cores (eq. 11):
//   q_i = sum_j a_j^T H_i b_j = sum_k h_ik x_i^T M_k x_i - sum_j (h_i.a_ij)(h_i.b_ij),
//   M_k = sum_j A_j[:,k] B_j[:,k]^T,  a_ijk = x_i.A_j[:,k],  b_ijk = x_i.B_j[:,k].
// A and B are first projected onto N^perp (class means removed): H_i vanishes on N, so the
// value is unchanged, and bf16 rounding of h cannot act on the near-null directions.
// term1 = rowdot(x (x) x, H . M~) with the symmetric part of M_k (alpha-GEMM, MODE 2);
// term2 from the alpha-GEMM on [A; B] with f32 output (MODE 1).
// ------------------------------------------------------------------------------------------
// Coefficient rows of the feature-contracted quadratic forms: row ((j nkc + kc) 2 + hl) 128 + r
// holds, over the features e < dp, the class-mean-projected A_j (r < 64, class 64 kc + r) or
// B_j (r >= 64, class 64 kc + r - 64), as bf16 hi (hl = 0) or lo (hl = 1); zero for classes
// >= c or e >= d.  means: [A; B] class means, (2 s) x pools x d.
__global__ void k_build_coef(bf16* Cf, const float* A, const float* B, const float* mean, int s,
                             int c, int d, int dp, int64_t D, int nkc, PoolTab pt) {
  const int rb = blockIdx.x;                 // ((j nkc + kc) 2 + hl)
  const int hl = rb & 1, kc = (rb >> 1) % nkc, j = (rb >> 1) / nkc;
  const int Qe = pool_count(pt);
  for (int idx = threadIdx.x; idx < 128 * dp; idx += blockDim.x) {
    const int r = idx / dp, e = idx - r * dp;
    const bool isb = r >= 64;
    const int k = kc * 64 + (isb ? r - 64 : r);
    const float* src = isb ? B : A;
    const int jm = isb ? s + j : j;
    float v = 0.0f;
    if (k < c && e < d)
      v = src[(int64_t)j * D + (int64_t)k * d + e] - mean[(jm * Qe + pool_of(pt, k)) * d + e];
    const bf16 hi = __float2bfloat16_rn(v);
    Cf[((int64_t)rb * 128 + r) * dp + e] = hl ? __float2bfloat16_rn(v - __bfloat162float(hi)) : hi;
  }
}

__global__ void k_build_mpairs(bf16* Mt, const float* A, const float* B, const float* meanA,
                               const float* meanB, int s, int c, int d, int64_t D, int cp,
                               int npairs, PoolTab pt) {
  extern __shared__ float Msh[];   // d*d
  const int k = blockIdx.x;
  const int Qe = pool_count(pt), pk = pool_of(pt, k);
  for (int t = threadIdx.x; t < d * d; t += blockDim.x) {
    const int e = t / d, e2 = t - e * d;
    double acc = 0.0;
    for (int j = 0; j < s; ++j) {
      const float a = A[(int64_t)j * D + (int64_t)k * d + e] - meanA[(j * Qe + pk) * d + e];
      const float b = B[(int64_t)j * D + (int64_t)k * d + e2] - meanB[(j * Qe + pk) * d + e2];
      acc += (double)a * (double)b;
    }
    Msh[t] = (float)acc;
  }
  __syncthreads();
  for (int p = threadIdx.x; p < npairs; p += blockDim.x) {
    int e, e2;
    pair_of(p, d, e, e2);
    const float v = e == e2 ? Msh[e * d + e] : Msh[e * d + e2] + Msh[e2 * d + e];
    const bf16 hi = __float2bfloat16_rn(v);
    const bf16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
    const int nt = p / 128, pl = p - nt * 128;
    Mt[((int64_t)nt * 256 + pl) * cp + k] = hi;
    Mt[((int64_t)nt * 256 + 128 + pl) * cp + k] = lo;
  }
}

__global__ void k_quad_combine(const float* part1, int n_nt1, const float* a32, int s,
                               int64_t m, int64_t N, int64_t Np, double scale, float* g) {
  for (int64_t i = m + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    double t1 = 0.0, t2 = 0.0;
    for (int nt = 0; nt < n_nt1; ++nt) t1 += part1[(int64_t)nt * Np + i];
    for (int j = 0; j < s; ++j)
      t2 += (double)a32[(int64_t)j * Np + i] * (double)a32[(int64_t)(s + j) * Np + i];
    g[i - m] = (float)(-scale / s * (t1 - t2));
  }
}

// bf16(h - bf16(h)), the low part of h, for the pair-form gradient GEMMs only (the
// feature-contracted form reads f32 h): made on first use
static int32_t ensure_hlo(firal_problem* P) {
  const size_t bytes = (size_t)P->Np * P->cp * 2;
  if (P->Hlo.p && P->Hlo.bytes >= bytes && P->hlo_ready) return FIRAL_OK;
  FIRAL_TRY(P->Hlo.ensure(bytes));
  ProfScope ps(P->H->stream, PF_PREP);
  count_launch();
  dim3 g, b;
  bf16_pad_grid(P->Np, P->cp, g, b);
  k_bf16_pad<1><<<g, b, 0, P->H->stream>>>(P->Hlo.as<bf16>(), P->Ha.as<float>(), nullptr, P->N,
                                           P->c, P->Np, P->cp);
  FIRAL_CUDA_TRY(cudaGetLastError());
  P->hlo_ready = true;
  return FIRAL_OK;
}

// ------------------------------------------------------------------------------------------
// Per-point quadratic forms (eq. 11) at d <= 64 with many classes, s <= 16: class-chunk-major,
// two probes per MMA.  For point tile i and 64-class chunk kc, the probes run in pairs
// (j, j'), one unit each:
//   S_A = x [A_j | A_j'][:, chunk]^T,  S_B = x [B_j | B_j'][:, chunk]^T      (N = 128 each)
// with A~ and B~ as bf16 hi + lo, except an A that is the probe block itself: its entries
// (+-1) are exact in bf16 and it needs neither a low part nor the class-mean projection (the
// forms are unchanged by adding a per-row constant to a, since the row's h sums to one).
// Epilogue: 8 warps; per probe the running sums sum_k h a b, sum_k h a, sum_k h b over the
// chunks stay in registers, and after the last chunk q = sum_j (sum h a b - (sum h a)(sum h b)).
// Each row's q reaches g as two atomic adds on zeroed memory (the sum of two addends does not
// depend on order).  General A: warp (quarter, half) takes TMEM lanes of its quarter and
// probe 2 jp + half, reading the chunk's h tile from shared memory for each pair.  Exact A:
// warp (quarter, box) takes class box `box` (32 classes) of both probes, with the box's h in
// registers for all the chunk's pairs, so the h tile is released as soon as it is read and one
// h buffer suffices; the freed space holds a third coefficient stage (three units in flight:
// each 48 KB block feeds only 768 MMA cycles) and the boxes' exchange of per-probe sums.
// Pipeline: x tile and TMEM accumulators double-buffered; coefficient blocks 2 (general A)
// or 3 (exact A) deep.
// ------------------------------------------------------------------------------------------
namespace qf_cfg {
constexpr int NP2MAX = 8;                     // probe pairs (s <= 16)
constexpr int CBLK = 512 * 128;               // coefficient block: up to 4 x 128 rows of 128 B
constexpr int HT = 128 * 64 * 4;              // f32 h tile, two 128-byte-swizzled boxes
constexpr int XT = 128 * 128;                 // x tile
constexpr int QX = 2 * 2 * NP2MAX * 128 * 4;  // box 1's per-probe sums (exact A)
template <bool AEXACT> struct L {
  static constexpr int CST = AEXACT ? 384 * 128 : CBLK;   // coefficient stage
  static constexpr int NCS = AEXACT ? 3 : 2;              // coefficient stages
  static constexpr int NHB = AEXACT ? 1 : 2;              // h buffers
  static constexpr int OFF_C = 0, OFF_H = NCS * CST, OFF_X = OFF_H + NHB * HT;
  static constexpr int OFF_Q = OFF_X + 2 * XT;
  static constexpr int OFF_CTL = OFF_Q + (AEXACT ? QX : 0);
  static constexpr int SMEM = OFF_CTL + 256 + 1024;
};
static_assert(L<true>::SMEM <= 232448 && L<false>::SMEM <= 232448, "shared memory per CTA");
}  // namespace qf_cfg

struct QfCtl {   // < 256 bytes
  uint64_t x_full[2], x_empty[2], h_full[2], h_empty[2], c_full[3], c_empty[3], s_full[2],
      s_empty[2], drain, q_full, q_empty;
  uint32_t tmem_base;
  int abort_w;
};
static_assert(sizeof(QfCtl) <= 256, "control block must fit in 256 bytes");

// h of 32 classes (box of the tile) times 32 a and b columns: the running sums of one probe
__device__ __forceinline__ void qf_box(const uint32_t (&ra)[32], const uint32_t (&rb)[32],
                                       const unsigned char* hrow, int r, float& sab, float& sa,
                                       float& sb) {
  uint64_t pab = 0, pa = 0, pb = 0;
#pragma unroll
  for (int ch = 0; ch < 8; ++ch) {
    const ulonglong2 h4 = *reinterpret_cast<const ulonglong2*>(hrow + ((ch ^ (r & 7)) << 4));
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const uint64_t h2 = v ? h4.y : h4.x;
      const int t = 4 * ch + 2 * v;
      const uint64_t a2 = f2_pack_u(ra[t], ra[t + 1]), b2 = f2_pack_u(rb[t], rb[t + 1]);
      const uint64_t ha2 = f2_mul(h2, a2);
      pab = f2_fma(ha2, b2, pab);
      pa = f2_add(pa, ha2);
      pb = f2_fma(h2, b2, pb);
    }
  }
  float x0, x1;
  f2_unpack(pab, x0, x1);
  sab += x0 + x1;
  f2_unpack(pa, x0, x1);
  sa += x0 + x1;
  f2_unpack(pb, x0, x1);
  sb += x0 + x1;
}

// The same sums with h of the box in registers (16 packed pairs), for probe pairs whose box
// of 32 classes is handled by one thread: sab over all probes, sa and sb per probe.
__device__ __forceinline__ void qf_box_reg(const uint32_t (&ra)[32], const uint32_t (&rb)[32],
                                           const uint64_t (&h2)[16], float& sab, float& sa,
                                           float& sb) {
  uint64_t pab = 0, pa = 0, pb = 0;
#pragma unroll
  for (int t = 0; t < 16; ++t) {
    const uint64_t a2 = f2_pack_u(ra[2 * t], ra[2 * t + 1]), b2 = f2_pack_u(rb[2 * t], rb[2 * t + 1]);
    const uint64_t ha2 = f2_mul(h2[t], a2);
    pab = f2_fma(ha2, b2, pab);
    pa = f2_add(pa, ha2);
    pb = f2_fma(h2[t], b2, pb);
  }
  float x0, x1;
  f2_unpack(pab, x0, x1);
  sab += x0 + x1;
  f2_unpack(pa, x0, x1);
  sa += x0 + x1;
  f2_unpack(pb, x0, x1);
  sb += x0 + x1;
}

template <bool AEXACT>
__global__ void __launch_bounds__(384, 1)
    k_tc_qf(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapC,
            const __grid_constant__ CUtensorMap mapH, float* __restrict__ g, int64_t N,
            int64_t m, int n_mt, int nkc, int np2, float gscale, int32_t* err) {
  using namespace qf_cfg;
  using Lc = L<AEXACT>;
  constexpr int NR = AEXACT ? 384 : 512;      // coefficient rows per unit
  constexpr int NCS = Lc::NCS, NHB = Lc::NHB, CST = Lc::CST;
  constexpr int OFF_C = Lc::OFF_C, OFF_H = Lc::OFF_H, OFF_X = Lc::OFF_X, OFF_CTL = Lc::OFF_CTL;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  QfCtl* ctl = (QfCtl*)(sm + OFF_CTL);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int b = 0; b < 2; ++b) {
      mbar_init(&ctl->x_full[b], 1);
      mbar_init(&ctl->x_empty[b], 1);
      mbar_init(&ctl->h_full[b], 1);
      mbar_init(&ctl->h_empty[b], 8);
      mbar_init(&ctl->s_full[b], 1);
      mbar_init(&ctl->s_empty[b], 8);
    }
    for (int b = 0; b < NCS; ++b) {
      mbar_init(&ctl->c_full[b], 1);
      mbar_init(&ctl->c_empty[b], 1);
    }
    mbar_init(&ctl->q_full, 4);
    mbar_init(&ctl->q_empty, 4);
    mbar_init(&ctl->drain, 1);
    ctl->abort_w = 0;
    mbar_fence_init();
  }
  if (warp == 2) {
    tmem_alloc(&ctl->tmem_base, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = ctl->tmem_base;
  volatile int* abort_w = &ctl->abort_w;
  auto give_up = [&](int code) {
    ctl->abort_w = 1;
    atomicExch(err, code);
  };
  const int rot = (int)(blockIdx.x % nkc);   // CTAs start on different chunks

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer
    tma_prefetch(&mapX);
    tma_prefetch(&mapC);
    tma_prefetch(&mapH);
    uint32_t nx = 0, nh = 0, nc = 0;
    bool ok = true;
    for (int mt = blockIdx.x; mt < n_mt && ok && !*abort_w; mt += gridDim.x) {
      {
        const int b = nx & 1;
        if (!mbar_wait(&ctl->x_empty[b], ((nx >> 1) & 1) ^ 1, abort_w)) { give_up(61); break; }
        mbar_expect_tx(&ctl->x_full[b], XT);
        tma_load_2d(sm + OFF_X + b * XT, &mapX, &ctl->x_full[b], 0, mt * 128);
        ++nx;
      }
      for (int kk = 0; kk < nkc && ok; ++kk) {
        const int kc = kk + rot < nkc ? kk + rot : kk + rot - nkc;
        {
          const int b = (int)(nh % NHB);
          if (!mbar_wait(&ctl->h_empty[b], ((nh / NHB) & 1) ^ 1, abort_w)) { give_up(62); ok = false; break; }
          unsigned char* hb = sm + OFF_H + b * HT;
          mbar_expect_tx(&ctl->h_full[b], HT);
          tma_load_2d(hb, &mapH, &ctl->h_full[b], kc * 64, mt * 128);
          tma_load_2d(hb + HT / 2, &mapH, &ctl->h_full[b], kc * 64 + 32, mt * 128);
          ++nh;
        }
        for (int jp = 0; jp < np2; ++jp) {
          const int b = (int)(nc % NCS);
          if (!mbar_wait(&ctl->c_empty[b], ((nc / NCS) & 1) ^ 1, abort_w)) { give_up(63); ok = false; break; }
          unsigned char* cb = sm + OFF_C + b * CST;
          mbar_expect_tx(&ctl->c_full[b], NR * 128);
          const int y0 = (kc * np2 + jp) * 512;
          // exact A: [A hi | B hi] then B lo (global rows 384-511) as the third part
#pragma unroll
          for (int r = 0; r < NR; r += 128)
            tma_load_2d(cb + r * 128, &mapC, &ctl->c_full[b], 0, y0 + (AEXACT && r == 256 ? 384 : r));
          ++nc;
        }
      }
    }
    // let the last load into every buffer land before the CTA can exit
    auto drain = [&](uint64_t* full, int K, uint32_t n) {
      for (int i = 0; i < K; ++i)
        if (n > (uint32_t)i) mbar_wait_drain(&full[i], ((n - i + K - 1) / K - 1) & 1);
    };
    drain(ctl->x_full, 2, nx);
    drain(ctl->h_full, NHB, nh);
    drain(ctl->c_full, NCS, nc);
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer
    constexpr uint32_t idesc = idesc_bf16_f32(128, 128), idesc256 = idesc_bf16_f32(128, 256);
    uint32_t nx = 0, nc = 0;
    bool ok = true;
    for (int mt = blockIdx.x; mt < n_mt && ok && !*abort_w; mt += gridDim.x) {
      const int bx = nx & 1;
      if (!mbar_wait(&ctl->x_full[bx], (nx >> 1) & 1, abort_w)) { give_up(64); break; }
      const uint32_t xa = smem_u32(sm + OFF_X + bx * XT);
      const int units = nkc * np2;
      for (int un = 0; un < units && ok; ++un) {
        const int cs = (int)(nc % NCS), b = nc & 1;
        if (!mbar_wait(&ctl->c_full[cs], (nc / NCS) & 1, abort_w) ||
            !mbar_wait(&ctl->s_empty[b], ((nc >> 1) & 1) ^ 1, abort_w)) { give_up(65); ok = false; break; }
        tc_fence_after();
        const uint32_t cb = smem_u32(sm + OFF_C + cs * CST);
        const uint32_t ta = tmem + 256 * b, tb = ta + 128;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const uint64_t ad = sdesc_sw128(xa + k * 32);
          // rows [A hi | B hi] are contiguous: one N = 256 product fills both accumulators;
          // then B lo alone (exact A) or [A lo | B lo] (general A)
          umma_bf16(ta, ad, sdesc_sw128(cb + k * 32), idesc256, k > 0 ? 1u : 0u);
          if (AEXACT)
            umma_bf16(tb, ad, sdesc_sw128(cb + 2 * 16384 + k * 32), idesc, 1u);
          else
            umma_bf16(ta, ad, sdesc_sw128(cb + 2 * 16384 + k * 32), idesc256, 1u);
        }
        umma_commit(&ctl->c_empty[cs]);
        umma_commit(&ctl->s_full[b]);
        ++nc;
      }
      umma_commit(&ctl->x_empty[bx]);
      ++nx;
    }
    umma_commit(&ctl->drain);
    mbar_wait_drain(&ctl->drain, 0);
  } else if (warp >= 4 && AEXACT) {
    // ---------------- epilogue, exact first operand: row r = TMEM lane, class box `box` (32
    // classes) of every chunk for both probes of each pair.  The box's h stays in registers
    // for all the chunk's pairs.  Per row the box sums are split, q = sum_j (sab_j - sa_j sb_j)
    // with sa_j = sa0_j + sa1_j (likewise sb): box 1 adds sum_j (sab1_j - sa1_j sb1_j) to g and
    // hands sa1, sb1 over in shared memory (the part of each coefficient buffer past its 384
    // rows, never written in this form); box 0 adds the rest.
    const int quad = warp & 3, box = (warp - 4) >> 2;
    const int r = quad * 32 + lane;
    const uint32_t lanes = (uint32_t)(quad * 32) << 16;
    uint32_t nh = 0, nc = 0, nq = 0;
    bool ok = true;
    for (int mt = blockIdx.x; mt < n_mt && ok && !*abort_w; mt += gridDim.x) {
      float sab = 0.0f, sa[2 * NP2MAX], sb[2 * NP2MAX];
#pragma unroll
      for (int j = 0; j < 2 * NP2MAX; ++j) sa[j] = sb[j] = 0.0f;
      for (int kk = 0; kk < nkc && ok; ++kk) {
        const int hb = (int)(nh % NHB);
        if (!mbar_wait(&ctl->h_full[hb], (nh / NHB) & 1, abort_w)) {
          give_up(66);
          ok = false;
          break;
        }
        uint64_t h2[16];
        {
          const unsigned char* hrow = sm + OFF_H + hb * HT + box * (HT / 2) + r * 128;
#pragma unroll
          for (int ch = 0; ch < 8; ++ch) {
            const ulonglong2 h4 = *reinterpret_cast<const ulonglong2*>(hrow + ((ch ^ (r & 7)) << 4));
            h2[2 * ch] = h4.x;
            h2[2 * ch + 1] = h4.y;
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&ctl->h_empty[hb]);
        ++nh;
#pragma unroll
        for (int jp = 0; jp < NP2MAX; ++jp) {
          if (jp < np2 && ok) {
            const int b = nc & 1;
            if (!mbar_wait(&ctl->s_full[b], (nc >> 1) & 1, abort_w)) {
              give_up(67);
              ok = false;
            } else {
              ++nc;
              tc_fence_after();
              const uint32_t ta = tmem + lanes + 256 * b + 32 * box, tb = ta + 128;
              uint32_t ra[32], rb[32];
              tmem_ld32_async(ta, ra);
              tmem_ld32_async(tb, rb);
              tmem_wait_ld();
              qf_box_reg(ra, rb, h2, sab, sa[2 * jp], sb[2 * jp]);
              tmem_ld32_async(ta + 64, ra);
              tmem_ld32_async(tb + 64, rb);
              tmem_wait_ld();
              tc_fence_before();
              __syncwarp();
              if (lane == 0) mbar_arrive(&ctl->s_empty[b]);
              qf_box_reg(ra, rb, h2, sab, sa[2 * jp + 1], sb[2 * jp + 1]);
            }
          }
        }
      }
      if (!ok) break;
      float* xq = reinterpret_cast<float*>(sm + Lc::OFF_Q);
      float q = sab;
      if (box == 1) {
        if (!mbar_wait(&ctl->q_empty, (nq & 1) ^ 1, abort_w)) {
          give_up(68);
          break;
        }
#pragma unroll
        for (int j = 0; j < 2 * NP2MAX; ++j) {
          xq[j * 128 + r] = sa[j];
          xq[(2 * NP2MAX + j) * 128 + r] = sb[j];
          q -= sa[j] * sb[j];
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&ctl->q_full);
      } else {
        if (!mbar_wait(&ctl->q_full, nq & 1, abort_w)) {
          give_up(69);
          break;
        }
#pragma unroll
        for (int j = 0; j < 2 * NP2MAX; ++j) {
          const float a1 = xq[j * 128 + r], b1 = xq[(2 * NP2MAX + j) * 128 + r];
          q -= sa[j] * (sb[j] + b1) + a1 * sb[j];
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&ctl->q_empty);
      }
      ++nq;
      const int64_t row = (int64_t)mt * 128 + r;
      if (row >= m && row < N) atomicAdd(g + (row - m), -gscale * q);
    }
  } else if (warp >= 4) {
    // ---------------- epilogue: row r = TMEM lane, probe 2 jp + half of every pair
    const int quad = warp & 3, half = (warp - 4) >> 2;
    const int r = quad * 32 + lane;
    const uint32_t lanes = (uint32_t)(quad * 32) << 16;
    uint32_t nh = 0, nc = 0;
    bool ok = true;
    for (int mt = blockIdx.x; mt < n_mt && ok && !*abort_w; mt += gridDim.x) {
      float sum[NP2MAX][3];
#pragma unroll
      for (int jp = 0; jp < NP2MAX; ++jp) sum[jp][0] = sum[jp][1] = sum[jp][2] = 0.0f;
      for (int kk = 0; kk < nkc && ok; ++kk) {
        const int hb = (int)(nh % NHB);
        if (!mbar_wait(&ctl->h_full[hb], (nh / NHB) & 1, abort_w)) {
          give_up(66);
          ok = false;
          break;
        }
        const unsigned char* hrow = sm + OFF_H + hb * HT + r * 128;
#pragma unroll
        for (int jp = 0; jp < NP2MAX; ++jp) {
          if (jp < np2 && ok) {
            const int b = nc & 1;
            if (!mbar_wait(&ctl->s_full[b], (nc >> 1) & 1, abort_w)) {
              give_up(67);
              ok = false;
            } else {
              ++nc;
              tc_fence_after();
              const uint32_t ta = tmem + lanes + 256 * b + 64 * half, tb = ta + 128;
#pragma unroll
              for (int box = 0; box < 2; ++box) {
                uint32_t ra[32], rb[32];
                tmem_ld32_async(ta + box * 32, ra);
                tmem_ld32_async(tb + box * 32, rb);
                tmem_wait_ld();
                qf_box(ra, rb, hrow + box * (HT / 2), r, sum[jp][0], sum[jp][1], sum[jp][2]);
              }
              tc_fence_before();
              __syncwarp();
              if (lane == 0) mbar_arrive(&ctl->s_empty[b]);
            }
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&ctl->h_empty[hb]);
        ++nh;
      }
      if (!ok) break;
      float q = 0.0f;
#pragma unroll
      for (int jp = 0; jp < NP2MAX; ++jp)
        if (jp < np2) q += sum[jp][0] - sum[jp][1] * sum[jp][2];
      const int64_t row = (int64_t)mt * 128 + r;
      if (row >= m && row < N) atomicAdd(g + (row - m), -gscale * q);
    }
  }
  __syncthreads();
  if (warp == 2) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// Coefficient blocks of k_tc_qf, block (kc, jp) = 512 rows of 64 bf16 features:
//   rows [0, 128) A hi | [128, 256) B hi | [256, 384) A lo | [384, 512) B lo; in each part rows
//   0-63 are probe 2 jp, 64-127 probe 2 jp + 1, class kc 64 + (row mod 64).
// A~ = A minus its class mean (amean; A as is when amean is null), B~ likewise; zero for classes
// >= c, probes >= s and features >= d.
__global__ void k_build_qcoef(bf16* Cf, const float* A, const float* B, const float* amean,
                              const float* bmean, int s, int c, int d, int64_t D, int np2) {
  const int blk = blockIdx.x;
  const int kc = blk / np2, jp = blk - kc * np2;
  for (int idx = threadIdx.x; idx < 512 * 64; idx += blockDim.x) {
    const int row = idx >> 6, e = idx & 63;
    const int part = row >> 7, rr = row & 127;
    const int j = 2 * jp + (rr >> 6), k = kc * 64 + (rr & 63);
    const bool isb = part == 1 || part == 3;
    float v = 0.0f;
    if (j < s && k < c && e < d) {
      const float* src = isb ? B : A;
      const float* mn = isb ? bmean : amean;
      v = src[(int64_t)j * D + (int64_t)k * d + e] - (mn ? mn[j * d + e] : 0.0f);
    }
    const bf16 hi = __float2bfloat16_rn(v);
    Cf[((int64_t)blk * 512 + row) * 64 + e] =
        (part == 2 || part == 3) ? __float2bfloat16_rn(v - __bfloat162float(hi)) : hi;
  }
}

// q via k_tc_qf (d <= 64, not pooled, c a multiple of 4, s <= 16).  aexact: A is the problem's
// probe block (entries +-1, exact in bf16).
static int32_t tc_quad_qf(firal_problem* P, const float* A, const float* B, int s, double scale,
                          float* g, bool aexact) {
  using namespace qf_cfg;
  cudaStream_t st = P->H->stream;
  const int c = P->c, d = P->d;
  const int64_t Np = P->Np;
  const int nkc = P->cp / 64, np2 = (s + 1) / 2;
  FIRAL_TRY(P->vmean.ensure((size_t)2 * s * d * sizeof(float)));
  float* meanA = P->vmean.as<float>();
  float* meanB = meanA + (size_t)s * d;
  const int64_t crow = (int64_t)nkc * np2 * 512;
  FIRAL_TRY(P->gq_m.ensure((size_t)crow * 64 * 2));
  ProfScope ps(st, PF_QUAD);
  count_launch(aexact ? 3 : 4);
  if (!aexact) FIRAL_TRY(class_mean(P, A, s, meanA, st));
  FIRAL_TRY(class_mean(P, B, s, meanB, st));
  k_build_qcoef<<<(unsigned)(nkc * np2), 256, 0, st>>>(P->gq_m.as<bf16>(), A, B,
                                                      aexact ? nullptr : meanA, meanB, s, c, d,
                                                      P->D, np2);
  FIRAL_CUDA_TRY(cudaGetLastError());
  static bool attr[2] = {false, false};
  if (!attr[aexact]) {
    if (aexact)
      FIRAL_CUDA_TRY(cudaFuncSetAttribute(k_tc_qf<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          L<true>::SMEM));
    else
      FIRAL_CUDA_TRY(cudaFuncSetAttribute(k_tc_qf<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          L<false>::SMEM));
    attr[aexact] = true;
  }
  CUtensorMap mX, mC, mH;
  FIRAL_TRY(make_map(&mX, P->Xb.p, Np, 64, 128, 64, true));
  FIRAL_TRY(make_map(&mC, P->gq_m.p, crow, 64, 128, 64, true));
  FIRAL_TRY(make_map_f32(&mH, P->Ha.p, P->N, c, 128));
  FIRAL_CUDA_TRY(cudaMemsetAsync(g, 0, (size_t)P->n * sizeof(float), st));
  const int n_mt = (int)(Np / 128);
  const int grid = std::min(n_mt, P->sms);
  if (aexact)
    k_tc_qf<true><<<grid, 384, L<true>::SMEM, st>>>(mX, mC, mH, g, P->N, P->m, n_mt, nkc, np2,
                                           (float)(scale / s), tc_error_word(P));
  else
    k_tc_qf<false><<<grid, 384, L<false>::SMEM, st>>>(mX, mC, mH, g, P->N, P->m, n_mt, nkc, np2,
                                            (float)(scale / s), tc_error_word(P));
  FIRAL_CUDA_TRY(cudaGetLastError());
  return FIRAL_OK;
}

template <int DP>
static int32_t tc_quad_t(firal_problem* P, const float* A, const float* B, int s, double scale,
                         float* g) {
  using namespace alpha_cfg;
  cudaStream_t st = P->H->stream;
  const int64_t Np = P->Np;
  const int cp = P->cp, c = P->c, d = P->d;
  const int64_t D = P->D;
  const int sms = P->sms;
  // d <= 64, many classes, s <= 16: probe pairs per MMA (k_tc_qf); the MD step's first
  // operand is the probe block itself, exact in bf16
  if (DP == 64 && !P->pt.Q && (c % 4) == 0 && s <= qf_cfg::NP2MAX * 2)
    return tc_quad_qf(P, A, B, s, scale, g, A == P->V.as<float>());
  // probe block [A; B] (2s columns) and its class means
  FIRAL_TRY(P->gq_ab.ensure((size_t)2 * s * D * sizeof(float)));
  float* AB = P->gq_ab.as<float>();
  FIRAL_CUDA_TRY(cudaMemcpyAsync(AB, A, (size_t)s * D * 4, cudaMemcpyDeviceToDevice, st));
  FIRAL_CUDA_TRY(cudaMemcpyAsync(AB + (size_t)s * D, B, (size_t)s * D * 4,
                                 cudaMemcpyDeviceToDevice, st));
  const int Qe = pool_count(P->pt);
  FIRAL_TRY(P->vmean.ensure((size_t)2 * s * Qe * d * sizeof(float)));
  ProfScope ps(st, PF_QUAD);
  count_launch(1);
  FIRAL_TRY(class_mean(P, AB, 2 * s, P->vmean.as<float>(), st));
  if (DP >= 64 && !P->pt.Q && (c % 4) == 0) {
    // a_ijk = x_i.A_j[:,k], b_ijk = x_i.B_j[:,k] on tensor cores (K = features, x exact in
    // bf16, A and B as hi + lo); the epilogue forms sum_k h a b - (sum_k h a)(sum_k h b)
    // with the exact f32 h row and accumulates over the probes (MODE 3)
    const int nkc = cp / 64;
    const int64_t crow = (int64_t)s * nkc * 2 * 128;
    FIRAL_TRY(P->gq_m.ensure((size_t)crow * DP * 2));
    count_launch(2);
    k_build_coef<<<(unsigned)(s * nkc * 2), 256, 0, st>>>(P->gq_m.as<bf16>(), AB, AB + (size_t)s * D,
                                                         P->vmean.as<float>(), s, c, d, DP, D,
                                                         nkc, P->pt);
    FIRAL_CUDA_TRY(cudaGetLastError());
    // s <= 16: class-chunk-major order (MODE 4), each h tile loaded once per chunk
    const bool kcm = s <= S4MAX;
    static bool attr3[4] = {false, false, false, false};
    const int a3 = (DP == 64 ? 0 : 2) + (kcm ? 1 : 0);
    if (!attr3[a3]) {
      if (kcm)
        FIRAL_CUDA_TRY(cudaFuncSetAttribute(k_tc_alpha<DP, 4, 2, 0>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            SMEM4(DP)));
      else
        FIRAL_CUDA_TRY(cudaFuncSetAttribute(k_tc_alpha<DP, 3, 2, 0>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            SMEM3(DP)));
      attr3[a3] = true;
    }
    CUtensorMap mX, mC, mHf;
    FIRAL_TRY(make_map(&mX, P->Xb.p, Np, DP, BM, BK, true));
    FIRAL_TRY(make_map(&mC, P->gq_m.p, crow, DP, 128, BK, true));
    FIRAL_TRY(make_map_f32(&mHf, P->Ha.p, P->N, c, BM));
    const int n_mt = (int)(Np / BM), n_nt = s * nkc;
    if (kcm) {
      // two epilogue groups add their shares of g
      FIRAL_CUDA_TRY(cudaMemsetAsync(g, 0, (size_t)P->n * sizeof(float), st));
      k_tc_alpha<DP, 4, 2, 0><<<std::min(n_mt, sms), 384, SMEM4(DP), st>>>(
          mX, mC, mHf, P->Xb.as<bf16>(), nullptr, nullptr, g, P->N, Np, s, DP / BK, n_mt, n_nt,
          0, d, tc_error_word(P), nullptr, P->Ha.as<float>(), c, P->m, (float)(scale / s));
    } else {
      k_tc_alpha<DP, 3, 2, 0><<<std::min(n_mt, sms), 256, SMEM3(DP), st>>>(
          mX, mC, mHf, P->Xb.as<bf16>(), nullptr, nullptr, g, P->N, Np, s, DP / BK, n_mt, n_nt,
          0, d, tc_error_word(P), nullptr, P->Ha.as<float>(), c, P->m, (float)(scale / s));
    }
    FIRAL_CUDA_TRY(cudaGetLastError());
    return FIRAL_OK;
  }
  FIRAL_TRY(ensure_hlo(P));
  // term 1: M~ pairs (hi | lo per 128-pair tile) and the quadratic alpha-GEMM
  const int npairs = d * (d + 1) / 2;
  const int n_nt1 = (npairs + 127) / 128;
  const int64_t mrows = (int64_t)n_nt1 * 256;
  FIRAL_TRY(P->gq_m.ensure((size_t)mrows * cp * 2));
  FIRAL_CUDA_TRY(cudaMemsetAsync(P->gq_m.p, 0, (size_t)mrows * cp * 2, st));
  FIRAL_CUDA_TRY(cudaFuncSetAttribute(k_build_mpairs, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      128 * 128 * 4));
  count_launch(1);
  k_build_mpairs<<<c, 256, (size_t)d * d * sizeof(float), st>>>(
      P->gq_m.as<bf16>(), AB, AB + (size_t)s * D, P->vmean.as<float>(),
      P->vmean.as<float>() + (size_t)s * Qe * d, s, c, d, D, cp, npairs, P->pt);
  FIRAL_CUDA_TRY(cudaGetLastError());
  FIRAL_TRY(P->gq_part.ensure((size_t)(n_nt1 + 2 * s) * Np * sizeof(float)));
  float* part1 = P->gq_part.as<float>();
  float* a32 = part1 + (size_t)n_nt1 * Np;
  static bool attr[4] = {false, false, false, false};
  const int ai = DP == 16 ? 0 : DP == 32 ? 1 : DP == 64 ? 2 : 3;
  if (!attr[ai]) {
    FIRAL_CUDA_TRY(cudaFuncSetAttribute(k_tc_alpha<DP, 1, 2, 1>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_H));
    FIRAL_CUDA_TRY(cudaFuncSetAttribute(k_tc_alpha<DP, 2, 2, 1>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        SMEM_QUAD_H(DP)));
    attr[ai] = true;
  }
  const int n_mt = (int)(Np / BM);
  {
    CUtensorMap mH, mM, mHL;
    FIRAL_TRY(make_map(&mH, P->Hb.p, Np, cp, BM, BK, true));
    FIRAL_TRY(make_map(&mHL, P->Hlo.p, Np, cp, BM, BK, true));
    FIRAL_TRY(make_map(&mM, P->gq_m.p, mrows, cp, BN, BK, true));
    count_launch(1);
    k_tc_alpha<DP, 2, 2, 1><<<std::min(n_mt * n_nt1, sms), 256, SMEM_QUAD_H(DP), st>>>(
        mH, mM, mHL, P->Xb.as<bf16>(), nullptr, nullptr, part1, P->N, Np, 0, cp / BK, n_mt,
        n_nt1, npairs, d, tc_error_word(P), P->kr_alpha.as<int2>());
    FIRAL_CUDA_TRY(cudaGetLastError());
  }
  // term 2: h.a_ij and h.b_ij for the projected [A; B]
  {
    const int s2 = 2 * s;
    const int64_t prow = (int64_t)s2 * 2 * DP;
    const int64_t prow_p = (prow + BN - 1) / BN * BN;
    FIRAL_TRY(P->Pb.ensure((size_t)prow_p * cp * 2));
    if (prow_p > prow)
      FIRAL_CUDA_TRY(cudaMemsetAsync(P->Pb.as<bf16>() + prow * cp, 0, (prow_p - prow) * cp * 2, st));
    count_launch(1);
    k_split_probes<2><<<dim3((unsigned)(cp + 31) / 32, DP / 32 > 0 ? DP / 32 : 1, s2), dim3(32, 8), 0,
                     st>>>(P->Pb.as<bf16>(), AB, P->vmean.as<float>(), s2, c, d, DP, cp, D,
                           P->pt);
    FIRAL_CUDA_TRY(cudaGetLastError());
    CUtensorMap mH, mP, mHL;
    FIRAL_TRY(make_map(&mH, P->Hb.p, Np, cp, BM, BK, true));
    FIRAL_TRY(make_map(&mHL, P->Hlo.p, Np, cp, BM, BK, true));
    FIRAL_TRY(make_map(&mP, P->Pb.p, prow_p, cp, BN, BK, true));
    const int n_nt2 = (int)(prow_p / BN);
    count_launch(1);
    k_tc_alpha<DP, 1, 2, 1><<<std::min(n_mt * n_nt2, sms), 256, SMEM_H, st>>>(
        mH, mP, mHL, P->Xb.as<bf16>(), nullptr, nullptr, a32, P->N, Np, s2, cp / BK, n_mt,
        n_nt2, 0, d, tc_error_word(P), P->kr_alpha.as<int2>());
    FIRAL_CUDA_TRY(cudaGetLastError());
  }
  count_launch(1);
  k_quad_combine<<<(unsigned)std::min<int64_t>((P->n + 255) / 256, 4096), 256, 0, st>>>(
      part1, n_nt1, a32, s, P->m, P->N, Np, scale, g);
  FIRAL_CUDA_TRY(cudaGetLastError());
  return FIRAL_OK;
}

template <int DP>
static int32_t tc_round_scores_t(firal_problem* P, const float* M1, const float* M2,
                                 const uint8_t* mask, const double* etas, int n_chain,
                                 double* pv, int64_t* pi, int* np_out) {
  using namespace r_cfg;
  cudaStream_t st = P->H->stream;
  const int d = P->d, c = P->c;
  const int sms = P->sms;
  // 8-pair chunk table (e, first e') with e' running over [8 floor(e/8), d8)
  if (P->rtab_d != d) {
    std::vector<short2> tab;
    const int d8 = (d + 7) / 8 * 8;
    for (int e = 0; e < d; ++e)
      for (int e2 = (e / 8) * 8; e2 < d8; e2 += 8) tab.push_back(make_short2((short)e, (short)e2));
    while (tab.size() % 8) tab.push_back(make_short2(-1, 0));
    FIRAL_TRY(P->rtab.ensure(tab.size() * sizeof(short2)));
    FIRAL_CUDA_TRY(cudaMemcpyAsync(P->rtab.p, tab.data(), tab.size() * sizeof(short2),
                                   cudaMemcpyHostToDevice, st));
    FIRAL_CUDA_TRY(cudaStreamSynchronize(st));
    P->rtab_d = d;
    P->rtab_chunks = (int)tab.size();
  }
  const int kblocks = P->rtab_chunks / 8;
  const int kpad = kblocks * BK;
  const int n_kc = (c + 127) / 128;
  if (n_chain < 1 || n_chain > RC_MAX) return fail(FIRAL_ERR_ARG, "1 to 8 Round chains per launch");
  const int rows = n_chain * n_kc * BN;
  const size_t mbytes = (size_t)rows * kpad * 2;
  FIRAL_TRY(P->rM.ensure(2 * mbytes));
  bf16* Mh = P->rM.as<bf16>();
  bf16* Ml = Mh + mbytes / 2;
  ProfScope ps(st, PF_ROUND);
  count_launch(2);
  k_round_mpairs<float><<<rows, 256, 0, st>>>(Mh, Ml, M1, M2, P->rtab.as<short2>(), c, d, kpad,
                                              n_kc);
  FIRAL_CUDA_TRY(cudaGetLastError());
  CUtensorMap mX, mMh, mMl;
  FIRAL_TRY(make_map(&mX, P->Xb.p, P->Np, DP, BM, DP, false));
  FIRAL_TRY(make_map(&mMh, Mh, (uint64_t)rows, kpad, BN, BK, true));
  FIRAL_TRY(make_map(&mMl, Ml, (uint64_t)rows, kpad, BN, BK, true));
  RoundChains rc{};
  rc.n = n_chain;
  rc.mask_stride = P->n;
  for (int e = 0; e < n_chain; ++e) rc.eta[e] = etas[e];
  static bool attr[4] = {false, false, false, false};
  const int ai = DP == 16 ? 0 : DP == 32 ? 1 : DP == 64 ? 2 : 3;
  if (!attr[ai]) {
    FIRAL_CUDA_TRY(cudaFuncSetAttribute(k_tc_round<DP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        L<DP>::SMEM));
    attr[ai] = true;
  }
  const int n_mt = (int)((P->n + BM - 1) / BM);
  const int grid = std::min(n_mt, sms);
  k_tc_round<DP><<<grid, 256, L<DP>::SMEM, st>>>(mX, mMh, mMl, P->rtab.as<short2>(),
                                                  P->Ha.as<float>(), mask, P->m, P->n, c, n_kc,
                                                  kblocks, rc, pv, pi, tc_error_word(P));
  FIRAL_CUDA_TRY(cudaGetLastError());
  *np_out = grid;
  return FIRAL_OK;
}

// Scores of n_chain Round chains in one launch: chain e has eta etas[e], M1/M2 blocks at
// M1 + e c d d, mask at mask + e n, and its CTA winners at pv/pi + e * (*np_out).
int32_t tc_round_scores(firal_problem* P, const void* M1, const void* M2, const uint8_t* mask,
                        const double* etas, int n_chain, double* pv, int64_t* pi, int* np_out) {
  const float* a = (const float*)M1;
  const float* b = (const float*)M2;
  switch (P->dp) {
    case 16: return tc_round_scores_t<16>(P, a, b, mask, etas, n_chain, pv, pi, np_out);
    case 32: return tc_round_scores_t<32>(P, a, b, mask, etas, n_chain, pv, pi, np_out);
    case 64: return tc_round_scores_t<64>(P, a, b, mask, etas, n_chain, pv, pi, np_out);
    default: return tc_round_scores_t<128>(P, a, b, mask, etas, n_chain, pv, pi, np_out);
  }
}

// ------------------------------------------------------------------------------------------
// At most 32 classes per pool: the Hessian apply in the per-point form of Lemma 1, fused into
// one persistent kernel.  For the rows of one pool q (weights w_i, probabilities h_i over the
// pool's c_q classes, direction P~ with the pool's class means removed):
//   a_ikj = x_i . P~_j[:, k]                      MMA1: 128 rows x (probe, class), K = features
//   alpha_ij = sum_k h_ik a_ikj,   psi_ikj = w_i h_ik (a_ikj - alpha_ij)     f32, CUDA cores
//   out_j[:, k] += sum_i psi_ikj x_i              MMA2: features x (probe, class), K = rows
// P~ and psi enter as bf16 hi + lo (x is exact in bf16), so both products carry about 2^-17
// relative rounding, and nothing cancels: each psi is the row's own contribution.  Column
// (probe j, class k) is j cpad + k, cpad = the pool's class count rounded up to 8, 16 or 32,
// so one 32-column TMEM load holds whole probes; a probe group of at most 128 columns is one
// unit of work, so a pool with cpad s > 128 runs as several groups.  MMA2 takes x^T (the
// staged x^T tile, K-major, 128 rows of which the first dp are features) and psi as an
// MN-major operand, so each epilogue thread writes its row's psi values as 16-byte runs.
// Work list: segments of at most SEG_TILES 128-row tiles of one pool's rows (its labelled
// rows and its pool rows are separate segments); the host deals the segments to the CTAs
// longest first (sched: per-CTA offsets, then segment indices), and a CTA takes every probe
// group of each of its segments (an item).  A tile that also holds rows of another pool runs once per pool with
// the other rows masked.  An item accumulates out in TMEM and writes one partial; a
// per-class combine adds a pool's partials in segment order.
// Pipeline: the x and x^T tiles, the S accumulator (TMEM), the psi operand (shared memory) and
// the D accumulator are double-buffered: the TMA loads of tile t+1, MMA1 of tile t+1, the
// epilogue of tile t and MMA2 of tile t-1 overlap.  Each epilogue thread loads its row's h for
// the next tile while it works on the current one, from the class-major copy of h (one
// coalesced run of 128 rows per class).
// Roles (384 threads): warp 0 TMA producer, warp 1 MMA issuer, warp 2 TMEM owner, warps 4-11
// epilogue (warp & 3 = TMEM lane quarter, (warp - 4) >> 2 = which 32-column chunks).
// ------------------------------------------------------------------------------------------
namespace pw_cfg {
constexpr int NU = 128;                           // columns per unit (probe group)
constexpr int SEG_TILES = 8;                      // tiles per segment: 128 adds per accumulator
constexpr int PT_HALF = NU * 128;                 // P~ hi (then lo) of one group: 16 KB
constexpr int XA_BYTES = 128 * 128;               // x tile: 128 rows x 64 features
constexpr int XT_BYTES = 2 * 64 * 128;            // x^T tile: 2 K-blocks x (<= 64 features)
constexpr int PSI_ATOM = 128 * 128;               // psi: 128 rows x 64 columns (one MN atom)
constexpr int PSI_BUF = 4 * PSI_ATOM;             // hi | lo, 2 MN atoms each: 64 KB
constexpr int OFF_PT = 0, OFF_XA = 2 * PT_HALF, OFF_XT = OFF_XA + 2 * XA_BYTES;
constexpr int OFF_PSI = OFF_XT + 2 * XT_BYTES, OFF_CTL = OFF_PSI + 2 * PSI_BUF;
constexpr int SMEM = OFF_CTL + 256 + 1024;
constexpr uint32_t TS = 0, TD = 256;              // TMEM columns: S (2 x 128) | D (2 x 128)
}  // namespace pw_cfg

struct PwCtl {   // < 256 bytes
  uint64_t x_full[2], x_empty[2], xt_full[2], xt_empty[2], s_full[2], s_empty[2], psi_full[2],
      psi_empty[2], d_full[2], d_empty[2], pt_full, pt_empty, drain;
  uint32_t tmem_base;
  int abort_w;
};
static_assert(sizeof(PwCtl) <= 256, "control block must fit in 256 bytes");

// Probe groups of a pool (cpad, sp): ceil(cpad sp / 128); columns of group grp.
__device__ __forceinline__ int pw_ngrp(int cpad, int sp) {
  return (cpad * sp + pw_cfg::NU - 1) / pw_cfg::NU;
}
__device__ __forceinline__ int pw_ncols(int cpad, int sp, int grp) {
  const int r = cpad * sp - grp * pw_cfg::NU;
  return r < pw_cfg::NU ? r : pw_cfg::NU;
}

// psi for one 32-column chunk (32 / CPAD whole probes) of the thread's row, written as bf16
// hi and lo into the row's four 16-byte chunks cb .. cb + 3 of the MN-major psi operand
// (swizzled: chunk u of row i at (u ^ (i mod 8)) 16 bytes).  wh2 = w h of classes (2m, 2m+1)
// as packed pairs (zero on masked rows and padding classes); alpha = (sum_k wh_k a_k) / w.
// The f32 arithmetic runs on packed pairs (f32x2), each lane rounded as the scalar form.
template <int CPAD>
__device__ __forceinline__ void pw_psi_chunk(const uint32_t (&ra)[32],
                                             const uint64_t (&wh2)[CPAD / 2], float winv,
                                             unsigned char* hi, unsigned char* lo, int cb,
                                             int sw) {
  const uint64_t m1 = f2_pack(-1.0f, -1.0f);
  uint32_t ph[16], pl[16];
#pragma unroll
  for (int pg = 0; pg < 32 / CPAD; ++pg) {
    uint64_t acc = 0;
#pragma unroll
    for (int k = 0; k < CPAD; k += 2)
      acc = f2_fma(wh2[k / 2], f2_pack_u(ra[pg * CPAD + k], ra[pg * CPAD + k + 1]), acc);
    float x0, x1;
    f2_unpack(acc, x0, x1);
    const float al = (x0 + x1) * winv;
    const uint64_t nal = f2_pack(-al, -al);
#pragma unroll
    for (int k = 0; k < CPAD; k += 2) {
      const int t = pg * CPAD + k;
      const uint64_t p2 = f2_mul(wh2[k / 2], f2_add(f2_pack_u(ra[t], ra[t + 1]), nal));
      float p0, p1;
      f2_unpack(p2, p0, p1);
      const __nv_bfloat162 h2 = __floats2bfloat162_rn(p0, p1);
      const float2 f2 = __bfloat1622float2(h2);
      float r0, r1;
      f2_unpack(f2_fma(f2_pack(f2.x, f2.y), m1, p2), r0, r1);   // p - bf16(p), per lane
      const __nv_bfloat162 l2 = __floats2bfloat162_rn(r0, r1);
      ph[t >> 1] = *reinterpret_cast<const uint32_t*>(&h2);
      pl[t >> 1] = *reinterpret_cast<const uint32_t*>(&l2);
    }
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int o = ((cb + u) ^ sw) << 4;
    *reinterpret_cast<uint4*>(hi + o) = make_uint4(ph[4 * u], ph[4 * u + 1], ph[4 * u + 2], ph[4 * u + 3]);
    *reinterpret_cast<uint4*>(lo + o) = make_uint4(pl[4 * u], pl[4 * u + 1], pl[4 * u + 2], pl[4 * u + 3]);
  }
}

// loads of the thread's row for a tile: h over the pool's CPAD padded classes from the
// class-major copy HaT (N rows per class; zero beyond c_q and on masked rows) and w
template <int CPAD>
__device__ __forceinline__ void pw_load_row_c(float (&hn)[CPAD], float& wn, const float* HaT,
                                              const float* w, int64_t row, bool valid, int64_t N,
                                              int coff, int cq) {
  const float* q = HaT + (int64_t)coff * N + row;   // class coff + k at q + k N
  const int kmax = valid ? cq : 0;
#pragma unroll
  for (int k = 0; k < CPAD; ++k) {
    hn[k] = k < kmax ? *q : 0.0f;
    q += N;
  }
  wn = valid ? w[row] : 0.0f;
}

// the same for 32 classes (the gradient kernel)
__device__ __forceinline__ void pw_load_row(float (&hn)[32], float& wn, const float* HaT,
                                            const float* w, int64_t row, bool valid, int64_t N,
                                            int coff, int cq) {
  const float* q = HaT + (int64_t)coff * N + row;   // class coff + k at q + k N
  const int kmax = valid ? cq : 0;
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    hn[k] = k < kmax ? *q : 0.0f;
    q += N;
  }
  wn = valid ? w[row] : 0.0f;
}

// Epilogue context of the fused apply kernel (one thread: row i of the tile = TMEM lane,
// half = which 32-column chunks it takes)
struct PwEpi {
  PwCtl* ctl;
  unsigned char* sm;
  uint32_t tmem, lanes;
  int i, half, lane;
  volatile int* abort_w;
  int32_t* err;
  const float* HaT;
  const float* w;
  float* part;
  int64_t N;
  int s, sp, d;
};

// One work item (segment sg of pool pq, probe group grp of nc columns) of the epilogue, with
// the pool's classes padded to CPAD: per tile, psi into the MN-major operand; at the end, the
// item's partial rows from the D accumulator.  u counts the units seen; false when a wait gave
// up (the abort word and the error word are set).
template <int CPAD, int DP>
__device__ __forceinline__ bool pw_epi_item(const PwEpi& E, uint32_t& u, uint32_t item,
                                            const int4& sg, const int4& pq, int grp, int nc) {
  using namespace pw_cfg;
  const int i = E.i, lane = E.lane, cq = pq.y;
  const int t0 = sg.y >> 7, t1 = (sg.z - 1) >> 7;
  auto give_up = [&](int code) {
    E.ctl->abort_w = 1;
    atomicExch(E.err, code);
  };
  float hn[CPAD], wn;
  {
    const int64_t row = (int64_t)t0 * 128 + i;
    pw_load_row_c<CPAD>(hn, wn, E.HaT, E.w, row, row >= sg.y && row < sg.z, E.N, pq.x, cq);
  }
  for (int t = t0; t <= t1; ++t) {
    uint64_t wh2[CPAD / 2];
    const uint64_t w2 = f2_pack(wn, wn);
#pragma unroll
    for (int k = 0; k < CPAD; k += 2) wh2[k / 2] = f2_mul(w2, f2_pack(hn[k], hn[k + 1]));
    const float winv = wn != 0.0f ? 1.0f / wn : 0.0f;
    if (t < t1) {   // the next tile's row, while this one is worked on
      const int64_t rn = (int64_t)(t + 1) * 128 + i;
      pw_load_row_c<CPAD>(hn, wn, E.HaT, E.w, rn, rn >= sg.y && rn < sg.z, E.N, pq.x, cq);
    }
    const int b = u & 1;
    const uint32_t ph = (u >> 1) & 1;
    if (!mbar_wait(&E.ctl->s_full[b], ph, E.abort_w) ||
        !mbar_wait(&E.ctl->psi_empty[b], ph ^ 1, E.abort_w)) {
      give_up(47);
      return false;
    }
    ++u;
    tc_fence_after();
    unsigned char* psi_row = E.sm + OFF_PSI + b * PSI_BUF + i * 128;
    for (int ch = E.half; ch < nc / 32; ch += 2) {
      uint32_t ra[32];
      tmem_ld32_async(E.tmem + E.lanes + TS + b * NU + ch * 32, ra);
      tmem_wait_ld();
      unsigned char* hi = psi_row + (ch >> 1) * PSI_ATOM;   // 64-column atom of the chunk
      pw_psi_chunk<CPAD>(ra, wh2, winv, hi, hi + 2 * PSI_ATOM, (ch & 1) * 4, i & 7);
    }
    tc_fence_before();
    fence_async_smem();
    __syncwarp();
    if (lane == 0) {
      mbar_arrive(&E.ctl->s_empty[b]);
      mbar_arrive(&E.ctl->psi_full[b]);
    }
  }
  // item end: D -> the item's partial rows, [class][probe][feature]; the thread holds feature
  // e (its TMEM lane) of the columns of its half
  const int db = item & 1;
  if (!mbar_wait(&E.ctl->d_full[db], (item >> 1) & 1, E.abort_w)) {
    give_up(48);
    return false;
  }
  tc_fence_after();
  {
    constexpr int LC = CPAD == 8 ? 3 : CPAD == 16 ? 4 : 5;
    const int e = i;
    for (int c0 = E.half * 64; c0 < E.half * 64 + 64; c0 += 32) {
      if (c0 >= nc) break;
      uint32_t v[32];
      tmem_ld32_async(E.tmem + E.lanes + TD + db * NU + c0, v);
      tmem_wait_ld();
      if (e < E.d) {
#pragma unroll
        for (int t = 0; t < 32; ++t) {
          const int col = c0 + t, jl = col >> LC, kl = col - (jl << LC);
          const int j = grp * (NU >> LC) + jl;
          if (kl < cq && j < E.s)
            E.part[((int64_t)(sg.w + kl) * E.sp + j) * E.d + e] = __uint_as_float(v[t]);
        }
      }
    }
  }
  tc_fence_before();
  __syncwarp();
  if (lane == 0) mbar_arrive(&E.ctl->d_empty[db]);
  return true;
}

template <int DP>
__global__ void __launch_bounds__(384, 1)
    k_tc_pw(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapXT,
            const __grid_constant__ CUtensorMap mapPT, const float* __restrict__ HaT,
            const float* __restrict__ w, float* __restrict__ part,
            const int4* __restrict__ pool_tab, const int4* __restrict__ seg_tab,
            const int* __restrict__ sched, int64_t N, int s, int sp, int d, int32_t* err) {
  using namespace pw_cfg;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  PwCtl* ctl = (PwCtl*)(sm + OFF_CTL);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int b = 0; b < 2; ++b) {
      mbar_init(&ctl->x_full[b], 1);
      mbar_init(&ctl->x_empty[b], 1);
      mbar_init(&ctl->xt_full[b], 1);
      mbar_init(&ctl->xt_empty[b], 1);
      mbar_init(&ctl->s_full[b], 1);
      mbar_init(&ctl->s_empty[b], 8);
      mbar_init(&ctl->psi_full[b], 8);
      mbar_init(&ctl->psi_empty[b], 1);
      mbar_init(&ctl->d_full[b], 1);
      mbar_init(&ctl->d_empty[b], 8);
    }
    mbar_init(&ctl->pt_full, 1);
    mbar_init(&ctl->pt_empty, 1);
    mbar_init(&ctl->drain, 1);
    ctl->abort_w = 0;
    mbar_fence_init();
  }
  if (warp == 2) {
    tmem_alloc(&ctl->tmem_base, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = ctl->tmem_base;
  volatile int* abort_w = &ctl->abort_w;
  auto give_up = [&](int code) {
    ctl->abort_w = 1;
    atomicExch(err, code);
  };

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer: P~ of each item, x and x^T of each of its tiles
    tma_prefetch(&mapX);
    tma_prefetch(&mapXT);
    tma_prefetch(&mapPT);
    uint32_t nt = 0, ni = 0;   // tiles and items loaded
    bool ok = true;
    for (int it = sched[blockIdx.x]; it < sched[blockIdx.x + 1] && ok && !*abort_w; ++it) {
      const int4 sg = seg_tab[sched[gridDim.x + 1 + it]];
      const int4 pq = pool_tab[sg.x];
      const int n1 = pq.z * sp, pbase = 2 * sp * pq.w;
      const int ng = pw_ngrp(pq.z, sp);
      for (int grp = 0; grp < ng && ok; ++grp) {
        const int nc = pw_ncols(pq.z, sp, grp);
        if (!mbar_wait(&ctl->pt_empty, (ni & 1) ^ 1, abort_w)) { give_up(41); ok = false; break; }
        mbar_expect_tx(&ctl->pt_full, 2 * nc * 128);
        for (int part = 0; part < 2; ++part)
          for (int r = 0; r < nc; r += 64)
            tma_load_2d(sm + OFF_PT + part * PT_HALF + r * 128, &mapPT, &ctl->pt_full, 0,
                        pbase + part * n1 + grp * NU + r);
        ++ni;
        for (int t = sg.y >> 7; t <= (sg.z - 1) >> 7; ++t) {
          const int b = nt & 1;
          const uint32_t ph = (nt >> 1) & 1;
          // both buffers free before either load is issued: a wait that gives up leaves no
          // load of this tile in flight
          if (!mbar_wait(&ctl->x_empty[b], ph ^ 1, abort_w) ||
              !mbar_wait(&ctl->xt_empty[b], ph ^ 1, abort_w)) {
            give_up(42);
            ok = false;
            break;
          }
          mbar_expect_tx(&ctl->x_full[b], XA_BYTES);
          tma_load_2d(sm + OFF_XA + b * XA_BYTES, &mapX, &ctl->x_full[b], 0, t * 128);
          mbar_expect_tx(&ctl->xt_full[b], 2 * DP * 128);
          unsigned char* xt = sm + OFF_XT + b * XT_BYTES;
          tma_load_2d(xt, &mapXT, &ctl->xt_full[b], 0, (2 * t) * DP);
          tma_load_2d(xt + DP * 128, &mapXT, &ctl->xt_full[b], 0, (2 * t + 1) * DP);
          ++nt;
        }
      }
    }
    // every issued load lands before the CTA can exit (buffer b took loads nt = b, b + 2, ...)
    for (int b = 0; b < 2; ++b) {
      const uint32_t cnt = (nt + 1 - b) / 2;
      if (cnt) {
        mbar_wait_drain(&ctl->x_full[b], (cnt - 1) & 1);
        mbar_wait_drain(&ctl->xt_full[b], (cnt - 1) & 1);
      }
    }
    if (ni) mbar_wait_drain(&ctl->pt_full, (ni - 1) & 1);
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer: MMA1 of unit u, then MMA2 of unit u - 1
    struct Pend {
      uint32_t u, item;
      bool first, last;
      int nc;
    };
    Pend pend{0, 0, false, false, 0};
    bool have = false;
    uint32_t nt = 0, ni = 0;
    bool ok = true;
    auto mma2 = [&](const Pend& p) -> bool {
      const int b = p.u & 1, db = p.item & 1;
      const uint32_t ph = (p.u >> 1) & 1;
      if (!mbar_wait(&ctl->psi_full[b], ph, abort_w) || !mbar_wait(&ctl->xt_full[b], ph, abort_w) ||
          (p.first && !mbar_wait(&ctl->d_empty[db], ((p.item >> 1) & 1) ^ 1, abort_w)))
        return false;
      tc_fence_after();
      // D (lanes = features, columns = the unit's (probe, class) columns) += x^T psi:
      // A = the x^T tile (K-major; rows past dp are not features and their D rows are unused),
      // B = psi (MN-major: rows = the tile's rows, 64-column atoms 16 KB apart)
      const uint32_t ps = smem_u32(sm + OFF_PSI + b * PSI_BUF),
                     xt = smem_u32(sm + OFF_XT + b * XT_BYTES);
      const uint32_t idesc2 = idesc_bf16_f32_bmn(128, p.nc);
#pragma unroll
      for (int kb = 0; kb < 2; ++kb)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const uint64_t ad = sdesc_sw128(xt + kb * DP * 128 + k * 32);
          const uint32_t b0 = ps + (kb * 64 + k * 16) * 128;
          const uint32_t acc = (p.first && kb == 0 && k == 0) ? 0u : 1u;
          umma_bf16(tmem + TD + db * NU, ad, sdesc_sw128_mn(b0, PSI_ATOM), idesc2, acc);
          umma_bf16(tmem + TD + db * NU, ad, sdesc_sw128_mn(b0 + 2 * PSI_ATOM, PSI_ATOM), idesc2,
                    1u);
        }
      umma_commit(&ctl->psi_empty[b]);
      umma_commit(&ctl->xt_empty[b]);
      if (p.last) umma_commit(&ctl->d_full[db]);
      return true;
    };
    for (int it = sched[blockIdx.x]; it < sched[blockIdx.x + 1] && ok && !*abort_w; ++it) {
      const int4 sg = seg_tab[sched[gridDim.x + 1 + it]];
      const int4 pq = pool_tab[sg.x];
      const int ng = pw_ngrp(pq.z, sp);
      const int t0 = sg.y >> 7, t1 = (sg.z - 1) >> 7;
      for (int grp = 0; grp < ng && ok; ++grp) {
        const uint32_t idesc1 = idesc_bf16_f32(128, pw_ncols(pq.z, sp, grp));
        if (!mbar_wait(&ctl->pt_full, ni & 1, abort_w)) { give_up(44); ok = false; break; }
        const uint32_t item = ni++;
        for (int t = t0; t <= t1; ++t) {
          const uint32_t u = nt;
          const int b = u & 1;
          const uint32_t ph = (u >> 1) & 1;
          if (!mbar_wait(&ctl->x_full[b], ph, abort_w) ||
              !mbar_wait(&ctl->s_empty[b], ph ^ 1, abort_w)) { give_up(45); ok = false; break; }
          tc_fence_after();
          const uint32_t xa = smem_u32(sm + OFF_XA + b * XA_BYTES), pt = smem_u32(sm + OFF_PT);
#pragma unroll
          for (int k = 0; k < DP / 16; ++k) {
            const uint64_t ad = sdesc_sw128(xa + k * 32);
            umma_bf16(tmem + TS + b * NU, ad, sdesc_sw128(pt + k * 32), idesc1, k > 0 ? 1u : 0u);
            umma_bf16(tmem + TS + b * NU, ad, sdesc_sw128(pt + PT_HALF + k * 32), idesc1, 1u);
          }
          umma_commit(&ctl->s_full[b]);
          umma_commit(&ctl->x_empty[b]);
          if (t == t1) umma_commit(&ctl->pt_empty);
          ++nt;
          if (have && !mma2(pend)) { give_up(46); ok = false; break; }
          pend = Pend{u, item, t == t0, t == t1, pw_ncols(pq.z, sp, grp)};
          have = true;
        }
      }
    }
    if (ok && have && !*abort_w && !mma2(pend)) give_up(46);
    umma_commit(&ctl->drain);
    mbar_wait_drain(&ctl->drain, 0);
  } else if (warp >= 4) {
    // ---------------- epilogue
    const int quad = warp & 3;
    const PwEpi E{ctl, sm, tmem, (uint32_t)(quad * 32) << 16, quad * 32 + lane, (warp - 4) >> 2,
                  lane, abort_w, err, HaT, w, part, N, s, sp, d};
    uint32_t u = 0, ni = 0;
    bool ok = true;
    for (int it = sched[blockIdx.x]; it < sched[blockIdx.x + 1] && ok && !*abort_w; ++it) {
      const int4 sg = seg_tab[sched[gridDim.x + 1 + it]];
      const int4 pq = pool_tab[sg.x];
      const int ng = pw_ngrp(pq.z, sp);
      for (int grp = 0; grp < ng && ok; ++grp) {
        const int nc = pw_ncols(pq.z, sp, grp);
        const uint32_t item = ni++;
        if (pq.z == 8) ok = pw_epi_item<8, DP>(E, u, item, sg, pq, grp, nc);
        else if (pq.z == 16) ok = pw_epi_item<16, DP>(E, u, item, sg, pq, grp, nc);
        else ok = pw_epi_item<32, DP>(E, u, item, sg, pq, grp, nc);
      }
    }
  }
  __syncthreads();
  if (warp == 2) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

// Packed direction of the fused kernel (sp = s rounded up to 8 probes), one block per (pool q,
// probe j): the pool's class mean of V_j (over its c_q classes, in double, groups combined in
// a fixed order; written to vmean[j][q]), then rows 2 sp cpre_q + part n1_q + j cpad_q + k
// (part 0 = bf16 hi, 1 = lo of V_j[:, k] minus that mean; zero for k >= c_q and for the
// padding probes j >= s); 64 bf16 features per row, zero for e >= d.
__global__ void __launch_bounds__(256) k_pw_pack(bf16* Pk, const float* V, float* vmean,
                                                 const int4* pool_tab, int s, int sp, int d,
                                                 int64_t D, int Qe) {
  __shared__ double red[4][64];
  __shared__ float mean[64];
  const int q = blockIdx.x, j = blockIdx.y;
  const int4 pq = pool_tab[q];   // first class, classes, padded classes, padded classes before
  const int64_t n1 = (int64_t)pq.z * sp;
  const int64_t r0 = 2LL * sp * pq.w + (int64_t)j * pq.z;
  {
    const int e = threadIdx.x & 63, gr = threadIdx.x >> 6;
    double acc = 0.0;
    if (j < s && e < d)
      for (int kl = gr; kl < pq.y; kl += 4) acc += (double)V[(int64_t)j * D + (int64_t)(pq.x + kl) * d + e];
    red[gr][e] = acc;
    __syncthreads();
    if (threadIdx.x < 64) {
      const double t = ((red[0][e] + red[1][e]) + red[2][e]) + red[3][e];
      const float m = (j < s && e < d) ? (float)(t / pq.y) : 0.0f;
      mean[e] = m;
      if (j < s && e < d) vmean[(j * Qe + q) * d + e] = m;
    }
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < pq.z * 64; idx += blockDim.x) {
    const int kl = idx >> 6, e = idx & 63;
    float v = 0.0f;
    if (kl < pq.y && e < d && j < s) v = V[(int64_t)j * D + (int64_t)(pq.x + kl) * d + e] - mean[e];
    const bf16 hi = __float2bfloat16_rn(v);
    Pk[(r0 + kl) * 64 + e] = hi;
    Pk[(r0 + n1 + kl) * 64 + e] = __float2bfloat16_rn(v - __bfloat162float(hi));
  }
}

// The apply's last steps for one (pool q, probe j), in shared memory:
//   t_k = lam (V_j[:, k] - vmean) + the pool's segment partials in segment order
//   out_j[:, k] = t_k - mean_k' t_k' + lam_null vmean      (the class-mean projection)
//   pq[j c + k] = <V_j[:, k], out_j[:, k]>                 (the CG dot products)
// lam is the diagonal-part lambda (rank 0 of a row-sharded group only: such a group takes the
// separate combine / allreduce / projection path instead).
constexpr int PWF_THREADS = 512;   // eight 64-thread groups: segment partials in flight
__global__ void __launch_bounds__(PWF_THREADS) k_pw_finish(float* out, const float* V,
                                                           const float* vmean, const float* part,
                                                           const int4* pool_tab,
                                                           const int2* pseg, const int4* seg_tab,
                                                           float lam, double lam_null, int s,
                                                           int sp, int c, int d, int64_t D,
                                                           int Qe, double* pq) {
  constexpr int NG = PWF_THREADS / 64;
  __shared__ float t[32 * 64];
  __shared__ double red[NG][64];
  __shared__ float qm[64];
  const int q = blockIdx.x, j = blockIdx.y;
  const int4 pt = pool_tab[q];
  const int2 sr = pseg[q];
  const int cq = pt.y;
  const float* vm = vmean + (j * Qe + q) * d;
  for (int idx = threadIdx.x; idx < cq * d; idx += blockDim.x) {
    const int kl = idx / d, e = idx - kl * d;
    const int64_t o = (int64_t)j * D + (int64_t)(pt.x + kl) * d + e;
    float acc = lam * (V[o] - vm[e]);
    for (int g = sr.x; g < sr.y; ++g) acc += part[((int64_t)(seg_tab[g].w + kl) * sp + j) * d + e];
    t[kl * 64 + e] = acc;
  }
  __syncthreads();
  {
    const int e = threadIdx.x & 63, gr = threadIdx.x >> 6;
    double acc = 0.0;
    if (e < d)
      for (int kl = gr; kl < cq; kl += NG) acc += (double)t[kl * 64 + e];
    red[gr][e] = acc;
    __syncthreads();
    if (threadIdx.x < 64 && e < d) {
      double tot = 0.0;
      for (int g = 0; g < NG; ++g) tot += red[g][e];
      qm[e] = (float)(tot / cq);
    }
    __syncthreads();
  }
  // one warp per class: the projected block and its dot product with V_j[:, k]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int kl = warp; kl < cq; kl += (int)(blockDim.x >> 5)) {
    double dot = 0.0;
    for (int e = lane; e < d; e += 32) {
      const int64_t o = (int64_t)j * D + (int64_t)(pt.x + kl) * d + e;
      const float v = t[kl * 64 + e] - qm[e] + (float)(lam_null * (double)vm[e]);
      out[o] = v;
      dot += (double)V[o] * (double)v;
    }
    if (pq) {
      for (int o2 = 16; o2 > 0; o2 >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o2);
      if (lane == 0) pq[(int64_t)j * c + pt.x + kl] = dot;
    }
  }
}

// out_j[:, k] = lam (V_j[:, k] - pool mean) + the pool's segment partials in segment order
__global__ void k_pw_combine(float* out, const float* V, const float* vmean, const float* part,
                             const int4* pool_tab, const int2* pseg, const int4* seg_tab,
                             float lam, int s, int sp, int d, int64_t D, PoolTab pt) {
  const int k = blockIdx.x;
  const int q = pool_of(pt, k), Qe = pool_count(pt);
  const int kl = k - pool_tab[q].x;
  const int2 sr = pseg[q];
  for (int idx = threadIdx.x; idx < s * d; idx += blockDim.x) {
    const int j = idx / d, e = idx - j * d;
    const int64_t o = (int64_t)j * D + (int64_t)k * d + e;
    float acc = lam * (V[o] - vmean[(j * Qe + q) * d + e]);
    for (int g = sr.x; g < sr.y; ++g) acc += part[((int64_t)(seg_tab[g].w + kl) * sp + j) * d + e];
    out[o] = acc;
  }
}

// x padded to 64 features (the fused kernel's MMA1 operand when dp < 64)
__global__ void k_pad_x64(bf16* X64, const bf16* Xb, int64_t Np, int dp) {
  const int64_t total = Np * 64;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = idx >> 6;
    const int e = (int)(idx & 63);
    X64[idx] = e < dp ? Xb[r * dp + e] : __float2bfloat16(0.0f);
  }
}

// Work list of the fused kernel (mixed precision, dp <= 64, every pool with at most 32
// classes; a problem that is not pooled is one pool): pool table, segments of at most
// SEG_TILES tiles of each row range (labelled rows loff, pool rows M + poff), each pool's
// segment range.  Leaves the problem on the general path otherwise.
int32_t tc_setup_pw(firal_problem* P, const std::vector<int>& coff,
                    const std::vector<int64_t>& loff, const std::vector<int64_t>& poff) {
  using namespace pw_cfg;
  const int Q = (int)coff.size() - 1;
  P->pw = false;
  if (Q < 1 || P->dp > 64 || !is_mixed(P->prec)) return FIRAL_OK;
  std::vector<int4> ptab(Q);
  int cmax = 0;
  int64_t cpre = 0;
  for (int q = 0; q < Q; ++q) {
    const int cq = coff[q + 1] - coff[q];
    const int cpad = cq <= 8 ? 8 : cq <= 16 ? 16 : 32;
    if (cq > 32) return FIRAL_OK;   // more classes: the general path
    ptab[q] = make_int4(coff[q], cq, cpad, (int)cpre);
    cpre += cpad;
    cmax = std::max(cmax, cpad);
  }
  const int64_t M = loff[Q];
  std::vector<int4> segs;
  std::vector<int2> pseg(Q);
  int64_t segcls = 0;
  for (int q = 0; q < Q; ++q) {
    pseg[q].x = (int)segs.size();
    const int64_t ranges[2][2] = {{loff[q], loff[q + 1]}, {M + poff[q], M + poff[q + 1]}};
    for (const auto& rg : ranges) {
      for (int64_t a = rg[0]; a < rg[1];) {
        const int64_t tend = (a / 128 + SEG_TILES) * 128;
        const int64_t b = std::min<int64_t>(rg[1], tend);
        segs.push_back(make_int4(q, (int)a, (int)b, (int)segcls));
        segcls += ptab[q].y;
        a = b;
      }
    }
    pseg[q].y = (int)segs.size();
  }
  cudaStream_t st = P->H->stream;
  FIRAL_TRY(P->pw_pool.ensure(ptab.size() * sizeof(int4)));
  FIRAL_TRY(P->pw_seg.ensure(std::max<size_t>(1, segs.size()) * sizeof(int4)));
  FIRAL_TRY(P->pw_pseg.ensure(pseg.size() * sizeof(int2)));
  FIRAL_CUDA_TRY(cudaMemcpyAsync(P->pw_pool.p, ptab.data(), ptab.size() * sizeof(int4),
                                 cudaMemcpyHostToDevice, st));
  if (!segs.empty())
    FIRAL_CUDA_TRY(cudaMemcpyAsync(P->pw_seg.p, segs.data(), segs.size() * sizeof(int4),
                                   cudaMemcpyHostToDevice, st));
  FIRAL_CUDA_TRY(cudaMemcpyAsync(P->pw_pseg.p, pseg.data(), pseg.size() * sizeof(int2),
                                 cudaMemcpyHostToDevice, st));
  if (P->dp < 64) {
    FIRAL_TRY(P->X64.ensure((size_t)P->Np * 64 * 2));
    count_launch();
    k_pad_x64<<<(unsigned)std::min<int64_t>((P->Np * 64 + 255) / 256, 1 << 20), 256, 0, st>>>(
        P->X64.as<bf16>(), P->Xb.as<bf16>(), P->Np, P->dp);
    FIRAL_CUDA_TRY(cudaGetLastError());
  }
  // h read class-major by the fused kernels (one coalesced run of a tile's rows per class)
  FIRAL_TRY(class_major_h(P));
  // the host vectors are read by the copies
  FIRAL_CUDA_TRY(cudaStreamSynchronize(st));
  P->pw_pool_h = ptab;
  P->pw_seg_h = segs;
  for (auto& sc : P->pw_sched) sc.buf.release();
  P->pw_sched.clear();
  P->pw = true;
  P->pw_cpad_max = cmax;
  P->pw_cpad_total = cpre;
  P->pw_nseg = (int)segs.size();
  P->pw_segcls_total = segcls;
  return FIRAL_OK;
}

// The CTAs' segment lists for sp padded probes (quad: the gradient, which skips the labelled
// rows' segments): each segment costs (tiles + 1) x probe groups, and the segments go longest
// first to the least-loaded CTA (ties to the lowest index), which keeps the slowest CTA within
// a few percent of the mean where striding left it up to 2x.  Made once per (sp, quad), before
// any graph capture (the first MD step runs eagerly); each CTA walks its list in pool order.
static int32_t pw_schedule(firal_problem* P, int sp, bool quad, int* grid_out,
                           const int** sched_out) {
  for (auto& sc : P->pw_sched)
    if (sc.sp == sp && sc.quad == quad) {
      *grid_out = sc.grid;
      *sched_out = sc.buf.as<int>();
      return FIRAL_OK;
    }
  std::vector<std::pair<int64_t, int>> items;
  for (int g = 0; g < (int)P->pw_seg_h.size(); ++g) {
    const int4 sg = P->pw_seg_h[g];
    if (quad && (int64_t)sg.z <= P->m) continue;
    const int4 pq = P->pw_pool_h[sg.x];
    const int64_t ng = ((int64_t)pq.z * sp + pw_cfg::NU - 1) / pw_cfg::NU;
    const int64_t tiles = (sg.z - 1) / 128 - sg.y / 128 + 1;
    items.push_back({(tiles + 1) * ng, g});
  }
  const int grid = std::max(1, std::min<int>(P->sms, (int)items.size()));
  std::stable_sort(items.begin(), items.end(),
                   [](const std::pair<int64_t, int>& a, const std::pair<int64_t, int>& b) {
                     return a.first > b.first;
                   });
  std::vector<std::vector<int>> lists(grid);
  std::vector<int64_t> load(grid, 0);
  for (const auto& it : items) {
    int best = 0;
    for (int b = 1; b < grid; ++b)
      if (load[b] < load[best]) best = b;
    lists[best].push_back(it.second);
    load[best] += it.first;
  }
  std::vector<int> tab(grid + 1, 0);
  for (int b = 0; b < grid; ++b) {
    std::sort(lists[b].begin(), lists[b].end());
    tab[b + 1] = tab[b] + (int)lists[b].size();
  }
  for (int b = 0; b < grid; ++b) tab.insert(tab.end(), lists[b].begin(), lists[b].end());
  firal_problem::PwSched sc;
  sc.sp = sp;
  sc.quad = quad;
  sc.grid = grid;
  FIRAL_TRY(sc.buf.ensure(tab.size() * sizeof(int)));
  cudaStream_t st = P->H->stream;
  cudaError_t e = cudaMemcpyAsync(sc.buf.p, tab.data(), tab.size() * sizeof(int),
                                  cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // tab is read by the copy
  if (e != cudaSuccess) {
    sc.buf.release();
    return fail(FIRAL_ERR_CUDA, cudaGetErrorString(e));
  }
  P->pw_sched.push_back(sc);
  *grid_out = grid;
  *sched_out = P->pw_sched.back().buf.as<int>();
  return FIRAL_OK;
}

template <int DP>
static int32_t tc_apply_pw_t(firal_problem* P, const float* w, const float* V, int s, float* out,
                             double* pq, double lam) {
  using namespace pw_cfg;
  cudaStream_t st = P->H->stream;
  const int c = P->c, d = P->d;
  const int Qe = pool_count(P->pt);
  FIRAL_TRY(P->vmean.ensure((size_t)s * Qe * d * sizeof(float)));
  FIRAL_TRY(P->qmean.ensure((size_t)s * Qe * d * sizeof(float)));
  const int sp = (s + 7) / 8 * 8;
  const int64_t prows = 2LL * sp * P->pw_cpad_total;
  FIRAL_TRY(P->pw_pk.ensure((size_t)prows * 64 * 2));
  FIRAL_TRY(P->pw_part.ensure((size_t)std::max<int64_t>(1, P->pw_segcls_total) * sp * d *
                              sizeof(float)));
  {
    ProfScope ps(st, PF_SPLIT);
    count_launch();
    k_pw_pack<<<dim3((unsigned)Qe, (unsigned)sp), 256, 0, st>>>(
        P->pw_pk.as<bf16>(), V, P->vmean.as<float>(), P->pw_pool.as<int4>(), s, sp, d, P->D, Qe);
    FIRAL_CUDA_TRY(cudaGetLastError());
  }
  static bool attr[3] = {false, false, false};
  const int ai = DP == 16 ? 0 : DP == 32 ? 1 : 2;
  if (!attr[ai]) {
    FIRAL_CUDA_TRY(cudaFuncSetAttribute(k_tc_pw<DP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        SMEM));
    attr[ai] = true;
  }
  CUtensorMap mX, mXT, mPT;
  const int64_t Np = P->Np;
  FIRAL_TRY(make_map(&mX, DP < 64 ? P->X64.p : P->Xb.p, Np, 64, 128, 64, true));
  FIRAL_TRY(make_map(&mXT, P->Xb.as<bf16>() + Np * DP, (uint64_t)(Np / 64) * DP, 64, DP, 64,
                     true));
  FIRAL_TRY(make_map(&mPT, P->pw_pk.p, prows, 64, 64, 64, true));
  {
    ProfScope ps(st, PF_ALPHA);
    count_launch();
    int grid = 0;
    const int* sched = nullptr;
    FIRAL_TRY(pw_schedule(P, sp, false, &grid, &sched));
    k_tc_pw<DP><<<grid, 384, SMEM, st>>>(mX, mXT, mPT, P->HaT.as<float>(), w,
                                         P->pw_part.as<float>(), P->pw_pool.as<int4>(),
                                         P->pw_seg.as<int4>(), sched, P->N, s, sp, d,
                                         tc_error_word(P));
    FIRAL_CUDA_TRY(cudaGetLastError());
  }
  ProfScope ps(st, PF_COMBINE);
  if (!sharded(P)) {
    count_launch();
    k_pw_finish<<<dim3((unsigned)Qe, (unsigned)s), PWF_THREADS, 0, st>>>(
        out, V, P->vmean.as<float>(), P->pw_part.as<float>(), P->pw_pool.as<int4>(),
        P->pw_pseg.as<int2>(), P->pw_seg.as<int4>(), (float)lam, lam, s, sp, c, d, P->D, Qe, pq);
    FIRAL_CUDA_TRY(cudaGetLastError());
    return FIRAL_OK;
  }
  // a row-sharded group: lambda I counts once (rank 0), and the projection and the dots act
  // on the summed result
  count_launch(3);
  k_pw_combine<<<c, 256, 0, st>>>(out, V, P->vmean.as<float>(), P->pw_part.as<float>(),
                                  P->pw_pool.as<int4>(), P->pw_pseg.as<int2>(),
                                  P->pw_seg.as<int4>(), P->comm.rank == 0 ? (float)lam : 0.0f,
                                  s, sp, d, P->D, P->pt);
  FIRAL_CUDA_TRY(cudaGetLastError());
  FIRAL_TRY(shard_allreduce(P, out, (int64_t)s * P->D, FIRAL_DT_F32, 0));
  const int mthreads = (d + 31) / 32 * 32;
  FIRAL_TRY(class_mean(P, out, s, P->qmean.as<float>(), st));
  k_project<<<dim3(c, (s + 3) / 4), mthreads, 0, st>>>(out, P->qmean.as<float>(),
                                                       P->vmean.as<float>(), V, lam, s, c, d,
                                                       P->D, pq, P->pt);
  FIRAL_CUDA_TRY(cudaGetLastError());
  return FIRAL_OK;
}

static int32_t tc_apply_pw(firal_problem* P, const float* w, const float* V, int s, float* out,
                           double* pq, double lam) {
  switch (P->dp) {
    case 16: return tc_apply_pw_t<16>(P, w, V, s, out, pq, lam);
    case 32: return tc_apply_pw_t<32>(P, w, V, s, out, pq, lam);
    default: return tc_apply_pw_t<64>(P, w, V, s, out, pq, lam);
  }
}

// ------------------------------------------------------------------------------------------
// Per-point quadratic forms (eq. 11) on the same work list, for at most 32 classes per pool:
//   a_ikj = x_i . A~_j[:, k],  b_ikj = x_i . B~_j[:, k]      two MMA1s (hi + lo each) per tile
//   q_i = sum_j [sum_k h_ik a_ikj b_ikj - (sum_k h_ik a_ikj)(sum_k h_ik b_ikj)]
// with A~, B~ the probe blocks minus their pool class means (H_i vanishes on those means).
// Only the pool rows' segments run.  Same pipeline as the apply (double-buffered x tile and
// S_A, S_B accumulators, h loaded a tile ahead).  The two epilogue halves of a row meet in
// shared memory (an mbarrier hand-off); the first probe group writes g and later groups add
// to it, all from the same thread, so g is written in a fixed order.
// ------------------------------------------------------------------------------------------
namespace pwq_cfg {
constexpr int PT_HALF = pw_cfg::PT_HALF;
constexpr int OFF_PA = 0, OFF_PB = 2 * PT_HALF, OFF_XA = 4 * PT_HALF;
constexpr int OFF_RED = OFF_XA + 2 * pw_cfg::XA_BYTES, OFF_CTL = OFF_RED + 1024;
constexpr int SMEM = OFF_CTL + 256 + 1024;
// TMEM columns: S_A of buffer b at 256 b, S_B at 256 b + 128
}  // namespace pwq_cfg

template <int CPAD>
__device__ __forceinline__ float pw_quad_chunk(const uint32_t (&ra)[32], const uint32_t (&rb)[32],
                                               const float (&h)[32]) {
  float q = 0.0f;
#pragma unroll
  for (int pl = 0; pl < 32 / CPAD; ++pl) {
    float sab = 0.0f, sa = 0.0f, sb = 0.0f;
#pragma unroll
    for (int k = 0; k < CPAD; ++k) {
      const int t = pl * CPAD + k;
      const float ha = h[k] * __uint_as_float(ra[t]);
      sab = fmaf(ha, __uint_as_float(rb[t]), sab);
      sa += ha;
      sb = fmaf(h[k], __uint_as_float(rb[t]), sb);
    }
    q += sab - sa * sb;
  }
  return q;
}

template <int DP>
__global__ void __launch_bounds__(384, 1)
    k_tc_pwq(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapPA,
             const __grid_constant__ CUtensorMap mapPB, const float* __restrict__ HaT,
             float* __restrict__ g, const int4* __restrict__ pool_tab,
             const int4* __restrict__ seg_tab, const int* __restrict__ sched, int64_t N, int sp,
             int64_t m, float gscale, int32_t* err) {
  using namespace pwq_cfg;
  using pw_cfg::NU;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  PwCtl* ctl = (PwCtl*)(sm + OFF_CTL);
  float* red = (float*)(sm + OFF_RED);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int b = 0; b < 2; ++b) {
      mbar_init(&ctl->x_full[b], 1);
      mbar_init(&ctl->x_empty[b], 1);
      mbar_init(&ctl->s_full[b], 1);
      mbar_init(&ctl->s_empty[b], 8);
    }
    mbar_init(&ctl->psi_full[0], 4);    // here: half 1's shares of the tile's rows are in red
    mbar_init(&ctl->psi_empty[0], 4);   // here: half 0 has read them
    mbar_init(&ctl->pt_full, 1);
    mbar_init(&ctl->pt_empty, 1);
    mbar_init(&ctl->drain, 1);
    ctl->abort_w = 0;
    mbar_fence_init();
  }
  if (warp == 2) {
    tmem_alloc(&ctl->tmem_base, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = ctl->tmem_base;
  volatile int* abort_w = &ctl->abort_w;
  auto give_up = [&](int code) {
    ctl->abort_w = 1;
    atomicExch(err, code);
  };
  // the labelled rows' segments carry no gradient
  auto skip = [&](const int4& sg) { return (int64_t)sg.z <= m; };

  if (warp == 0 && lane == 0) {
    tma_prefetch(&mapX);
    tma_prefetch(&mapPA);
    tma_prefetch(&mapPB);
    uint32_t nt = 0, ni = 0;
    bool ok = true;
    for (int it = sched[blockIdx.x]; it < sched[blockIdx.x + 1] && ok && !*abort_w; ++it) {
      const int4 sg = seg_tab[sched[gridDim.x + 1 + it]];
      if (skip(sg)) continue;
      const int4 pq = pool_tab[sg.x];
      const int n1 = pq.z * sp, pbase = 2 * sp * pq.w;
      const int ng = pw_ngrp(pq.z, sp);
      for (int grp = 0; grp < ng && ok; ++grp) {
        const int nc = pw_ncols(pq.z, sp, grp);
        if (!mbar_wait(&ctl->pt_empty, (ni & 1) ^ 1, abort_w)) { give_up(51); ok = false; break; }
        mbar_expect_tx(&ctl->pt_full, 4 * nc * 128);
        for (int part = 0; part < 2; ++part)
          for (int r = 0; r < nc; r += 64) {
            const int y = pbase + part * n1 + grp * NU + r;
            tma_load_2d(sm + OFF_PA + part * PT_HALF + r * 128, &mapPA, &ctl->pt_full, 0, y);
            tma_load_2d(sm + OFF_PB + part * PT_HALF + r * 128, &mapPB, &ctl->pt_full, 0, y);
          }
        ++ni;
        for (int t = sg.y >> 7; t <= (sg.z - 1) >> 7; ++t) {
          const int b = nt & 1;
          if (!mbar_wait(&ctl->x_empty[b], ((nt >> 1) & 1) ^ 1, abort_w)) {
            give_up(52);
            ok = false;
            break;
          }
          mbar_expect_tx(&ctl->x_full[b], pw_cfg::XA_BYTES);
          tma_load_2d(sm + OFF_XA + b * pw_cfg::XA_BYTES, &mapX, &ctl->x_full[b], 0, t * 128);
          ++nt;
        }
      }
    }
    for (int b = 0; b < 2; ++b) {
      const uint32_t cnt = (nt + 1 - b) / 2;
      if (cnt) mbar_wait_drain(&ctl->x_full[b], (cnt - 1) & 1);
    }
    if (ni) mbar_wait_drain(&ctl->pt_full, (ni - 1) & 1);
  } else if (warp == 1 && lane == 0) {
    uint32_t nt = 0, ni = 0;
    bool ok = true;
    for (int it = sched[blockIdx.x]; it < sched[blockIdx.x + 1] && ok && !*abort_w; ++it) {
      const int4 sg = seg_tab[sched[gridDim.x + 1 + it]];
      if (skip(sg)) continue;
      const int4 pq = pool_tab[sg.x];
      const int ng = pw_ngrp(pq.z, sp);
      const int t0 = sg.y >> 7, t1 = (sg.z - 1) >> 7;
      for (int grp = 0; grp < ng && ok; ++grp) {
        const uint32_t idesc1 = idesc_bf16_f32(128, pw_ncols(pq.z, sp, grp));
        if (!mbar_wait(&ctl->pt_full, ni & 1, abort_w)) { give_up(53); ok = false; break; }
        ++ni;
        for (int t = t0; t <= t1; ++t) {
          const int b = nt & 1;
          const uint32_t ph = (nt >> 1) & 1;
          if (!mbar_wait(&ctl->x_full[b], ph, abort_w) ||
              !mbar_wait(&ctl->s_empty[b], ph ^ 1, abort_w)) { give_up(54); ok = false; break; }
          tc_fence_after();
          const uint32_t xa = smem_u32(sm + OFF_XA + b * pw_cfg::XA_BYTES),
                         pa = smem_u32(sm + OFF_PA), pb = smem_u32(sm + OFF_PB);
          const uint32_t ta = tmem + 256 * b, tb = ta + 128;
#pragma unroll
          for (int k = 0; k < DP / 16; ++k) {
            const uint64_t ad = sdesc_sw128(xa + k * 32);
            umma_bf16(ta, ad, sdesc_sw128(pa + k * 32), idesc1, k > 0 ? 1u : 0u);
            umma_bf16(ta, ad, sdesc_sw128(pa + PT_HALF + k * 32), idesc1, 1u);
            umma_bf16(tb, ad, sdesc_sw128(pb + k * 32), idesc1, k > 0 ? 1u : 0u);
            umma_bf16(tb, ad, sdesc_sw128(pb + PT_HALF + k * 32), idesc1, 1u);
          }
          umma_commit(&ctl->s_full[b]);
          umma_commit(&ctl->x_empty[b]);
          if (t == t1) umma_commit(&ctl->pt_empty);
          ++nt;
        }
      }
    }
    umma_commit(&ctl->drain);
    mbar_wait_drain(&ctl->drain, 0);
  } else if (warp >= 4) {
    const int quad = warp & 3, half = (warp - 4) >> 2;
    const int i = quad * 32 + lane;
    const uint32_t lanes = (uint32_t)(quad * 32) << 16;
    uint32_t nt = 0, nr = 0;
    bool ok = true;
    for (int it = sched[blockIdx.x]; it < sched[blockIdx.x + 1] && ok && !*abort_w; ++it) {
      const int4 sg = seg_tab[sched[gridDim.x + 1 + it]];
      if (skip(sg)) continue;
      const int4 pq = pool_tab[sg.x];
      const int cpad = pq.z, cq = pq.y;
      const int ng = pw_ngrp(cpad, sp);
      const int t0 = sg.y >> 7, t1 = (sg.z - 1) >> 7;
      for (int grp = 0; grp < ng && ok; ++grp) {
        const int nc = pw_ncols(cpad, sp, grp);
        float hn[32];
        {
          const int64_t row = (int64_t)t0 * 128 + i;
          const bool v0 = row >= sg.y && row < sg.z && row >= m;
          float wd;
          pw_load_row(hn, wd, HaT, HaT, row, v0, N, pq.x, cq);
        }
        for (int t = t0; t <= t1; ++t) {
          const int64_t row = (int64_t)t * 128 + i;
          const bool valid = row >= sg.y && row < sg.z && row >= m;
          float h[32];
#pragma unroll
          for (int k = 0; k < 32; ++k) h[k] = hn[k];
          if (t < t1) {   // the next tile's row, while this one is worked on
            const int64_t rn = row + 128;
            const bool vn = rn >= sg.y && rn < sg.z && rn >= m;
            float wd;
            pw_load_row(hn, wd, HaT, HaT, rn, vn, N, pq.x, cq);
          }
          const int b = nt & 1;
          if (!mbar_wait(&ctl->s_full[b], (nt >> 1) & 1, abort_w)) {
            give_up(55);
            ok = false;
            break;
          }
          ++nt;
          tc_fence_after();
          float q = 0.0f;
          for (int ch = half; ch < nc / 32; ch += 2) {
            uint32_t ra[32], rb[32];
            tmem_ld32_async(tmem + lanes + 256 * b + ch * 32, ra);
            tmem_ld32_async(tmem + lanes + 256 * b + 128 + ch * 32, rb);
            tmem_wait_ld();
            if (cpad == 8) q += pw_quad_chunk<8>(ra, rb, h);
            else if (cpad == 16) q += pw_quad_chunk<16>(ra, rb, h);
            else q += pw_quad_chunk<32>(ra, rb, h);
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&ctl->s_empty[b]);
          // the two halves of the row: half 1 leaves its share, half 0 writes the sum
          if (half == 1) {
            if (!mbar_wait(&ctl->psi_empty[0], (nr & 1) ^ 1, abort_w)) {
              give_up(56);
              ok = false;
              break;
            }
            red[i] = q;
            __syncwarp();
            if (lane == 0) mbar_arrive(&ctl->psi_full[0]);
          } else {
            if (!mbar_wait(&ctl->psi_full[0], nr & 1, abort_w)) {
              give_up(57);
              ok = false;
              break;
            }
            if (valid) {
              const float v = -gscale * (q + red[i]);
              g[row - m] = grp > 0 ? g[row - m] + v : v;
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&ctl->psi_empty[0]);
          }
          ++nr;
        }
      }
    }
  }
  __syncthreads();
  if (warp == 2) {
    __syncwarp();
    tc_fence_after();
    tmem_dealloc(tmem, 512);
  }
}

template <int DP>
static int32_t tc_quad_pw_t(firal_problem* P, const float* A, const float* B, int s, double scale,
                            float* g) {
  using namespace pwq_cfg;
  cudaStream_t st = P->H->stream;
  const int d = P->d;
  const int Qe = pool_count(P->pt);
  const int sp = (s + 7) / 8 * 8;
  FIRAL_TRY(P->vmean.ensure((size_t)2 * s * Qe * d * sizeof(float)));
  float* meanA = P->vmean.as<float>();
  float* meanB = meanA + (size_t)s * Qe * d;
  const int64_t prows = 2LL * sp * P->pw_cpad_total;
  FIRAL_TRY(P->pw_pk.ensure((size_t)2 * prows * 64 * 2));
  bf16* pkA = P->pw_pk.as<bf16>();
  bf16* pkB = pkA + prows * 64;
  ProfScope ps(st, PF_QUAD);
  count_launch(3);
  k_pw_pack<<<dim3((unsigned)Qe, (unsigned)sp), 256, 0, st>>>(pkA, A, meanA, P->pw_pool.as<int4>(),
                                                               s, sp, d, P->D, Qe);
  k_pw_pack<<<dim3((unsigned)Qe, (unsigned)sp), 256, 0, st>>>(pkB, B, meanB, P->pw_pool.as<int4>(),
                                                               s, sp, d, P->D, Qe);
  FIRAL_CUDA_TRY(cudaGetLastError());
  static bool attr[3] = {false, false, false};
  const int ai = DP == 16 ? 0 : DP == 32 ? 1 : 2;
  if (!attr[ai]) {
    FIRAL_CUDA_TRY(cudaFuncSetAttribute(k_tc_pwq<DP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        SMEM));
    attr[ai] = true;
  }
  CUtensorMap mX, mA, mB;
  FIRAL_TRY(make_map(&mX, DP < 64 ? P->X64.p : P->Xb.p, P->Np, 64, 128, 64, true));
  FIRAL_TRY(make_map(&mA, pkA, prows, 64, 64, 64, true));
  FIRAL_TRY(make_map(&mB, pkB, prows, 64, 64, 64, true));
  int grid = 0;
  const int* sched = nullptr;
  FIRAL_TRY(pw_schedule(P, sp, true, &grid, &sched));
  k_tc_pwq<DP><<<grid, 384, SMEM, st>>>(mX, mA, mB, P->HaT.as<float>(), g, P->pw_pool.as<int4>(),
                                        P->pw_seg.as<int4>(), sched, P->N, sp, P->m,
                                        (float)(scale / s), tc_error_word(P));
  FIRAL_CUDA_TRY(cudaGetLastError());
  return FIRAL_OK;
}

static int32_t tc_quad_pw(firal_problem* P, const float* A, const float* B, int s, double scale,
                          float* g) {
  switch (P->dp) {
    case 16: return tc_quad_pw_t<16>(P, A, B, s, scale, g);
    case 32: return tc_quad_pw_t<32>(P, A, B, s, scale, g);
    default: return tc_quad_pw_t<64>(P, A, B, s, scale, g);
  }
}

template <int NPART>
static int32_t tc_apply_dp(firal_problem* P, const void* w, const void* Sblk, const void* V, int s,
                           void* out, double* pq, double lam_null) {
  const float* ww = (const float*)w;
  const float* sb = (const float*)Sblk;
  const float* vv = (const float*)V;
  float* o = (float*)out;
  switch (P->dp) {
    case 16: return tc_apply_t<16, NPART>(P, ww, sb, vv, s, o, pq, lam_null);
    case 32: return tc_apply_t<32, NPART>(P, ww, sb, vv, s, o, pq, lam_null);
    case 64: return tc_apply_t<64, NPART>(P, ww, sb, vv, s, o, pq, lam_null);
    default: return tc_apply_t<128, NPART>(P, ww, sb, vv, s, o, pq, lam_null);
  }
}

int32_t tc_hessian_apply(firal_problem* P, const void* w, const void* Sblk, const void* V, int s,
                         void* out, double* pq, double lam_null) {
  // at most 32 classes per pool: the fused per-point kernel (its lambda I term is lam_null,
  // added on rank 0 of a row-sharded group)
  if (P->pw) return tc_apply_pw(P, (const float*)w, (const float*)V, s, (float*)out, pq, lam_null);
  // the bf16 direction's rounding (2^-9 per entry) enters only the low-rank term, whose size
  // next to the result is the rows' mean low-rank share; above 0.1 (errors above ~2e-4 per
  // apply) the problem takes the hi + lo direction in both modes (fast_rounding)
  if (fast_rounding(P)) return tc_apply_dp<1>(P, w, Sblk, V, s, out, pq, lam_null);
  return tc_apply_dp<2>(P, w, Sblk, V, s, out, pq, lam_null);
}

int32_t tc_quad_forms(firal_problem* P, const void* A, const void* B, int s, double scale,
                      void* g) {
  const float* a = (const float*)A;
  const float* b = (const float*)B;
  float* gg = (float*)g;
  if (P->pw && !sharded(P)) return tc_quad_pw(P, a, b, s, scale, gg);
  switch (P->dp) {
    case 16: return tc_quad_t<16>(P, a, b, s, scale, gg);
    case 32: return tc_quad_t<32>(P, a, b, s, scale, gg);
    case 64: return tc_quad_t<64>(P, a, b, s, scale, gg);
    default: return tc_quad_t<128>(P, a, b, s, scale, gg);
  }
}

}  // namespace firal
