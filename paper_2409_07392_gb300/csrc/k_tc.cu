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
// P_lo = P - P_hi, so the contraction sees P to ~2^-17 relative.  X is stored in bf16 and h
// is rounded to bf16 (independent per-element rounding, averaged by the sums over points).
//
// Warp roles (256 threads): warp 0 = TMA producer, warp 1 = MMA issuer (+ TMEM owner),
// warps 2..7 = Y builders (D-GEMM), warps 4..7 = epilogue (TMEM lanes 32*(warp%4)..+31).
// Every mbarrier wait is bounded; on timeout the CTA raises a device flag, drains its
// in-flight MMAs, releases TMEM and exits (FIRAL_ERR_TIMEOUT on the host).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

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

static int32_t* tc_error_word(firal_problem* P) { return &P->H->flags.as<DevFlags>()->pad[0]; }

// ------------------------------------------------------------------------------------------
// preparation: padded bf16 copies (rows x cols -> rows_p x cols_p) and transposes
// ------------------------------------------------------------------------------------------
__global__ void k_to_bf16_pad(bf16* dst, const float* src, int64_t rows, int cols,
                              int64_t rows_p, int cols_p) {
  const int64_t total = rows_p * cols_p;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = idx / cols_p;
    const int cc = (int)(idx - r * cols_p);
    dst[idx] = __float2bfloat16_rn((r < rows && cc < cols) ? src[r * cols + cc] : 0.0f);
  }
}

// dst[cols_p x rows_p] = transpose of a padded bf16 matrix src[rows_p x cols_p]
__global__ void k_transpose_bf16(bf16* dst, const bf16* src, int64_t rows_p, int cols_p) {
  __shared__ bf16 tile[32][34];
  const int64_t rb = (int64_t)blockIdx.x * 32;
  const int cb = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int64_t r = rb + i;
    const int col = cb + threadIdx.x;
    if (r < rows_p && col < cols_p) tile[i][threadIdx.x] = src[r * cols_p + col];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int col = cb + i;
    const int64_t r = rb + threadIdx.x;
    if (r < rows_p && col < cols_p) dst[(int64_t)col * rows_p + r] = tile[threadIdx.x][i];
  }
}

// P (s x [c][d], f32) -> P~ rows (j, part, e), columns k (bf16, K-major), part 0 = hi, 1 = lo
__global__ void k_split_probes(bf16* Pt, const float* P, const float* vmean, int s, int c, int d,
                               int dp, int cp, int64_t D) {
  __shared__ float tile[32][33];
  const int j = blockIdx.z;
  const int k0 = blockIdx.x * 32, e0 = blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int k = k0 + i, e = e0 + threadIdx.x;
    tile[i][threadIdx.x] =
        (k < c && e < d) ? P[(int64_t)j * D + (int64_t)k * d + e] - vmean[j * d + e] : 0.0f;
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int e = e0 + i, k = k0 + threadIdx.x;
    if (e >= dp || k >= cp) continue;
    const float v = tile[threadIdx.x][i];
    const bf16 hi = __float2bfloat16_rn(v);
    const bf16 lo = __float2bfloat16_rn(v - __bfloat162float(hi));
    Pt[((int64_t)(j * 2 + 0) * dp + e) * cp + k] = hi;
    Pt[((int64_t)(j * 2 + 1) * dp + e) * cp + k] = lo;
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
__global__ void k_class_mean(const float* V, int s, int c, int d, int64_t D, float* mean) {
  const int j = blockIdx.x, e = threadIdx.x;
  if (e >= d) return;
  double acc = 0.0;
  for (int k = 0; k < c; ++k) acc += (double)V[(int64_t)j * D + (int64_t)k * d + e];
  mean[j * d + e] = (float)(acc / c);
}

// out = out - qmean + lam_null * vmean (per class block); pq[j c + k] = <V_j[k], out_j[k]>
__global__ void k_project(float* out, const float* qmean, const float* vmean, const float* V,
                          double lam_null, int s, int c, int d, int64_t D, double* pq) {
  __shared__ double red[32];
  const int k = blockIdx.x, e = threadIdx.x;
  for (int jj = 0; jj < 4; ++jj) {
    const int j = blockIdx.y * 4 + jj;
    if (j >= s) break;
    double contrib = 0.0;
    if (e < d) {
      const int64_t o = (int64_t)j * D + (int64_t)k * d + e;
      const float q = out[o] - qmean[j * d + e] + (float)(lam_null * (double)vmean[j * d + e]);
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

// ------------------------------------------------------------------------------------------
// alpha-GEMM
// ------------------------------------------------------------------------------------------
namespace alpha_cfg {
constexpr int BM = 128, BN = 256, BK = 64, STAGES = 4;
constexpr int A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2;
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int SMEM = STAGES * STAGE_BYTES + 1024 + 256;
}  // namespace alpha_cfg

struct TcCtl {
  uint64_t full[4], empty[4], yfull[4], tfull[2], tempty[2], drain;
  uint32_t tmem_base;
  int abort_w;
};

__device__ __forceinline__ void raise_abort(TcCtl* ctl, int32_t* err, int code) {
  ctl->abort_w = 1;
  atomicExch(err, code);
}

template <int DP>
__global__ void __launch_bounds__(256, 1)
    k_tc_alpha(const __grid_constant__ CUtensorMap mapH, const __grid_constant__ CUtensorMap mapP,
               const bf16* __restrict__ Xb, const float* __restrict__ w, bf16* __restrict__ aT,
               int64_t N, int64_t Np, int s, int kblocks, int n_mt, int n_nt, int32_t* err) {
  using namespace alpha_cfg;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  TcCtl* ctl = (TcCtl*)(sm + STAGES * STAGE_BYTES);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int PPN = BN / (2 * DP);   // probes per N tile
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
  const int ntiles = n_mt * n_nt;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer
    tma_prefetch(&mapH);
    tma_prefetch(&mapP);
    int stage = 0;
    uint32_t phase = 0;
    for (int tile = blockIdx.x; tile < ntiles && !*abort_w; tile += gridDim.x) {
      const int mt = tile / n_nt, nt = tile % n_nt;
      for (int kb = 0; kb < kblocks; ++kb) {
        if (!mbar_wait(&ctl->empty[stage], phase ^ 1, abort_w)) {
          raise_abort(ctl, err, 1);
          break;
        }
        unsigned char* st = sm + stage * STAGE_BYTES;
        mbar_expect_tx(&ctl->full[stage], STAGE_BYTES);
        tma_load_2d(st, &mapH, &ctl->full[stage], kb * BK, mt * BM);
        tma_load_2d(st + A_BYTES, &mapP, &ctl->full[stage], kb * BK, nt * BN);
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
    int acc = 0;
    uint32_t acc_phase = 0;
    for (int tile = blockIdx.x; tile < ntiles && !*abort_w; tile += gridDim.x) {
      if (!mbar_wait(&ctl->tempty[acc], acc_phase ^ 1, abort_w)) {
        raise_abort(ctl, err, 2);
        break;
      }
      tc_fence_after();
      const uint32_t d = tmem + acc * BN;
      bool ok = true;
      for (int kb = 0; kb < kblocks; ++kb) {
        if (!mbar_wait(&ctl->full[stage], phase, abort_w)) {
          raise_abort(ctl, err, 3);
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t a0 = smem_u32(sm + stage * STAGE_BYTES);
        const uint32_t b0 = a0 + A_BYTES;
#pragma unroll
        for (int k = 0; k < BK / 16; ++k)
          umma_bf16(d, sdesc_sw128(a0 + k * 32), sdesc_sw128(b0 + k * 32), idesc,
                    (kb | k) != 0);
        umma_commit(&ctl->empty[stage]);
        if (++stage == STAGES) {
          stage = 0;
          phase ^= 1;
        }
      }
      if (!ok) break;
      umma_commit(&ctl->tfull[acc]);
      acc ^= 1;
      if (acc == 0) acc_phase ^= 1;
    }
    // drain: the commit below fires once every MMA issued above has completed
    umma_commit(&ctl->drain);
    mbar_wait_drain(&ctl->drain, 0);
  } else if (warp >= 4) {
    // ---------------- epilogue: one pool row per thread
    const int q = warp & 3;
    int acc = 0;
    uint32_t acc_phase = 0;
    for (int tile = blockIdx.x; tile < ntiles && !*abort_w; tile += gridDim.x) {
      const int mt = tile / n_nt, nt = tile % n_nt;
      if (!mbar_wait(&ctl->tfull[acc], acc_phase, abort_w)) {
        raise_abort(ctl, err, 4);
        break;
      }
      tc_fence_after();
      const int64_t row = (int64_t)mt * BM + q * 32 + lane;
      const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + acc * BN;
      const float wi = row < N ? w[row] : 0.0f;
#pragma unroll 1
      for (int jj = 0; jj < PPN; ++jj) {
        const int j = nt * PPN + jj;
        float sum = 0.0f;
#pragma unroll 1
        for (int part = 0; part < 2; ++part) {
#pragma unroll 1
          for (int ec = 0; ec < DP; ec += (DP < 32 ? DP : 32)) {
            float v[32];
            float xv[32];
            const int cw = DP < 32 ? DP : 32;
            const uint32_t col = (uint32_t)((jj * 2 + part) * DP + ec);
            if (cw == 32) tmem_ld32(tbase + col, v);
            else tmem_ld16(tbase + col, v);
            const bf16* xr = Xb + (row < Np ? row : 0) * DP + ec;
#pragma unroll
            for (int t = 0; t < 32; t += 8) {
              if (t < cw) {
                const uint4 u = *reinterpret_cast<const uint4*>(xr + t);
                const __nv_bfloat162* p2 = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                  const float2 f = __bfloat1622float2(p2[h]);
                  xv[t + 2 * h] = f.x;
                  xv[t + 2 * h + 1] = f.y;
                }
              }
            }
#pragma unroll
            for (int t = 0; t < 32; ++t)
              if (t < cw) sum = fmaf(xv[t], v[t], sum);
          }
        }
        if (row < N && j < s) aT[(int64_t)j * Np + row] = __float2bfloat16_rn(wi * sum);
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
constexpr int BM = 128, BN = 256, BK = 64, STAGES = 3;
constexpr int A_BYTES = BM * BK * 2;      // H^T tile
constexpr int Y_BYTES = BN * BK * 2;      // built operand
constexpr int XT_MAX = 128 * BK * 2;      // x^T tile (dp rows)
constexpr int AT_MAX = 16 * BK * 2;       // walpha^T tile (<= 16 probes)
constexpr int STAGE_BYTES = A_BYTES + Y_BYTES + XT_MAX + AT_MAX;
constexpr int SMEM = STAGES * STAGE_BYTES + 1024 + 256;
constexpr int NBUILD = 6;                 // builder warps (2..7)
}  // namespace d_cfg

template <int DP>
__global__ void __launch_bounds__(256, 1)
    k_tc_dterm(const __grid_constant__ CUtensorMap mapHT, const __grid_constant__ CUtensorMap mapXT,
               const __grid_constant__ CUtensorMap mapAT, float* __restrict__ Dpart, int64_t N,
               int c, int d, int s, int n_mt, int n_nt, int splits, int64_t kb_per_split,
               int64_t kb_total, int32_t* err) {
  using namespace d_cfg;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* sm = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  TcCtl* ctl = (TcCtl*)(sm + STAGES * STAGE_BYTES);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int PPN = BN / DP;                 // probes per N tile
  constexpr int XT_BYTES = DP * BK * 2;
  constexpr int AT_BYTES = PPN * BK * 2;
  constexpr uint32_t TX = A_BYTES + XT_BYTES + AT_BYTES;
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
    tmem_alloc(&ctl->tmem_base, 256);
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
    kb0 = (int64_t)sp * kb_per_split;
    kb1 = kb0 + kb_per_split < kb_total ? kb0 + kb_per_split : kb_total;
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
        const int x = (int)(kb * BK);
        tma_load_2d(st, &mapHT, &ctl->full[stage], x, mt * BM);
        tma_load_2d(st + A_BYTES + Y_BYTES, &mapXT, &ctl->full[stage], x, 0);
        tma_load_2d(st + A_BYTES + Y_BYTES + XT_MAX, &mapAT, &ctl->full[stage], x, nt * PPN);
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
        const uint32_t y0 = a0 + A_BYTES;
#pragma unroll
        for (int k = 0; k < BK / 16; ++k)
          umma_bf16(tmem, sdesc_sw128(a0 + k * 32), sdesc_sw128(y0 + k * 32), idesc,
                    (kb != kb0) || k != 0);
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
        unsigned char* Y = st + A_BYTES;
        const unsigned char* XT = st + A_BYTES + Y_BYTES;
        const unsigned char* AT = XT + XT_MAX;
        // chunk = (row r of Y, 8 consecutive points c8); 8 threads share a row
        for (int ch = bw * 32 + lane; ch < BN * 8; ch += NBUILD * 32) {
          const int r = ch >> 3, c8 = ch & 7;
          const int jl = r / DP, e = r - jl * DP;
          const uint4 xv = *reinterpret_cast<const uint4*>(XT + e * (BK * 2) + c8 * 16);
          const uint4 av = *reinterpret_cast<const uint4*>(AT + jl * (BK * 2) + c8 * 16);
          uint4 yv;
          const __nv_bfloat162* x2 = reinterpret_cast<const __nv_bfloat162*>(&xv);
          const __nv_bfloat162* a2 = reinterpret_cast<const __nv_bfloat162*>(&av);
          __nv_bfloat162* y2 = reinterpret_cast<__nv_bfloat162*>(&yv);
#pragma unroll
          for (int h = 0; h < 4; ++h) y2[h] = __hmul2(x2[h], a2[h]);
          *reinterpret_cast<uint4*>(Y + r * 128 + ((c8 ^ (r & 7)) << 4)) = yv;
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
      if (warp >= 4) {
        const int q = warp & 3;
        if (!mbar_wait(&ctl->tfull[0], acc_phase, abort_w)) {
          raise_abort(ctl, err, 15);
          break;
        }
        tc_fence_after();
        const int k = mt * BM + q * 32 + lane;           // class row of this thread
        const int sp = (u / n_nt) / n_mt;
        const int sd = s * d;
        float* out = Dpart + ((int64_t)sp * c + k) * sd;
        for (int cc = 0; cc < BN; cc += 32) {
          float v[32];
          tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + cc, v);
          if (k < c) {
#pragma unroll
            for (int t = 0; t < 32; ++t) {
              const int col = nt * BN + cc + t;
              const int j = col / DP, e = col - j * DP;
              if (j < s && e < d) out[j * d + e] = v[t];
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
    tmem_dealloc(tmem, 256);
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

int32_t tc_prepare(firal_problem* P) {
  cudaStream_t st = P->H->stream;
  if (P->d > 128) return fail(FIRAL_ERR_UNSUPPORTED, "mixed path supports d <= 128");
  P->dp = pow2_dim(P->d);
  P->cp = (int32_t)((P->c + 63) / 64 * 64);
  P->Np = (P->N + 127) / 128 * 128;
  const int64_t Np = P->Np;
  FIRAL_TRY(P->Hb.ensure((size_t)Np * P->cp * 2));
  FIRAL_TRY(P->HbT.ensure((size_t)Np * P->cp * 2));
  FIRAL_TRY(P->Xb.ensure((size_t)Np * P->dp * 2 * 2));   // X (Np x dp) then X^T (dp x Np)
  const int64_t tot_h = Np * P->cp, tot_x = Np * P->dp;
  ProfScope ps(st, PF_PREP);
  count_launch(4);
  k_to_bf16_pad<<<(unsigned)std::min<int64_t>((tot_h + 255) / 256, 1 << 20), 256, 0, st>>>(
      P->Hb.as<bf16>(), P->Ha.as<float>(), P->N, P->c, Np, P->cp);
  k_to_bf16_pad<<<(unsigned)std::min<int64_t>((tot_x + 255) / 256, 1 << 20), 256, 0, st>>>(
      P->Xb.as<bf16>(), P->Xa.as<float>(), P->N, P->d, Np, P->dp);
  FIRAL_CUDA_TRY(cudaGetLastError());
  k_transpose_bf16<<<dim3((unsigned)(Np / 32), (unsigned)((P->cp + 31) / 32)), dim3(32, 8), 0,
                     st>>>(P->HbT.as<bf16>(), P->Hb.as<bf16>(), Np, P->cp);
  k_transpose_bf16<<<dim3((unsigned)(Np / 32), (unsigned)((P->dp + 31) / 32)), dim3(32, 8), 0,
                     st>>>(P->Xb.as<bf16>() + tot_x, P->Xb.as<bf16>(), Np, P->dp);
  FIRAL_CUDA_TRY(cudaGetLastError());
  return FIRAL_OK;
}

template <int DP>
static int32_t tc_apply_t(firal_problem* P, const float* w, const float* Sblk, const float* V,
                          int s, float* out, double* pq, double lam_null) {
  using namespace alpha_cfg;
  cudaStream_t st = P->H->stream;
  const int64_t Np = P->Np;
  const int cp = P->cp;
  const int sp16 = (s + 15) / 16 * 16;
  // P~ (hi/lo) and walpha^T buffers
  const int64_t prow = (int64_t)s * 2 * DP;
  const int64_t prow_p = (prow + BN - 1) / BN * BN;
  FIRAL_TRY(P->Pb.ensure((size_t)prow_p * cp * 2));
  FIRAL_TRY(P->walpha.ensure((size_t)sp16 * Np * 2));
  if (prow_p > prow)
    FIRAL_CUDA_TRY(cudaMemsetAsync(P->Pb.as<bf16>() + prow * cp, 0, (prow_p - prow) * cp * 2, st));
  FIRAL_TRY(P->vmean.ensure((size_t)s * P->d * sizeof(float)));
  FIRAL_TRY(P->qmean.ensure((size_t)s * P->d * sizeof(float)));
  const int mthreads = (P->d + 31) / 32 * 32;
  {
  ProfScope ps(st, PF_ALPHA);
  count_launch(2);
  k_class_mean<<<s, mthreads, 0, st>>>(V, s, P->c, P->d, P->D, P->vmean.as<float>());
  k_split_probes<<<dim3((unsigned)(cp + 31) / 32, DP / 32 > 0 ? DP / 32 : 1, s), dim3(32, 8), 0,
                   st>>>(P->Pb.as<bf16>(), V, P->vmean.as<float>(), s, P->c, P->d, DP, cp,
                           P->D);
  }
  FIRAL_CUDA_TRY(cudaGetLastError());
  CUtensorMap mH, mP;
  FIRAL_TRY(make_map(&mH, P->Hb.p, Np, cp, BM, BK, true));
  FIRAL_TRY(make_map(&mP, P->Pb.p, prow_p, cp, BN, BK, true));
  const int n_mt = (int)(Np / BM), n_nt = (int)(prow_p / BN);
  const int sms = P->H->sm_count;
  const int grid = std::min(n_mt * n_nt, sms);
  static bool attr[4] = {false, false, false, false};
  const int ai = DP == 16 ? 0 : DP == 32 ? 1 : DP == 64 ? 2 : 3;
  if (!attr[ai]) {
    FIRAL_CUDA_TRY(cudaFuncSetAttribute(k_tc_alpha<DP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        SMEM));
    FIRAL_CUDA_TRY(cudaFuncSetAttribute(k_tc_dterm<DP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        d_cfg::SMEM));
    attr[ai] = true;
  }
  {
  ProfScope ps(st, PF_ALPHA);
  count_launch();
  k_tc_alpha<DP><<<grid, 256, SMEM, st>>>(mH, mP, P->Xb.as<bf16>(), w, P->walpha.as<bf16>(),
                                          P->N, Np, s, cp / BK, n_mt, n_nt, tc_error_word(P));
  }
  FIRAL_CUDA_TRY(cudaGetLastError());
  // D-GEMM
  {
    constexpr int PPN = d_cfg::BN / DP;
    const int sd = s * P->d;
    const int n_mt2 = cp / d_cfg::BM + (cp % d_cfg::BM ? 1 : 0);
    const int n_nt2 = (s * DP + d_cfg::BN - 1) / d_cfg::BN;
    const int64_t kb_total = Np / d_cfg::BK;
    const int tiles = n_mt2 * n_nt2;
    int splits = (int)std::max<int64_t>(1, std::min<int64_t>((4LL * sms + tiles - 1) / tiles,
                                                            kb_total / 4 > 0 ? kb_total / 4 : 1));
    const int64_t kbps = (kb_total + splits - 1) / splits;
    splits = (int)((kb_total + kbps - 1) / kbps);
    FIRAL_TRY(P->Dpart.ensure((size_t)splits * P->c * sd * sizeof(float)));
    CUtensorMap mHT, mXT, mAT;
    FIRAL_TRY(make_map(&mHT, P->HbT.p, cp, Np, d_cfg::BM, d_cfg::BK, true));
    FIRAL_TRY(make_map(&mXT, P->Xb.as<bf16>() + Np * DP, DP, Np, DP, d_cfg::BK, false));
    FIRAL_TRY(make_map(&mAT, P->walpha.p, sp16, Np, PPN, d_cfg::BK, false));
    const int units = tiles * splits;
    const int grid2 = std::min(units, sms);
    {
    ProfScope ps(st, PF_DTERM);
    count_launch();
    k_tc_dterm<DP><<<grid2, 256, d_cfg::SMEM, st>>>(mHT, mXT, mAT, P->Dpart.as<float>(), P->N, P->c,
                                             P->d, s, n_mt2, n_nt2, splits, kbps, kb_total,
                                             tc_error_word(P));
    }
    FIRAL_CUDA_TRY(cudaGetLastError());
    FIRAL_TRY(combine_f32(P, Sblk, V, splits, s, out, nullptr, P->vmean.as<float>()));
    ProfScope ps(st, PF_COMBINE);
    count_launch(2);
    k_class_mean<<<s, mthreads, 0, st>>>(out, s, P->c, P->d, P->D, P->qmean.as<float>());
    k_project<<<dim3(P->c, (s + 3) / 4), mthreads, 0, st>>>(
        out, P->qmean.as<float>(), P->vmean.as<float>(), V, lam_null, s, P->c, P->d, P->D, pq);
    FIRAL_CUDA_TRY(cudaGetLastError());
    return FIRAL_OK;
  }
}

int32_t tc_hessian_apply(firal_problem* P, const void* w, const void* Sblk, const void* V, int s,
                         void* out, double* pq, double lam_null) {
  switch (P->dp) {
    case 16: return tc_apply_t<16>(P, (const float*)w, (const float*)Sblk, (const float*)V, s, (float*)out, pq, lam_null);
    case 32: return tc_apply_t<32>(P, (const float*)w, (const float*)Sblk, (const float*)V, s, (float*)out, pq, lam_null);
    case 64: return tc_apply_t<64>(P, (const float*)w, (const float*)Sblk, (const float*)V, s, (float*)out, pq, lam_null);
    default: return tc_apply_t<128>(P, (const float*)w, (const float*)Sblk, (const float*)V, s, (float*)out, pq, lam_null);
  }
}

int32_t tc_quad_forms(firal_problem* P, const void* A, const void* B, int s, double scale,
                      void* g) {
  return quad_forms_simt(P, A, B, s, scale, g);
}

}  // namespace firal
