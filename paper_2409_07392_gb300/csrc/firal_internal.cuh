// Internal declarations of the Approx-FIRAL GB300 library (not part of the C-ABI).
#pragma once

#include <cuda_runtime.h>
#include <atomic>
#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "firal.h"

namespace firal {

inline bool is_mixed(int32_t prec) {
  return prec == FIRAL_MIXED_BF16 || prec == FIRAL_MIXED_BF16_FAST;
}


// ------------------------------------------------------------------------------------------
// Error plumbing: every host helper returns a firal_status; CUDA failures carry a detail.
// ------------------------------------------------------------------------------------------
struct Err {
  int32_t code = FIRAL_OK;
  std::string msg;
};

#define FIRAL_CUDA_TRY(expr)                                                              \
  do {                                                                                    \
    cudaError_t e_ = (expr);                                                              \
    if (e_ != cudaSuccess) {                                                              \
      return ::firal::fail(FIRAL_ERR_CUDA, std::string(#expr) + ": " +                    \
                                               cudaGetErrorString(e_));                   \
    }                                                                                     \
  } while (0)

#define FIRAL_TRY(expr)                \
  do {                                 \
    int32_t s_ = (expr);               \
    if (s_ != FIRAL_OK) return s_;     \
  } while (0)

int32_t fail(int32_t code, const std::string& msg);   // records the detail in thread-local storage
const std::string& last_detail();

// ------------------------------------------------------------------------------------------
// Device memory owned by the library.
// ------------------------------------------------------------------------------------------
struct DBuf {
  void* p = nullptr;
  size_t bytes = 0;
  int32_t ensure(size_t nbytes);   // grow (never shrink); contents not preserved
  void release();                  // cudaFree
  void park();                     // to the block cache (no kernel may still use the buffer)
  template <class T> T* as() const { return static_cast<T*>(p); }
};

// Per-column PCG state kept on the device (one entry per right-hand side).
struct CGCol {
  double rho;       // r^T z
  double bnorm2;    // ||b||^2
  double alpha;     // step of the current iteration (0 when inactive)
  double beta;
  double relres;    // ||r|| / ||b|| after the last update
  int32_t active;   // 1 while the column iterates
  int32_t iters;    // iterations taken
};

// Device-side status words written by kernels and read by the host on synchronising calls.
struct DevFlags {
  int32_t not_spd;     // set by a Cholesky that met a non-positive pivot
  int32_t nonfinite;   // set when a reduction meets NaN/Inf
  int32_t pad[2];
};

}  // namespace firal

namespace firal {
// Kernel-class timers and the launch counter (see firal_profile* in firal.h).
enum ProfId {
  PF_PREP = 0, PF_PROBES, PF_SYRK, PF_CHOL, PF_ALPHA, PF_DTERM, PF_COMBINE, PF_CG, PF_QUAD,
  PF_MD, PF_DOT, PF_ROUND, PF_SPLIT, PF_EXACT_BUILD, PF_EXACT_FACTOR, PF_EXACT_GEMM,
  PF_EXACT_QUAD, PF_EXACT_SCORE, PF_LR, PF_COUNT
};
extern std::atomic<long long> g_launches;
inline void count_launch(int n = 1) { g_launches.fetch_add(n, std::memory_order_relaxed); }
// Split-count override for tests of the row partition (0 = automatic).
int forced_splits();
int forced_sm_budget();
struct ProfScope {
  ProfScope(cudaStream_t st, int id);
  ~ProfScope();
  cudaStream_t st;
  int id;
  cudaEvent_t a = nullptr;
};
}  // namespace firal

namespace firal {
// Launch tuning of a prepared problem (firal_tuning in firal.h; 0 = the built-in shape rule).
struct Tuning {
  int dterm_splits = 0;    // point-range splits of the Hessian apply's D-GEMM
  int bsum_splits = 0;     // point-range splits of the block sums
  int sm_budget = 0;       // CTAs the problem's grids spread over
};
}  // namespace firal

struct firal_handle {
  int device = 0;
  int sm_count = 148;
  int sm_budget = 0;       // > 0: CTAs a problem created on this handle may spread over
  firal::Tuning tune;      // default tuning of problems created on this handle
  cudaStream_t stream = nullptr;
  firal::DBuf flags;       // firal::DevFlags
  firal::DBuf scratch;     // small reductions
  std::string err;
};

namespace firal {
// Pooled problem: Q independent pools stacked into one problem.  Classes and pool rows are
// grouped by pool and every h row is zero outside its pool's classes, so the Hessians, the
// preconditioner blocks and Sigma_z are block diagonal over pools; only the reductions that
// define per-pool scalars (CG alpha/beta, class means, the MD normalisation) see the tables.
// Q = 0: an ordinary problem (one pool, tables unused).
struct PoolTab {
  int Q = 0;
  const int* cpool = nullptr;    // class -> pool (c entries)
  const int* coff = nullptr;     // first class of each pool (Q + 1)
  const int* pdim = nullptr;     // true feature dimension of each pool (Q); features above are 0
};
__host__ __device__ inline int pool_count(const PoolTab& t) { return t.Q > 0 ? t.Q : 1; }
#ifdef __CUDACC__
__device__ __forceinline__ int pool_of(const PoolTab& t, int k) { return t.Q ? t.cpool[k] : 0; }
#endif
}  // namespace firal

namespace firal {
// Dense d~ x d~ workspace of Exact-FIRAL (Algorithm 1), allocated on first use.
enum ExactMat {
  EX_HO = 0, EX_HP, EX_A, EX_W, EX_S, EX_T, EX_M,   // Relax (objective and gradient)
  EX_MATS_RELAX,
  EX_SIG = EX_MATS_RELAX, EX_LINV, EX_HSUM, EX_HHO, EX_MHAT,   // Round
  EX_MATS
};
struct ExactWs {
  DBuf m[EX_MATS];
  DBuf pairs;           // int2 (k, l), k <= l, row by row
  int npairs = 0;
  bool ho_ready = false, hp_ready = false;
  DBuf part, gpart;     // class-pair partial sums / gradient partials per pair group
  DBuf K, YZ;           // Round: c x c matrices per candidate chunk; rank-c factors (d~ x c)
  DBuf negr, mask, argp;
  DBuf flag, scal;      // not-SPD flag; device scalars and reduction partials
};
}  // namespace firal

struct firal_problem {
  firal::ExactWs* ex = nullptr;   // Exact-FIRAL dense workspace (null until used)
  firal::Tuning tune;             // requested launch tuning (0 = shape rule)
  firal::Tuning tune_used;        // what the last launches used
  int sms = 0;            // SM budget for grids and split counts (<= H->sm_count)
  firal::PoolTab pt;      // pooled problems only (device tables below)
  firal::DBuf pool_tabs;  // cpool | coff | pdim (int32) for pt
  firal::DBuf pool_z;     // pooled: per-pool budgets (f64, Q) and pool-row offsets (i64, Q + 1)
  firal::DBuf md_part;    // pooled: per-block partials of the MD step (max, then sum)
  std::vector<int64_t> pool_zoff_h;   // pooled: pool-row offsets, host copy
  firal::DBuf kr_alpha, kr_dterm, kr_bsum;  // pooled: K ranges of the tensor-core GEMM tiles
  int kbL = 0;                   // pooled: K-steps holding the labelled rows (every class tile)
  int64_t kr_dterm_Lmax = 0, kr_bsum_Lmax = 0;   // pooled: longest class-tile K list
  firal_handle* H = nullptr;
  int32_t prec = FIRAL_FP32;
  bool dbl = false;            // vec type is double
  int64_t n = 0, m = 0, N = 0; // pool, labelled, total rows (labelled first)
  int32_t d = 0, c = 0;
  int64_t D = 0;               // d * c
  double lambda = 0.0;

  // SIMT layout, vec type: X (N x d), h (N x c), h^T (c x N)
  firal::DBuf Xa, Ha, HaT;
  // weights over all N rows: Sigma_z (1 on labelled, z on pool) and H_p (0 / 1/n)
  firal::DBuf w_sig, w_p;
  // block matrices (c x d x d): H_p diagonal-part operator, Sigma_z diagonal-part operator,
  // preconditioner blocks (double), their inverse (vec type), B(H_o) (double)
  firal::DBuf S_p, S_sig, Pblk, Minv, HoBlk;
  bool S_p_ready = false;
  // scratch of the Hessian apply
  firal::DBuf walpha, Dpart, syrk_part;
  // PCG
  firal::DBuf cgX, cgR, cgP, cgQ, cgZ, cgcols, cgpart1, cgpart2;
  firal::DBuf bcg;               // block PCG: class partials, s x s matrices, breakdown flag
  // Relax iteration buffers
  firal::DBuf V, U, W, HU, g, red, zsave;

  // tensor-core layout (FIRAL_MIXED_BF16): bf16 X (N x dp), bf16 h (Np x cp), its transpose
  firal::DBuf Xb, Hb, HbT, Pb;   // Pb: bf16 (hi/lo) operand of the probe block
  firal::DBuf Hlo;               // bf16(h - bf16(h)), row-major like Hb (pair-form gradient,
  bool hlo_ready = false;        // made on first use)
  firal::DBuf vmean, qmean;      // class means of the probe block / of the raw apply (s x d)
  firal::DBuf Aw;                // block sums: (w h)^T hi, lo and (w h (1 - h))^T (3 x cp x Np)
  firal::DBuf Zp;                // block sums: x (x) x on the pair triangle, bf16 hi and lo
  firal::DBuf gq_ab, gq_m, gq_part;  // tensor-core quadratic forms: [A;B], M~ pairs, partials
  firal::DBuf rtab, rM;          // Round on tensor cores: 8-pair chunk table, M~ hi/lo rows
  firal::DBuf tdev;              // device-resident MD step counter (graph replays)
  // row sharding (firal_problem_set_comm): allreduce callback, rank, world, total pool size
  firal_comm comm{0, 1, nullptr, nullptr};
  int64_t n_total = 0;
  // confident rows (max_k h_ik > 1/2), centred at their class m: u_i = h_i - e_m in the
  // Hessian apply (cen[i] = m or -1; rows grouped by class in cen_idx, cen_off per class);
  // bf16 u row-major and K-block-major; a_m and w (u . a) per (row, probe) of an apply
  int64_t n_cen = 0;
  double lowrank_share = 0.0;   // mean over rows of sum_k h_ik^2 (1 on centred rows)
  // (the labelled rows of such a problem are applied on CUDA cores: cen_lab, m x s x c)
  // (cen_items: the grouped rows cut into work items, cen_off then holds each class's first
  // item; cen_part: per-item partial sums)
  firal::DBuf cen, cen_off, cen_idx, Ub, UbT, cen_am, cen_rho, cen_lab, cen_items, cen_part;
  int n_cen_items = 0;
  // pooled problems with few classes per pool: the fused per-point apply and gradient
  // (pw_pool: per pool {first class, classes, padded classes, padded classes before it};
  // pw_seg: segments {pool, first row, end row, classes of the segments before it};
  // pw_pseg: each pool's segment range; pw_pk: packed bf16 direction; pw_part: partials;
  // X64: x padded to 64 features when dp < 64)
  bool pw = false;
  int pw_cpad_max = 0, pw_nseg = 0;
  int64_t pw_cpad_total = 0, pw_segcls_total = 0;
  firal::DBuf pw_pool, pw_seg, pw_pseg, pw_pk, pw_part, X64;
  // host copies of the pool table and segments; per (padded probe count, apply or gradient):
  // the CTAs' segment lists (offsets per CTA, then segment indices), longest first
  std::vector<int4> pw_pool_h, pw_seg_h;
  struct PwSched {
    int sp = 0;
    bool quad = false;
    int grid = 0;
    firal::DBuf buf;
  };
  std::vector<PwSched> pw_sched;
  // fast mixed mode: the labelled rows' diagonal-part block sums (weight 1 in every Sigma_z,
  // so computed once, as three bf16 products) and their weights (1 on those rows, 0 after)
  firal::DBuf S_lab, w_lab;
  firal::DBuf cm_scr;   // class means over many classes: split partials (f64), then tickets
  int cm_np = 0;        // probes cm_scr has room for
  bool slab_ready = false;
  int rtab_d = -1, rtab_chunks = 0;
  int32_t dp = 0, cp = 0;
  int64_t Np = 0;
};

namespace firal {
// ---- capi.cu: row sharding (no-op on a problem that is alone)
bool sharded(const firal_problem* P);
int32_t shard_allreduce(firal_problem* P, void* buf, int64_t count, int32_t dtype, int32_t op);
// ---- k_simt.cu
int32_t copy_rows(bool dbl, void* dst, const void* a, int64_t ma, const void* b, int64_t nb,
                  int cols, int32_t src_dtype, cudaStream_t st);
int32_t transpose(bool dbl, void* dst, const void* src, int64_t rows, int cols, cudaStream_t st);
int32_t class_major_h(firal_problem* P);
int32_t fill_weights(bool dbl, void* w, int64_t m, double lab_val, const void* z, double zconst,
                     int64_t n, cudaStream_t st);
int32_t probes(bool dbl, void* V, uint64_t seed, int64_t t, int s, int64_t D, cudaStream_t st,
               const int64_t* t_dev = nullptr, const PoolTab* pt = nullptr, int d = 0);
int32_t md_step_pooled(firal_problem* P, void* z, const void* g, double beta0, cudaStream_t st);
int32_t selected_weights(firal_problem* P, const int32_t* sel, int32_t b, cudaStream_t st);
int32_t identity_blocks(double* L, int c, int d, cudaStream_t st);
int32_t block_gram(firal_problem* P, const void* A, const void* B, int s, double* part,
                   double* G);
int32_t small_spd_solve(const double* A, const double* Y, int s, double* X, int* flag,
                        cudaStream_t st);
int32_t block_axpy(firal_problem* P, void* Y, const void* Z, const void* Pm, const double* M,
                   double sign, int s);
int32_t precond_apply(firal_problem* P, const void* R, int s, void* Z);
int32_t tick(int64_t* t_dev, cudaStream_t st);
int32_t set_step(int64_t* t_dev, int64_t v, cudaStream_t st);
int32_t syrk_blocks(firal_problem* P, const void* w, double lamS, void* outS, double lamP,
                    double* outP);
int32_t syrk_reduce_f32(firal_problem* P, const float* partS, const float* partP, int splits,
                        double lamS, float* outS, double lamP, double* outP,
                        const float* addS = nullptr);
int32_t hessian_apply_simt(firal_problem* P, const void* w, const void* Sblk, const void* V,
                           int s, void* out, double* pq);
int32_t combine_f32(firal_problem* P, const float* Sblk, const float* V, int splits, int s,
                    float* out, double* pq, const float* vmean);
int32_t cg_init(firal_problem* P, const void* B, int s, double tol, int fixed);
int32_t cg_iterate_tail(firal_problem* P, int s, double tol, int fixed);
int32_t quad_forms_simt(firal_problem* P, const void* A, const void* B, int s, double scale,
                        void* g);
int32_t dot_scaled(bool dbl, const void* a, const void* b, int64_t total, double scale,
                   double* part, double* out, cudaStream_t st);
int32_t md_step_simt(bool dbl, void* z, const void* g, int64_t n, double budget, double beta0,
                     double* red, cudaStream_t st);
int32_t md_step_sharded(firal_problem* P, void* z, const void* g, double budget, double beta0,
                        double* red, cudaStream_t st);
int32_t block_dots(firal_problem* P, const void* V, const void* out, int s, double* pq);
// ---- k_linalg.cu
int32_t chol_inv(bool dbl, const double* A, int c, int d, void* inv_t, double* inv_d,
                 double* L_out, int32_t* not_spd, cudaStream_t st);
int32_t tilde_eigvals(const double* L, const double* H, int c, int d, double* eig,
                      cudaStream_t st);
int32_t tilde_nu(const double* L, const double* H, int c, int d, double eta, double* tri,
                 double* gb, double* nu_out, cudaStream_t st);
int32_t sym_tri_nu(const double* Ht, int c, int d, double eta, double* tri, double* gb,
                   double* nu_out, cudaStream_t st);
int32_t sym_tri(const double* Ht, int nblocks, int d, double* tri, double* gb, cudaStream_t st);
int32_t nu_of_tri(const double* tri, const double* gb, int c, int d, double eta, double* work,
                  double* nu_out, cudaStream_t st);
int32_t similarity_blocks(const double* L, const double* H, int c, int d, double* out,
                          cudaStream_t st);
int32_t nu_bisect_dev(const double* lam, int64_t count, double scale, double* nu_out,
                      cudaStream_t st);
int32_t round_scores(firal_problem* P, const void* M1, const void* M2, const uint8_t* mask,
                     double eta, double* pv, int64_t* pi, int np);
int32_t round_pick(const double* pv, const int64_t* pi, int np, uint8_t* mask, int32_t* sel,
                   int32_t t, double* score_out, cudaStream_t st);
int32_t round_m(bool dbl, const double* Binv, const double* Sig, int c, int d, void* M1, void* M2,
                double* Tg, cudaStream_t st, int n_chain = 1);
int32_t round_hupdate(firal_problem* P, double* H, const double* Ho, double invb,
                      const int32_t* sel, int32_t t, const double* L = nullptr,
                      double* Ht = nullptr, const double* Hot = nullptr);
int32_t lincomb(double* out, double a, const double* X, double b, const double* Y, double cc,
                const double* Z, int64_t total, cudaStream_t st);
int32_t lincomb_nu(double* out, const double* nu, const double* X, double b, const double* Y,
                   double cc, const double* Z, int64_t total, cudaStream_t st);
// ---- k_exact.cu (Exact-FIRAL, dense d~ x d~)
int32_t exact_objective(firal_problem* P, const void* z, double* f_host, void* g);
int32_t exact_relax(firal_problem* P, double budget, int T, double beta0, const void* z0,
                    void* z, double* hist);
int32_t exact_round(firal_problem* P, const void* zd, int b, double eta, int exclude,
                    int32_t* sel, double* r_host, double* nu_host, int* evals);
void exact_release(firal_problem* P);
int32_t dense_gemm(bool dbl, cudaStream_t st, bool ta, bool tb, int M, int N, int K,
                   double alpha, const void* A, int64_t lda, const void* B, int64_t ldb,
                   double beta, void* C, int64_t ldc);
// ---- k_al.cu (classifier refit and gathers of the active-learning loop)
int32_t lr_probs(bool dbl, const void* X, const void* W, int64_t rows, int d, int c, void* h,
                 cudaStream_t st);
int32_t lr_grad(bool dbl, const void* X, const int32_t* y, const void* h, const void* W,
                int64_t m, int d, int c, double gamma, void* R, void* g, cudaStream_t st);
int32_t lr_nll(bool dbl, const void* h, const int32_t* y, int64_t m, int c, double* part,
               double* out, cudaStream_t st);
int32_t axpby(bool dbl, void* out, double a, const void* X, double b, const void* Y, int64_t n,
              cudaStream_t st);
int32_t gather_rows(bool dbl, bool labels, const void* src, const int32_t* idx, int64_t rows,
                    int cols, void* dst, cudaStream_t st);
}  // namespace firal
