// C-ABI entry points (include/firal.h) and host orchestration of the Relax and Round steps.
#include <algorithm>
#include <cmath>
#include <map>
#include <tuple>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "firal_internal.cuh"

namespace firal {

static thread_local std::string g_detail;

int32_t fail(int32_t code, const std::string& msg) {
  g_detail = msg;
  return code;
}
const std::string& last_detail() { return g_detail; }

// ---------------------------------------------------------------------------- profiling
std::atomic<long long> g_launches{0};

// FIRAL_SPLITS=p forces p point-range partitions in the split-K reductions (row sharding of the
// pool, Section 3.3); used by the virtual-shard tests.
int forced_splits() {
  static int v = [] {
    const char* e = std::getenv("FIRAL_SPLITS");
    return e ? std::atoi(e) : 0;
  }();
  return v;
}

// FIRAL_SM_BUDGET=k caps the CTAs every problem spreads over (0 or unset: no cap)
int forced_sm_budget() {
  static int v = [] {
    const char* e = std::getenv("FIRAL_SM_BUDGET");
    return e ? std::atoi(e) : 0;
  }();
  return v;
}

namespace {
struct Pending {
  int id;
  cudaEvent_t a, b;
};
struct Profiler {
  std::mutex mu;
  bool on = false;
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  double ms[PF_COUNT] = {};
  long long calls[PF_COUNT] = {};
  cudaEvent_t get() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  void drain() {
    for (auto& p : pending) {
      float t = 0.f;
      if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) {
        ms[p.id] += t;
        calls[p.id] += 1;
      }
      pool.push_back(p.a);
      pool.push_back(p.b);
    }
    pending.clear();
  }
};
Profiler& prof() {
  static Profiler* p = new Profiler();   // never destroyed: no CUDA calls at process exit
  return *p;
}
}  // namespace

ProfScope::ProfScope(cudaStream_t s, int i) : st(s), id(i) {
  Profiler& P = prof();
  if (!P.on) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
  std::lock_guard<std::mutex> g(P.mu);
  a = P.get();
  cudaEventRecord(a, st);
}
ProfScope::~ProfScope() {
  if (!a) return;
  Profiler& P = prof();
  std::lock_guard<std::mutex> g(P.mu);
  cudaEvent_t b = P.get();
  cudaEventRecord(b, st);
  P.pending.push_back({id, a, b});
  if (P.pending.size() > 4096) P.drain();
}

// ---------------------------------------------------------------------------- block cache
// Buffers of destroyed problems are parked here and handed to later allocations on the same
// device instead of going back to the driver: freeing a large problem's buffers costs about
// 20 ms, and a caller that builds one problem per call (firal_relax, firal_round) pays it
// every time.  Only firal_problem_destroy parks, after synchronising the problem's stream, so
// a parked block has no kernel in flight; every other release still calls cudaFree (which
// synchronises the device).  Bounded by FIRAL_CACHE_BYTES (default 64 GiB, 0 disables);
// firal_cache_trim returns every parked block.
namespace {
struct ParkedBlock {
  void* p;
  size_t bytes;
  int dev;
};
struct BlockCache {
  std::mutex mu;
  std::vector<ParkedBlock> blocks;
  size_t held = 0;
  size_t cap = [] {
    const char* e = std::getenv("FIRAL_CACHE_BYTES");
    return e ? (size_t)std::strtoull(e, nullptr, 10) : ((size_t)64 << 30);
  }();
};
BlockCache& block_cache() {
  static BlockCache* c = new BlockCache();   // never destroyed: no CUDA calls at process exit
  return *c;
}
// The smallest parked block of this device holding nbytes, if it is at most twice that size.
void* cache_take(size_t nbytes, size_t* got) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  BlockCache& c = block_cache();
  std::lock_guard<std::mutex> g(c.mu);
  int best = -1;
  for (int i = 0; i < (int)c.blocks.size(); ++i) {
    const ParkedBlock& b = c.blocks[i];
    if (b.dev == dev && b.bytes >= nbytes && b.bytes <= 2 * nbytes + (1u << 20) &&
        (best < 0 || b.bytes < c.blocks[best].bytes))
      best = i;
  }
  if (best < 0) return nullptr;
  void* p = c.blocks[best].p;
  *got = c.blocks[best].bytes;
  c.held -= *got;
  c.blocks.erase(c.blocks.begin() + best);
  return p;
}
// Park a block whose last use has completed; false when the cache is full (caller frees).
bool cache_park(void* p, size_t bytes) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  BlockCache& c = block_cache();
  std::lock_guard<std::mutex> g(c.mu);
  if (c.held + bytes > c.cap) return false;
  c.blocks.push_back({p, bytes, dev});
  c.held += bytes;
  return true;
}
}  // namespace

int32_t DBuf::ensure(size_t nbytes) {
  if (nbytes <= bytes && p) return FIRAL_OK;
  if (p) {
    cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  if (nbytes == 0) nbytes = 16;
  size_t got = 0;
  if (void* q = cache_take(nbytes, &got)) {
    p = q;
    bytes = got;
    return FIRAL_OK;
  }
  cudaError_t e = cudaMalloc(&p, nbytes);
  if (e != cudaSuccess) {
    p = nullptr;
    return fail(FIRAL_ERR_NOMEM, std::string("cudaMalloc(") + std::to_string(nbytes) +
                                     "): " + cudaGetErrorString(e));
  }
  bytes = nbytes;
  return FIRAL_OK;
}

void DBuf::release() {
  if (p) cudaFree(p);
  p = nullptr;
  bytes = 0;
}

void DBuf::park() {
  if (p && !cache_park(p, bytes)) cudaFree(p);
  p = nullptr;
  bytes = 0;
}

// tensor-core entry points (k_tc.cu); return FIRAL_ERR_UNSUPPORTED when not built
int32_t tc_prepare(firal_problem* P);
int32_t tc_hessian_apply(firal_problem* P, const void* w, const void* Sblk, const void* V, int s,
                         void* out, double* pq, double lam_null);
int32_t tc_quad_forms(firal_problem* P, const void* A, const void* B, int s, double scale,
                      void* g);
int32_t tc_syrk_blocks(firal_problem* P, const void* w, double lamS, void* outS, double lamP,
                       double* outP);
int32_t tc_setup_pw(firal_problem* P, const std::vector<int>& coff,
                    const std::vector<int64_t>& loff, const std::vector<int64_t>& poff);
int32_t tc_round_scores(firal_problem* P, const void* M1, const void* M2, const uint8_t* mask,
                        const double* etas, int n_chain, double* pv, int64_t* pi, int* np_out);
bool tc_available();

}  // namespace firal

using namespace firal;

namespace {

inline size_t vsize(const firal_problem* P) { return P->dbl ? sizeof(double) : sizeof(float); }

int32_t record(firal_handle* H, int32_t code) {
  if (H && code != FIRAL_OK) H->err = last_detail();
  return code;
}

int32_t read_flags(firal_handle* H) {
  DevFlags f;
  FIRAL_CUDA_TRY(cudaMemcpyAsync(&f, H->flags.p, sizeof(f), cudaMemcpyDeviceToHost, H->stream));
  FIRAL_CUDA_TRY(cudaStreamSynchronize(H->stream));
  if (f.not_spd || f.nonfinite || f.pad[0]) {
    FIRAL_CUDA_TRY(cudaMemsetAsync(H->flags.p, 0, sizeof(DevFlags), H->stream));
    if (f.pad[0])
      return fail(FIRAL_ERR_TIMEOUT, "a tensor-core kernel wait gave up (site " +
                                         std::to_string(f.pad[0]) + ")");
    if (f.not_spd) return fail(FIRAL_ERR_NOT_SPD, "a block Cholesky met a non-positive pivot");
    return fail(FIRAL_ERR_NONFINITE, "non-finite value in a reduction");
  }
  return FIRAL_OK;
}

int32_t* not_spd_flag(firal_handle* H) { return &H->flags.as<DevFlags>()->not_spd; }

// lambda of H_o = sum_labelled H_i + lambda I counts once over a row-sharded group (rank 0)
double lam_r(const firal_problem* P) { return P->comm.rank == 0 ? P->lambda : 0.0; }

// Hessian apply dispatch (tensor cores for FIRAL_MIXED_BF16)
int32_t apply(firal_problem* P, const void* w, const void* Sblk, const void* V, int s, void* out,
              double* pq) {
  // (the tensor-core apply adds the partials of a row-sharded group itself, before its
  // null-space projection; lambda_N of that projection acts on the summed result)
  if (is_mixed(P->prec))
    return tc_hessian_apply(P, w, Sblk, V, s, out, pq, w == P->w_sig.p ? P->lambda : 0.0);
  if (!sharded(P)) return hessian_apply_simt(P, w, Sblk, V, s, out, pq);
  FIRAL_TRY(hessian_apply_simt(P, w, Sblk, V, s, out, nullptr));
  FIRAL_TRY(shard_allreduce(P, out, (int64_t)s * P->D, P->dbl ? FIRAL_DT_F64 : FIRAL_DT_F32, 0));
  return pq ? block_dots(P, V, out, s, pq) : FIRAL_OK;
}

int32_t quad(firal_problem* P, const void* A, const void* B, int s, double scale, void* g) {
  if (is_mixed(P->prec)) return tc_quad_forms(P, A, B, s, scale, g);
  return quad_forms_simt(P, A, B, s, scale, g);
}

// weighted block sums of the Relax operators (tensor cores for FIRAL_MIXED_BF16)
int32_t blocks(firal_problem* P, const void* w, double lamS, void* outS, double lamP,
               double* outP) {
  if (is_mixed(P->prec)) return tc_syrk_blocks(P, w, lamS, outS, lamP, outP);
  return syrk_blocks(P, w, lamS, outS, lamP, outP);
}

// w_sig = [1 (labelled), z (pool)]; S_sig = diag-part operator with lambda; optional blocks
int32_t setup_sigma(firal_problem* P, const void* z, bool want_precond) {
  cudaStream_t st = P->H->stream;
  if (z) {
    FIRAL_CUDA_TRY(cudaMemcpyAsync((char*)P->w_sig.p + P->m * vsize(P), z, P->n * vsize(P),
                                   cudaMemcpyDeviceToDevice, st));
  }
  FIRAL_TRY(blocks(P, P->w_sig.p, lam_r(P), P->S_sig.p, lam_r(P),
                   want_precond ? P->Pblk.as<double>() : nullptr));
  // a row-sharded group sums the preconditioner blocks of eq. 13 over all rows; the
  // diagonal-part operator S stays this rank's own (each rank's apply adds S_rank V to its
  // partial, and the partials are summed)
  if (sharded(P) && want_precond)
    FIRAL_TRY(shard_allreduce(P, P->Pblk.p, (int64_t)P->c * P->d * P->d, FIRAL_DT_F64, 0));
  if (want_precond)
    FIRAL_TRY(chol_inv(P->dbl, P->Pblk.as<double>(), P->c, P->d, P->Minv.p, nullptr, nullptr,
                       not_spd_flag(P->H), st));
  return FIRAL_OK;
}

int32_t ensure_sp(firal_problem* P) {
  if (P->S_p_ready) return FIRAL_OK;
  FIRAL_TRY(blocks(P, P->w_p.p, 0.0, P->S_p.p, 0.0, nullptr));
  P->S_p_ready = true;
  return FIRAL_OK;
}

int32_t ensure_cg(firal_problem* P, int s) {
  const size_t vb = (size_t)s * P->D * vsize(P);
  FIRAL_TRY(P->cgX.ensure(vb));
  FIRAL_TRY(P->cgR.ensure(vb));
  FIRAL_TRY(P->cgP.ensure(vb));
  FIRAL_TRY(P->cgQ.ensure(vb));
  FIRAL_TRY(P->cgZ.ensure(vb));
  FIRAL_TRY(P->cgcols.ensure((size_t)s * pool_count(P->pt) * sizeof(CGCol)));
  FIRAL_TRY(P->cgpart1.ensure((size_t)s * P->c * sizeof(double)));
  FIRAL_TRY(P->cgpart2.ensure((size_t)s * P->c * sizeof(double)));
  // block PCG: c * s * s partials, six s x s matrices, flag
  FIRAL_TRY(P->bcg.ensure(((size_t)P->c * s * s + 6 * (size_t)s * s + 1) * sizeof(double)));
  return FIRAL_OK;
}

struct CGResult {
  int32_t max_iters = 0;
  double max_relres = 0.0;
  bool converged = true;
};

// Block PCG (O'Leary 1980) on Sigma_z: one Krylov space for all s columns, s x s step
// matrices in FP64 (oracle: approx.block_pcg).  Fixed-iteration mode reads nothing back.
int32_t block_pcg_run(firal_problem* P, const void* B, int s, const firal_cg_opts& cg,
                      void* X_out, bool want_result, CGResult* res,
                      std::vector<CGCol>* cols_out) {
  if (s > 32) return fail(FIRAL_ERR_UNSUPPORTED, "block CG supports s <= 32");
  if (P->pt.Q) return fail(FIRAL_ERR_UNSUPPORTED, "block CG is not available on pooled problems");
  cudaStream_t st = P->H->stream;
  FIRAL_TRY(ensure_cg(P, s));
  const int fixed = cg.fixed_iters > 0 ? 1 : 0;
  const int iters = fixed ? cg.fixed_iters : (cg.maxit > 0 ? cg.maxit : 100);
  const size_t vb = (size_t)s * P->D * vsize(P);
  const size_t ss = (size_t)s * s;
  double* part = P->bcg.as<double>();
  double* gam = part + (size_t)P->c * ss;
  double* gnew = gam + ss;
  double* pq = gnew + ss;
  double* alpha = pq + ss;
  double* beta = alpha + ss;
  double* rr = beta + ss;
  int* flag = reinterpret_cast<int*>(rr + ss);
  FIRAL_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int), st));
  FIRAL_CUDA_TRY(cudaMemsetAsync(P->cgX.p, 0, vb, st));
  FIRAL_CUDA_TRY(cudaMemcpyAsync(P->cgR.p, B, vb, cudaMemcpyDeviceToDevice, st));
  FIRAL_TRY(precond_apply(P, P->cgR.p, s, P->cgZ.p));
  FIRAL_CUDA_TRY(cudaMemcpyAsync(P->cgP.p, P->cgZ.p, vb, cudaMemcpyDeviceToDevice, st));
  FIRAL_TRY(block_gram(P, P->cgZ.p, P->cgR.p, s, part, gam));
  std::vector<double> bn2(s, 0.0), rn2(s, 0.0), hmat(ss);
  auto diag_rr = [&](std::vector<double>& out) -> int32_t {
    FIRAL_TRY(block_gram(P, P->cgR.p, P->cgR.p, s, part, rr));
    FIRAL_CUDA_TRY(cudaMemcpyAsync(hmat.data(), rr, ss * sizeof(double), cudaMemcpyDeviceToHost, st));
    FIRAL_CUDA_TRY(cudaStreamSynchronize(st));
    for (int j = 0; j < s; ++j) out[j] = hmat[(size_t)j * s + j];
    return FIRAL_OK;
  };
  if (!fixed || want_result) FIRAL_TRY(diag_rr(bn2));
  int it = 0;
  for (; it < iters; ++it) {
    if (!fixed) {
      FIRAL_TRY(diag_rr(rn2));
      int hflag = 0;
      FIRAL_CUDA_TRY(cudaMemcpy(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost));
      bool done = hflag != 0;
      if (!done) {
        done = true;
        for (int j = 0; j < s; ++j) done &= rn2[j] <= cg.tol * cg.tol * bn2[j];
      }
      if (done) break;
    }
    FIRAL_TRY(apply(P, P->w_sig.p, P->S_sig.p, P->cgP.p, s, P->cgQ.p, nullptr));
    FIRAL_TRY(block_gram(P, P->cgP.p, P->cgQ.p, s, part, pq));
    FIRAL_TRY(small_spd_solve(pq, gam, s, alpha, flag, st));            // alpha = (P^T A P)^-1 gamma
    FIRAL_TRY(block_axpy(P, P->cgX.p, P->cgX.p, P->cgP.p, alpha, 1.0, s));   // X += P alpha
    FIRAL_TRY(block_axpy(P, P->cgR.p, P->cgR.p, P->cgQ.p, alpha, -1.0, s));  // R -= Q alpha
    FIRAL_TRY(precond_apply(P, P->cgR.p, s, P->cgZ.p));                 // Z = M^-1 R
    FIRAL_TRY(block_gram(P, P->cgZ.p, P->cgR.p, s, part, gnew));        // gamma_new = Z^T R
    FIRAL_TRY(small_spd_solve(gam, gnew, s, beta, flag, st));           // beta = gamma^-1 gamma_new
    FIRAL_TRY(block_axpy(P, P->cgP.p, P->cgZ.p, P->cgP.p, beta, 1.0, s));    // P = Z + P beta
    std::swap(gam, gnew);
  }
  FIRAL_CUDA_TRY(cudaMemcpyAsync(X_out, P->cgX.p, vb, cudaMemcpyDeviceToDevice, st));
  if (want_result || !fixed) {
    FIRAL_TRY(diag_rr(rn2));
    std::vector<CGCol> cols(s);
    if (res) {
      res->max_iters = it;
      res->max_relres = 0.0;
      res->converged = true;
    }
    for (int j = 0; j < s; ++j) {
      const double rel = bn2[j] > 0 ? std::sqrt(rn2[j] / bn2[j]) : 0.0;
      cols[j].iters = it;
      cols[j].relres = rel;
      cols[j].bnorm2 = bn2[j];
      cols[j].active = 0;
      if (res) {
        res->max_relres = std::max(res->max_relres, rel);
        if (!fixed && rel > cg.tol && bn2[j] > 0) res->converged = false;
      }
    }
    if (cols_out) *cols_out = cols;
  }
  return FIRAL_OK;
}

// PCG on Sigma_z (w_sig, S_sig, Minv already set up).  X_out may alias nothing of the CG state.
int32_t pcg_run(firal_problem* P, const void* B, int s, const firal_cg_opts& cg, void* X_out,
                bool want_result, CGResult* res, std::vector<CGCol>* cols_out) {
  if (cg.block) return block_pcg_run(P, B, s, cg, X_out, want_result, res, cols_out);
  cudaStream_t st = P->H->stream;
  FIRAL_TRY(ensure_cg(P, s));
  const int fixed = cg.fixed_iters > 0 ? 1 : 0;
  const int iters = fixed ? cg.fixed_iters : (cg.maxit > 0 ? cg.maxit : 100);
  const double tol = cg.tol;
  FIRAL_TRY(cg_init(P, B, s, tol, fixed));
  const int ns = s * pool_count(P->pt);   // one CG scalar set per (column, pool)
  std::vector<CGCol> cols(ns);
  for (int it = 0; it < iters; ++it) {
    if (!fixed) {
      FIRAL_CUDA_TRY(cudaMemcpyAsync(cols.data(), P->cgcols.p, ns * sizeof(CGCol),
                                     cudaMemcpyDeviceToHost, st));
      FIRAL_CUDA_TRY(cudaStreamSynchronize(st));
      bool any = false;
      for (int j = 0; j < ns; ++j) any |= cols[j].active != 0;
      if (!any) break;
    }
    FIRAL_TRY(apply(P, P->w_sig.p, P->S_sig.p, P->cgP.p, s, P->cgQ.p, P->cgpart1.as<double>()));
    FIRAL_TRY(cg_iterate_tail(P, s, tol, fixed));
  }
  FIRAL_CUDA_TRY(cudaMemcpyAsync(X_out, P->cgX.p, (size_t)s * P->D * vsize(P),
                                 cudaMemcpyDeviceToDevice, st));
  if (want_result || !fixed) {
    FIRAL_CUDA_TRY(cudaMemcpyAsync(cols.data(), P->cgcols.p, ns * sizeof(CGCol),
                                   cudaMemcpyDeviceToHost, st));
    FIRAL_CUDA_TRY(cudaStreamSynchronize(st));
    if (res) {
      res->max_iters = 0;
      res->max_relres = 0.0;
      res->converged = true;
      for (int j = 0; j < ns; ++j) {
        res->max_iters = std::max(res->max_iters, cols[j].iters);
        res->max_relres = std::max(res->max_relres, cols[j].relres);
        if (!fixed && cols[j].relres > tol && cols[j].bnorm2 > 0) res->converged = false;
      }
    }
    if (cols_out) *cols_out = cols;
  }
  return FIRAL_OK;
}

int32_t validate_pool(const firal_pool* pool, const firal_hess0* h0) {
  if (!pool || !pool->X || !pool->h) return fail(FIRAL_ERR_ARG, "pool, X and h must be non-null");
  if (pool->n < 1) return fail(FIRAL_ERR_ARG, "pool size n must be >= 1");
  if (pool->d < 1 || pool->d > 128) return fail(FIRAL_ERR_UNSUPPORTED, "d must be in [1, 128]");
  if (pool->c < 2 || pool->c > 4096) return fail(FIRAL_ERR_UNSUPPORTED, "c must be in [2, 4096]");
  if (pool->x_dtype < 0 || pool->x_dtype > 2) return fail(FIRAL_ERR_ARG, "bad x_dtype");
  if (pool->h_dtype != FIRAL_DT_F32 && pool->h_dtype != FIRAL_DT_F64)
    return fail(FIRAL_ERR_ARG, "h_dtype must be F32 or F64");
  if (h0 && h0->m > 0 && (!h0->Xo || !h0->ho))
    return fail(FIRAL_ERR_ARG, "labelled set pointers must be non-null when m > 0");
  if (h0 && (h0->m < 0 || !(h0->lambda >= 0.0)))
    return fail(FIRAL_ERR_ARG, "m must be >= 0 and lambda >= 0");
  return FIRAL_OK;
}

int32_t problem_create_impl(firal_handle* H, const firal_pool* pool, const firal_hess0* h0,
                            int32_t precision, firal_problem** out) {
  if (!H || !out) return fail(FIRAL_ERR_ARG, "handle and out must be non-null");
  FIRAL_TRY(validate_pool(pool, h0));
  if (precision < FIRAL_FP64 || precision > FIRAL_MIXED_BF16_FAST)
    return fail(FIRAL_ERR_ARG, "unknown precision");
  if (is_mixed(precision) && !tc_available())
    return fail(FIRAL_ERR_UNSUPPORTED, "tensor-core path not built");
  FIRAL_CUDA_TRY(cudaSetDevice(H->device));
  auto* P = new firal_problem();
  P->H = H;
  P->prec = precision;
  P->dbl = precision == FIRAL_FP64;
  P->n = pool->n;
  P->m = h0 ? h0->m : 0;
  P->N = P->n + P->m;
  P->d = pool->d;
  P->c = pool->c;
  P->D = (int64_t)P->d * P->c;
  P->lambda = h0 ? h0->lambda : 0.0;
  P->tune = H->tune;
  {
    int b = forced_sm_budget() > 0 ? forced_sm_budget()
                                   : (P->tune.sm_budget > 0 ? P->tune.sm_budget : H->sm_budget);
    P->sms = (b > 0 && b < H->sm_count) ? b : H->sm_count;
  }
  P->tune_used.sm_budget = P->sms;
  cudaStream_t st = H->stream;
  const size_t vs = vsize(P);
  auto cleanup = [&](int32_t code) {
    firal_problem_destroy(P);
    return code;
  };
  int32_t rc;
#define TRYC(x)                     \
  do {                              \
    rc = (x);                       \
    if (rc != FIRAL_OK) return cleanup(rc); \
  } while (0)
  TRYC(P->Xa.ensure((size_t)P->N * P->d * vs));
  TRYC(P->Ha.ensure((size_t)P->N * P->c * vs));
  TRYC(copy_rows(P->dbl, P->Xa.p, h0 ? h0->Xo : nullptr, P->m, pool->X, P->n, P->d,
                 pool->x_dtype, st));
  TRYC(copy_rows(P->dbl, P->Ha.p, h0 ? h0->ho : nullptr, P->m, pool->h, P->n, P->c,
                 pool->h_dtype, st));
  // class-major copy of h for the CUDA-core kernels; the tensor-core path reads its own bf16
  // operands, prepared below, and makes this copy only if Round asks for it
  if (!is_mixed(precision)) TRYC(class_major_h(P));
  TRYC(P->w_sig.ensure((size_t)P->N * vs));
  TRYC(P->w_p.ensure((size_t)P->N * vs));
  TRYC(P->zsave.ensure((size_t)P->N * vs));
  TRYC(fill_weights(P->dbl, P->w_sig.p, P->m, 1.0, nullptr, 1.0 / P->n, P->n, st));
  TRYC(fill_weights(P->dbl, P->w_p.p, P->m, 0.0, nullptr, 1.0 / P->n, P->n, st));
  const size_t blk = (size_t)P->c * P->d * P->d;
  TRYC(P->S_p.ensure(blk * vs));
  TRYC(P->S_sig.ensure(blk * vs));
  TRYC(P->Minv.ensure(blk * vs));
  TRYC(P->Pblk.ensure(blk * sizeof(double)));
  TRYC(P->HoBlk.ensure(blk * sizeof(double)));
  TRYC(P->red.ensure(2048 * sizeof(double)));
  TRYC(P->g.ensure((size_t)P->n * vs));
  if (is_mixed(precision)) TRYC(tc_prepare(P));
  // at most 32 classes: the fused per-point apply (one pool; a pooled problem replaces these
  // tables with its pools')
  if (is_mixed(precision))
    TRYC(tc_setup_pw(P, std::vector<int>{0, (int)P->c}, std::vector<int64_t>{0, P->m},
                     std::vector<int64_t>{0, P->n}));
#undef TRYC
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cleanup(fail(FIRAL_ERR_CUDA, cudaGetErrorString(e)));
  *out = P;
  return FIRAL_OK;
}

int32_t relax_step_impl(firal_problem* P, const firal_relax_opts* o, int32_t t, double budget,
                        void* z, firal_step_stats* stats, bool device_t = false) {
  if (!P || !o || !z) return fail(FIRAL_ERR_ARG, "problem, opts and z must be non-null");
  if (o->s < 1 || o->s > 256) return fail(FIRAL_ERR_ARG, "s must be in [1, 256]");
  if (!(budget > 0)) return fail(FIRAL_ERR_ARG, "budget must be > 0");
  cudaStream_t st = P->H->stream;
  const int s = o->s;
  const size_t vb = (size_t)s * P->D * vsize(P);
  FIRAL_TRY(P->V.ensure(vb));
  FIRAL_TRY(P->U.ensure(vb));
  FIRAL_TRY(P->W.ensure(vb));
  FIRAL_TRY(P->HU.ensure(vb));
  // line 4: probes (step index from the device counter when replayed from a graph)
  if (device_t) FIRAL_TRY(P->tdev.ensure(sizeof(int64_t)));
  FIRAL_TRY(probes(P->dbl, P->V.p, o->seed, t, s, P->D, st,
                   device_t ? P->tdev.as<int64_t>() : nullptr, &P->pt, P->d));
  // line 5: preconditioner from Sigma_z (z copied into the pool part of w_sig)
  FIRAL_TRY(setup_sigma(P, z, true));
  FIRAL_TRY(ensure_sp(P));
  CGResult r1, r2;
  const bool want = stats != nullptr;
  // line 6: U = Sigma^{-1} V
  FIRAL_TRY(pcg_run(P, P->V.p, s, o->cg, P->U.p, want, &r1, nullptr));
  // line 7: HU = H_p U, f^ = <V, HU>/s
  FIRAL_TRY(apply(P, P->w_p.p, P->S_p.p, P->U.p, s, P->HU.p, nullptr));
  double* red = P->red.as<double>();
  FIRAL_TRY(dot_scaled(P->dbl, P->V.p, P->HU.p, (int64_t)s * P->D, 1.0 / s, red + 1024,
                       red + 1536, st));
  // line 8 (paper estimator) or the derivative of f^ (estimator 1)
  const void* first;
  if (o->estimator == 0) {
    FIRAL_TRY(pcg_run(P, P->HU.p, s, o->cg, P->W.p, want, &r2, nullptr));
    first = P->V.p;
  } else {
    FIRAL_TRY(apply(P, P->w_p.p, P->S_p.p, P->V.p, s, P->HU.p, nullptr));
    FIRAL_TRY(pcg_run(P, P->HU.p, s, o->cg, P->W.p, want, &r2, nullptr));
    first = P->U.p;
  }
  // line 9: gradient
  FIRAL_TRY(quad(P, first, P->W.p, s, 1.0, P->g.p));
  // lines 10-11: MD update on the budget simplex (in the pool part of w_sig), then copy out
  void* zdev = (char*)P->w_sig.p + P->m * vsize(P);
  if (P->pt.Q) FIRAL_TRY(md_step_pooled(P, zdev, P->g.p, o->beta0, st));   // per-pool simplex
  else if (sharded(P)) FIRAL_TRY(md_step_sharded(P, zdev, P->g.p, budget, o->beta0, red, st));
  else FIRAL_TRY(md_step_simt(P->dbl, zdev, P->g.p, P->n, budget, o->beta0, red, st));
  FIRAL_CUDA_TRY(cudaMemcpyAsync(z, zdev, P->n * vsize(P), cudaMemcpyDeviceToDevice, st));
  if (device_t) FIRAL_TRY(tick(P->tdev.as<int64_t>(), st));
  if (stats) {
    double h[4];
    FIRAL_CUDA_TRY(cudaMemcpyAsync(h, red + 1536, sizeof(double), cudaMemcpyDeviceToHost, st));
    FIRAL_CUDA_TRY(cudaMemcpyAsync(h + 1, red + 512, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                                   st));
    FIRAL_CUDA_TRY(cudaStreamSynchronize(st));
    stats->fhat = h[0];
    stats->gmax = h[1];
    stats->zmax = h[2];
    stats->cg_iters[0] = r1.max_iters;
    stats->cg_iters[1] = r2.max_iters;
    stats->cg_relres[0] = r1.max_relres;
    stats->cg_relres[1] = r2.max_relres;
    FIRAL_TRY(read_flags(P->H));
    if (!std::isfinite(h[0]) || !std::isfinite(h[1]))
      return fail(FIRAL_ERR_NONFINITE, "non-finite objective or gradient");
  }
  return FIRAL_OK;
}

// The eta-independent part of Round (Algorithm 3 line 3): B(H_o), the Sigma_diamond blocks and
// their Cholesky factors, shared by every eta of a sweep.
struct RoundSetup {
  DBuf Sig, L;
  ~RoundSetup() {
    Sig.release();
    L.release();
  }
};

int32_t round_setup(firal_problem* P, const void* zr, RoundSetup& rs) {
  cudaStream_t st = P->H->stream;
  const size_t blk = (size_t)P->c * P->d * P->d;
  FIRAL_TRY(rs.Sig.ensure(blk * 8));
  FIRAL_TRY(rs.L.ensure(blk * 8));
  // B(H_o): weights 1 on labelled rows, 0 on the pool; Sigma_diamond: z on the pool (C-15)
  FIRAL_TRY(fill_weights(P->dbl, P->zsave.p, P->m, 1.0, nullptr, 0.0, P->n, st));
  FIRAL_TRY(syrk_blocks(P, P->zsave.p, 0.0, nullptr, P->lambda, P->HoBlk.as<double>()));
  FIRAL_TRY(fill_weights(P->dbl, P->zsave.p, P->m, 1.0, zr, 0.0, P->n, st));
  FIRAL_TRY(syrk_blocks(P, P->zsave.p, 0.0, nullptr, P->lambda, rs.Sig.as<double>()));
  FIRAL_TRY(chol_inv(P->dbl, rs.Sig.as<double>(), P->c, P->d, nullptr, nullptr, rs.L.as<double>(),
                     not_spd_flag(P->H), st));
  return FIRAL_OK;
}

// Round chains (Algorithm 3 lines 4-12) for n_chain values of eta on one prepared set-up, run
// side by side pick by pick: one eq. 14 score launch covers every chain (tensor-core path),
// and each per-pick block step (update, tridiagonal forms, Cholesky, M1/M2) is one launch over
// the stacked c x n_chain blocks; only the scalar root nu and the pick are per chain.
// sel: n_chain x b picks (row e = eta etas[e]).  stats (chain 0) may be NULL.
int32_t round_chains(firal_problem* P, const RoundSetup& rs, int32_t b, const double* etas,
                     int ne, int32_t* sel, firal_round_stats* stats) {
  cudaStream_t st = P->H->stream;
  const int c = P->c, d = P->d;
  const int64_t D = P->D;
  const size_t blk = (size_t)c * d * d;
  const double* Sig = rs.Sig.as<double>();
  const double* L = rs.L.as<double>();
  DBuf Bm, Binv, Hk, M1, M2, eig, nu, mask, pv, pi, score, Tg, Ht, Hot, Sig3;
  auto rel = [&]() {
    for (DBuf* bf : {&Bm, &Binv, &Hk, &M1, &M2, &eig, &nu, &mask, &pv, &pi, &score, &Tg, &Ht,
                     &Hot, &Sig3})
      bf->release();
  };
  const int np = (int)std::max<int64_t>((P->n + 127) / 128, P->sms);
  // per chain: tridiagonal forms (2 c d), Gershgorin bounds (2 c), nu step state and
  // per-SM partials (4 + 3 * 1024)
  const size_t tri_sz = (size_t)2 * c * d, gb_sz = (size_t)2 * c, work_sz = 4 + 3 * 1024;
  int32_t rc = FIRAL_OK;
#define TRYR(x)                    \
  do {                             \
    rc = (x);                      \
    if (rc != FIRAL_OK) {          \
      rel();                       \
      return rc;                   \
    }                              \
  } while (0)
  TRYR(Bm.ensure(ne * blk * 8));
  TRYR(Binv.ensure(ne * blk * 8));
  TRYR(Hk.ensure(ne * blk * 8));
  TRYR(M1.ensure(ne * blk * vsize(P)));
  TRYR(M2.ensure(ne * blk * vsize(P)));
  TRYR(eig.ensure(ne * (tri_sz + gb_sz + work_sz) * 8));
  TRYR(nu.ensure(ne * 8));
  TRYR(mask.ensure((size_t)ne * P->n));
  TRYR(pv.ensure((size_t)ne * np * 8));
  TRYR(pi.ensure((size_t)ne * np * 8));
  TRYR(score.ensure(ne * 8));
  TRYR(Tg.ensure(ne * blk * 8));
  // H~ = L^{-1} H L^{-T} kept up to date pick by pick (rank one plus L^{-1} H_o L^{-T} / b)
  TRYR(Ht.ensure(ne * blk * 8));
  TRYR(Hot.ensure(blk * 8));
  const int64_t tot = (int64_t)blk;
  double* tri = eig.as<double>();
  double* gb = tri + ne * tri_sz;
  double* work = gb + ne * gb_sz;
  auto Bm_e = [&](int e) { return Bm.as<double>() + e * blk; };
  auto Hk_e = [&](int e) { return Hk.as<double>() + e * blk; };
  auto Ht_e = [&](int e) { return Ht.as<double>() + e * blk; };
  auto M_e = [&](DBuf& M, int e) { return (void*)((char*)M.p + e * blk * vsize(P)); };
  // line 4: B_1 = sqrt(d~) Sigma + (eta/b) H_o, for every chain
  for (int e = 0; e < ne; ++e)
    TRYR(lincomb(Bm_e(e), std::sqrt((double)D), Sig, etas[e] / b, P->HoBlk.as<double>(), 0.0,
                 nullptr, tot, st));
  TRYR(chol_inv(P->dbl, Bm.as<double>(), c * ne, d, nullptr, Binv.as<double>(), nullptr,
                not_spd_flag(P->H), st));
  TRYR(round_m(P->dbl, Binv.as<double>(), Sig, c, d, M1.p, M2.p, Tg.as<double>(), st, ne));
  FIRAL_CUDA_TRY(cudaMemsetAsync(Hk.p, 0, ne * blk * 8, st));
  FIRAL_CUDA_TRY(cudaMemsetAsync(Ht.p, 0, ne * blk * 8, st));
  TRYR(similarity_blocks(L, P->HoBlk.as<double>(), c, d, Hot.as<double>(), st));
  FIRAL_CUDA_TRY(cudaMemsetAsync(mask.p, 0, (size_t)ne * P->n, st));
  for (int t = 0; t < b; ++t) {
    // line 7: eq. 14 scores and the masked argmax of every chain (one tensor-core launch for
    // FIRAL_MIXED_BF16*)
    int npart = np;
    if (is_mixed(P->prec)) {
      TRYR(tc_round_scores(P, M1.p, M2.p, mask.as<uint8_t>(), etas, ne, pv.as<double>(),
                           pi.as<int64_t>(), &npart));
    } else {
      for (int e = 0; e < ne; ++e)
        TRYR(round_scores(P, M_e(M1, e), M_e(M2, e), mask.as<uint8_t>() + (size_t)e * P->n,
                          etas[e], pv.as<double>() + (size_t)e * np,
                          pi.as<int64_t>() + (size_t)e * np, np));
    }
    for (int e = 0; e < ne; ++e) {
      TRYR(round_pick(pv.as<double>() + (size_t)e * npart, pi.as<int64_t>() + (size_t)e * npart,
                      npart, mask.as<uint8_t>() + (size_t)e * P->n, sel + (size_t)e * b, t,
                      score.as<double>() + e, st));
      // line 8: H_k += B_k(H_o)/b + w x x^T (and H~_k alongside)
      TRYR(round_hupdate(P, Hk_e(e), P->HoBlk.as<double>(), 1.0 / b, sel + (size_t)e * b, t, L,
                         Ht_e(e), Hot.as<double>()));
    }
    // lines 9-10: nu with sum_j (nu + eta lambda_j(H~_k))^-2 = 1, from the tridiagonal forms
    // of H~_k (the eigenvalues enter only through that trace)
    TRYR(sym_tri(Ht.as<double>(), c * ne, d, tri, gb, st));
    for (int e = 0; e < ne; ++e)
      TRYR(nu_of_tri(tri + e * tri_sz, gb + e * gb_sz, c, d, etas[e], work + e * work_sz,
                     nu.as<double>() + e, st));
    // line 11: B = nu Sigma + eta H + (eta/b) H_o, inverted
    for (int e = 0; e < ne; ++e)
      TRYR(lincomb_nu(Bm_e(e), nu.as<double>() + e, Sig, etas[e], Hk_e(e), etas[e] / b,
                      P->HoBlk.as<double>(), tot, st));
    TRYR(chol_inv(P->dbl, Bm.as<double>(), c * ne, d, nullptr, Binv.as<double>(), nullptr,
                  not_spd_flag(P->H), st));
    TRYR(round_m(P->dbl, Binv.as<double>(), Sig, c, d, M1.p, M2.p, Tg.as<double>(), st, ne));
  }
  if (stats) {
    double h[2];
    FIRAL_CUDA_TRY(cudaMemcpyAsync(h, nu.p, 8, cudaMemcpyDeviceToHost, st));
    FIRAL_CUDA_TRY(cudaMemcpyAsync(h + 1, score.p, 8, cudaMemcpyDeviceToHost, st));
    FIRAL_CUDA_TRY(cudaStreamSynchronize(st));
    stats->nu_last = h[0];
    stats->score_last = h[1];
  }
  FIRAL_CUDA_TRY(cudaStreamSynchronize(st));
  rel();
#undef TRYR
  return FIRAL_OK;
}

int32_t round_impl(firal_problem* P, const void* zr, int32_t b, const firal_round_opts* o,
                   int32_t* sel, firal_round_stats* stats) {
  if (!P || !zr || !sel) return fail(FIRAL_ERR_ARG, "problem, z and selected_out must be non-null");
  if (sharded(P)) return fail(FIRAL_ERR_UNSUPPORTED, "Round does not take a row-sharded problem");
  if (b < 1 || b > P->n) return fail(FIRAL_ERR_ARG, "budget must be in [1, n]");
  if (P->dbl && P->d > 90) return fail(FIRAL_ERR_UNSUPPORTED, "FP64 Round supports d <= 90");
  RoundSetup rs;
  FIRAL_TRY(round_setup(P, zr, rs));
  const double eta = (o && o->eta > 0) ? o->eta : 8.0 * std::sqrt((double)P->D);
  FIRAL_TRY(round_chains(P, rs, b, &eta, 1, sel, stats));
  return read_flags(P->H);
}

// ------------------------------------------------------------------------------------------
// CUDA-graph replay of MD iterations.  One step runs eagerly (it sizes every workspace), the
// next is captured with the step index read from the device counter, and the graph is
// replayed for the remaining iterations.  Only fixed-iteration CG (no host reads) qualifies.
// ------------------------------------------------------------------------------------------
struct StreamSet {
  std::vector<cudaStream_t> st;
  std::vector<cudaEvent_t> ev;
  ~StreamSet() {
    for (auto e : ev) cudaEventDestroy(e);
    for (auto s : st) cudaStreamDestroy(s);
  }
  int32_t make(int n) {
    for (int i = 0; i < n; ++i) {
      cudaStream_t s;
      cudaEvent_t e;
      FIRAL_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
      st.push_back(s);
      FIRAL_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      ev.push_back(e);
    }
    return FIRAL_OK;
  }
};

// Run MD iterations t_begin+1 .. t_end-1 of every problem (step t_begin already run eagerly)
// by capturing one batched iteration into a graph on `cap` and replaying it.
int32_t replay_steps(firal_handle* H, std::vector<firal_problem*>& probs,
                     const std::vector<firal_relax_opts>& opts, const std::vector<double>& budgets,
                     const std::vector<void*>& zs, int32_t t_next, int32_t t_end) {
  if (t_next >= t_end) return FIRAL_OK;
  cudaStream_t user = H->stream;
  const int np = (int)probs.size();
  const int nstreams = np < 64 ? np : 64;
  StreamSet ss;
  FIRAL_TRY(ss.make(nstreams + 1));
  cudaStream_t cap = ss.st[nstreams];
  cudaEvent_t fork = ss.ev[nstreams];
  // device step counters start at t_next; wait for the eager work first
  FIRAL_CUDA_TRY(cudaEventRecord(fork, user));
  FIRAL_CUDA_TRY(cudaStreamWaitEvent(cap, fork, 0));
  for (int p = 0; p < np; ++p) {
    FIRAL_TRY(probs[p]->tdev.ensure(sizeof(int64_t)));
    FIRAL_TRY(set_step(probs[p]->tdev.as<int64_t>(), t_next, cap));
  }
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int32_t rc = FIRAL_OK;
  FIRAL_CUDA_TRY(cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed));
  cudaEventRecord(fork, cap);
  for (int i = 0; i < nstreams; ++i) cudaStreamWaitEvent(ss.st[i], fork, 0);
  for (int p = 0; p < np && rc == FIRAL_OK; ++p) {
    H->stream = ss.st[p % nstreams];
    rc = relax_step_impl(probs[p], &opts[p], 0, budgets[p], zs[p], nullptr, true);
  }
  H->stream = user;
  for (int i = 0; i < nstreams; ++i) {
    cudaEventRecord(ss.ev[i], ss.st[i]);
    cudaStreamWaitEvent(cap, ss.ev[i], 0);
  }
  cudaError_t e = cudaStreamEndCapture(cap, &graph);
  if (rc != FIRAL_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return fail(FIRAL_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return fail(FIRAL_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  for (int t = t_next; t < t_end && e == cudaSuccess; ++t) e = cudaGraphLaunch(exec, cap);
  if (e == cudaSuccess) {
    cudaEventRecord(fork, cap);
    e = cudaStreamWaitEvent(user, fork, 0);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(cap);
  cudaGraphExecDestroy(exec);
  if (e != cudaSuccess) return fail(FIRAL_ERR_CUDA, std::string("graph replay: ") + cudaGetErrorString(e));
  return FIRAL_OK;
}

firal_relax_opts default_relax_opts() {
  firal_relax_opts o;
  o.s = 10;
  o.T = 20;
  o.cg.tol = 0.1;
  o.cg.maxit = 100;
  o.cg.fixed_iters = 0;
  o.cg.block = 0;
  o.cg.reserved = 0;
  o.beta0 = 1.0;
  o.seed = 1;
  o.precision = FIRAL_FP32;
  o.estimator = 0;
  o.md_tol = 0.0;
  return o;
}

// ------------------------------------------------------------------------------------------
// Pooled problems: the pools idx[0..Q) (one padded feature width, one lambda, one storage type)
// stacked into a single problem.  Rows: all labelled rows (pool by pool), then all pool rows
// (pool by pool); classes pool by pool; features padded with zeros to the widest pool; each
// h row holds its pool's probabilities in that pool's class columns and zeros elsewhere, so
// every Hessian, Sigma_z and the preconditioner are block diagonal over pools.
// ------------------------------------------------------------------------------------------
static size_t dtype_size(int32_t dt) {
  return dt == FIRAL_DT_BF16 ? 2 : dt == FIRAL_DT_F32 ? 4 : 8;
}

int32_t pooled_create(firal_handle* H, const std::vector<int>& idx, const firal_pool* pools,
                      const firal_hess0* h0s, const double* budgets, int32_t prec,
                      firal_problem** out) {
  const int Q = (int)idx.size();
  cudaStream_t st = H->stream;
  const firal_pool& p0 = pools[idx[0]];
  const size_t xs = dtype_size(p0.x_dtype), hs = dtype_size(p0.h_dtype);
  int dg = 0;
  int64_t C = 0, M = 0, n = 0;
  std::vector<int> coff(Q + 1), pdim(Q);
  std::vector<int64_t> loff(Q + 1), poff(Q + 1);
  for (int q = 0; q < Q; ++q) {
    const firal_pool& pl = pools[idx[q]];
    FIRAL_TRY(validate_pool(&pl, h0s ? &h0s[idx[q]] : nullptr));
    dg = std::max(dg, (int)pl.d);
    coff[q] = (int)C;
    C += pl.c;
    pdim[q] = pl.d;
    loff[q] = M;
    M += h0s ? h0s[idx[q]].m : 0;
    poff[q] = n;
    n += pl.n;
  }
  coff[Q] = (int)C;
  loff[Q] = M;
  poff[Q] = n;
  if (C > 4096) return fail(FIRAL_ERR_UNSUPPORTED, "pooled classes exceed 4096");
  // stacked inputs (temporaries)
  DBuf Xs, Hs, Xos, Hos;
  auto rel = [&]() {
    Xs.release();
    Hs.release();
    Xos.release();
    Hos.release();
  };
  int32_t rc = FIRAL_OK;
#define TRYP(x)                    \
  do {                             \
    rc = (x);                      \
    if (rc != FIRAL_OK) {          \
      rel();                       \
      return rc;                   \
    }                              \
  } while (0)
#define CUDP(x)                                                           \
  do {                                                                    \
    cudaError_t e_ = (x);                                                 \
    if (e_ != cudaSuccess) {                                              \
      rel();                                                              \
      return fail(FIRAL_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
    }                                                                     \
  } while (0)
  TRYP(Xs.ensure((size_t)n * dg * xs));
  TRYP(Hs.ensure((size_t)n * C * hs));
  CUDP(cudaMemsetAsync(Xs.p, 0, (size_t)n * dg * xs, st));
  CUDP(cudaMemsetAsync(Hs.p, 0, (size_t)n * C * hs, st));
  if (M > 0) {
    TRYP(Xos.ensure((size_t)M * dg * xs));
    TRYP(Hos.ensure((size_t)M * C * hs));
    CUDP(cudaMemsetAsync(Xos.p, 0, (size_t)M * dg * xs, st));
    CUDP(cudaMemsetAsync(Hos.p, 0, (size_t)M * C * hs, st));
  }
  for (int q = 0; q < Q; ++q) {
    const firal_pool& pl = pools[idx[q]];
    CUDP(cudaMemcpy2DAsync((char*)Xs.p + (size_t)poff[q] * dg * xs, dg * xs, pl.X, pl.d * xs,
                           pl.d * xs, pl.n, cudaMemcpyDeviceToDevice, st));
    CUDP(cudaMemcpy2DAsync((char*)Hs.p + ((size_t)poff[q] * C + coff[q]) * hs, C * hs, pl.h,
                           pl.c * hs, pl.c * hs, pl.n, cudaMemcpyDeviceToDevice, st));
    const int64_t mq = loff[q + 1] - loff[q];
    if (mq > 0) {
      const firal_hess0& h0 = h0s[idx[q]];
      CUDP(cudaMemcpy2DAsync((char*)Xos.p + (size_t)loff[q] * dg * xs, dg * xs, h0.Xo,
                             pl.d * xs, pl.d * xs, mq, cudaMemcpyDeviceToDevice, st));
      CUDP(cudaMemcpy2DAsync((char*)Hos.p + ((size_t)loff[q] * C + coff[q]) * hs, C * hs, h0.ho,
                             pl.c * hs, pl.c * hs, mq, cudaMemcpyDeviceToDevice, st));
    }
  }
  firal_pool sp{Xs.p, Hs.p, n, dg, (int32_t)C, p0.x_dtype, p0.h_dtype};
  firal_hess0 sh{Xos.p, Hos.p, M, h0s ? h0s[idx[0]].lambda : 0.0};
  firal_problem* P = nullptr;
  TRYP(problem_create_impl(H, &sp, &sh, prec, &P));
  rel();
#undef TRYP
#undef CUDP
  auto bail = [&](int32_t code) {
    firal_problem_destroy(P);
    return code;
  };
  // pool tables
  std::vector<int> cpool(C);
  for (int q = 0; q < Q; ++q)
    for (int k = coff[q]; k < coff[q + 1]; ++k) cpool[k] = q;
  std::vector<int> tabs;
  tabs.insert(tabs.end(), cpool.begin(), cpool.end());
  tabs.insert(tabs.end(), coff.begin(), coff.end());
  tabs.insert(tabs.end(), pdim.begin(), pdim.end());
  if ((rc = P->pool_tabs.ensure(tabs.size() * sizeof(int))) != FIRAL_OK) return bail(rc);
  cudaError_t e = cudaMemcpyAsync(P->pool_tabs.p, tabs.data(), tabs.size() * sizeof(int),
                                  cudaMemcpyHostToDevice, st);
  P->pt.Q = Q;
  P->pt.cpool = P->pool_tabs.as<int>();
  P->pt.coff = P->pt.cpool + C;
  P->pt.pdim = P->pt.coff + Q + 1;
  // budgets (f64, Q) | pool-row offsets (i64, Q + 1)
  std::vector<double> bz(Q + (Q + 1));
  for (int q = 0; q < Q; ++q) bz[q] = budgets[idx[q]];
  std::memcpy(bz.data() + Q, poff.data(), (Q + 1) * sizeof(int64_t));
  if ((rc = P->pool_z.ensure(bz.size() * sizeof(double))) != FIRAL_OK) return bail(rc);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(P->pool_z.p, bz.data(), bz.size() * sizeof(double), cudaMemcpyHostToDevice,
                        st);
  P->pool_zoff_h = poff;
  // H_p = (1/n_q) sum over pool q's rows, per pool
  for (int q = 0; q < Q && rc == FIRAL_OK; ++q) {
    const int64_t nq = poff[q + 1] - poff[q];
    rc = fill_weights(P->dbl, (char*)P->w_p.p + (size_t)(M + poff[q]) * vsize(P), 0, 0.0, nullptr,
                      1.0 / nq, nq, st);
  }
  if (rc != FIRAL_OK) return bail(rc);
  // K ranges of the tensor-core GEMM tiles (pool of every row: labelled rows, then pool rows)
  const int64_t N = M + n;
  auto pool_of_row = [&](int64_t r) {
    const std::vector<int64_t>& off = r < M ? loff : poff;
    const int64_t x = r < M ? r : r - M;
    return (int)(std::upper_bound(off.begin(), off.end(), x) - off.begin()) - 1;
  };
  if (is_mixed(prec)) {
    const int64_t ntiles = P->Np / 128;
    std::vector<int2> ka(ntiles);
    for (int64_t t = 0; t < ntiles; ++t) {
      int qmin = Q, qmax = -1;
      for (int64_t r = t * 128; r < std::min<int64_t>(N, t * 128 + 128); ++r) {
        const int q = pool_of_row(r);
        qmin = std::min(qmin, q);
        qmax = std::max(qmax, q);
      }
      ka[t] = make_int2(coff[qmin] / 64, (coff[qmax + 1] + 63) / 64);
    }
    const int kbL = (int)((M + 63) / 64);
    P->kbL = kbL;
    auto klist = [&](int width, int ntile, std::vector<int4>& out, int64_t& Lmax) {
      out.resize(ntile);
      Lmax = kbL;
      for (int t = 0; t < ntile; ++t) {
        const int k0 = t * width, k1 = std::min<int64_t>(C, (int64_t)t * width + width);
        int4 v = make_int4(kbL, kbL, kbL, 0);
        if (k0 < k1) {
          const int qa = cpool[k0], qb = cpool[k1 - 1];
          const int64_t lo = (M + poff[qa]) / 64, hi = (M + poff[qb + 1] + 63) / 64;
          const int64_t lo2 = std::max<int64_t>(lo, kbL);
          v = make_int4((int)lo2, (int)hi, (int)(kbL + std::max<int64_t>(0, hi - lo2)), 0);
        }
        out[t] = v;
        Lmax = std::max<int64_t>(Lmax, v.z);
      }
    };
    std::vector<int4> kd, kbs;
    klist(256, (P->cp + 255) / 256, kd, P->kr_dterm_Lmax);
    klist(128, (P->cp + 127) / 128, kbs, P->kr_bsum_Lmax);
    if ((rc = P->kr_alpha.ensure(ka.size() * sizeof(int2))) != FIRAL_OK ||
        (rc = P->kr_dterm.ensure(kd.size() * sizeof(int4))) != FIRAL_OK ||
        (rc = P->kr_bsum.ensure(kbs.size() * sizeof(int4))) != FIRAL_OK)
      return bail(rc);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(P->kr_alpha.p, ka.data(), ka.size() * sizeof(int2),
                          cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(P->kr_dterm.p, kd.data(), kd.size() * sizeof(int4),
                          cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(P->kr_bsum.p, kbs.data(), kbs.size() * sizeof(int4),
                          cudaMemcpyHostToDevice, st);
    // pools of at most 32 classes (and dp <= 64): the fused per-point apply
    if (e == cudaSuccess && (rc = tc_setup_pw(P, coff, loff, poff)) != FIRAL_OK) return bail(rc);
  }
  // the host vectors above are read by the copies: wait for them before they go out of scope
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return bail(fail(FIRAL_ERR_CUDA, cudaGetErrorString(e)));
  *out = P;
  return FIRAL_OK;
}

// Batched Relax over pooled problems: pools grouped by padded feature width, lambda and storage
// types (at most 4096 classes per group); each group is one problem whose MD iterations are
// replayed, together with the other groups', from one CUDA graph.
int32_t replay_steps(firal_handle* H, std::vector<firal_problem*>& probs,
                     const std::vector<firal_relax_opts>& opts, const std::vector<double>& budgets,
                     const std::vector<void*>& zs, int32_t t_next, int32_t t_end);

int32_t batched_pooled(firal_handle* H, int32_t nq, const firal_pool* pools,
                       const firal_hess0* hess0s, const double* budgets,
                       const firal_relax_opts* opts, void* const* z_outs) {
  const firal_relax_opts& o = *opts;
  cudaStream_t st = H->stream;
  for (int q = 0; q < nq; ++q) {
    if (!z_outs[q] || !(budgets[q] > 0)) return fail(FIRAL_ERR_ARG, "bad z_out or budget");
    FIRAL_TRY(validate_pool(&pools[q], hess0s ? &hess0s[q] : nullptr));
  }
  // groups
  std::map<std::tuple<int, double, int, int>, std::vector<std::vector<int>>> groups;
  for (int q = 0; q < nq; ++q) {
    int dp = 16;
    while (dp < pools[q].d) dp <<= 1;
    auto& g = groups[std::make_tuple(dp, hess0s ? hess0s[q].lambda : 0.0, pools[q].x_dtype,
                                     pools[q].h_dtype)];
    int cl = 0;
    if (!g.empty())
      for (int i : g.back()) cl += pools[i].c;
    if (g.empty() || cl + pools[q].c > 4096) g.emplace_back();
    g.back().push_back(q);
  }
  std::vector<firal_problem*> probs;
  std::vector<std::vector<int>> members;
  std::vector<DBuf> zcat;
  auto destroy_all = [&]() {
    for (auto* p : probs) firal_problem_destroy(p);
    for (auto& z : zcat) z.release();
  };
  int32_t rc = FIRAL_OK;
  for (auto& kv : groups)
    for (auto& idx : kv.second) {
      firal_problem* P = nullptr;
      rc = pooled_create(H, idx, pools, hess0s, budgets, o.precision, &P);
      if (rc != FIRAL_OK) {
        destroy_all();
        return rc;
      }
      probs.push_back(P);
      members.push_back(idx);
    }
  const int G = (int)probs.size();
  zcat.resize(G);
  std::vector<void*> zs(G);
  for (int g = 0; g < G && rc == FIRAL_OK; ++g) {
    firal_problem* P = probs[g];
    rc = zcat[g].ensure((size_t)P->n * vsize(P));
    // z starts at b_q / n_q on every pool (the uniform point of each simplex)
    for (size_t i = 0; i < members[g].size() && rc == FIRAL_OK; ++i) {
      const int q = members[g][i];
      const int64_t a = P->pool_zoff_h[i], b = P->pool_zoff_h[i + 1];
      rc = fill_weights(P->dbl, (char*)zcat[g].p + a * vsize(P), 0, 0.0, nullptr,
                        budgets[q] / (double)(b - a), b - a, st);
    }
    zs[g] = zcat[g].p;
  }
  std::vector<firal_relax_opts> os(G, o);
  std::vector<double> ones(G, 1.0);   // pooled problems take each pool's budget from their table
  for (int g = 0; g < G && rc == FIRAL_OK && o.T > 0; ++g)
    rc = relax_step_impl(probs[g], &o, 0, 1.0, zs[g], nullptr);
  if (rc == FIRAL_OK && o.T > 1) rc = replay_steps(H, probs, os, ones, zs, 1, o.T);
  // scatter each pool's z back to the caller's buffer
  for (int g = 0; g < G && rc == FIRAL_OK; ++g) {
    firal_problem* P = probs[g];
    for (size_t i = 0; i < members[g].size() && rc == FIRAL_OK; ++i) {
      const int q = members[g][i];
      const int64_t a = P->pool_zoff_h[i], b = P->pool_zoff_h[i + 1];
      const cudaError_t e = cudaMemcpyAsync(z_outs[q], (char*)zs[g] + a * vsize(P),
                                            (b - a) * vsize(P), cudaMemcpyDeviceToDevice, st);
      if (e != cudaSuccess) rc = fail(FIRAL_ERR_CUDA, cudaGetErrorString(e));
    }
  }
  if (rc == FIRAL_OK) {
    const cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = fail(FIRAL_ERR_CUDA, cudaGetErrorString(e));
  }
  if (rc == FIRAL_OK) rc = read_flags(H);
  destroy_all();
  return rc;
}

// min_k lambda_min of the block-diagonal Hessian sum of the selected points (eta criterion)
int32_t selected_min_eig(firal_problem* P, const int32_t* sel, int32_t b, double* out) {
  cudaStream_t st = P->H->stream;
  const int c = P->c, d = P->d;
  const size_t blk = (size_t)c * d * d;
  DBuf Hs, Lid, eig;
  auto rel = [&]() {
    Hs.release();
    Lid.release();
    eig.release();
  };
  int32_t rc = FIRAL_OK;
  if ((rc = Hs.ensure(blk * 8)) != FIRAL_OK || (rc = Lid.ensure(blk * 8)) != FIRAL_OK ||
      (rc = eig.ensure((size_t)c * d * 8)) != FIRAL_OK) {
    rel();
    return rc;
  }
  if (rc == FIRAL_OK) rc = selected_weights(P, sel, b, st);
  // FP64/FP32 SIMT block sums (not the bf16 tensor-core ones: the smallest eigenvalue of a
  // sum of b rank-one terms needs the full precision)
  if (rc == FIRAL_OK) rc = syrk_blocks(P, P->zsave.p, 0.0, nullptr, 0.0, Hs.as<double>());
  if (rc == FIRAL_OK) rc = identity_blocks(Lid.as<double>(), c, d, st);
  if (rc == FIRAL_OK) rc = tilde_eigvals(Lid.as<double>(), Hs.as<double>(), c, d, eig.as<double>(), st);
  if (rc == FIRAL_OK) {
    std::vector<double> h((size_t)c * d);
    cudaError_t e = cudaMemcpyAsync(h.data(), eig.p, h.size() * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = fail(FIRAL_ERR_CUDA, cudaGetErrorString(e));
    else *out = *std::min_element(h.begin(), h.end());
  }
  rel();
  return rc;
}

int32_t round_sweep_impl(firal_problem* P, const void* zr, int32_t b, const double* etas,
                         int32_t neta, const firal_round_opts* o, int32_t* sel, double* crit,
                         int32_t* best) {
  if (!P || !zr || !sel || !etas || !crit || !best)
    return fail(FIRAL_ERR_ARG, "problem, z, etas, selected_out, criteria and best must be non-null");
  if (neta < 1 || neta > 64) return fail(FIRAL_ERR_ARG, "n_eta must be in [1, 64]");
  for (int e = 0; e < neta; ++e)
    if (!(etas[e] > 0)) return fail(FIRAL_ERR_ARG, "every eta must be > 0");
  if (b < 1 || b > P->n) return fail(FIRAL_ERR_ARG, "budget must be in [1, n]");
  if (sharded(P)) return fail(FIRAL_ERR_UNSUPPORTED, "Round does not take a row-sharded problem");
  if (P->dbl && P->d > 90) return fail(FIRAL_ERR_UNSUPPORTED, "FP64 Round supports d <= 90");
  // the eta-independent set-up once, then one chain per eta
  RoundSetup rs;
  FIRAL_TRY(round_setup(P, zr, rs));
  // the chains of up to 8 values of eta side by side (one score launch per pick for all)
  for (int e0 = 0; e0 < neta; e0 += 8) {
    const int ne = std::min(8, neta - e0);
    FIRAL_TRY(round_chains(P, rs, b, etas + e0, ne, sel + (size_t)e0 * b, nullptr));
  }
  for (int e = 0; e < neta; ++e) FIRAL_TRY(selected_min_eig(P, sel + (size_t)e * b, b, &crit[e]));
  int bi = 0;
  for (int e = 1; e < neta; ++e)
    if (crit[e] > crit[bi]) bi = e;
  *best = bi;
  return read_flags(P->H);
}

}  // namespace

// =========================================================================================
// C-ABI
// =========================================================================================
extern "C" {

const char* firal_status_string(int32_t s) {
  switch (s) {
    case FIRAL_OK: return "FIRAL_OK";
    case FIRAL_ERR_ARG: return "FIRAL_ERR_ARG";
    case FIRAL_ERR_CUDA: return "FIRAL_ERR_CUDA";
    case FIRAL_ERR_NOT_SPD: return "FIRAL_ERR_NOT_SPD";
    case FIRAL_ERR_CG_NOT_CONVERGED: return "FIRAL_ERR_CG_NOT_CONVERGED";
    case FIRAL_ERR_NONFINITE: return "FIRAL_ERR_NONFINITE";
    case FIRAL_ERR_TIMEOUT: return "FIRAL_ERR_TIMEOUT";
    case FIRAL_ERR_NOMEM: return "FIRAL_ERR_NOMEM";
    case FIRAL_ERR_UNSUPPORTED: return "FIRAL_ERR_UNSUPPORTED";
    case FIRAL_ERR_COMM: return "FIRAL_ERR_COMM";
    default: return "FIRAL_ERR_UNKNOWN";
  }
}

int32_t firal_build_info(void) { return 1 | (tc_available() ? 2 : 0); }

int64_t firal_launch_count(void) { return g_launches.load(); }

int32_t firal_profile(int32_t enable) {
  Profiler& P = prof();
  std::lock_guard<std::mutex> g(P.mu);
  P.drain();
  for (int i = 0; i < PF_COUNT; ++i) {
    P.ms[i] = 0.0;
    P.calls[i] = 0;
  }
  P.on = enable != 0;
  return FIRAL_OK;
}

int32_t firal_profile_read(double* ms_out, int64_t* calls_out, int32_t count) {
  if (count < 0) return FIRAL_ERR_ARG;
  Profiler& P = prof();
  std::lock_guard<std::mutex> g(P.mu);
  P.drain();
  for (int i = 0; i < count && i < PF_COUNT; ++i) {
    if (ms_out) ms_out[i] = P.ms[i];
    if (calls_out) calls_out[i] = P.calls[i];
  }
  return PF_COUNT;
}

const char* firal_profile_name(int32_t id) {
  static const char* names[PF_COUNT] = {"prep", "probes", "syrk_blocks", "chol_inv",
                                        "apply_alpha", "apply_dterm", "apply_combine", "cg_vec",
                                        "quad_forms", "md_step", "dot", "round",
                                        "apply_split", "exact_build", "exact_factor",
                                        "exact_gemm", "exact_quad", "exact_score",
                                        "lr_refit"};
  return (id >= 0 && id < PF_COUNT) ? names[id] : "unknown";
}

int32_t firal_create(firal_handle** out, void* stream) {
  if (!out) return fail(FIRAL_ERR_ARG, "out must be non-null");
  auto* H = new firal_handle();
  cudaError_t e = cudaGetDevice(&H->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&H->sm_count, cudaDevAttrMultiProcessorCount, H->device);
  if (e != cudaSuccess) {
    delete H;
    return fail(FIRAL_ERR_CUDA, cudaGetErrorString(e));
  }
  H->stream = (cudaStream_t)stream;
  int32_t rc = H->flags.ensure(sizeof(DevFlags));
  if (rc == FIRAL_OK) rc = H->scratch.ensure(4096);
  if (rc != FIRAL_OK) {
    delete H;
    return rc;
  }
  e = cudaMemsetAsync(H->flags.p, 0, sizeof(DevFlags), H->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(H->stream);
  if (e != cudaSuccess) {
    H->flags.release();
    H->scratch.release();
    delete H;
    return fail(FIRAL_ERR_CUDA, cudaGetErrorString(e));
  }
  *out = H;
  return FIRAL_OK;
}

int32_t firal_destroy(firal_handle* H) {
  if (!H) return FIRAL_OK;
  cudaStreamSynchronize(H->stream);
  H->flags.release();
  H->scratch.release();
  delete H;
  return FIRAL_OK;
}

int32_t firal_set_stream(firal_handle* H, void* stream) {
  if (!H) return fail(FIRAL_ERR_ARG, "handle must be non-null");
  H->stream = (cudaStream_t)stream;
  return FIRAL_OK;
}

int32_t firal_last_error(firal_handle* H, char* buf, size_t len) {
  if (!buf || len == 0) return FIRAL_ERR_ARG;
  const std::string& s = H ? H->err : last_detail();
  std::strncpy(buf, s.c_str(), len - 1);
  buf[len - 1] = 0;
  return FIRAL_OK;
}

int32_t firal_problem_create(firal_handle* H, const firal_pool* pool, const firal_hess0* h0,
                             int32_t precision, firal_problem** out) {
  return record(H, problem_create_impl(H, pool, h0, precision, out));
}

int32_t firal_problem_destroy(firal_problem* P) {
  if (!P) return FIRAL_OK;
  // every kernel of the problem ran on the handle's stream (graph replays join it before
  // returning): after this synchronisation its buffers can be parked for reuse
  const bool synced = cudaStreamSynchronize(P->H->stream) == cudaSuccess;
  exact_release(P);
  for (DBuf* b : {&P->Xa, &P->Ha, &P->HaT, &P->w_sig, &P->w_p, &P->S_p, &P->S_sig, &P->Pblk,
                  &P->Minv, &P->HoBlk, &P->walpha, &P->Dpart, &P->syrk_part, &P->cgX, &P->cgR,
                  &P->cgP, &P->cgQ, &P->cgZ, &P->cgcols, &P->cgpart1, &P->cgpart2, &P->V, &P->U,
                  &P->W, &P->HU, &P->g, &P->red, &P->zsave, &P->Xb, &P->Hb, &P->HbT, &P->Pb, &P->vmean, &P->qmean, &P->Aw, &P->Zp, &P->Hlo, &P->gq_ab,
                  &P->gq_m, &P->gq_part, &P->rtab, &P->rM, &P->tdev, &P->cen, &P->cen_off,
                  &P->cen_idx, &P->Ub, &P->UbT, &P->cen_am, &P->cen_rho, &P->cen_lab, &P->cen_items, &P->cen_part,
                  &P->pool_tabs, &P->pool_z, &P->md_part, &P->kr_alpha, &P->kr_dterm,
                  &P->kr_bsum, &P->bcg, &P->pw_pool, &P->pw_seg, &P->pw_pseg, &P->pw_pk,
                  &P->pw_part, &P->X64, &P->S_lab, &P->w_lab, &P->cm_scr}) {
    if (synced) b->park();
    else b->release();
  }
  for (auto& sc : P->pw_sched) {
    if (synced) sc.buf.park();
    else sc.buf.release();
  }
  delete P;
  return FIRAL_OK;
}

int32_t firal_relax_step(firal_problem* P, const firal_relax_opts* o, int32_t t, double budget,
                         void* z, firal_step_stats* stats) {
  return record(P ? P->H : nullptr, relax_step_impl(P, o, t, budget, z, stats));
}

int32_t firal_relax(firal_handle* H, const firal_pool* pool, const firal_hess0* h0, double budget,
                    const void* z0, const firal_relax_opts* opts, void* z_out, double* fhat_hist,
                    firal_relax_stats* stats) {
  if (!H || !z_out) return record(H, fail(FIRAL_ERR_ARG, "handle and z_out must be non-null"));
  firal_relax_opts o = opts ? *opts : default_relax_opts();
  if (o.T < 0) return record(H, fail(FIRAL_ERR_ARG, "T must be >= 0"));
  firal_problem* P = nullptr;
  int32_t rc = problem_create_impl(H, pool, h0, o.precision, &P);
  if (rc != FIRAL_OK) return record(H, rc);
  const size_t vs = P->dbl ? 8 : 4;
  if (z0) {
    rc = cudaMemcpyAsync(z_out, z0, P->n * vs, cudaMemcpyDeviceToDevice, H->stream) == cudaSuccess
             ? FIRAL_OK
             : fail(FIRAL_ERR_CUDA, "copy of z0 failed");
  } else {
    rc = fill_weights(P->dbl, z_out, 0, 0.0, nullptr, budget / P->n, P->n, H->stream);
  }
  firal_step_stats ss{};
  const bool need_stats = fhat_hist || stats || o.md_tol > 0;
  int it = 0, cg_total = 0;
  double prev = 0.0, last = 0.0;
  if (rc == FIRAL_OK && !need_stats && o.cg.fixed_iters > 0 && o.T > 1) {
    // first iteration eagerly, the rest replayed from a CUDA graph
    rc = relax_step_impl(P, &o, 0, budget, z_out, nullptr);
    std::vector<firal_problem*> ps{P};
    std::vector<firal_relax_opts> os{o};
    std::vector<double> bs{budget};
    std::vector<void*> zs{z_out};
    if (rc == FIRAL_OK) rc = replay_steps(H, ps, os, bs, zs, 1, o.T);
    it = o.T;
  }
  for (; rc == FIRAL_OK && it < o.T; ++it) {
    rc = relax_step_impl(P, &o, it, budget, z_out, need_stats ? &ss : nullptr);
    if (rc != FIRAL_OK) break;
    if (need_stats) {
      if (fhat_hist) fhat_hist[it] = ss.fhat;
      cg_total += ss.cg_iters[0] + ss.cg_iters[1];
      last = ss.fhat;
      if (o.md_tol > 0 && it > 0 && std::fabs(ss.fhat - prev) <= o.md_tol * std::fabs(prev)) {
        ++it;
        break;
      }
      prev = ss.fhat;
    }
  }
  if (rc == FIRAL_OK) rc = read_flags(H);
  if (stats) {
    stats->iters_done = it;
    stats->fhat_last = last;
    stats->cg_iters_total = cg_total;
  }
  firal_problem_destroy(P);
  return record(H, rc);
}

int32_t firal_batched_relax(firal_handle* H, int32_t nproblems, const firal_pool* pools,
                            const firal_hess0* hess0s, const double* budgets,
                            const firal_relax_opts* opts, void* const* z_outs) {
  if (!H || nproblems < 1 || !pools || !budgets || !opts || !z_outs)
    return record(H, fail(FIRAL_ERR_ARG, "bad batched_relax arguments"));
  const firal_relax_opts& o = *opts;
  if (is_mixed(o.precision) && o.cg.fixed_iters > 0 && nproblems > 1)
    return record(H, batched_pooled(H, nproblems, pools, hess0s, budgets, opts, z_outs));
  std::vector<firal_problem*> probs(nproblems, nullptr);
  auto destroy_all = [&]() {
    for (auto* p : probs) firal_problem_destroy(p);
  };
  int32_t rc = FIRAL_OK;
  for (int p = 0; p < nproblems && rc == FIRAL_OK; ++p) {
    if (!z_outs[p] || !(budgets[p] > 0)) rc = fail(FIRAL_ERR_ARG, "bad z_out or budget");
    if (rc == FIRAL_OK)
      rc = problem_create_impl(H, &pools[p], hess0s ? &hess0s[p] : nullptr, o.precision, &probs[p]);
    if (rc == FIRAL_OK)
      rc = fill_weights(probs[p]->dbl, z_outs[p], 0, 0.0, nullptr, budgets[p] / probs[p]->n,
                        probs[p]->n, H->stream);
  }
  std::vector<firal_relax_opts> os(nproblems, o);
  std::vector<double> bs(budgets, budgets + nproblems);
  std::vector<void*> zs(z_outs, z_outs + nproblems);
  // iteration 0 eagerly (sizes the workspaces), on the handle's stream
  for (int p = 0; p < nproblems && rc == FIRAL_OK && o.T > 0; ++p)
    rc = relax_step_impl(probs[p], &o, 0, bs[p], zs[p], nullptr);
  if (rc == FIRAL_OK && o.T > 1) {
    if (o.cg.fixed_iters > 0) {
      rc = replay_steps(H, probs, os, bs, zs, 1, o.T);
    } else {
      for (int t = 1; t < o.T && rc == FIRAL_OK; ++t)
        for (int p = 0; p < nproblems && rc == FIRAL_OK; ++p)
          rc = relax_step_impl(probs[p], &o, t, bs[p], zs[p], nullptr);
    }
  }
  if (rc == FIRAL_OK) rc = read_flags(H);
  destroy_all();
  return record(H, rc);
}

int32_t firal_round_problem(firal_problem* P, const void* zr, int32_t b,
                            const firal_round_opts* o, int32_t* sel, firal_round_stats* stats) {
  return record(P ? P->H : nullptr, round_impl(P, zr, b, o, sel, stats));
}

int32_t firal_round_sweep(firal_problem* P, const void* zr, int32_t b, const double* etas,
                          int32_t neta, const firal_round_opts* o, int32_t* sel, double* crit,
                          int32_t* best) {
  return record(P ? P->H : nullptr, round_sweep_impl(P, zr, b, etas, neta, o, sel, crit, best));
}

int32_t firal_round(firal_handle* H, const firal_pool* pool, const firal_hess0* h0,
                    const void* zr, int32_t b, const firal_round_opts* o, int32_t* sel,
                    firal_round_stats* stats) {
  const int32_t prec = o ? o->precision : FIRAL_FP32;
  firal_problem* P = nullptr;
  int32_t rc = problem_create_impl(H, pool, h0, prec, &P);
  if (rc != FIRAL_OK) return record(H, rc);
  rc = round_impl(P, zr, b, o, sel, stats);
  firal_problem_destroy(P);
  return record(H, rc);
}

int32_t firal_probes(firal_problem* P, uint64_t seed, int32_t t, int32_t s, void* V) {
  if (!P || !V || s < 1 || t < 0) return record(P ? P->H : nullptr, fail(FIRAL_ERR_ARG, "bad probe arguments"));
  return record(P->H, probes(P->dbl, V, seed, t, s, P->D, P->H->stream));
}

int32_t firal_hessian_apply(firal_problem* P, int32_t op, const void* z, const void* V, int32_t s,
                            void* out) {
  firal_handle* H = P ? P->H : nullptr;
  if (!P || !V || !out || s < 1 || (op == 0 && !z) || op < 0 || op > 1)
    return record(H, fail(FIRAL_ERR_ARG, "bad hessian_apply arguments"));
  if (V == out) return record(H, fail(FIRAL_ERR_ARG, "out must not alias V"));
  int32_t rc;
  if (op == 0) {
    rc = setup_sigma(P, z, false);
    if (rc == FIRAL_OK) rc = apply(P, P->w_sig.p, P->S_sig.p, V, s, out, nullptr);
  } else {
    rc = ensure_sp(P);
    if (rc == FIRAL_OK) rc = apply(P, P->w_p.p, P->S_p.p, V, s, out, nullptr);
  }
  return record(H, rc);
}

int32_t firal_precond_blocks(firal_problem* P, const void* z, double* out) {
  firal_handle* H = P ? P->H : nullptr;
  if (!P || !out) return record(H, fail(FIRAL_ERR_ARG, "bad precond_blocks arguments"));
  cudaStream_t st = P->H->stream;
  int32_t rc = fill_weights(P->dbl, P->zsave.p, P->m, 1.0, z, 0.0, P->n, st);
  if (rc == FIRAL_OK) rc = syrk_blocks(P, P->zsave.p, 0.0, nullptr, P->lambda, out);
  return record(H, rc);
}

int32_t firal_pcg(firal_problem* P, const void* z, const void* B, int32_t s,
                  const firal_cg_opts* cg, void* X_out, int32_t* iters_out, double* relres_out) {
  firal_handle* H = P ? P->H : nullptr;
  if (!P || !z || !B || !X_out || !cg || s < 1)
    return record(H, fail(FIRAL_ERR_ARG, "bad pcg arguments"));
  int32_t rc = setup_sigma(P, z, true);
  CGResult res;
  std::vector<CGCol> cols;
  const bool want = iters_out || relres_out;
  if (rc == FIRAL_OK) rc = pcg_run(P, B, s, *cg, X_out, want, &res, &cols);
  if (rc == FIRAL_OK && want) {
    for (int j = 0; j < s; ++j) {
      if (iters_out) iters_out[j] = cols[j].iters;
      if (relres_out) relres_out[j] = cols[j].relres;
    }
    rc = read_flags(P->H);
    if (rc == FIRAL_OK && cg->fixed_iters <= 0 && !res.converged)
      rc = fail(FIRAL_ERR_CG_NOT_CONVERGED, "PCG reached maxit above tolerance");
  }
  return record(H, rc);
}

int32_t firal_quad_forms(firal_problem* P, const void* A, const void* B, int32_t s, double scale,
                         void* g) {
  firal_handle* H = P ? P->H : nullptr;
  if (!P || !A || !B || !g || s < 1) return record(H, fail(FIRAL_ERR_ARG, "bad quad_forms arguments"));
  return record(H, quad(P, A, B, s, scale, g));
}

int32_t firal_md_step(firal_problem* P, void* z, const void* g, double budget, double beta0) {
  firal_handle* H = P ? P->H : nullptr;
  if (!P || !z || !g || !(budget > 0)) return record(H, fail(FIRAL_ERR_ARG, "bad md_step arguments"));
  return record(H, md_step_simt(P->dbl, z, g, P->n, budget, beta0, P->red.as<double>(),
                                P->H->stream));
}

int32_t firal_objective_fwd(firal_problem* P, const void* z, uint64_t seed, int32_t t, int32_t s,
                            const firal_cg_opts* cg, double* fhat_out, void* U_out, void* Y_out) {
  firal_handle* H = P ? P->H : nullptr;
  if (!P || !z || !cg || !fhat_out || s < 1 || s > 128)
    return record(H, fail(FIRAL_ERR_ARG, "bad objective_fwd arguments"));
  cudaStream_t st = P->H->stream;
  const size_t vs = vsize(P);
  const int64_t sD = (int64_t)s * P->D;
  int32_t rc = FIRAL_OK;
#define TRYF(x)                          \
  do {                                   \
    rc = (x);                            \
    if (rc != FIRAL_OK) return record(H, rc); \
  } while (0)
  TRYF(P->V.ensure(2 * sD * vs));
  TRYF(P->U.ensure(2 * sD * vs));
  TRYF(P->HU.ensure(2 * sD * vs));
  TRYF(probes(P->dbl, P->V.p, seed, t, s, P->D, st));
  TRYF(setup_sigma(P, z, true));
  TRYF(ensure_sp(P));
  // right-hand sides [V, H_p V] solved together as one 2s-column PCG
  FIRAL_CUDA_TRY(cudaMemcpyAsync(P->HU.p, P->V.p, sD * vs, cudaMemcpyDeviceToDevice, st));
  TRYF(apply(P, P->w_p.p, P->S_p.p, P->V.p, s, (char*)P->HU.p + sD * vs, nullptr));
  CGResult res;
  TRYF(pcg_run(P, P->HU.p, 2 * s, *cg, P->U.p, true, &res, nullptr));
  double* red = P->red.as<double>();
  // f^ = (1/s) sum_j <H_p v_j, u_j>
  TRYF(dot_scaled(P->dbl, (char*)P->HU.p + sD * vs, P->U.p, sD, 1.0 / s, red + 1024, red + 1536,
                  st));
  FIRAL_CUDA_TRY(cudaMemcpyAsync(fhat_out, red + 1536, 8, cudaMemcpyDeviceToHost, st));
  if (U_out) FIRAL_CUDA_TRY(cudaMemcpyAsync(U_out, P->U.p, sD * vs, cudaMemcpyDeviceToDevice, st));
  if (Y_out)
    FIRAL_CUDA_TRY(cudaMemcpyAsync(Y_out, (char*)P->U.p + sD * vs, sD * vs,
                                   cudaMemcpyDeviceToDevice, st));
  FIRAL_CUDA_TRY(cudaStreamSynchronize(st));
#undef TRYF
  return record(H, read_flags(P->H));
}

int32_t firal_objective_bwd(firal_problem* P, const void* z, uint64_t seed, int32_t t, int32_t s,
                            const firal_cg_opts* cg, const void* U, const void* Y, double grad_out,
                            void* g_out) {
  firal_handle* H = P ? P->H : nullptr;
  if (!P || !g_out || s < 1) return record(H, fail(FIRAL_ERR_ARG, "bad objective_bwd arguments"));
  if ((U == nullptr) != (Y == nullptr))
    return record(H, fail(FIRAL_ERR_ARG, "pass both U and Y, or neither"));
  if (U) return record(H, quad(P, U, Y, s, grad_out, g_out));
  // recompute the probe solves
  double fh = 0.0;
  int32_t rc = firal_objective_fwd(P, z, seed, t, s, cg, &fh, nullptr, nullptr);
  if (rc != FIRAL_OK) return rc;
  const size_t off = (size_t)s * P->D * vsize(P);
  return record(H, quad(P, P->U.p, (char*)P->U.p + off, s, grad_out, g_out));
}

int32_t firal_block_eigvals(firal_handle* H, int32_t c, int32_t d, const double* Sig,
                            const double* Hm, double* eig) {
  if (!H || !Sig || !Hm || !eig || c < 1 || d < 1 || d > 128)
    return record(H, fail(FIRAL_ERR_ARG, "bad block_eigvals arguments"));
  DBuf L;
  int32_t rc = L.ensure((size_t)c * d * d * 8);
  if (rc == FIRAL_OK)
    rc = chol_inv(true, Sig, c, d, nullptr, nullptr, L.as<double>(), not_spd_flag(H), H->stream);
  if (rc == FIRAL_OK) rc = tilde_eigvals(L.as<double>(), Hm, c, d, eig, H->stream);
  if (rc == FIRAL_OK) rc = read_flags(H);
  L.release();
  return record(H, rc);
}

int32_t firal_nu_bisect(firal_handle* H, const double* mu, int64_t count, double* nu_out) {
  if (!H || !mu || !nu_out || count < 1) return record(H, fail(FIRAL_ERR_ARG, "bad nu arguments"));
  int32_t rc = nu_bisect_dev(mu, count, 1.0, H->scratch.as<double>(), H->stream);
  if (rc == FIRAL_OK) {
    if (cudaMemcpyAsync(nu_out, H->scratch.p, 8, cudaMemcpyDeviceToHost, H->stream) != cudaSuccess ||
        cudaStreamSynchronize(H->stream) != cudaSuccess)
      rc = fail(FIRAL_ERR_CUDA, "nu readback failed");
  }
  return record(H, rc);
}

}  // extern "C"

// ------------------------------------------------------------------------------------------
// Exact-FIRAL (Algorithm 1) on dense d~ x d~ matrices
// ------------------------------------------------------------------------------------------
namespace firal {
namespace {
constexpr int64_t kExactMaxDim = 16384;
int32_t exact_check(firal_problem* P) {
  if (!P) return fail(FIRAL_ERR_ARG, "problem must be non-null");
  if (P->pt.Q) return fail(FIRAL_ERR_UNSUPPORTED, "Exact-FIRAL does not take pooled problems");
  if (sharded(P)) return fail(FIRAL_ERR_UNSUPPORTED, "Exact-FIRAL does not take a row-sharded problem");
  if (P->D > kExactMaxDim) return fail(FIRAL_ERR_UNSUPPORTED, "Exact-FIRAL needs d c <= 16384");
  return FIRAL_OK;
}
}  // namespace
}  // namespace firal

int32_t firal_exact_objective(firal_problem* P, const void* z, double* f_out, void* g_out) {
  firal_handle* H = P ? P->H : nullptr;
  int32_t rc = exact_check(P);
  if (rc == FIRAL_OK && !z) rc = fail(FIRAL_ERR_ARG, "z must be non-null");
  if (rc == FIRAL_OK) rc = exact_objective(P, z, f_out, g_out);
  return record(H, rc);
}

int32_t firal_exact_relax(firal_problem* P, double budget, int32_t T, double beta0,
                          const void* z0, void* z_out, double* f_hist) {
  firal_handle* H = P ? P->H : nullptr;
  int32_t rc = exact_check(P);
  if (rc == FIRAL_OK && (!z_out || !(budget > 0) || T < 0 || !(beta0 > 0)))
    rc = fail(FIRAL_ERR_ARG, "bad exact_relax arguments");
  if (rc == FIRAL_OK) rc = exact_relax(P, budget, T, beta0, z0, z_out, f_hist);
  if (rc == FIRAL_OK) {
    cudaError_t e = cudaStreamSynchronize(P->H->stream);
    if (e != cudaSuccess) rc = fail(FIRAL_ERR_CUDA, cudaGetErrorString(e));
  }
  return record(H, rc);
}

int32_t firal_exact_round(firal_problem* P, const void* z_relaxed, int32_t budget, double eta,
                          int32_t exclude_selected, int32_t* selected_out, double* r_out,
                          double* nu_out) {
  firal_handle* H = P ? P->H : nullptr;
  int32_t rc = exact_check(P);
  if (rc == FIRAL_OK && (!z_relaxed || !selected_out))
    rc = fail(FIRAL_ERR_ARG, "z_relaxed and selected_out must be non-null");
  if (rc == FIRAL_OK && (budget < 1 || budget > P->n))
    rc = fail(FIRAL_ERR_ARG, "budget must be in [1, n]");
  if (rc == FIRAL_OK && P->c > 112)
    rc = fail(FIRAL_ERR_UNSUPPORTED, "exact Round needs c <= 112");
  if (rc == FIRAL_OK) {
    const double e = eta > 0 ? eta : 8.0 * std::sqrt((double)P->D);
    int evals = 0;
    rc = exact_round(P, z_relaxed, budget, e, exclude_selected ? 1 : 0, selected_out, r_out,
                     nu_out, &evals);
  }
  if (rc == FIRAL_OK) {
    cudaError_t e = cudaStreamSynchronize(P->H->stream);
    if (e != cudaSuccess) rc = fail(FIRAL_ERR_CUDA, cudaGetErrorString(e));
  }
  return record(H, rc);
}

// ------------------------------------------------------------------------------------------
// Active learning (the outer loop of Section 5): classifier refit and the round driver
// ------------------------------------------------------------------------------------------
namespace {

int32_t labels_in_range(const int32_t* y, int64_t m, int c, cudaStream_t st) {
  if (m <= 0) return FIRAL_OK;
  std::vector<int32_t> hy((size_t)m);
  FIRAL_CUDA_TRY(cudaMemcpyAsync(hy.data(), y, (size_t)m * sizeof(int32_t),
                                 cudaMemcpyDeviceToHost, st));
  FIRAL_CUDA_TRY(cudaStreamSynchronize(st));
  for (int32_t v : hy)
    if (v < 0 || v >= c) return fail(FIRAL_ERR_ARG, "labels must lie in [0, c)");
  return FIRAL_OK;
}

// Damped Newton for W = argmin sum_i -log softmax(W x_i)_{y_i} + (gamma / 2) ||W||^2 on the
// labelled rows Xv (m x d, vec type).  Each step solves (sum_i H_i(W) + gamma I) dW = grad
// with the block-Jacobi PCG (a problem whose pool is the labelled set with unit weights),
// then backtracks along -dW until the Armijo condition holds.
int32_t lr_fit_impl(firal_handle* H, const void* Xv, const int32_t* y, int64_t m, int d, int c,
                    double gamma, bool dbl, int max_newton, double tol, void* W, int* iters_out,
                    double* gnorm_out) {
  cudaStream_t st = H->stream;
  const size_t vs = dbl ? 8 : 4;
  const int64_t D = (int64_t)c * d;
  DBuf h, R, g, dW, Wt, ones, part;
  auto rel = [&] {
    for (DBuf* b : {&h, &R, &g, &dW, &Wt, &ones, &part}) b->release();
  };
  int32_t rc = FIRAL_OK;
#define TRYL(x)          \
  do {                   \
    rc = (x);            \
    if (rc != FIRAL_OK) { \
      rel();             \
      return rc;         \
    }                    \
  } while (0)
  TRYL(h.ensure((size_t)m * c * vs));
  TRYL(R.ensure((size_t)m * c * vs));
  TRYL(g.ensure((size_t)D * vs));
  TRYL(dW.ensure((size_t)D * vs));
  TRYL(Wt.ensure((size_t)D * vs));
  TRYL(ones.ensure((size_t)m * vs));
  TRYL(part.ensure(272 * sizeof(double)));
  TRYL(fill_weights(dbl, ones.p, 0, 0.0, nullptr, 1.0, m, st));
  double* pp = part.as<double>();
  double* dv = pp + 256;
  auto read = [&](double* host, int k) -> int32_t {
    FIRAL_CUDA_TRY(cudaMemcpyAsync(host, dv, k * sizeof(double), cudaMemcpyDeviceToHost, st));
    FIRAL_CUDA_TRY(cudaStreamSynchronize(st));
    return FIRAL_OK;
  };
  auto loss = [&](const void* Wc, double* out) -> int32_t {
    FIRAL_TRY(lr_probs(dbl, Xv, Wc, m, d, c, h.p, st));
    FIRAL_TRY(lr_nll(dbl, h.p, y, m, c, pp, dv, st));
    FIRAL_TRY(dot_scaled(dbl, Wc, Wc, D, 1.0, pp, dv + 1, st));
    double hv[2];
    FIRAL_TRY(read(hv, 2));
    *out = hv[0] + 0.5 * gamma * hv[1];
    return FIRAL_OK;
  };
  // a float gradient stops shrinking near 1e-5 of its start: do not ask for more
  if (!dbl) tol = std::max(tol, 2e-5);
  int it = 0;
  double gn = 0.0, gn0 = 0.0;
  for (; it < max_newton; ++it) {
    double f0 = 0.0;
    TRYL(loss(W, &f0));
    TRYL(lr_grad(dbl, Xv, y, h.p, W, m, d, c, gamma, R.p, g.p, st));
    TRYL(dot_scaled(dbl, g.p, g.p, D, 1.0, pp, dv, st));
    double g2 = 0.0;
    TRYL(read(&g2, 1));
    gn = std::sqrt(g2);
    if (it == 0) gn0 = gn;
    if (!(gn == gn)) TRYL(fail(FIRAL_ERR_NONFINITE, "classifier gradient is not finite"));
    if (gn <= tol * std::max(1.0, gn0)) break;
    firal_pool pool{Xv, h.p, m, d, c, dbl ? FIRAL_DT_F64 : FIRAL_DT_F32,
                    dbl ? FIRAL_DT_F64 : FIRAL_DT_F32};
    firal_hess0 h0{nullptr, nullptr, 0, gamma};
    firal_problem* P = nullptr;
    TRYL(problem_create_impl(H, &pool, &h0, dbl ? FIRAL_FP64 : FIRAL_FP32, &P));
    firal_cg_opts cg{dbl ? 1e-11 : 1e-6, 4000, 0, 0, 0};
    CGResult res;
    rc = setup_sigma(P, ones.p, true);
    if (rc == FIRAL_OK) rc = pcg_run(P, g.p, 1, cg, dW.p, true, &res, nullptr);
    firal_problem_destroy(P);
    if (rc != FIRAL_OK) {
      rel();
      return rc;
    }
    TRYL(dot_scaled(dbl, g.p, dW.p, D, 1.0, pp, dv, st));
    double gd = 0.0;
    TRYL(read(&gd, 1));
    double step = 1.0;
    bool ok = false;
    for (int ls = 0; ls < 40 && gd > 0.0; ++ls) {
      TRYL(axpby(dbl, Wt.p, 1.0, W, -step, dW.p, D, st));
      double ft = 0.0;
      TRYL(loss(Wt.p, &ft));
      if (ft <= f0 - 1e-4 * step * gd) {
        ok = true;
        break;
      }
      step *= 0.5;
    }
    if (!ok) break;
    FIRAL_CUDA_TRY(cudaMemcpyAsync(W, Wt.p, (size_t)D * vs, cudaMemcpyDeviceToDevice, st));
  }
#undef TRYL
  if (iters_out) *iters_out = it;
  if (gnorm_out) *gnorm_out = gn;
  FIRAL_CUDA_TRY(cudaStreamSynchronize(st));
  rel();
  return read_flags(H);
}

int32_t al_impl(firal_handle* H, const void* Xp, const int32_t* yp, int64_t n, const void* Xl0,
                const int32_t* yl0, int64_t m, int d, int c, int32_t x_dtype,
                const firal_al_opts& o, int32_t* sel_out, void* W_out, double* fhat_out) {
  cudaStream_t st = H->stream;
  const bool dbl = o.relax.precision == FIRAL_FP64;
  const size_t vs = dbl ? 8 : 4;
  const int32_t vdt = dbl ? FIRAL_DT_F64 : FIRAL_DT_F32;
  const int R = o.rounds, b = o.budget;
  const int64_t mt = m + (int64_t)R * b;
  const int newton = o.lr_max_newton > 0 ? o.lr_max_newton : 30;
  const double ltol = o.lr_tol > 0 ? o.lr_tol : 1e-8;
  FIRAL_TRY(labels_in_range(yp, n, c, st));
  FIRAL_TRY(labels_in_range(yl0, m, c, st));
  DBuf Xpv, Xl, yl, Xr, hr, hl, W, z, idx, sl;
  auto rel = [&] {
    for (DBuf* bf : {&Xpv, &Xl, &yl, &Xr, &hr, &hl, &W, &z, &idx, &sl}) bf->release();
  };
  int32_t rc = FIRAL_OK;
#define TRYA(x)          \
  do {                   \
    rc = (x);            \
    if (rc != FIRAL_OK) { \
      rel();             \
      return rc;         \
    }                    \
  } while (0)
  TRYA(Xpv.ensure((size_t)n * d * vs));
  TRYA(Xl.ensure((size_t)mt * d * vs));
  TRYA(yl.ensure((size_t)mt * sizeof(int32_t)));
  TRYA(Xr.ensure((size_t)n * d * vs));
  TRYA(hr.ensure((size_t)n * c * vs));
  TRYA(hl.ensure((size_t)mt * c * vs));
  TRYA(W.ensure((size_t)c * d * vs));
  TRYA(z.ensure((size_t)n * vs));
  TRYA(idx.ensure((size_t)n * sizeof(int32_t)));
  TRYA(sl.ensure((size_t)b * sizeof(int32_t)));
  // the pool and the initial labelled rows in the vec type
  TRYA(copy_rows(dbl, Xpv.p, nullptr, 0, Xp, n, d, x_dtype, st));
  if (m > 0) {
    TRYA(copy_rows(dbl, Xl.p, nullptr, 0, Xl0, m, d, x_dtype, st));
    FIRAL_CUDA_TRY(cudaMemcpyAsync(yl.p, yl0, (size_t)m * sizeof(int32_t),
                                   cudaMemcpyDeviceToDevice, st));
  }
  FIRAL_CUDA_TRY(cudaMemsetAsync(W.p, 0, (size_t)c * d * vs, st));
  std::vector<int32_t> remaining((size_t)n), picks((size_t)b), orig((size_t)b);
  for (int64_t i = 0; i < n; ++i) remaining[(size_t)i] = (int32_t)i;
  for (int r = 0; r < R; ++r) {
    const int64_t ml = m + (int64_t)r * b, nr = n - (int64_t)r * b;
    // remaining pool rows, in index order
    FIRAL_CUDA_TRY(cudaMemcpyAsync(idx.p, remaining.data(), (size_t)nr * sizeof(int32_t),
                                   cudaMemcpyHostToDevice, st));
    TRYA(gather_rows(dbl, false, Xpv.p, idx.as<int32_t>(), nr, d, Xr.p, st));
    // classifier refit on the labelled set (warm start from the previous round), then h
    if (ml > 0)
      TRYA(lr_fit_impl(H, Xl.p, yl.as<int32_t>(), ml, d, c, o.lr_gamma, dbl, newton, ltol, W.p,
                       nullptr, nullptr));
    TRYA(lr_probs(dbl, Xl.p, W.p, ml, d, c, hl.p, st));
    TRYA(lr_probs(dbl, Xr.p, W.p, nr, d, c, hr.p, st));
    // Relax (Algorithm 2) and Round (Algorithm 3) on the remaining pool
    firal_pool pool{Xr.p, hr.p, nr, d, c, vdt, vdt};
    firal_hess0 h0{ml > 0 ? Xl.p : nullptr, ml > 0 ? hl.p : nullptr, ml, o.lambda};
    firal_relax_opts ro = o.relax;
    ro.seed = o.relax.seed + (uint64_t)r;
    firal_relax_stats rs{};
    TRYA(firal_relax(H, &pool, &h0, (double)b, nullptr, &ro, z.p, nullptr, &rs));
    if (fhat_out) fhat_out[r] = rs.fhat_last;
    firal_round_opts rop{o.eta, 1, o.relax.precision};
    TRYA(firal_round(H, &pool, &h0, z.p, b, &rop, sl.as<int32_t>(), nullptr));
    FIRAL_CUDA_TRY(cudaMemcpyAsync(picks.data(), sl.p, (size_t)b * sizeof(int32_t),
                                   cudaMemcpyDeviceToHost, st));
    FIRAL_CUDA_TRY(cudaStreamSynchronize(st));
    for (int j = 0; j < b; ++j) {
      if (picks[j] < 0 || picks[j] >= nr) TRYA(fail(FIRAL_ERR_NONFINITE, "Round pick out of range"));
      orig[j] = remaining[(size_t)picks[j]];
    }
    FIRAL_CUDA_TRY(cudaMemcpyAsync(sel_out + (size_t)r * b, orig.data(), (size_t)b * sizeof(int32_t),
                                   cudaMemcpyHostToDevice, st));
    // the picked points join the labelled set, in selection order
    FIRAL_CUDA_TRY(cudaMemcpyAsync(idx.p, orig.data(), (size_t)b * sizeof(int32_t),
                                   cudaMemcpyHostToDevice, st));
    TRYA(gather_rows(dbl, false, Xpv.p, idx.as<int32_t>(), b, d, (char*)Xl.p + ml * d * vs, st));
    TRYA(gather_rows(dbl, true, yp, idx.as<int32_t>(), b, 1, yl.as<int32_t>() + ml, st));
    FIRAL_CUDA_TRY(cudaStreamSynchronize(st));
    std::vector<char> taken((size_t)n, 0);
    for (int j = 0; j < b; ++j) taken[(size_t)orig[j]] = 1;
    std::vector<int32_t> next;
    next.reserve((size_t)(nr - b));
    for (int64_t q = 0; q < nr; ++q)
      if (!taken[(size_t)remaining[(size_t)q]]) next.push_back(remaining[(size_t)q]);
    remaining.swap(next);
  }
  if (W_out) {
    TRYA(lr_fit_impl(H, Xl.p, yl.as<int32_t>(), mt, d, c, o.lr_gamma, dbl, newton, ltol, W.p,
                     nullptr, nullptr));
    FIRAL_CUDA_TRY(cudaMemcpyAsync(W_out, W.p, (size_t)c * d * vs, cudaMemcpyDeviceToDevice, st));
  }
  FIRAL_CUDA_TRY(cudaStreamSynchronize(st));
#undef TRYA
  rel();
  return FIRAL_OK;
}

bool valid_shape(int64_t rows, int d, int c) { return rows >= 0 && d >= 1 && d <= 128 && c >= 2 && c <= 4096; }

}  // namespace

int32_t firal_lr_probs(firal_handle* H, const void* X, int32_t x_dtype, const void* W,
                       int64_t rows, int32_t d, int32_t c, int32_t precision, void* h_out) {
  if (!H || !X || !W || !h_out || !valid_shape(rows, d, c) || x_dtype < 0 || x_dtype > 2)
    return record(H, fail(FIRAL_ERR_ARG, "bad lr_probs arguments"));
  const bool dbl = precision == FIRAL_FP64;
  const size_t vs = dbl ? 8 : 4;
  DBuf Xv;
  int32_t rc = Xv.ensure((size_t)rows * d * vs);
  if (rc == FIRAL_OK) rc = copy_rows(dbl, Xv.p, nullptr, 0, X, rows, d, x_dtype, H->stream);
  if (rc == FIRAL_OK) rc = lr_probs(dbl, Xv.p, W, rows, d, c, h_out, H->stream);
  if (rc == FIRAL_OK && cudaStreamSynchronize(H->stream) != cudaSuccess)
    rc = fail(FIRAL_ERR_CUDA, "lr_probs failed");
  Xv.release();
  return record(H, rc);
}

int32_t firal_lr_fit(firal_handle* H, const void* X, int32_t x_dtype, const int32_t* y, int64_t m,
                     int32_t d, int32_t c, double gamma, int32_t precision, int32_t max_newton,
                     double tol, void* W, int32_t* iters_out, double* gnorm_out) {
  if (!H || !X || !y || !W || m < 1 || !valid_shape(m, d, c) || x_dtype < 0 || x_dtype > 2 ||
      !(gamma > 0) || max_newton < 0)
    return record(H, fail(FIRAL_ERR_ARG, "bad lr_fit arguments"));
  const bool dbl = precision == FIRAL_FP64;
  const size_t vs = dbl ? 8 : 4;
  int32_t rc = labels_in_range(y, m, c, H->stream);
  DBuf Xv;
  if (rc == FIRAL_OK) rc = Xv.ensure((size_t)m * d * vs);
  if (rc == FIRAL_OK) rc = copy_rows(dbl, Xv.p, nullptr, 0, X, m, d, x_dtype, H->stream);
  int it = 0;
  double gn = 0.0;
  if (rc == FIRAL_OK)
    rc = lr_fit_impl(H, Xv.p, y, m, d, c, gamma, dbl, max_newton, tol > 0 ? tol : 1e-8, W, &it,
                     &gn);
  if (iters_out) *iters_out = it;
  if (gnorm_out) *gnorm_out = gn;
  Xv.release();
  return record(H, rc);
}

int32_t firal_active_learning(firal_handle* H, const void* X_pool, const int32_t* y_pool,
                              int64_t n, const void* X_lab, const int32_t* y_lab, int64_t m,
                              int32_t d, int32_t c, int32_t x_dtype, const firal_al_opts* opts,
                              int32_t* selected_out, void* W_out, double* fhat_out) {
  if (!H || !X_pool || !y_pool || !opts || !selected_out || !valid_shape(n, d, c) || n < 1 ||
      m < 0 || (m > 0 && (!X_lab || !y_lab)) || x_dtype < 0 || x_dtype > 2)
    return record(H, fail(FIRAL_ERR_ARG, "bad active_learning arguments"));
  if (opts->rounds < 1 || opts->budget < 1 || (int64_t)opts->rounds * opts->budget >= n ||
      !(opts->lr_gamma > 0) || !(opts->lambda >= 0))
    return record(H, fail(FIRAL_ERR_ARG, "rounds, budget, lr_gamma or lambda out of range"));
  if (opts->relax.precision < FIRAL_FP64 || opts->relax.precision > FIRAL_MIXED_BF16_FAST)
    return record(H, fail(FIRAL_ERR_ARG, "unknown precision"));
  return record(H, al_impl(H, X_pool, y_pool, n, X_lab, y_lab, m, d, c, x_dtype, *opts,
                           selected_out, W_out, fhat_out));
}

// ------------------------------------------------------------------------------------------
// Launch tuning (set by the autotuner)
// ------------------------------------------------------------------------------------------
namespace {
int32_t tuning_check(const firal_tuning* t) {
  if (!t) return fail(FIRAL_ERR_ARG, "tuning must be non-null");
  if (t->dterm_splits < 0 || t->bsum_splits < 0 || t->sm_budget < 0 || t->reserved != 0)
    return fail(FIRAL_ERR_ARG, "tuning values must be >= 0 (reserved = 0)");
  return FIRAL_OK;
}
}  // namespace

int32_t firal_problem_set_tuning(firal_problem* P, const firal_tuning* t) {
  firal_handle* H = P ? P->H : nullptr;
  if (!P) return record(H, fail(FIRAL_ERR_ARG, "problem must be non-null"));
  int32_t rc = tuning_check(t);
  if (rc != FIRAL_OK) return record(H, rc);
  P->tune.dterm_splits = t->dterm_splits;
  P->tune.bsum_splits = t->bsum_splits;
  P->tune.sm_budget = t->sm_budget;
  const int b = forced_sm_budget() > 0 ? forced_sm_budget()
                                       : (t->sm_budget > 0 ? t->sm_budget : H->sm_budget);
  P->sms = (b > 0 && b < H->sm_count) ? b : H->sm_count;
  P->tune_used.sm_budget = P->sms;
  return FIRAL_OK;
}

int32_t firal_problem_get_tuning(firal_problem* P, firal_tuning* out) {
  firal_handle* H = P ? P->H : nullptr;
  if (!P || !out) return record(H, fail(FIRAL_ERR_ARG, "problem and out must be non-null"));
  out->dterm_splits = P->tune_used.dterm_splits;
  out->bsum_splits = P->tune_used.bsum_splits;
  out->sm_budget = P->tune_used.sm_budget;
  out->reserved = 0;
  return FIRAL_OK;
}

int32_t firal_set_default_tuning(firal_handle* H, const firal_tuning* t) {
  if (!H) return fail(FIRAL_ERR_ARG, "handle must be non-null");
  int32_t rc = tuning_check(t);
  if (rc != FIRAL_OK) return record(H, rc);
  H->tune.dterm_splits = t->dterm_splits;
  H->tune.bsum_splits = t->bsum_splits;
  H->tune.sm_budget = t->sm_budget;
  return FIRAL_OK;
}

int32_t firal_cache_trim(void) {
  BlockCache& c = block_cache();
  std::vector<ParkedBlock> blocks;
  {
    std::lock_guard<std::mutex> g(c.mu);
    blocks.swap(c.blocks);
    c.held = 0;
  }
  int cur = 0;
  cudaGetDevice(&cur);
  for (const ParkedBlock& b : blocks) {
    cudaSetDevice(b.dev);
    cudaFree(b.p);
  }
  cudaSetDevice(cur);
  return FIRAL_OK;
}

int64_t firal_cache_bytes(void) {
  BlockCache& c = block_cache();
  std::lock_guard<std::mutex> g(c.mu);
  return (int64_t)c.held;
}

// ------------------------------------------------------------------------------------------
// Row sharding (Section 3.3 of the paper): the problem holds this process's rows; the partial
// sums over points are added across the group by the caller's allreduce.
// ------------------------------------------------------------------------------------------
namespace firal {
bool sharded(const firal_problem* P) { return P->comm.world > 1 && P->comm.allreduce; }

int32_t shard_allreduce(firal_problem* P, void* buf, int64_t count, int32_t dtype, int32_t op) {
  if (!sharded(P)) return FIRAL_OK;
  const int32_t rc = P->comm.allreduce(buf, count, dtype, op, P->H->stream, P->comm.user);
  if (rc != 0)
    return fail(FIRAL_ERR_COMM, "allreduce callback returned " + std::to_string(rc) + " (rank " +
                                    std::to_string(P->comm.rank) + " of " +
                                    std::to_string(P->comm.world) + ")");
  return FIRAL_OK;
}
}  // namespace firal

int32_t firal_problem_set_comm(firal_problem* P, const firal_comm* comm) {
  firal_handle* H = P ? P->H : nullptr;
  if (!P) return record(H, fail(FIRAL_ERR_ARG, "problem must be non-null"));
  if (P->pt.Q) return record(H, fail(FIRAL_ERR_UNSUPPORTED, "pooled problems are not sharded"));
  firal_comm c = comm ? *comm : firal_comm{0, 1, nullptr, nullptr};
  if (c.world < 1 || c.rank < 0 || c.rank >= c.world || (c.world > 1 && !c.allreduce))
    return record(H, fail(FIRAL_ERR_ARG, "need 0 <= rank < world and an allreduce for world > 1"));
  if (c.world == 1) c = firal_comm{0, 1, nullptr, nullptr};
  cudaStream_t st = H->stream;
  P->comm = c;
  // total pool size over the group
  double* red = P->red.as<double>();
  const double nl = (double)P->n;
  int32_t rc = FIRAL_OK;
  if (cudaMemcpyAsync(red + 2000, &nl, sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess)
    rc = fail(FIRAL_ERR_CUDA, "copy of the pool size failed");
  if (rc == FIRAL_OK) rc = shard_allreduce(P, red + 2000, 1, FIRAL_DT_F64, 0);
  double nt = nl;
  if (rc == FIRAL_OK &&
      (cudaMemcpyAsync(&nt, red + 2000, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
       cudaStreamSynchronize(st) != cudaSuccess))
    rc = fail(FIRAL_ERR_CUDA, "read of the total pool size failed");
  if (rc != FIRAL_OK) {
    P->comm = firal_comm{0, 1, nullptr, nullptr};
    return record(H, rc);
  }
  P->n_total = (int64_t)std::llround(nt);
  // H_p = (1/n_total) sum over the pool rows; labelled rows (and lambda) only on rank 0
  rc = fill_weights(P->dbl, P->w_p.p, P->m, 0.0, nullptr, 1.0 / (double)P->n_total, P->n, st);
  if (rc == FIRAL_OK)
    rc = fill_weights(P->dbl, P->w_sig.p, P->m, P->comm.rank == 0 ? 1.0 : 0.0, nullptr,
                      1.0 / (double)P->n_total, P->n, st);
  P->S_p_ready = false;
  if (rc == FIRAL_OK && cudaStreamSynchronize(st) != cudaSuccess)
    rc = fail(FIRAL_ERR_CUDA, "set_comm synchronisation failed");
  return record(H, rc);
}
