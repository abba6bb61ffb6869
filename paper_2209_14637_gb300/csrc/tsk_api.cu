// Host side of the C ABI declared in include/tsk.h: handles, argument
// checks, plans (workspace + schedule + CUDA graph), the eigensolver loop
// of the training side and the dispatch to the kernels.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "tsk_internal.cuh"

// NVTX ranges name each entry point on a profiler's timeline (no cost when
// no tool is attached); without the header they compile to nothing.
#if defined(__has_include)
#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
#define TSK_NVTX 1
#endif
#endif
namespace {
struct NvtxRange {
  explicit NvtxRange(const char* name) {
#ifdef TSK_NVTX
    nvtxRangePushA(name);
#else
    (void)name;
#endif
  }
  ~NvtxRange() {
#ifdef TSK_NVTX
    nvtxRangePop();
#endif
  }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};
}  // namespace
#define TSK_NVTX_RANGE(name) NvtxRange tsk_nvtx_range_(name)

using namespace tsk;

struct tsk_plan_s {
  tsk_handle h = nullptr;
  int count = 0;
  tsk_prec prec = TSK_FP32;
  int kp = 16;
  int kmax = 1;
  bool dbl = false;
  bool use_tc = false;   // some matrices take the tensor-core sketch
  bool use_simt = true;  // some matrices take the CUDA-core sketch
  bool small64 = false;  // FP32 / BF16 plan with the FP64 small-factor route
  void* ws = nullptr;
  size_t ws_bytes = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int launches = 0;
  TcPlan* tc = nullptr;
  std::vector<unsigned char> key;
  // what a (re-)capture needs
  bool any_out = false;
  int nx = 0, ny = 0, nio = 0;
  unsigned char* base = nullptr;
  size_t o_mats = 0, o_ix = 0, o_iy = 0, o_io = 0, o_pan = 0, o_X = 0, o_Y = 0,
         o_RX = 0, o_RY = 0, o_W = 0, o_flag = 0, o_U2 = 0, o_V2 = 0, o_e2 = 0,
         o_pan64 = 0, o_RX64 = 0, o_RY64 = 0, o_W64 = 0;
  // BF16 matrices copied to 16-byte aligned rows before the sketch pass
  int npack_items = 0;
  size_t o_pk = 0, o_pki = 0;
  // FP32 / BF16 small factors: matrix ids grouped by k rounded up to 8, one
  // launch per group (kc, first id, count)
  size_t o_fids = 0;
  std::vector<int3> fin_cls;
  // Gram route (FP32 / BF16)
  double* d_norm = nullptr;
  double* d_err = nullptr;
  cudaGraphNode_t probe_begin = nullptr, probe_end = nullptr;
};

struct tsk_handle_s {
  int device = 0;
  tsk_options opts{};
  char last_error[512] = {0};
  int* d_status = nullptr;
  cudaStream_t cap_stream = nullptr;
  // branches of a captured plan: the sketch pass of each cluster-size class
  // of the tensor-core kernel and the CUDA-core kernels run concurrently
  static constexpr int kBranches = 8;
  cudaStream_t branch[kBranches] = {nullptr};
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_join[kBranches] = {nullptr};
  std::vector<tsk_plan> cache;
  GramCache* gram_cache = nullptr;  // tensor maps of the last BF16 training set
  // Autotuned rows of A per CTA of the tensor-core sketch, by size class:
  // (cluster size at 512 rows per CTA, k rounded up to 8) -> 256 or 512.
  std::map<std::pair<int, int>, int> tune;
  std::map<std::pair<int, int>, std::vector<double>> tune_us;  // us / matrix at 512, 256, 384
  int tune_version = 0;
  int force_mc = 0;  // while tuning: every matrix takes this shape
};

// Size class of a matrix for the autotuner: the cluster size it needs at
// 512 rows per CTA, and k rounded up to 8 (the kernel's X~ rows).
static std::pair<int, int> tune_key(int64_t m, int32_t k) {
  int c = 1;
  while ((int64_t)c * 512 < m) c *= 2;
  return {c, (k + 7) / 8 * 8};
}

static thread_local char g_create_error[512] = "no error";

static void set_err(tsk_handle h, const char* fmt, ...) {
  char* dst = h ? h->last_error : g_create_error;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(dst, 512, fmt, ap);
  va_end(ap);
}

void tsk::set_thread_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_create_error, sizeof(g_create_error), fmt, ap);
  va_end(ap);
}

#define TSK_CUDA(h, call)                                                   \
  do {                                                                      \
    cudaError_t e_ = (call);                                                \
    if (e_ != cudaSuccess) {                                                \
      set_err((h), "%s failed: %s", #call, cudaGetErrorString(e_));         \
      return e_ == cudaErrorMemoryAllocation ? TSK_ENOMEM : TSK_ECUDA;      \
    }                                                                       \
  } while (0)

static size_t elt_size(tsk_prec p) {
  return p == TSK_FP64 ? 8 : (p == TSK_FP32 ? 4 : 2);
}
static size_t compute_size(tsk_prec p) { return p == TSK_FP64 ? 8 : 4; }
static size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// An integer (or, for env_real, a number) from environment variable `name`,
// when it is set, parses completely and lies in [lo, hi].
static bool env_int(const char* name, long long lo, long long hi, long long* v) {
  const char* s = getenv(name);
  if (!s || !*s) return false;
  char* end = nullptr;
  const long long x = strtoll(s, &end, 10);
  if (*end != '\0' || x < lo || x > hi) return false;
  *v = x;
  return true;
}
static bool env_real(const char* name, double lo, double hi, double* v) {
  const char* s = getenv(name);
  if (!s || !*s) return false;
  char* end = nullptr;
  const double x = strtod(s, &end);
  if (*end != '\0' || !(x >= lo && x <= hi)) return false;
  *v = x;
  return true;
}

extern "C" void tsk_default_options(tsk_options* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->kernel = TSK_KERNEL_AUTO;
  o->refine_q = 2;
  o->max_iter = 300;
  o->eig_tol = 0.0;
  o->err_mode = 0;
  o->spin_limit = 1ll << 24;
  o->small_fp64 = 0;
  o->gram_tile = 0;
  long long v = 0;
  if (env_int("TSK_KERNEL", 0, 2, &v)) o->kernel = (int32_t)v;
  if (env_int("TSK_REFINE_Q", 0, 2, &v)) o->refine_q = (int32_t)v;
  if (env_int("TSK_MAX_ITER", 1, 1000000, &v)) o->max_iter = (int32_t)v;
  if (env_int("TSK_ERR_MODE", 0, 2, &v)) o->err_mode = (int32_t)v;
  if (env_int("TSK_SPIN_LIMIT", 1, 1ll << 40, &v)) o->spin_limit = v;
  if (env_int("TSK_SMALL_FP64", 0, 1, &v)) o->small_fp64 = (int32_t)v;
  if (env_int("TSK_GRAM_TILE", 0, 1, &v)) o->gram_tile = (int32_t)v;
  double t = 0.0;
  if (env_real("TSK_EIG_TOL", 0.0, 1.0, &t)) o->eig_tol = t;
}

extern "C" tsk_status tsk_create(tsk_handle* out, const tsk_options* opts) {
  if (!out) {
    set_err(nullptr, "tsk_create: out is NULL");
    return TSK_EINVAL;
  }
  *out = nullptr;
  int dev = 0, ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev == 0) {
    set_err(nullptr, "tsk_create: no CUDA device (%s)", cudaGetErrorString(e));
    return TSK_ECUDA;
  }
  if (cudaGetDevice(&dev) != cudaSuccess) {
    set_err(nullptr, "tsk_create: cudaGetDevice failed");
    return TSK_ECUDA;
  }
  tsk_handle h = new (std::nothrow) tsk_handle_s();
  if (!h) return TSK_ENOMEM;
  h->device = dev;
  tsk_default_options(&h->opts);
  if (opts) h->opts = *opts;
  if (h->opts.max_iter <= 0) h->opts.max_iter = 300;
  if (h->opts.spin_limit <= 0) h->opts.spin_limit = 1ll << 24;
  e = cudaMalloc(&h->d_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(h->d_status, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
  for (int b = 0; e == cudaSuccess && b < tsk_handle_s::kBranches; ++b) {
    e = cudaStreamCreateWithFlags(&h->branch[b], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_join[b], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    set_err(nullptr, "tsk_create: %s", cudaGetErrorString(e));
    for (int b = 0; b < tsk_handle_s::kBranches; ++b) {
      if (h->ev_join[b]) cudaEventDestroy(h->ev_join[b]);
      if (h->branch[b]) cudaStreamDestroy(h->branch[b]);
    }
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->d_status) cudaFree(h->d_status);
    delete h;
    return TSK_ECUDA;
  }
  *out = h;
  return TSK_OK;
}

static void plan_free(tsk_plan p) {
  if (!p) return;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  if (p->tc) tc_destroy(p->tc);
  if (p->ws) cudaFree(p->ws);
  delete p;
}

extern "C" tsk_status tsk_destroy(tsk_handle h) {
  if (!h) return TSK_EINVAL;
  cudaDeviceSynchronize();
  for (tsk_plan p : h->cache) plan_free(p);
  h->cache.clear();
  gram_cache_destroy(h->gram_cache);
  for (int b = 0; b < tsk_handle_s::kBranches; ++b) {
    if (h->ev_join[b]) cudaEventDestroy(h->ev_join[b]);
    if (h->branch[b]) cudaStreamDestroy(h->branch[b]);
  }
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->d_status) cudaFree(h->d_status);
  delete h;
  return TSK_OK;
}

extern "C" const char* tsk_last_error(tsk_handle h) {
  return h ? h->last_error : g_create_error;
}

extern "C" tsk_status tsk_sync_status(tsk_handle h, tsk_stream stream) {
  if (!h) return TSK_EINVAL;
  TSK_CUDA(h, cudaStreamSynchronize((cudaStream_t)stream));
  int st = 0;
  TSK_CUDA(h, cudaMemcpy(&st, h->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  TSK_CUDA(h, cudaMemset(h->d_status, 0, sizeof(int)));
  if (st & kStatusTimeout) {
    set_err(h, "a bounded device wait ran out (status word 0x%x)", st);
    return TSK_ETIMEOUT;
  }
  if (st & kStatusRankDef) {
    set_err(h, "S A had rank < k for at least one matrix");
    return TSK_ERANKDEF;
  }
  return TSK_OK;
}

// ---------------------------------------------------------------------------
// argument checks
// ---------------------------------------------------------------------------
static tsk_status check_desc(tsk_handle h, const tsk_mat_desc& d, int64_t i,
                             tsk_prec prec) {
  if (!d.A || !d.S) {
    set_err(h, "matrix %lld: A or S is NULL", (long long)i);
    return TSK_EINVAL;
  }
  if (d.m < 1 || d.n < 1 || d.lda < d.n) {
    set_err(h, "matrix %lld: need m, n >= 1 and lda >= n (m=%lld n=%lld lda=%lld)",
            (long long)i, (long long)d.m, (long long)d.n, (long long)d.lda);
    return TSK_EINVAL;
  }
  const int64_t mn = std::min(d.m, d.n);
  if (d.r < 1 || d.r > d.k || d.k > mn || d.k > TSK_MAX_K) {
    set_err(h, "matrix %lld: need 1 <= r <= k <= min(m, n) and k <= %d "
               "(r=%d k=%d m=%lld n=%lld)",
            (long long)i, TSK_MAX_K, d.r, d.k, (long long)d.m, (long long)d.n);
    return TSK_EINVAL;
  }
  const size_t es = elt_size(prec);
  if (((uintptr_t)d.A) % es != 0 || ((uintptr_t)d.S) % compute_size(prec) != 0) {
    set_err(h, "matrix %lld: A or S is not aligned to its element size", (long long)i);
    return TSK_EINVAL;
  }
  return TSK_OK;
}

// The tensor-core kernel takes k <= 48 and m <= 4096 (clusters of at most 8
// CTAs of 512 rows) and needs 16-byte aligned rows for TMA; S is read
// through a pre-swizzled image the plan builds, so it needs no alignment.
static bool tc_eligible_one(const tsk_mat_desc& d) {
  return tc_matrix_eligible(d.A, d.m, d.lda, d.k);
}
// Padded leading dimension of the aligned copy: n rounded up to 8 elements.
static long long pack_ld(long long n) { return (n + 7) / 8 * 8; }
// Eligible once copied to rows with that leading dimension (an aligned base).
static bool tc_eligible_packed(const tsk_mat_desc& d) {
  return tc_matrix_eligible((const void*)256, d.m, pack_ld(d.n), d.k);
}

// ---------------------------------------------------------------------------
// plans
// ---------------------------------------------------------------------------
struct Carve {
  size_t off = 0;
  size_t take(size_t bytes) {
    off = align_up(off, 256);
    size_t o = off;
    off += bytes;
    return o;
  }
};

// Records one execution of the plan into a CUDA graph.  With events given,
// event-record nodes bracket the sketch pass (the stage that streams A).
static cudaError_t capture_plan(tsk_plan p, cudaEvent_t evb, cudaEvent_t eve) {
  tsk_handle h = p->h;
  unsigned char* base = p->base;
  const int kp = p->kp;
  const int count = p->count;
  const int in_type = (int)p->prec;
  const MatDev* d_mats = (const MatDev*)(base + p->o_mats);
  double* d_norm = p->d_norm;
  double* d_err = p->d_err;
  cudaStream_t s = h->cap_stream;
  if (p->exec) {
    cudaGraphExecDestroy(p->exec);
    p->exec = nullptr;
  }
  if (p->graph) {
    cudaGraphDestroy(p->graph);
    p->graph = nullptr;
  }
  p->probe_begin = p->probe_end = nullptr;
  cudaError_t ce = cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed);
  if (ce != cudaSuccess) return ce;
  int launches = 0;
  ce = cudaMemsetAsync(d_norm, 0, sizeof(double) * count, s);
  if (ce == cudaSuccess && evb) ce = cudaEventRecordWithFlags(evb, s, cudaEventRecordExternal);
  // The sketch pass: one branch of the graph per cluster-size class of the
  // tensor-core kernel and one for the CUDA-core kernels (the matrices the
  // tensor-core kernel cannot take); the branches run concurrently and join
  // before the small factors.
  if (ce == cudaSuccess && p->use_tc) {
    ce = tc_launch_prep(p->tc, s);  // the S images, read by every class
    ++launches;
  }
  if (ce == cudaSuccess && p->npack_items > 0) {  // aligned copies, before every branch
    ce = launch_pack_rows((const PackDev*)(base + p->o_pk), (const int2*)(base + p->o_pki),
                          p->npack_items, s);
    ++launches;
  }
  const int ncls = p->use_tc ? tc_classes(p->tc) : 0;
  const int nbr = ncls + (p->use_simt ? 1 : 0);
  if (nbr > tsk_handle_s::kBranches + 1 && ce == cudaSuccess) ce = cudaErrorInvalidValue;
  int forked = 0;
  if (ce == cudaSuccess && nbr > 1) {
    ce = cudaEventRecord(h->ev_fork, s);
    for (int b = 0; ce == cudaSuccess && b < nbr - 1; ++b, ++forked)
      ce = cudaStreamWaitEvent(h->branch[b], h->ev_fork, 0);
  }
  // branch j runs on s for j == 0 and on h->branch[j - 1] otherwise
  auto br = [&](int j) { return j == 0 ? s : h->branch[j - 1]; };
  for (int j = 0; ce == cudaSuccess && j < ncls; ++j) {
    ce = tc_launch_class(p->tc, j, br(j));
    ++launches;
  }
  if (ce == cudaSuccess && p->use_simt) {
    cudaStream_t s2 = br(ncls);
    ce = launch_sketch_x(in_type, kp, d_mats, (const int2*)(base + p->o_ix),
                         p->nx, base + p->o_X, d_norm, s2);
    if (ce == cudaSuccess)
      ce = launch_sketch_y(in_type, kp, d_mats, (const int2*)(base + p->o_iy),
                           p->ny, base + p->o_X, base + p->o_Y, s2);
    launches += 2;
  }
  // join every forked branch, even after an error, so the capture can end
  for (int b = 0; b < forked; ++b) {
    cudaError_t je = cudaEventRecord(h->ev_join[b], h->branch[b]);
    if (je == cudaSuccess) je = cudaStreamWaitEvent(s, h->ev_join[b], 0);
    if (ce == cudaSuccess) ce = je;
  }
  if (ce == cudaSuccess && eve) ce = cudaEventRecordWithFlags(eve, s, cudaEventRecordExternal);
  const double tau = p->dbl ? 1e-6 : 1e-4;
  if (ce == cudaSuccess && p->dbl) {
    // FP64: blockwise Householder R factors of X and Y, SVD of R_Y R_X^{-1}
    ce = launch_tsqr(p->dbl, kp, (const PanelDev*)(base + p->o_pan), 2 * count,
                     h->opts.refine_q ? 1 : 0, h->d_status, s);
    ++launches;
    if (ce == cudaSuccess)
      ce = launch_small_svd(p->dbl, kp, d_mats, count, base + p->o_RX,
                            base + p->o_RY, base + p->o_W, d_norm, d_err,
                            (int*)(base + p->o_flag), h->opts.err_mode, tau,
                            h->d_status, s);
    ++launches;
  } else if (ce == cudaSuccess && p->small64) {
    // FP32 / BF16 panels, small factors in double: Householder R factors of
    // X and Y (with one refinement pass on X when refine_q != 0), the SVD of
    // R_Y R_X^{-1}, then W back to float for the outputs and the fallback.
    ce = launch_tsqr_f32_in_f64(kp, (const PanelDev*)(base + p->o_pan64), 2 * count,
                                h->opts.refine_q ? 1 : 0, s);
    ++launches;
    if (ce == cudaSuccess)
      ce = launch_small_svd(true, kp, d_mats, count, base + p->o_RX64, base + p->o_RY64,
                            base + p->o_W64, d_norm, d_err, (int*)(base + p->o_flag),
                            h->opts.err_mode, tau, h->d_status, s, 1);
    ++launches;
    if (ce == cudaSuccess)
      ce = launch_convert_gram(false, (const double*)(base + p->o_W64), base + p->o_W,
                               (long long)count * kp * kp, s);
    ++launches;
  } else if (ce == cudaSuccess) {
    // FP32 / BF16: Cholesky of X^T X (+ one refinement), eigenpairs of M^T M,
    // one CTA per matrix, one launch per k class; the classes run
    // concurrently on branches of the graph
    const PanelDev* pan = (const PanelDev*)(base + p->o_pan);
    const int* fids = (const int*)(base + p->o_fids);
    const int nfc = (int)p->fin_cls.size();
    if (nfc > tsk_handle_s::kBranches + 1) ce = cudaErrorInvalidValue;
    int fforked = 0;
    if (ce == cudaSuccess && nfc > 1) {
      ce = cudaEventRecord(h->ev_fork, s);
      for (int b = 0; ce == cudaSuccess && b < nfc - 1; ++b, ++fforked)
        ce = cudaStreamWaitEvent(h->branch[b], h->ev_fork, 0);
    }
    for (int j = 0; ce == cudaSuccess && j < nfc; ++j) {
      const int3 c = p->fin_cls[(size_t)j];
      ce = launch_finish(kp, c.x, fids + c.y, c.z, d_mats, pan, pan + count,
                         (float*)(base + p->o_W), d_norm, d_err, (int*)(base + p->o_flag),
                         h->opts.err_mode, tau, h->opts.refine_q, h->d_status, br(j));
      ++launches;
    }
    for (int b = 0; b < fforked; ++b) {
      cudaError_t je = cudaEventRecord(h->ev_join[b], h->branch[b]);
      if (je == cudaSuccess) je = cudaStreamWaitEvent(s, h->ev_join[b], 0);
      if (ce == cudaSuccess) ce = je;
    }
  }
  if (ce == cudaSuccess && h->opts.err_mode != 1) {
    ce = cudaMemsetAsync(base + p->o_e2, 0, sizeof(double) * count, s);
    if (ce == cudaSuccess)
      ce = launch_direct_fallback(in_type, kp, d_mats, count, (const int*)(base + p->o_flag),
                                  base + p->o_X, base + p->o_Y, base + p->o_W,
                                  base + p->o_U2, base + p->o_V2, (double*)(base + p->o_e2),
                                  d_err, s);
    launches += 3;
  }
  if (ce == cudaSuccess && p->any_out) {
    ce = launch_project_out(p->dbl, kp, d_mats, (const int4*)(base + p->o_io),
                            p->nio, base + p->o_X, base + p->o_Y, base + p->o_W,
                            s);
    ++launches;
  }
  cudaGraph_t g = nullptr;
  cudaError_t ce2 = cudaStreamEndCapture(s, &g);
  if (ce == cudaSuccess) ce = ce2;
  p->graph = g;
  if (ce == cudaSuccess) ce = cudaGraphInstantiate(&p->exec, p->graph, 0);
  if (ce == cudaSuccess && evb && eve) {
    size_t nn = 0;
    ce = cudaGraphGetNodes(p->graph, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    if (ce == cudaSuccess && nn) ce = cudaGraphGetNodes(p->graph, nodes.data(), &nn);
    for (size_t i = 0; ce == cudaSuccess && i < nn; ++i) {
      cudaGraphNodeType t;
      if (cudaGraphNodeGetType(nodes[i], &t) != cudaSuccess) continue;
      if (t != cudaGraphNodeTypeEventRecord) continue;
      cudaEvent_t ev = nullptr;
      if (cudaGraphEventRecordNodeGetEvent(nodes[i], &ev) != cudaSuccess) continue;
      if (ev == evb) p->probe_begin = nodes[i];
      if (ev == eve) p->probe_end = nodes[i];
    }
  }
  p->launches = launches;
  return ce;
}

static tsk_status build_plan(tsk_handle h, int64_t count,
                             const tsk_mat_desc* mats, tsk_prec prec,
                             const tsk_mat_out* outs, double* err,
                             double* normA2, tsk_plan* out) {
  *out = nullptr;
  if (count < 1 || !mats) {
    set_err(h, "count must be >= 1 and mats non-NULL");
    return TSK_EINVAL;
  }
  if (prec != TSK_FP64 && prec != TSK_FP32 && prec != TSK_BF16) {
    set_err(h, "unknown precision %d", (int)prec);
    return TSK_EINVAL;
  }
  if (count > (1 << 22)) {
    set_err(h, "count too large");
    return TSK_EINVAL;
  }
  int kmax = 1;
  long long rows8 = 0, cols64 = 0;  // the largest item lists a plan launches over
  for (int64_t i = 0; i < count; ++i) {
    tsk_status st = check_desc(h, mats[i], i, prec);
    if (st != TSK_OK) return st;
    kmax = std::max(kmax, mats[i].k);
    rows8 += (mats[i].m + 7) / 8;
    cols64 += (mats[i].n + 63) / 64;
  }
  if (rows8 > 2147483647ll || cols64 > 2147483647ll) {
    set_err(h, "batch too large for one plan (its per-block work items exceed a launch's grid)");
    return TSK_EINVAL;
  }
  const int req = h->opts.kernel;
  // per matrix: tensor-core sketch (1) or CUDA-core sketch (0)
  // BF16 rows that TMA cannot address (not 16-byte aligned) are copied to
  // aligned rows in the workspace at every execution and take the
  // tensor-core kernel too
  std::vector<char> on_tc((size_t)count, 0);
  std::vector<int> tc_ids, pack_ids;
  if (prec == TSK_BF16 && req != TSK_KERNEL_SIMT && tc_supported()) {
    for (int64_t i = 0; i < count; ++i) {
      const bool direct = tc_eligible_one(mats[i]);
      if (direct || tc_eligible_packed(mats[i])) {
        on_tc[(size_t)i] = 1;
        tc_ids.push_back((int)i);
        if (!direct) pack_ids.push_back((int)i);
      }
    }
  }
  if (req == TSK_KERNEL_TC) {
    if (prec != TSK_BF16) {
      set_err(h, "the tensor-core kernel runs the TSK_BF16 path only");
      return TSK_EUNSUPPORTED;
    }
    if ((int64_t)tc_ids.size() != count) {
      set_err(h, "tensor-core kernel requested but unavailable for these "
                 "arguments (needs a GB300, k <= 48 and m <= 4096)");
      return TSK_EUNSUPPORTED;
    }
  }
  const bool use_tc = !tc_ids.empty();
  const bool use_simt = (int64_t)tc_ids.size() < count;

  tsk_plan p = new (std::nothrow) tsk_plan_s();
  if (!p) return TSK_ENOMEM;
  p->h = h;
  p->count = (int)count;
  p->prec = prec;
  p->dbl = (prec == TSK_FP64);
  p->kp = ((kmax + 15) / 16) * 16;
  p->kmax = kmax;
  p->use_tc = use_tc;
  p->use_simt = use_simt;
  p->small64 = (prec != TSK_FP64) && h->opts.small_fp64 != 0;
  const int kp = p->kp;
  const size_t cs = compute_size(prec);

  std::vector<MatDev> hm(count);
  std::vector<int2> ix, iy;
  std::vector<int4> io;
  long long offX = 0, offY = 0;
  bool any_out = false;
  for (int64_t i = 0; i < count; ++i) {
    MatDev& d = hm[i];
    d.A = mats[i].A;
    d.S = mats[i].S;
    d.m = mats[i].m;
    d.n = mats[i].n;
    d.lda = mats[i].lda;
    d.k = mats[i].k;
    d.r = mats[i].r;
    d.offX = offX;
    d.offY = offY;
    d.US = outs ? outs[i].US : nullptr;
    d.Vt = outs ? outs[i].Vt : nullptr;
    d.sigma = outs ? outs[i].sigma : nullptr;
    offX += d.n * kp;
    offY += d.m * kp;
    if (!on_tc[(size_t)i]) {  // CUDA-core sketch items: 64 columns (X) or rows (Y)
      for (long long t = 0; t < (d.n + 63) / 64; ++t) ix.push_back(make_int2((int)i, (int)t));
      for (long long t = 0; t < (d.m + 63) / 64; ++t) iy.push_back(make_int2((int)i, (int)t));
    }
    if (d.US)
      for (long long t = 0; t < (d.m + 255) / 256; ++t)
        io.push_back(make_int4((int)i, (int)t, 0, 0));
    if (d.Vt)
      for (long long t = 0; t < (d.n + 255) / 256; ++t)
        io.push_back(make_int4((int)i, (int)t, 1, 0));
    any_out |= (d.US || d.Vt);
  }
  Carve cv;
  const size_t o_mats = cv.take(sizeof(MatDev) * count);
  const size_t o_ix = cv.take(sizeof(int2) * std::max<size_t>(1, ix.size()));
  const size_t o_iy = cv.take(sizeof(int2) * std::max<size_t>(1, iy.size()));
  const size_t o_io = cv.take(sizeof(int4) * std::max<size_t>(1, io.size()));
  const size_t o_pan = cv.take(sizeof(PanelDev) * 2 * count);
  // aligned copies: descriptors and row-block items (uploaded with the
  // other descriptors), then the copies themselves
  std::vector<PackDev> hpk(pack_ids.size());
  std::vector<int2> pki;
  for (size_t q = 0; q < pack_ids.size(); ++q) {
    const tsk_mat_desc& d = mats[pack_ids[q]];
    for (long long t = 0; t < (d.m + 7) / 8; ++t) pki.push_back(make_int2((int)q, (int)t));
  }
  if (pki.size() > (size_t)INT32_MAX) {
    set_err(h, "too many rows to copy");
    delete p;
    return TSK_EINVAL;
  }
  std::vector<int> fids;
  std::vector<int3> fcls;
  // the widest class first, and within a class the longest panels (m + n)
  // first: the CTAs that run longest start first
  for (int kc = TSK_MAX_K; kc >= 8; kc -= 8) {
    const int first = (int)fids.size();
    for (int64_t i = 0; i < count; ++i)
      if (((mats[i].k + 7) & ~7) == kc) fids.push_back((int)i);
    std::stable_sort(fids.begin() + first, fids.end(), [&](int a, int b) {
      return mats[a].m + mats[a].n > mats[b].m + mats[b].n;
    });
    if ((int)fids.size() > first) fcls.push_back(make_int3(kc, first, (int)fids.size() - first));
  }
  const size_t o_fids = cv.take(sizeof(int) * fids.size());
  const size_t o_pk = cv.take(sizeof(PackDev) * std::max<size_t>(1, hpk.size()));
  const size_t o_pki = cv.take(sizeof(int2) * std::max<size_t>(1, pki.size()));
  const size_t o_X = cv.take(cs * offX);
  const size_t o_Y = cv.take(cs * offY);
  const size_t o_RX = cv.take(cs * count * kp * kp);
  const size_t o_RY = cv.take(cs * count * kp * kp);
  const size_t o_W = cv.take(cs * count * kp * kp);
  const size_t o_nrm = cv.take(sizeof(double) * count);
  const size_t o_err = cv.take(sizeof(double) * count);
  const bool fallback = h->opts.err_mode != 1;
  const size_t o_flag = cv.take(sizeof(int) * count);
  const size_t o_U2 = cv.take(fallback ? cs * offY : 0);
  const size_t o_V2 = cv.take(fallback ? cs * offX : 0);
  const size_t o_e2 = cv.take(sizeof(double) * count);
  // FP64 small-factor route: panel descriptors and double R_X, R_Y, W
  const bool s64 = p->small64;
  const size_t o_pan64 = cv.take(s64 ? sizeof(PanelDev) * 2 * count : 0);
  const size_t o_RX64 = cv.take(s64 ? 8 * (size_t)count * kp * kp : 0);
  const size_t o_RY64 = cv.take(s64 ? 8 * (size_t)count * kp * kp : 0);
  const size_t o_W64 = cv.take(s64 ? 8 * (size_t)count * kp * kp : 0);
  std::vector<size_t> o_copy(pack_ids.size());
  for (size_t q = 0; q < pack_ids.size(); ++q) {
    const tsk_mat_desc& d = mats[pack_ids[q]];
    o_copy[q] = cv.take(2 * (size_t)d.m * (size_t)pack_ld(d.n));
  }
  const size_t host_part = o_X;  // descriptors live before X
  p->ws_bytes = cv.off;
  cudaError_t ce = cudaMalloc(&p->ws, p->ws_bytes);
  if (ce != cudaSuccess) {
    set_err(h, "plan workspace of %zu bytes: %s", p->ws_bytes, cudaGetErrorString(ce));
    delete p;
    return TSK_ENOMEM;
  }
  unsigned char* base = (unsigned char*)p->ws;
  double* d_norm = normA2 ? normA2 : (double*)(base + o_nrm);
  double* d_err = err ? err : (double*)(base + o_err);
  std::vector<PanelDev> hp(2 * count);
  for (int64_t i = 0; i < count; ++i) {
    PanelDev& px = hp[i];
    px.P = base + o_X + cs * hm[i].offX;
    px.rows = hm[i].n;
    px.k = hm[i].k;
    px.ld = kp;
    px.R = base + o_RX + cs * i * kp * kp;
    PanelDev& py = hp[count + i];
    py.P = base + o_Y + cs * hm[i].offY;
    py.rows = hm[i].m;
    py.k = hm[i].k;
    py.ld = kp;
    py.R = base + o_RY + cs * i * kp * kp;
  }
  std::vector<unsigned char> staging(host_part, 0);
  memcpy(staging.data() + o_mats, hm.data(), sizeof(MatDev) * count);
  if (!ix.empty()) memcpy(staging.data() + o_ix, ix.data(), sizeof(int2) * ix.size());
  if (!iy.empty()) memcpy(staging.data() + o_iy, iy.data(), sizeof(int2) * iy.size());
  if (!io.empty()) memcpy(staging.data() + o_io, io.data(), sizeof(int4) * io.size());
  memcpy(staging.data() + o_pan, hp.data(), sizeof(PanelDev) * 2 * count);
  for (size_t q = 0; q < pack_ids.size(); ++q) {
    const tsk_mat_desc& d = mats[pack_ids[q]];
    hpk[q].src = d.A;
    hpk[q].dst = base + o_copy[q];
    hpk[q].m = d.m;
    hpk[q].n = d.n;
    hpk[q].lda = d.lda;
    hpk[q].ldp = pack_ld(d.n);
  }
  memcpy(staging.data() + o_fids, fids.data(), sizeof(int) * fids.size());
  if (!hpk.empty()) memcpy(staging.data() + o_pk, hpk.data(), sizeof(PackDev) * hpk.size());
  if (!pki.empty()) memcpy(staging.data() + o_pki, pki.data(), sizeof(int2) * pki.size());
  ce = cudaMemcpy(p->ws, staging.data(), host_part, cudaMemcpyHostToDevice);
  if (ce == cudaSuccess && s64) {
    // the same float panels, with double R factors
    std::vector<PanelDev> hp64(hp);
    for (int64_t i = 0; i < count; ++i) {
      hp64[i].R = base + o_RX64 + 8 * i * kp * kp;
      hp64[count + i].R = base + o_RY64 + 8 * i * kp * kp;
    }
    ce = cudaMemcpy(base + o_pan64, hp64.data(), sizeof(PanelDev) * 2 * count,
                    cudaMemcpyHostToDevice);
  }
  // The X and Y panels start zeroed: the kernels write columns < k (the
  // tensor-core kernel: < k rounded up to 8) and never the rest, which the
  // Gram kernel reads as zeros.
  if (ce == cudaSuccess) ce = cudaMemset(base + o_X, 0, cs * offX);
  if (ce == cudaSuccess) ce = cudaMemset(base + o_Y, 0, cs * offY);
  if (ce != cudaSuccess) {
    set_err(h, "plan upload: %s", cudaGetErrorString(ce));
    plan_free(p);
    return TSK_ECUDA;
  }
  const MatDev* d_mats = (const MatDev*)(base + o_mats);
  if (use_tc) {
    char msg[256] = {0};
    // rows of A per CTA: forced while tuning, else the tuned choice of the
    // matrix's size class, else the default shape
    std::vector<int> mcp((size_t)count, 0);
    for (int64_t i = 0; i < count; ++i) {
      if (h->force_mc) {
        mcp[(size_t)i] = h->force_mc;
      } else {
        auto it = h->tune.find(tune_key(mats[i].m, mats[i].k));
        if (it != h->tune.end()) mcp[(size_t)i] = it->second;
      }
    }
    // the tensor maps of copied matrices address the copies
    std::vector<MatDev> hmt(hm);
    for (size_t q = 0; q < pack_ids.size(); ++q) {
      hmt[(size_t)pack_ids[q]].A = hpk[q].dst;
      hmt[(size_t)pack_ids[q]].lda = hpk[q].ldp;
    }
    ce = tc_prepare(&p->tc, hmt.data(), d_mats, (int)count, tc_ids.data(), (int)tc_ids.size(),
                    mcp.data(), kp, base + o_X, base + o_Y, d_norm, h->d_status,
                    h->opts.spin_limit, msg, sizeof(msg));
    if (ce != cudaSuccess) {
      set_err(h, "tensor-core plan: %s (%s)", msg, cudaGetErrorString(ce));
      plan_free(p);
      return TSK_ECUDA;
    }
  }

  p->any_out = any_out;
  p->nx = (int)ix.size();
  p->ny = (int)iy.size();
  p->nio = (int)io.size();
  p->base = base;
  p->o_mats = o_mats;
  p->o_ix = o_ix;
  p->o_iy = o_iy;
  p->o_io = o_io;
  p->o_pan = o_pan;
  p->o_X = o_X;
  p->o_Y = o_Y;
  p->o_RX = o_RX;
  p->o_RY = o_RY;
  p->o_W = o_W;
  p->o_flag = o_flag;
  p->o_U2 = o_U2;
  p->o_V2 = o_V2;
  p->o_e2 = o_e2;
  p->o_pan64 = o_pan64;
  p->o_RX64 = o_RX64;
  p->o_RY64 = o_RY64;
  p->o_W64 = o_W64;
  p->npack_items = (int)pki.size();
  p->o_fids = o_fids;
  p->fin_cls = fcls;
  p->o_pk = o_pk;
  p->o_pki = o_pki;
  p->d_norm = d_norm;
  p->d_err = d_err;
  ce = capture_plan(p, nullptr, nullptr);
  if (ce != cudaSuccess) {
    set_err(h, "plan capture: %s", cudaGetErrorString(ce));
    cudaGetLastError();
    plan_free(p);
    return TSK_ECUDA;
  }
  *out = p;
  return TSK_OK;
}

extern "C" tsk_status tsk_plan_create(tsk_handle h, int64_t count,
                                      const tsk_mat_desc* mats, tsk_prec prec,
                                      const tsk_mat_out* outs, double* err,
                                      double* normA2, tsk_plan* plan) {
  TSK_NVTX_RANGE("tsk_plan_create");
  if (!h || !plan) return TSK_EINVAL;
  return build_plan(h, count, mats, prec, outs, err, normA2, plan);
}

extern "C" tsk_status tsk_plan_execute(tsk_plan p, tsk_stream stream) {
  TSK_NVTX_RANGE("tsk_plan_execute");
  if (!p || !p->exec) return TSK_EINVAL;
  TSK_CUDA(p->h, cudaGraphLaunch(p->exec, (cudaStream_t)stream));
  return TSK_OK;
}

extern "C" tsk_status tsk_plan_destroy(tsk_plan p) {
  if (!p) return TSK_EINVAL;
  cudaDeviceSynchronize();
  plan_free(p);
  return TSK_OK;
}

extern "C" tsk_status tsk_plan_set_probe(tsk_plan p, void* ev_begin,
                                         void* ev_end) {
  if (!p) return TSK_EINVAL;
  if (!ev_begin && !ev_end) {  // remove the probe
    if (!p->probe_begin && !p->probe_end) return TSK_OK;
    TSK_CUDA(p->h, cudaDeviceSynchronize());
    TSK_CUDA(p->h, capture_plan(p, nullptr, nullptr));
    return TSK_OK;
  }
  if (!ev_begin || !ev_end || ev_begin == ev_end) return TSK_EINVAL;
  cudaEvent_t b = (cudaEvent_t)ev_begin, e = (cudaEvent_t)ev_end;
  if (p->probe_begin && p->probe_end) {
    TSK_CUDA(p->h, cudaGraphExecEventRecordNodeSetEvent(p->exec, p->probe_begin, b));
    TSK_CUDA(p->h, cudaGraphExecEventRecordNodeSetEvent(p->exec, p->probe_end, e));
    return TSK_OK;
  }
  TSK_CUDA(p->h, cudaDeviceSynchronize());
  TSK_CUDA(p->h, capture_plan(p, b, e));
  if (!p->probe_begin || !p->probe_end) {
    set_err(p->h, "probe nodes not found in the captured graph");
    return TSK_ECUDA;
  }
  return TSK_OK;
}

extern "C" tsk_status tsk_plan_info(tsk_plan p, int64_t* ws, int32_t* launches) {
  if (!p) return TSK_EINVAL;
  if (ws) *ws = (int64_t)p->ws_bytes + (p->tc ? tc_workspace_bytes(p->tc) : 0);
  if (launches) *launches = p->launches;
  return TSK_OK;
}

static std::vector<unsigned char> plan_key(tsk_handle h, int64_t count,
                                           const tsk_mat_desc* mats,
                                           tsk_prec prec,
                                           const tsk_mat_out* outs,
                                           double* err, double* normA2) {
  std::vector<unsigned char> k;
  auto put = [&k](const void* src, size_t n) {
    const unsigned char* c = (const unsigned char*)src;
    k.insert(k.end(), c, c + n);
  };
  put(&count, sizeof(count));
  put(&prec, sizeof(prec));
  put(&err, sizeof(err));
  put(&normA2, sizeof(normA2));
  put(&h->opts.kernel, sizeof(h->opts.kernel));
  put(&h->opts.refine_q, sizeof(h->opts.refine_q));
  put(&h->opts.err_mode, sizeof(h->opts.err_mode));
  put(&h->opts.small_fp64, sizeof(h->opts.small_fp64));
  put(&h->tune_version, sizeof(h->tune_version));
  put(mats, sizeof(tsk_mat_desc) * count);
  const unsigned char has = outs ? 1 : 0;
  put(&has, 1);
  if (outs) put(outs, sizeof(tsk_mat_out) * count);
  return k;
}

extern "C" tsk_status tsk_approx_batch(tsk_handle h, int64_t count,
                                       const tsk_mat_desc* mats, tsk_prec prec,
                                       const tsk_mat_out* outs, double* err,
                                       double* normA2, tsk_stream stream) {
  TSK_NVTX_RANGE("tsk_approx_batch");
  if (!h) return TSK_EINVAL;
  if (count < 1 || !mats) {
    set_err(h, "count must be >= 1 and mats non-NULL");
    return TSK_EINVAL;
  }
  std::vector<unsigned char> key = plan_key(h, count, mats, prec, outs, err, normA2);
  tsk_plan found = nullptr;
  for (size_t i = 0; i < h->cache.size(); ++i) {
    if (h->cache[i]->key == key) {
      found = h->cache[i];
      h->cache.erase(h->cache.begin() + i);
      h->cache.push_back(found);  // most recently used last
      break;
    }
  }
  if (!found) {
    tsk_status st = build_plan(h, count, mats, prec, outs, err, normA2, &found);
    if (st != TSK_OK) return st;
    found->key = std::move(key);
    if (h->cache.size() >= 8) {
      cudaDeviceSynchronize();
      plan_free(h->cache.front());
      h->cache.erase(h->cache.begin());
    }
    h->cache.push_back(found);
  }
  return tsk_plan_execute(found, stream);
}

// ---------------------------------------------------------------------------
// direct error (one more pass over A)
// ---------------------------------------------------------------------------
extern "C" tsk_status tsk_error(tsk_handle h, int64_t count,
                                const tsk_mat_desc* mats, tsk_prec prec,
                                const tsk_mat_out* outs, double* err,
                                tsk_stream stream) {
  TSK_NVTX_RANGE("tsk_error");
  if (!h) return TSK_EINVAL;
  if (count < 1 || !mats || !outs || !err) {
    set_err(h, "tsk_error: count >= 1 and non-NULL mats, outs, err required");
    return TSK_EINVAL;
  }
  std::vector<MatDev> hm(count);
  std::vector<int2> items;
  for (int64_t i = 0; i < count; ++i) {
    tsk_status st = check_desc(h, mats[i], i, prec);
    if (st != TSK_OK) return st;
    if (!outs[i].US || !outs[i].Vt) {
      set_err(h, "tsk_error: matrix %lld has no US/Vt factors", (long long)i);
      return TSK_EINVAL;
    }
    MatDev& d = hm[i];
    memset(&d, 0, sizeof(d));
    d.A = mats[i].A;
    d.S = mats[i].S;
    d.m = mats[i].m;
    d.n = mats[i].n;
    d.lda = mats[i].lda;
    d.k = mats[i].k;
    d.r = mats[i].r;
    d.US = outs[i].US;
    d.Vt = outs[i].Vt;
    for (long long t = 0; t < (d.m + 15) / 16; ++t) items.push_back(make_int2((int)i, (int)t));
  }
  cudaStream_t s = (cudaStream_t)stream;
  const size_t b1 = align_up(sizeof(MatDev) * count, 256);
  const size_t bytes = b1 + sizeof(int2) * items.size();
  std::vector<unsigned char> staging(bytes);
  memcpy(staging.data(), hm.data(), sizeof(MatDev) * count);
  memcpy(staging.data() + b1, items.data(), sizeof(int2) * items.size());
  void* d = nullptr;
  TSK_CUDA(h, cudaMallocAsync(&d, bytes, s));
  TSK_CUDA(h, cudaMemcpyAsync(d, staging.data(), bytes, cudaMemcpyHostToDevice, s));
  TSK_CUDA(h, cudaMemsetAsync(err, 0, sizeof(double) * count, s));
  TSK_CUDA(h, launch_direct_error((int)prec, (const MatDev*)d,
                                  (const int2*)((unsigned char*)d + b1),
                                  (int)items.size(), err, s));
  TSK_CUDA(h, launch_sqrt_inplace(err, (int)count, s));
  TSK_CUDA(h, cudaFreeAsync(d, s));
  // The pageable staging buffer must outlive the copy.
  TSK_CUDA(h, cudaStreamSynchronize(s));
  return TSK_OK;
}

// ---------------------------------------------------------------------------
// training side
// ---------------------------------------------------------------------------
extern "C" tsk_status tsk_gram(tsk_handle h, const void* const* A, int64_t D,
                               int64_t m, int64_t n, int64_t lda,
                               tsk_prec prec, int32_t mode, double* G,
                               int32_t accumulate, tsk_stream stream) {
  TSK_NVTX_RANGE("tsk_gram");
  if (!h) return TSK_EINVAL;
  if (!A || !G || D < 1 || m < 1 || n < 1 || lda < n || (mode != 1 && mode != 2)) {
    set_err(h, "tsk_gram: need A, G non-NULL, D, m, n >= 1, lda >= n, mode 1 or 2");
    return TSK_EINVAL;
  }
  if (prec != TSK_FP64 && prec != TSK_FP32 && prec != TSK_BF16) {
    set_err(h, "tsk_gram: unknown precision");
    return TSK_EINVAL;
  }
  for (int64_t d = 0; d < D; ++d)
    if (!A[d] || ((uintptr_t)A[d]) % elt_size(prec) != 0) {
      set_err(h, "tsk_gram: A[%lld] is NULL or misaligned", (long long)d);
      return TSK_EINVAL;
    }
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t dim = (mode == 1) ? m : n;
  if (!accumulate) TSK_CUDA(h, cudaMemsetAsync(G, 0, sizeof(double) * dim * dim, s));
  if (h->opts.kernel != TSK_KERNEL_SIMT && gram_tc_eligible((int)prec, mode, A, D, m, n, lda)) {
    // BF16: tcgen05 SYRK (FP32 in TMEM, FP64 in G) on CTA pairs (or single
    // CTAs with gram_tile = 1), both modes; shapes whose tensor maps cannot
    // be encoded go to the CUDA-core kernel below
    const cudaError_t ge =
        launch_gram_tc(A, D, m, n, lda, mode, G, h->d_status, h->opts.spin_limit,
                       h->gram_cache ? h->gram_cache : (h->gram_cache = gram_cache_create()),
                       h->opts.gram_tile == 0, s);
    if (ge != cudaErrorNotSupported) {
      TSK_CUDA(h, ge);
      TSK_CUDA(h, cudaStreamSynchronize(s));
      return TSK_OK;
    }
  }
  void* dA = nullptr;
  TSK_CUDA(h, cudaMallocAsync(&dA, sizeof(void*) * D, s));
  TSK_CUDA(h, cudaMemcpyAsync(dA, A, sizeof(void*) * D, cudaMemcpyHostToDevice, s));
  TSK_CUDA(h, launch_gram((int)prec, (const void* const*)dA, D, m, n, lda, mode, G, s));
  TSK_CUDA(h, cudaFreeAsync(dA, s));
  TSK_CUDA(h, cudaStreamSynchronize(s));  // A (host array) must outlive the copy
  return TSK_OK;
}

extern "C" tsk_status tsk_sketch_from_gram(tsk_handle h, const double* G,
                                           int64_t dim, int32_t k,
                                           tsk_prec prec, void* S, double* eig,
                                           tsk_stream stream) {
  TSK_NVTX_RANGE("tsk_sketch_from_gram");
  if (!h) return TSK_EINVAL;
  if (!G || !S || dim < 1 || k < 1 || k > dim || k > TSK_MAX_K) {
    set_err(h, "tsk_sketch_from_gram: need G, S non-NULL and 1 <= k <= min(dim, %d)",
            TSK_MAX_K);
    return TSK_EINVAL;
  }
  const bool dbl = (prec == TSK_FP64);
  const size_t cs = dbl ? 8 : 4;
  // Oversampling: the block converges at the rate lambda_{p+1}/lambda_k per
  // iteration, and streams whose matrices drift have flat spectra there.
  int p = std::max(2 * k, k + 32);
  p = std::min<int64_t>(p, 96);
  p = std::max(p, (int)k);
  p = (int)std::min<int64_t>(p, dim);
  double tol = h->opts.eig_tol > 0 ? h->opts.eig_tol : (dbl ? 1e-13 : 2e-6);
  cudaStream_t s = (cudaStream_t)stream;
  Carve cv;
  const size_t o_Gc = dbl ? 0 : cv.take(cs * dim * dim);
  const size_t o_Z = cv.take(cs * dim * p);
  const size_t o_W = cv.take(cs * dim * p);
  const size_t o_U = cv.take(cs * dim * p);
  const size_t o_GU = cv.take(cs * dim * p);
  const size_t o_H = cv.take(cs * p * p);
  const size_t o_V = cv.take(cs * p * p);
  const size_t o_th = cv.take(cs * p);
  const size_t o_R = cv.take(cs * p * p);
  const size_t o_res = cv.take(sizeof(double) * k);
  const size_t o_pan = cv.take(sizeof(PanelDev));
  // partial products of the split-K GEMMs (up to 8 splits of dim x p, 64 of
  // p x p)
  const size_t part_bytes = cs * (size_t)std::max<int64_t>(8 * dim * p, 64 * (int64_t)p * p);
  const size_t o_part = cv.take(part_bytes);
  void* ws = nullptr;
  TSK_CUDA(h, cudaMallocAsync(&ws, cv.off, s));
  unsigned char* b = (unsigned char*)ws;
  const void* Gm = dbl ? (const void*)G : (const void*)(b + o_Gc);
  void *Z = b + o_Z, *W = b + o_W, *U = b + o_U, *GU = b + o_GU, *H = b + o_H,
       *V = b + o_V, *th = b + o_th, *R = b + o_R;
  double* res = (double*)(b + o_res);
  PanelDev* dpan = (PanelDev*)(b + o_pan);
  void* part = b + o_part;
  tsk_status result = TSK_OK;
#define TSK_E(call)                                                            \
  do {                                                                         \
    cudaError_t e_ = (call);                                                   \
    if (e_ != cudaSuccess) {                                                   \
      set_err(h, "%s failed: %s", #call, cudaGetErrorString(e_));              \
      cudaFreeAsync(ws, s);                                                    \
      return TSK_ECUDA;                                                        \
    }                                                                          \
  } while (0)
  if (!dbl) TSK_E(launch_convert_gram(false, G, b + o_Gc, dim * dim, s));
  // orth(P) in place through the panel descriptor: R = TSQR(P), P <- P R^{-1}
  auto orth = [&](void* P) -> cudaError_t {
    PanelDev pd;
    pd.P = P;
    pd.rows = dim;
    pd.k = p;
    pd.ld = p;
    pd.R = R;
    cudaError_t e = cudaMemcpyAsync(dpan, &pd, sizeof(pd), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // pd is on the stack
    if (e == cudaSuccess) e = launch_tsqr(dbl, p, dpan, 1, 1, h->d_status, s);
    if (e == cudaSuccess) e = launch_apply_rinv(dbl, P, R, P, dim, p, s);
    return e;
  };
  // FP32: CholeskyQR2 of the block (its Gram, Cholesky, Z <- Z R^{-1}, twice),
  // after scaling column c of G U by 1/theta_c, which leaves it close to
  // orthonormal (G u_c ~ theta_c u_c), so the Gram is well conditioned; R is
  // then close to the identity and Z R^{-1} is taken as a GEMM with the
  // explicit inverse (into U, which is free here, then back).  FP64 keeps the
  // blockwise Householder factorisation.
  auto orth2 = [&](void* P, const void* theta) -> cudaError_t {
    cudaError_t e = cudaSuccess;
    if (theta) e = launch_scale_cols(dbl, P, dim, p, theta, s);
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
      e = launch_gemm(dbl, 1, 0, p, p, dim, 1.0, P, p, P, p, 0.0, H, p, s, part, part_bytes);
      if (e == cudaSuccess) e = launch_chol_inv(dbl, H, p, H, s);
      if (e == cudaSuccess) e = launch_gemm(dbl, 0, 0, dim, p, p, 1.0, P, p, H, p, 0.0, U, p, s);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(P, U, cs * (size_t)dim * p, cudaMemcpyDeviceToDevice, s);
    }
    return e;
  };
  TSK_E(launch_random_fill(dbl, Z, dim * p, 0x5eed5eedull, s));
  TSK_E(dbl ? orth(Z) : orth2(Z, nullptr));
  std::vector<double> hres(k), hth(p);
  std::vector<float> hthf(p);
  double best = 1e300;
  int stall = 0;
  bool converged = false;
  for (int it = 0; it < h->opts.max_iter; ++it) {
    TSK_E(launch_gemm(dbl, 0, 0, dim, p, dim, 1.0, Gm, dim, Z, p, 0.0, W, p, s, part,
                      part_bytes));
    TSK_E(launch_gemm(dbl, 1, 0, p, p, dim, 1.0, Z, p, W, p, 0.0, H, p, s, part, part_bytes));
    TSK_E(launch_sym_eig(dbl, H, p, th, V, s));
    TSK_E(launch_gemm(dbl, 0, 0, dim, p, p, 1.0, Z, p, V, p, 0.0, U, p, s));
    TSK_E(launch_gemm(dbl, 0, 0, dim, p, p, 1.0, W, p, V, p, 0.0, GU, p, s));
    TSK_E(launch_ritz_residual(dbl, U, GU, th, res, dim, p, k, s));
    TSK_E(cudaMemcpyAsync(hres.data(), res, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
    if (dbl)
      TSK_E(cudaMemcpyAsync(hth.data(), th, sizeof(double) * p, cudaMemcpyDeviceToHost, s));
    else
      TSK_E(cudaMemcpyAsync(hthf.data(), th, sizeof(float) * p, cudaMemcpyDeviceToHost, s));
    TSK_E(cudaStreamSynchronize(s));
    if (!dbl)
      for (int c = 0; c < p; ++c) hth[c] = hthf[c];
    const double scale = std::max(std::fabs(hth[0]), 1e-300);
    double worst = 0.0;
    for (int c = 0; c < k; ++c) worst = std::max(worst, hres[c] / scale);
    if (worst <= tol) {
      converged = true;
      break;
    }
    // A residual that stopped improving has reached the rounding floor of
    // the compute type.
    if (worst < 0.999 * best) {
      best = worst;
      stall = 0;
    } else if (++stall >= 4 && worst < 1e3 * tol) {
      converged = true;
      break;
    }
    TSK_E(dbl ? orth(GU) : orth2(GU, th));
    std::swap(Z, GU);
  }
  TSK_E(launch_emit_sketch(dbl, U, dim, p, k, S, s));
  if (eig) {
    TSK_E(cudaMemcpyAsync(eig, hth.data(), sizeof(double) * k, cudaMemcpyHostToDevice, s));
  }
  TSK_E(cudaFreeAsync(ws, s));
  TSK_E(cudaStreamSynchronize(s));
#undef TSK_E
  if (!converged) {
    set_err(h, "eigensolver: residual above %g after %d iterations", tol,
            h->opts.max_iter);
    result = TSK_ENOCONV;
  }
  return result;
}

extern "C" tsk_status tsk_train_sketch(tsk_handle h, const void* const* A,
                                       int64_t D, int64_t m, int64_t n,
                                       int64_t lda, tsk_prec prec, int32_t k,
                                       int32_t l, void* S, void* W,
                                       double* eig, tsk_stream stream) {
  TSK_NVTX_RANGE("tsk_train_sketch");
  if (!h) return TSK_EINVAL;
  if (k < 1 || k > std::min(m, n) || k > TSK_MAX_K || l < 0 ||
      (l > 0 && (l > std::min(m, n) || l > TSK_MAX_K || !W)) || !S) {
    set_err(h, "tsk_train_sketch: need 1 <= k <= min(m, n, %d), 0 <= l <= "
               "min(m, n, %d), S (and W when l > 0) non-NULL", TSK_MAX_K, TSK_MAX_K);
    return TSK_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t dmax = (l > 0) ? std::max(m, n) : m;
  double* G = nullptr;
  TSK_CUDA(h, cudaMallocAsync((void**)&G, sizeof(double) * dmax * dmax, s));
  tsk_status st = tsk_gram(h, A, D, m, n, lda, prec, 1, G, 0, stream);
  tsk_status st2 = TSK_OK;
  if (st == TSK_OK) {
    st = tsk_sketch_from_gram(h, G, m, k, prec, S, eig, stream);
    if (st == TSK_ENOCONV) st2 = st, st = TSK_OK;
  }
  if (st == TSK_OK && l > 0) {
    st = tsk_gram(h, A, D, m, n, lda, prec, 2, G, 0, stream);
    if (st == TSK_OK) {
      st = tsk_sketch_from_gram(h, G, n, l, prec, W, eig ? eig + k : nullptr, stream);
      if (st == TSK_ENOCONV) st2 = st, st = TSK_OK;
    }
  }
  cudaFreeAsync(G, s);
  cudaStreamSynchronize(s);
  return st != TSK_OK ? st : st2;
}

// ---------------------------------------------------------------------------
// learned refiner: IVY loss (Eq. 2.1) gradient and the SGD loop
// ---------------------------------------------------------------------------
namespace {

// Device workspace for one forward + backward over a batch of `cap` matrices
// that share m, n, k and r (slot b always uses the same X / Y offsets).
struct GradWs {
  bool dbl = false;
  int cap = 0, kp = 16, kp2 = 16, k = 0, r = 0;
  long long m = 0, n = 0, zt_stride = 0;
  unsigned char* base = nullptr;
  size_t bytes = 0;
  int2 *ix = nullptr, *iy = nullptr, *ix2 = nullptr, *iy2 = nullptr;
  int nx = 0, ny = 0;
  PanelDev* pan = nullptr;
  void *X = nullptr, *Y = nullptr, *RX = nullptr, *RY = nullptr, *W = nullptr,
       *sig = nullptr, *Zt = nullptr, *X2 = nullptr, *Y2 = nullptr;
  double *norm = nullptr, *norm2 = nullptr, *err = nullptr, *e2 = nullptr;
  int* flags = nullptr;
};

cudaError_t gradws_alloc(GradWs& g, bool dbl, int cap, long long m, long long n, int k,
                         int r, cudaStream_t s) {
  g.dbl = dbl;
  g.cap = cap;
  g.m = m;
  g.n = n;
  g.k = k;
  g.r = r;
  g.kp = ((k + 15) / 16) * 16;
  g.kp2 = ((r + 15) / 16) * 16;
  g.zt_stride = (long long)r * m;
  const size_t cs = dbl ? 8 : 4;
  const int tx = (int)((n + 63) / 64), ty = (int)((m + 63) / 64);
  g.nx = tx * cap;
  g.ny = ty * cap;
  Carve cv;
  const size_t o_ix = cv.take(sizeof(int2) * g.nx), o_iy = cv.take(sizeof(int2) * g.ny);
  const size_t o_pan = cv.take(sizeof(PanelDev) * 2 * cap);
  const size_t o_X = cv.take(cs * cap * n * g.kp), o_Y = cv.take(cs * cap * m * g.kp);
  const size_t o_RX = cv.take(cs * cap * g.kp * g.kp), o_RY = cv.take(cs * cap * g.kp * g.kp);
  const size_t o_W = cv.take(cs * cap * g.kp * g.kp), o_sig = cv.take(cs * cap * g.kp);
  const size_t o_Zt = cv.take(cs * cap * g.zt_stride);
  const size_t o_X2 = cv.take(cs * cap * n * g.kp2), o_Y2 = cv.take(cs * cap * m * g.kp2);
  const size_t o_nrm = cv.take(8 * cap), o_nrm2 = cv.take(8 * cap), o_err = cv.take(8 * cap);
  const size_t o_e2 = cv.take(8 * cap), o_fl = cv.take(4 * cap);
  g.bytes = cv.off;
  cudaError_t e = cudaMallocAsync((void**)&g.base, g.bytes, s);
  if (e != cudaSuccess) return e;
  unsigned char* b = g.base;
  g.ix = (int2*)(b + o_ix);
  g.iy = (int2*)(b + o_iy);
  g.pan = (PanelDev*)(b + o_pan);
  g.X = b + o_X;
  g.Y = b + o_Y;
  g.RX = b + o_RX;
  g.RY = b + o_RY;
  g.W = b + o_W;
  g.sig = b + o_sig;
  g.Zt = b + o_Zt;
  g.X2 = b + o_X2;
  g.Y2 = b + o_Y2;
  g.norm = (double*)(b + o_nrm);
  g.norm2 = (double*)(b + o_nrm2);
  g.err = (double*)(b + o_err);
  g.e2 = (double*)(b + o_e2);
  g.flags = (int*)(b + o_fl);
  std::vector<int2> ix, iy;
  for (int sl = 0; sl < cap; ++sl) {
    for (int t = 0; t < tx; ++t) ix.push_back(make_int2(sl, t));
    for (int t = 0; t < ty; ++t) iy.push_back(make_int2(sl, t));
  }
  std::vector<PanelDev> pan(2 * cap);
  for (int sl = 0; sl < cap; ++sl) {
    pan[2 * sl] = PanelDev{(unsigned char*)g.X + cs * sl * n * g.kp, n, k, g.kp,
                           (unsigned char*)g.RX + cs * sl * g.kp * g.kp};
    pan[2 * sl + 1] = PanelDev{(unsigned char*)g.Y + cs * sl * m * g.kp, m, k, g.kp,
                               (unsigned char*)g.RY + cs * sl * g.kp * g.kp};
  }
  std::vector<unsigned char> host(o_X, 0);
  memcpy(host.data() + o_ix, ix.data(), sizeof(int2) * ix.size());
  memcpy(host.data() + o_iy, iy.data(), sizeof(int2) * iy.size());
  memcpy(host.data() + o_pan, pan.data(), sizeof(PanelDev) * pan.size());
  e = cudaMemcpyAsync(b, host.data(), o_X, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
}

// Forward and backward descriptors of one batch (A pointers of the slots).
void gradws_descs(const GradWs& g, const tsk_mat_desc* const* slots, int count,
                  const void* S, MatDev* fwd, MatDev* bwd) {
  const size_t cs = g.dbl ? 8 : 4;
  for (int sl = 0; sl < count; ++sl) {
    const tsk_mat_desc& d = *slots[sl];
    MatDev f;
    memset(&f, 0, sizeof(f));
    f.A = d.A;
    f.S = S;
    f.m = g.m;
    f.n = g.n;
    f.lda = d.lda;
    f.k = g.k;
    f.r = g.r;
    f.offX = (long long)sl * g.n * g.kp;
    f.offY = (long long)sl * g.m * g.kp;
    f.sigma = (unsigned char*)g.sig + cs * sl * g.kp;
    fwd[sl] = f;
    MatDev bb = f;
    bb.S = (unsigned char*)g.Zt + cs * sl * g.zt_stride;
    bb.k = g.r;
    bb.offX = (long long)sl * g.n * g.kp2;
    bb.offY = (long long)sl * g.m * g.kp2;
    bb.sigma = nullptr;
    bwd[sl] = bb;
  }
}

// One forward + backward: grad (k x m) = mean dL/dS over the batch, and the
// batch loss (device double) when loss != NULL.
cudaError_t gradws_run(const GradWs& g, int in_type, int count, const MatDev* fwd,
                       const MatDev* bwd, void* grad, double* loss, int* status,
                       cudaStream_t s) {
  const int tx = (int)((g.n + 63) / 64), ty = (int)((g.m + 63) / 64);
  cudaError_t e = cudaMemsetAsync(g.norm, 0, 8 * count, s);
  if (e == cudaSuccess) e = launch_sketch_x(in_type, g.kp, fwd, g.ix, tx * count, g.X, g.norm, s);
  if (e == cudaSuccess) e = launch_sketch_y(in_type, g.kp, fwd, g.iy, ty * count, g.X, g.Y, s);
  if (e == cudaSuccess) e = launch_tsqr(g.dbl, g.kp, g.pan, 2 * count, 1, status, s);
  if (e == cudaSuccess)
    e = launch_small_svd(g.dbl, g.kp, fwd, count, g.RX, g.RY, g.W, g.norm, g.err, g.flags, 1,
                         0.0, status, s);
  if (e == cudaSuccess) e = launch_zt(g.dbl, g.kp, fwd, count, g.Y, g.W, g.Zt, g.zt_stride, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(g.norm2, 0, 8 * count, s);
  if (e == cudaSuccess)
    e = launch_sketch_x(in_type, g.kp2, bwd, g.ix, tx * count, g.X2, g.norm2, s);
  if (e == cudaSuccess)
    e = launch_sketch_y(in_type, g.kp2, bwd, g.iy, ty * count, g.X2, g.Y2, s);
  if (e == cudaSuccess)
    e = launch_ivy_grad(g.dbl, g.kp, g.kp2, count, (long long)g.k * g.m, fwd, bwd, g.W, g.sig,
                        g.Zt, g.zt_stride, g.Y2, g.norm, 1.0 / count, grad, s);
  if (e == cudaSuccess && loss) e = launch_batch_loss(count, g.err, g.norm, loss, s);
  return e;
}

tsk_status check_refine_batch(tsk_handle h, const tsk_mat_desc* mats, int64_t count,
                              tsk_prec prec) {
  for (int64_t i = 0; i < count; ++i) {
    tsk_status st = check_desc(h, mats[i], i, prec);
    if (st != TSK_OK) return st;
    if (mats[i].m != mats[0].m || mats[i].n != mats[0].n || mats[i].k != mats[0].k ||
        mats[i].r != mats[0].r) {
      set_err(h, "refiner: every matrix must share m, n, k and r");
      return TSK_EINVAL;
    }
  }
  if (prec == TSK_BF16) {
    set_err(h, "refiner: TSK_FP32 or TSK_FP64 only");
    return TSK_EUNSUPPORTED;
  }
  return TSK_OK;
}

}  // namespace

extern "C" tsk_status tsk_ivy_grad(tsk_handle h, int64_t count, const tsk_mat_desc* mats,
                                   tsk_prec prec, const void* S, void* grad, double* loss,
                                   tsk_stream stream) {
  TSK_NVTX_RANGE("tsk_ivy_grad");
  if (!h) return TSK_EINVAL;
  if (count < 1 || !mats || !S || !grad) {
    set_err(h, "tsk_ivy_grad: count >= 1 and non-NULL mats, S, grad required");
    return TSK_EINVAL;
  }
  tsk_status st = check_refine_batch(h, mats, count, prec);
  if (st != TSK_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  GradWs g;
  TSK_CUDA(h, gradws_alloc(g, prec == TSK_FP64, (int)count, mats[0].m, mats[0].n, mats[0].k,
                           mats[0].r, s));
  std::vector<const tsk_mat_desc*> slots(count);
  for (int64_t i = 0; i < count; ++i) slots[i] = &mats[i];
  std::vector<MatDev> fwd(count), bwd(count);
  gradws_descs(g, slots.data(), (int)count, S, fwd.data(), bwd.data());
  MatDev* d = nullptr;
  TSK_CUDA(h, cudaMallocAsync((void**)&d, sizeof(MatDev) * 2 * count, s));
  TSK_CUDA(h, cudaMemcpyAsync(d, fwd.data(), sizeof(MatDev) * count, cudaMemcpyHostToDevice, s));
  TSK_CUDA(h, cudaMemcpyAsync(d + count, bwd.data(), sizeof(MatDev) * count,
                              cudaMemcpyHostToDevice, s));
  TSK_CUDA(h, gradws_run(g, (int)prec, (int)count, d, d + count, grad, loss, h->d_status, s));
  TSK_CUDA(h, cudaFreeAsync(d, s));
  TSK_CUDA(h, cudaFreeAsync(g.base, s));
  TSK_CUDA(h, cudaStreamSynchronize(s));
  return TSK_OK;
}

extern "C" void tsk_default_refine_options(tsk_refine_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->steps = 2000;
  o->batch = 16;
  o->lr = 1e-3;
  o->eval_every = 100;
  o->seed = 20220929ull;
  o->order = nullptr;
}

extern "C" tsk_status tsk_refine_sketch_steps(tsk_handle h, const tsk_mat_desc* train,
                                              int64_t ntrain, const tsk_mat_desc* val,
                                              int64_t nval, tsk_prec prec,
                                              const tsk_refine_opts* opts,
                                              const void* S_tensor, void* dS,
                                              tsk_refine_state* state, int32_t stop,
                                              double* history, tsk_stream stream) {
  TSK_NVTX_RANGE("tsk_refine_sketch_steps");
  if (!h) return TSK_EINVAL;
  tsk_refine_opts o;
  tsk_default_refine_options(&o);
  if (opts) o = *opts;
  if (!train || ntrain < 1 || !val || nval < 1 || !S_tensor || !dS || o.steps < 0 ||
      o.batch < 1 || o.eval_every < 1 || !state || !state->best || state->step < 0 ||
      state->step > stop || stop > o.steps) {
    set_err(h, "tsk_refine_sketch: bad arguments");
    return TSK_EINVAL;
  }
  tsk_status st = check_refine_batch(h, train, ntrain, prec);
  if (st != TSK_OK) return st;
  st = check_refine_batch(h, val, nval, prec);
  if (st != TSK_OK) return st;
  if (val[0].m != train[0].m || val[0].k != train[0].k || val[0].r != train[0].r) {
    set_err(h, "tsk_refine_sketch: validation and training shapes differ");
    return TSK_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const bool dbl = prec == TSK_FP64;
  const size_t cs = dbl ? 8 : 4;
  const int B = o.batch;
  const long long km = (long long)train[0].k * train[0].m;
  const int t0 = state->step;
  const int nrun = stop - t0;  // steps this call takes
  // batch order of the whole run (the method's random draws, passed in or
  // drawn here): step t takes its batch wherever the run was resumed
  std::vector<int32_t> order((size_t)o.steps * B);
  if (o.order) {
    for (size_t i = 0; i < order.size(); ++i) {
      if (o.order[i] < 0 || o.order[i] >= ntrain) {
        set_err(h, "tsk_refine_sketch: order[%zu] out of range", i);
        return TSK_EINVAL;
      }
      order[i] = o.order[i];
    }
  } else {
    unsigned long long x = o.seed ? o.seed : 1;
    for (size_t i = 0; i < order.size(); ++i) {
      x ^= x << 13;
      x ^= x >> 7;
      x ^= x << 17;
      order[i] = (int32_t)(x % (unsigned long long)ntrain);
    }
  }
  GradWs g;
  TSK_CUDA(h, gradws_alloc(g, dbl, B, train[0].m, train[0].n, train[0].k, train[0].r, s));
  // S_theta, grad, per-step descriptors, losses
  Carve cv;
  const size_t o_St = cv.take(cs * km), o_gr = cv.take(cs * km);
  const size_t o_desc = cv.take(sizeof(MatDev) * 2 * (size_t)std::max(1, nrun) * B);
  const size_t o_loss = cv.take(8 * (size_t)std::max(1, nrun));
  unsigned char* wb = nullptr;
  TSK_CUDA(h, cudaMallocAsync((void**)&wb, cv.off, s));
  void* St = wb + o_St;
  void* gr = wb + o_gr;
  void* best = state->best;
  MatDev* dd = (MatDev*)(wb + o_desc);
  double* dloss = (double*)(wb + o_loss);
  {
    std::vector<MatDev> all(2 * (size_t)std::max(1, nrun) * B);
    std::vector<const tsk_mat_desc*> slots(B);
    for (int i = 0; i < nrun; ++i) {
      const size_t t = (size_t)(t0 + i);
      for (int b = 0; b < B; ++b) slots[b] = &train[order[t * B + b]];
      gradws_descs(g, slots.data(), B, St, &all[(size_t)i * 2 * B], &all[(size_t)i * 2 * B + B]);
    }
    TSK_CUDA(h, cudaMemcpyAsync(dd, all.data(), sizeof(MatDev) * all.size(),
                                cudaMemcpyHostToDevice, s));
    TSK_CUDA(h, cudaStreamSynchronize(s));
  }
  // validation: a test-side plan over the held-out matrices reading S_theta
  std::vector<tsk_mat_desc> vd(val, val + nval);
  for (auto& v : vd) v.S = St;
  double* verr = nullptr;
  double* vnorm = nullptr;
  TSK_CUDA(h, cudaMalloc((void**)&verr, 16 * nval));
  vnorm = verr + nval;
  tsk_plan vplan = nullptr;
  const int save_mode = h->opts.err_mode;
  h->opts.err_mode = 1;
  st = build_plan(h, nval, vd.data(), prec, nullptr, verr, vnorm, &vplan);
  h->opts.err_mode = save_mode;
  if (st != TSK_OK) {
    cudaFree(verr);
    cudaFreeAsync(wb, s);
    cudaFreeAsync(g.base, s);
    return st;
  }
  std::vector<double> he(nval), hn(nval);
  auto validate = [&](double* out) -> tsk_status {
    TSK_CUDA(h, launch_add(dbl, km, S_tensor, dS, St, s));
    TSK_CUDA(h, cudaGraphLaunch(vplan->exec, s));
    TSK_CUDA(h, cudaMemcpyAsync(he.data(), verr, 8 * nval, cudaMemcpyDeviceToHost, s));
    TSK_CUDA(h, cudaMemcpyAsync(hn.data(), vnorm, 8 * nval, cudaMemcpyDeviceToHost, s));
    TSK_CUDA(h, cudaStreamSynchronize(s));
    double l = 0.0;
    for (int64_t i = 0; i < nval; ++i) l += he[i] * he[i] / hn[i];
    *out = l / nval;
    return TSK_OK;
  };
  if (t0 == 0) {
    // the starting dS (zero: the plain tensor sketch) is the reference the
    // result is never worse than
    double l = 0.0;
    st = validate(&l);
    if (st == TSK_OK) {
      state->best_loss = l;
      if (history) history[0] = l;
      cudaMemcpyAsync(best, dS, cs * km, cudaMemcpyDeviceToDevice, s);
    }
  }
  int t = t0;
  for (; st == TSK_OK && t < stop; ++t) {
    cudaError_t e = launch_add(dbl, km, S_tensor, dS, St, s);
    const MatDev* f = dd + (size_t)(t - t0) * 2 * B;
    if (e == cudaSuccess)
      e = gradws_run(g, (int)prec, B, f, f + B, gr, dloss + (t - t0), h->d_status, s);
    if (e == cudaSuccess) e = launch_axpy(dbl, km, -o.lr, gr, dS, s);
    if (e != cudaSuccess) {
      set_err(h, "refiner step %d: %s", t, cudaGetErrorString(e));
      st = TSK_ECUDA;
      break;
    }
    if ((t + 1) % o.eval_every == 0) {
      double l = 0.0;
      st = validate(&l);
      if (st != TSK_OK) break;
      if (history) history[(t + 1) / o.eval_every] = l;
      if (l < state->best_loss) {
        state->best_loss = l;
        cudaMemcpyAsync(best, dS, cs * km, cudaMemcpyDeviceToDevice, s);
      }
    }
  }
  state->step = t;
  cudaStreamSynchronize(s);
  plan_free(vplan);
  cudaFree(verr);
  cudaFreeAsync(wb, s);
  cudaFreeAsync(g.base, s);
  cudaStreamSynchronize(s);
  return st;
}

extern "C" tsk_status tsk_refine_sketch(tsk_handle h, const tsk_mat_desc* train,
                                        int64_t ntrain, const tsk_mat_desc* val, int64_t nval,
                                        tsk_prec prec, const tsk_refine_opts* opts,
                                        const void* S_tensor, void* dS, double* history,
                                        tsk_stream stream) {
  if (!h) return TSK_EINVAL;
  tsk_refine_opts o;
  tsk_default_refine_options(&o);
  if (opts) o = *opts;
  if (!train || ntrain < 1 || !S_tensor || !dS || o.steps < 0 || o.eval_every < 1) {
    set_err(h, "tsk_refine_sketch: bad arguments");
    return TSK_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const size_t cs = prec == TSK_FP64 ? 8 : 4;
  const long long km = (long long)train[0].k * train[0].m;
  if (km < 1) {
    set_err(h, "tsk_refine_sketch: bad arguments");
    return TSK_EINVAL;
  }
  const int nhist = o.steps / o.eval_every + 1;
  if (history)
    for (int i = 0; i < nhist; ++i) history[i] = NAN;
  tsk_refine_state state{};
  TSK_CUDA(h, cudaMallocAsync(&state.best, cs * km, s));
  tsk_status st = tsk_refine_sketch_steps(h, train, ntrain, val, nval, prec, &o, S_tensor, dS,
                                          &state, o.steps, history, stream);
  // keep the best validated dS ("never worse" than the plain tensor sketch)
  if (st == TSK_OK) cudaMemcpyAsync(dS, state.best, cs * km, cudaMemcpyDeviceToDevice, s);
  cudaFreeAsync(state.best, s);
  cudaStreamSynchronize(s);
  return st;
}

// ---------------------------------------------------------------------------
// two-sided sketching: Algorithm 3 (test side) and HOOI (Algorithm 5)
// ---------------------------------------------------------------------------
extern "C" tsk_status tsk_approx_two_sided(tsk_handle h, int64_t count,
                                           const tsk_mat2_desc* mats, tsk_prec prec,
                                           const tsk_mat_out* outs, double* err,
                                           double* normA2, tsk_stream stream) {
  TSK_NVTX_RANGE("tsk_approx_two_sided");
  if (!h) return TSK_EINVAL;
  if (count < 1 || !mats || count > (1 << 22)) {
    set_err(h, "tsk_approx_two_sided: count >= 1 and non-NULL mats required");
    return TSK_EINVAL;
  }
  if (prec != TSK_FP64 && prec != TSK_FP32 && prec != TSK_BF16) {
    set_err(h, "tsk_approx_two_sided: unknown precision");
    return TSK_EINVAL;
  }
  const bool dbl = prec == TSK_FP64;
  const size_t cs = compute_size(prec);
  int kmax = 1, lmax = 1;
  long long rows64 = 0, cols64 = 0;  // the item lists of the sketch kernels
  for (int64_t i = 0; i < count; ++i) {
    const tsk_mat2_desc& d = mats[i];
    if (!d.A || !d.S || !d.W || d.m < 1 || d.n < 1 || d.lda < d.n || d.k < 1 || d.l < 1 ||
        d.k > d.n || d.l > d.m || d.k > TSK_MAX_K || d.l > TSK_MAX_K || d.r < 1 ||
        d.r > std::min(d.k, d.l)) {
      set_err(h, "tsk_approx_two_sided: matrix %lld: need A, S, W non-NULL, lda >= n, "
                 "1 <= r <= min(k, l), k <= min(n, %d), l <= min(m, %d)",
              (long long)i, TSK_MAX_K, TSK_MAX_K);
      return TSK_EINVAL;
    }
    if (((uintptr_t)d.A) % elt_size(prec) || ((uintptr_t)d.S) % cs || ((uintptr_t)d.W) % cs) {
      set_err(h, "tsk_approx_two_sided: matrix %lld: misaligned pointer", (long long)i);
      return TSK_EINVAL;
    }
    kmax = std::max(kmax, d.k);
    lmax = std::max(lmax, d.l);
    rows64 += (d.m + 63) / 64;
    cols64 += (d.n + 63) / 64;
  }
  if (rows64 > 2147483647ll || cols64 > 2147483647ll) {
    set_err(h, "tsk_approx_two_sided: batch too large (its per-block work items exceed a "
               "launch's grid)");
    return TSK_EINVAL;
  }
  const int kp = (kmax + 15) / 16 * 16, lp = (lmax + 15) / 16 * 16;
  // per-matrix descriptors: xm for X (n x kp) and Y (m x kp); zm for the
  // W^T panel (offX, one per distinct W) and Z (m x lp)
  std::vector<MatDev> xm(count), zm(count);
  std::vector<int2> ix, iy;
  std::vector<int4> io_u, io_v;
  std::vector<std::pair<const void*, long long>> wkeys;
  std::vector<long long> woff_of;
  std::vector<int> wl;
  long long offX = 0, offY = 0, offZ = 0, offW = 0;
  for (int64_t i = 0; i < count; ++i) {
    const tsk_mat2_desc& d = mats[i];
    MatDev a;
    memset(&a, 0, sizeof(a));
    a.A = d.A;
    a.S = d.S;
    a.m = d.m;
    a.n = d.n;
    a.lda = d.lda;
    a.k = d.k;
    a.r = d.r;
    a.offX = offX;
    a.offY = offY;
    a.Vt = outs ? outs[i].Vt : nullptr;
    a.sigma = outs ? outs[i].sigma : nullptr;
    MatDev z = a;
    z.S = nullptr;
    z.k = d.l;
    z.offY = offZ;
    z.US = outs ? outs[i].US : nullptr;
    z.Vt = nullptr;
    z.sigma = nullptr;
    long long wo = -1;
    for (size_t t = 0; t < wkeys.size(); ++t)
      if (wkeys[t].first == d.W && wkeys[t].second == d.n && wl[t] == d.l) wo = woff_of[t];
    if (wo < 0) {
      wo = offW;
      wkeys.push_back({d.W, d.n});
      woff_of.push_back(wo);
      wl.push_back(d.l);
      offW += d.n * lp;
    }
    z.offX = wo;
    offX += d.n * kp;
    offY += d.m * kp;
    offZ += d.m * lp;
    for (long long t = 0; t < (d.n + 63) / 64; ++t) ix.push_back(make_int2((int)i, (int)t));
    for (long long t = 0; t < (d.m + 63) / 64; ++t) iy.push_back(make_int2((int)i, (int)t));
    if (z.US)
      for (long long t = 0; t < (d.m + 255) / 256; ++t)
        io_u.push_back(make_int4((int)i, (int)t, 0, 0));
    if (a.Vt)
      for (long long t = 0; t < (d.n + 255) / 256; ++t)
        io_v.push_back(make_int4((int)i, (int)t, 1, 0));
    xm[i] = a;
    zm[i] = z;
  }
  Carve cv;
  const size_t o_xm = cv.take(sizeof(MatDev) * count);
  const size_t o_zm = cv.take(sizeof(MatDev) * count);
  const size_t o_ix = cv.take(sizeof(int2) * ix.size());
  const size_t o_iy = cv.take(sizeof(int2) * iy.size());
  const size_t o_iu = cv.take(sizeof(int4) * std::max<size_t>(1, io_u.size()));
  const size_t o_iv = cv.take(sizeof(int4) * std::max<size_t>(1, io_v.size()));
  const size_t o_px = cv.take(sizeof(PanelDev) * count);
  const size_t o_pz = cv.take(sizeof(PanelDev) * count);
  const size_t host_part = cv.off;
  const size_t o_X = cv.take(cs * offX);
  const size_t o_Y = cv.take(cs * offY);
  const size_t o_Z = cv.take(cs * offZ);
  const size_t o_WT = cv.take(cs * offW);
  const size_t o_RX = cv.take(8 * (size_t)count * kp * kp);
  const size_t o_RZ = cv.take(8 * (size_t)count * lp * lp);
  const size_t o_WX = cv.take(cs * (size_t)count * kp * kp);
  const size_t o_WZ = cv.take(cs * (size_t)count * lp * lp);
  const size_t o_nrm = cv.take(8 * (size_t)count);
  const size_t o_err = cv.take(8 * (size_t)count);
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* base = nullptr;
  TSK_CUDA(h, cudaMallocAsync((void**)&base, cv.off, s));
  std::vector<PanelDev> px(count), pz(count);
  for (int64_t i = 0; i < count; ++i) {
    px[i] = PanelDev{base + o_X + cs * xm[i].offX, xm[i].n, xm[i].k, kp,
                     base + o_RX + 8 * (size_t)i * kp * kp};
    pz[i] = PanelDev{base + o_Z + cs * zm[i].offY, zm[i].m, zm[i].k, lp,
                     base + o_RZ + 8 * (size_t)i * lp * lp};
  }
  std::vector<unsigned char> host(host_part, 0);
  memcpy(host.data() + o_xm, xm.data(), sizeof(MatDev) * count);
  memcpy(host.data() + o_zm, zm.data(), sizeof(MatDev) * count);
  memcpy(host.data() + o_ix, ix.data(), sizeof(int2) * ix.size());
  memcpy(host.data() + o_iy, iy.data(), sizeof(int2) * iy.size());
  if (!io_u.empty()) memcpy(host.data() + o_iu, io_u.data(), sizeof(int4) * io_u.size());
  if (!io_v.empty()) memcpy(host.data() + o_iv, io_v.data(), sizeof(int4) * io_v.size());
  memcpy(host.data() + o_px, px.data(), sizeof(PanelDev) * count);
  memcpy(host.data() + o_pz, pz.data(), sizeof(PanelDev) * count);
  double* d_norm = normA2 ? normA2 : (double*)(base + o_nrm);
  double* d_err = err ? err : (double*)(base + o_err);
  const MatDev* dxm = (const MatDev*)(base + o_xm);
  const MatDev* dzm = (const MatDev*)(base + o_zm);
  cudaError_t e = cudaMemcpyAsync(base, host.data(), host_part, cudaMemcpyHostToDevice, s);
  // panels start zeroed: the kernels leave the padding columns alone
  if (e == cudaSuccess) e = cudaMemsetAsync(base + o_X, 0, o_RX - o_X, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_norm, 0, 8 * count, s);
  for (size_t t = 0; e == cudaSuccess && t < wkeys.size(); ++t)
    e = launch_wt_panel(dbl ? 0 : 1, wkeys[t].first, wl[t], wkeys[t].second, lp,
                        base + o_WT + cs * woff_of[t], s);
  if (e == cudaSuccess)
    e = launch_sketch_x((int)prec, kp, dxm, (const int2*)(base + o_ix), (int)ix.size(),
                        base + o_X, d_norm, s);
  if (e == cudaSuccess)
    e = launch_sketch_y((int)prec, kp, dxm, (const int2*)(base + o_iy), (int)iy.size(),
                        base + o_X, base + o_Y, s);
  if (e == cudaSuccess)  // Z = A W^T: the Y kernel with W^T's panel in place of X
    e = launch_sketch_y((int)prec, lp, dzm, (const int2*)(base + o_iy), (int)iy.size(),
                        base + o_WT, base + o_Z, s);
  if (e == cudaSuccess)
    e = dbl ? launch_tsqr(true, kp, (const PanelDev*)(base + o_px), (int)count, 1, h->d_status, s)
            : launch_tsqr_f32_in_f64(kp, (const PanelDev*)(base + o_px), (int)count, 1, s);
  if (e == cudaSuccess)
    e = dbl ? launch_tsqr(true, lp, (const PanelDev*)(base + o_pz), (int)count, 1, h->d_status, s)
            : launch_tsqr_f32_in_f64(lp, (const PanelDev*)(base + o_pz), (int)count, 1, s);
  if (e == cudaSuccess)
    e = launch_two_sided_small(dbl, kp, lp, dxm, dzm, (int)count, base + o_Y, base + o_Z,
                               (const double*)(base + o_RX), (const double*)(base + o_RZ),
                               base + o_WX, base + o_WZ, d_norm, d_err, h->d_status, s);
  if (e == cudaSuccess && !io_u.empty())  // US = Z (R_Z^{-1} U_r Sigma_r)
    e = launch_project_out(dbl, lp, dzm, (const int4*)(base + o_iu), (int)io_u.size(),
                           base + o_X, base + o_Z, base + o_WZ, s);
  if (e == cudaSuccess && !io_v.empty())  // Vt = (X R_X^{-1} V_r)^T
    e = launch_project_out(dbl, kp, dxm, (const int4*)(base + o_iv), (int)io_v.size(),
                           base + o_X, base + o_Y, base + o_WX, s);
  cudaFreeAsync(base, s);
  const cudaError_t se = cudaStreamSynchronize(s);  // host staging must outlive the copy
  if (e == cudaSuccess) e = se;
  if (e != cudaSuccess) {
    set_err(h, "tsk_approx_two_sided: %s", cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? TSK_ENOMEM : TSK_ECUDA;
  }
  return TSK_OK;
}

extern "C" tsk_status tsk_train_two_sided(tsk_handle h, const void* const* A, int64_t D,
                                          int64_t m, int64_t n, int64_t lda, tsk_prec prec,
                                          int32_t k, int32_t l, int32_t max_sweeps, double tol,
                                          void* S, void* W, double* core_energy,
                                          int32_t* sweeps_out, tsk_stream stream) {
  TSK_NVTX_RANGE("tsk_train_two_sided");
  if (!h) return TSK_EINVAL;
  if (!A || D < 1 || m < 1 || n < 1 || lda < n || k < 1 || l < 1 || k > std::min(m, n) ||
      l > std::min(m, n) || k > TSK_MAX_K || l > TSK_MAX_K || !S || !W || max_sweeps < 0) {
    set_err(h, "tsk_train_two_sided: need A, S, W non-NULL, D, m, n >= 1, lda >= n, "
               "1 <= k, l <= min(m, n, %d)", TSK_MAX_K);
    return TSK_EINVAL;
  }
  if (prec != TSK_FP64 && prec != TSK_FP32 && prec != TSK_BF16) {
    set_err(h, "tsk_train_two_sided: unknown precision");
    return TSK_EINVAL;
  }
  // the sketch kernels take one CTA per (matrix, 64-wide block): D times the
  // blocks of a matrix must fit a launch's grid
  if (D > 2147483647ll / std::max((m + 63) / 64, (n + 63) / 64)) {
    set_err(h, "tsk_train_two_sided: D * ceil(max(m, n) / 64) exceeds a launch's grid");
    return TSK_EINVAL;
  }
  for (int64_t d = 0; d < D; ++d)
    if (!A[d] || ((uintptr_t)A[d]) % elt_size(prec) != 0) {
      set_err(h, "tsk_train_two_sided: A[%lld] is NULL or misaligned", (long long)d);
      return TSK_EINVAL;
    }
  const bool dbl = prec == TSK_FP64;
  const size_t cs = compute_size(prec);
  const int ctype = dbl ? 0 : 1;  // element type of the projected panels
  if (tol <= 0) tol = dbl ? 1e-12 : 1e-7;
  const int kp = (k + 15) / 16 * 16, lp = (l + 15) / 16 * 16;
  cudaStream_t s = (cudaStream_t)stream;
  // HOSVD start: S from the mode-1 Gram, W from the mode-2 Gram
  const int64_t dmax = std::max(m, n);
  double* G = nullptr;
  TSK_CUDA(h, cudaMallocAsync((void**)&G, sizeof(double) * dmax * dmax, s));
  tsk_status st = tsk_gram(h, A, D, m, n, lda, prec, 1, G, 0, stream);
  tsk_status noconv = TSK_OK;
  auto eig_step = [&](int64_t dim, int32_t kk, void* out, double* eig) -> tsk_status {
    tsk_status r = tsk_sketch_from_gram(h, G, dim, kk, prec == TSK_BF16 ? TSK_FP32 : prec,
                                        out, eig, stream);
    if (r == TSK_ENOCONV) noconv = r, r = TSK_OK;
    return r;
  };
  if (st == TSK_OK) st = eig_step(m, k, S, nullptr);
  if (st == TSK_OK) st = tsk_gram(h, A, D, m, n, lda, prec, 2, G, 0, stream);
  double* d_eig = nullptr;
  if (st == TSK_OK && cudaMallocAsync((void**)&d_eig, sizeof(double) * 64, s) != cudaSuccess)
    st = TSK_ENOMEM;
  if (st == TSK_OK) st = eig_step(n, l, W, d_eig);
  double total = 0.0;
  {  // sum_d ||A_d||^2 = trace of the mode-2 Gram just formed
    std::vector<double> diag(n);
    if (st == TSK_OK &&
        cudaMemcpy2DAsync(diag.data(), sizeof(double), G, sizeof(double) * (n + 1),
                          sizeof(double), n, cudaMemcpyDeviceToHost, s) == cudaSuccess &&
        cudaStreamSynchronize(s) == cudaSuccess)
      for (double v : diag) total += v;
  }
  // projected panels of every training matrix: Z_d = A_d W^T (m x lp) and
  // X_d = A_d^T S^T (n x kp); descriptors for both
  Carve cv;
  const size_t o_md = cv.take(sizeof(MatDev) * D);
  const size_t o_mz = cv.take(sizeof(MatDev) * D);
  const size_t o_ix = cv.take(sizeof(int2) * D * ((n + 63) / 64));
  const size_t o_iy = cv.take(sizeof(int2) * D * ((m + 63) / 64));
  const size_t o_pz = cv.take(sizeof(void*) * D);
  const size_t o_px = cv.take(sizeof(void*) * D);
  const size_t host_part = cv.off;
  const size_t o_Z = cv.take(cs * (size_t)D * m * lp);
  const size_t o_X = cv.take(cs * (size_t)D * n * kp);
  const size_t o_WT = cv.take(cs * (size_t)n * lp);
  const size_t o_nrm = cv.take(8 * (size_t)D);
  unsigned char* base = nullptr;
  if (st == TSK_OK && cudaMallocAsync((void**)&base, cv.off, s) != cudaSuccess) st = TSK_ENOMEM;
  int sweeps = 0;
  double energy = 0.0;
  if (st == TSK_OK) {
    std::vector<unsigned char> host(host_part, 0);
    MatDev* md = (MatDev*)(host.data() + o_md);
    MatDev* mz = (MatDev*)(host.data() + o_mz);
    int2* ix = (int2*)(host.data() + o_ix);
    int2* iy = (int2*)(host.data() + o_iy);
    void** pz = (void**)(host.data() + o_pz);
    void** px = (void**)(host.data() + o_px);
    const long long tx = (n + 63) / 64, ty = (m + 63) / 64;
    for (int64_t d = 0; d < D; ++d) {
      MatDev a;
      memset(&a, 0, sizeof(a));
      a.A = A[d];
      a.S = S;
      a.m = m;
      a.n = n;
      a.lda = lda;
      a.k = k;
      a.r = 1;
      a.offX = d * n * kp;
      a.offY = 0;
      md[d] = a;
      MatDev z = a;
      z.S = nullptr;
      z.k = l;
      z.offX = 0;  // the one W^T panel
      z.offY = d * m * lp;
      mz[d] = z;
      for (long long t = 0; t < tx; ++t) ix[d * tx + t] = make_int2((int)d, (int)t);
      for (long long t = 0; t < ty; ++t) iy[d * ty + t] = make_int2((int)d, (int)t);
      pz[d] = base + o_Z + cs * (size_t)d * m * lp;
      px[d] = base + o_X + cs * (size_t)d * n * kp;
    }
    cudaError_t e = cudaMemcpyAsync(base, host.data(), host_part, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + o_Z, 0, o_nrm - o_Z, s);
    double prev = -1.0;
    std::vector<double> hl(64);
    for (int sw = 1; e == cudaSuccess && st == TSK_OK && sw <= max_sweeps; ++sw) {
      // mode 1: S <- top k eigenvectors of sum_d (A_d W^T)(A_d W^T)^T
      e = launch_wt_panel(dbl ? 0 : 1, W, l, n, lp, base + o_WT, s);
      if (e == cudaSuccess)
        e = launch_sketch_y((int)prec, lp, (const MatDev*)(base + o_mz),
                            (const int2*)(base + o_iy), (int)(D * ty), base + o_WT, base + o_Z,
                            s);
      if (e == cudaSuccess) e = cudaMemsetAsync(G, 0, sizeof(double) * m * m, s);
      if (e == cudaSuccess)
        e = launch_gram(ctype, (const void* const*)(base + o_pz), D, m, lp, lp, 1, G, s);
      if (e != cudaSuccess) break;
      st = eig_step(m, k, S, nullptr);
      if (st != TSK_OK) break;
      // mode 2: W <- top l eigenvectors of sum_d (S A_d)^T (S A_d)
      e = cudaMemsetAsync(base + o_nrm, 0, 8 * D, s);
      if (e == cudaSuccess)
        e = launch_sketch_x((int)prec, kp, (const MatDev*)(base + o_md),
                            (const int2*)(base + o_ix), (int)(D * tx), base + o_X,
                            (double*)(base + o_nrm), s);
      if (e == cudaSuccess) e = cudaMemsetAsync(G, 0, sizeof(double) * n * n, s);
      if (e == cudaSuccess)
        e = launch_gram(ctype, (const void* const*)(base + o_px), D, n, kp, kp, 1, G, s);
      if (e != cudaSuccess) break;
      st = eig_step(n, l, W, d_eig);
      if (st != TSK_OK) break;
      // core energy sum_d ||S A_d W^T||^2 = sum of the top l eigenvalues
      e = cudaMemcpyAsync(hl.data(), d_eig, sizeof(double) * l, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) break;
      energy = 0.0;
      for (int i = 0; i < l; ++i) energy += hl[i];
      sweeps = sw;
      if (prev >= 0.0 && std::fabs(energy - prev) < tol * total) break;
      prev = energy;
    }
    if (e != cudaSuccess && st == TSK_OK) {
      set_err(h, "tsk_train_two_sided: %s", cudaGetErrorString(e));
      st = TSK_ECUDA;
    }
  }
  if (base) cudaFreeAsync(base, s);
  if (d_eig) cudaFreeAsync(d_eig, s);
  cudaFreeAsync(G, s);
  cudaStreamSynchronize(s);
  if (core_energy) *core_energy = energy;
  if (sweeps_out) *sweeps_out = sweeps;
  return st != TSK_OK ? st : noconv;
}

// ---------------------------------------------------------------------------
// autotuner of the tensor-core sketch: rows of A per CTA by size class
// ---------------------------------------------------------------------------
extern "C" tsk_status tsk_autotune(tsk_handle h, int64_t count, const tsk_mat_desc* mats,
                                   tsk_prec prec, int32_t reps, tsk_stream stream) {
  TSK_NVTX_RANGE("tsk_autotune");
  if (!h) return TSK_EINVAL;
  if (count < 1 || !mats || prec != TSK_BF16) {
    set_err(h, "tsk_autotune: count >= 1, non-NULL mats and TSK_BF16 required");
    return TSK_EINVAL;
  }
  if (reps < 1) reps = 5;
  for (int64_t i = 0; i < count; ++i) {
    tsk_status st = check_desc(h, mats[i], i, prec);
    if (st != TSK_OK) return st;
  }
  if (!tc_supported()) return TSK_OK;  // nothing to tune
  // classes where more than one shape exists: 256 < m <= 2304 (CTAs of 256
  // rows up to m = 2048, of 384 rows up to 2304 when k <= 40, of 512 rows)
  std::map<std::pair<int, int>, std::vector<tsk_mat_desc>> byk;
  for (int64_t i = 0; i < count; ++i) {
    const tsk_mat_desc& d = mats[i];
    if (!tc_eligible_one(d) || d.m <= 256 || d.m > 2304) continue;
    // every matrix of the class (up to 2048): a shape's throughput depends on
    // how many SMs the class fills, so a small sample can rank the shapes
    // the wrong way round (wider clusters win while SMs are idle)
    auto& v = byk[tune_key(d.m, d.k)];
    if (v.size() < 2048) v.push_back(d);
  }
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  TSK_CUDA(h, cudaEventCreate(&e0));
  TSK_CUDA(h, cudaEventCreate(&e1));
  tsk_status result = TSK_OK;
  const int save_force = h->force_mc;
  for (auto& kv : byk) {
    const std::vector<tsk_mat_desc>& v = kv.second;
    int mmax = 0, kmax = 0;
    for (const tsk_mat_desc& d : v) {
      mmax = std::max<int>(mmax, (int)d.m);
      kmax = std::max(kmax, d.k);
    }
    const int shapes[3] = {512, 256, 384};
    bool valid[3] = {true, mmax <= 2048, (kmax + 7) / 8 * 8 <= 40};
    double us[3] = {0.0, 0.0, 0.0};
    for (int c = 0; c < 3 && result == TSK_OK; ++c) {
      if (!valid[c]) continue;
      h->force_mc = shapes[c];
      tsk_plan p = nullptr;
      result = build_plan(h, (int64_t)v.size(), v.data(), prec, nullptr, nullptr, nullptr, &p);
      if (result != TSK_OK) break;
      cudaError_t e = capture_plan(p, e0, e1);  // events around the sketch pass
      float best = 1e30f;
      for (int r = 0; e == cudaSuccess && r < reps + 1; ++r) {
        e = cudaGraphLaunch(p->exec, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && r > 0) best = std::min(best, ms);  // the first warms up
      }
      plan_free(p);
      if (e != cudaSuccess) {
        set_err(h, "tsk_autotune: %s", cudaGetErrorString(e));
        result = TSK_ECUDA;
        break;
      }
      us[c] = 1e3 * best / (double)v.size();
    }
    if (result != TSK_OK) break;
    int best = 0;
    for (int c = 1; c < 3; ++c)
      if (valid[c] && us[c] < us[best]) best = c;
    h->tune[kv.first] = shapes[best];
    h->tune_us[kv.first] = {us[0], valid[1] ? us[1] : 0.0, valid[2] ? us[2] : 0.0};
  }
  h->force_mc = save_force;
  ++h->tune_version;  // plans built from now on use the table
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (result == TSK_OK) {
    int st = 0;
    cudaMemcpy(&st, h->d_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (st & kStatusTimeout) {
      set_err(h, "tsk_autotune: a bounded device wait ran out");
      result = TSK_ETIMEOUT;
    }
  }
  return result;
}

extern "C" tsk_status tsk_autotune_save(tsk_handle h, const char* path) {
  if (!h || !path) return TSK_EINVAL;
  FILE* f = fopen(path, "w");
  if (!f) {
    set_err(h, "tsk_autotune_save: cannot open %s", path);
    return TSK_EINVAL;
  }
  fprintf(f, "{\"kernel\": \"sketch_tc\", \"classes\": [");
  bool first = true;
  for (auto& kv : h->tune) {
    std::vector<double> us = h->tune_us.count(kv.first) ? h->tune_us[kv.first]
                                                        : std::vector<double>(3, 0.0);
    us.resize(3, 0.0);
    // a shape that was not timed (not valid for the class) is written as 0
    fprintf(f, "%s\n  {\"cluster_at_512\": %d, \"k8\": %d, \"rows_per_cta\": %d, "
               "\"us_per_matrix_512\": %.4f, \"us_per_matrix_256\": %.4f, "
               "\"us_per_matrix_384\": %.4f}",
            first ? "" : ",", kv.first.first, kv.first.second, kv.second, us[0], us[1], us[2]);
    first = false;
  }
  fprintf(f, "\n]}\n");
  fclose(f);
  return TSK_OK;
}

extern "C" tsk_status tsk_autotune_load(tsk_handle h, const char* path) {
  if (!h || !path) return TSK_EINVAL;
  FILE* f = fopen(path, "r");
  if (!f) {
    set_err(h, "tsk_autotune_load: cannot open %s", path);
    return TSK_EINVAL;
  }
  std::string text;
  char buf[4096];
  size_t got;
  while ((got = fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, got);
  fclose(f);
  // the entries this library writes: one object per class, fields by name
  auto field = [](const std::string& obj, const char* name, double* out) {
    const std::string key = std::string("\"") + name + "\"";
    size_t p = obj.find(key);
    if (p == std::string::npos) return false;
    p = obj.find(':', p + key.size());
    if (p == std::string::npos) return false;
    char* end = nullptr;
    *out = strtod(obj.c_str() + p + 1, &end);
    return end != obj.c_str() + p + 1;
  };
  std::map<std::pair<int, int>, int> table;
  size_t pos = text.find("\"classes\"");
  if (pos == std::string::npos) {
    set_err(h, "tsk_autotune_load: %s has no \"classes\"", path);
    return TSK_EINVAL;
  }
  while ((pos = text.find('{', pos + 1)) != std::string::npos) {
    const size_t end = text.find('}', pos);
    if (end == std::string::npos) break;
    const std::string obj = text.substr(pos, end - pos + 1);
    double c = 0, k8 = 0, mc = 0;
    if (!field(obj, "cluster_at_512", &c) || !field(obj, "k8", &k8) ||
        !field(obj, "rows_per_cta", &mc) || (mc != 256 && mc != 384 && mc != 512)) {
      set_err(h, "tsk_autotune_load: malformed entry in %s", path);
      return TSK_EINVAL;
    }
    table[{(int)c, (int)k8}] = (int)mc;
    pos = end;
  }
  h->tune = table;
  h->tune_us.clear();
  ++h->tune_version;
  return TSK_OK;
}

// ---------------------------------------------------------------------------
// FP8 (E4M3) training Gram: quantization with per-(group, row) scales and the
// tensor-core Gram of the E4M3 copies
// ---------------------------------------------------------------------------
extern "C" tsk_status tsk_quantize_e4m3(tsk_handle h, const void* const* A, int64_t D,
                                        int64_t m, int64_t n, int64_t lda, tsk_prec prec,
                                        void* const* A8, int64_t ld8, float* scales,
                                        tsk_stream stream) {
  TSK_NVTX_RANGE("tsk_quantize_e4m3");
  if (!h) return TSK_EINVAL;
  if (!A || !A8 || !scales || D < 1 || D > 65535 || m < 1 || n < 1 || lda < n || ld8 < n ||
      (prec != TSK_FP32 && prec != TSK_BF16)) {
    set_err(h, "tsk_quantize_e4m3: need A, A8, scales non-NULL, 1 <= D <= 65535, m, n >= 1, "
               "lda >= n, ld8 >= n and TSK_FP32 or TSK_BF16 input");
    return TSK_EINVAL;
  }
  for (int64_t d = 0; d < D; ++d)
    if (!A[d] || !A8[d] || ((uintptr_t)A[d]) % elt_size(prec) != 0) {
      set_err(h, "tsk_quantize_e4m3: A[%lld] or A8[%lld] is NULL or misaligned", (long long)d,
              (long long)d);
      return TSK_EINVAL;
    }
  // 16-byte loads and 8-byte (BF16) or 4-byte (FP32) stores where every
  // row of every matrix starts aligned for them
  const int per = prec == TSK_BF16 ? 8 : 4;
  bool vec = (lda * elt_size(prec)) % 16 == 0 && ld8 % per == 0;
  for (int64_t d = 0; d < D && vec; ++d)
    vec = ((uintptr_t)A[d]) % 16 == 0 && ((uintptr_t)A8[d]) % per == 0;
  cudaStream_t s = (cudaStream_t)stream;
  void* dp = nullptr;
  TSK_CUDA(h, cudaMallocAsync(&dp, 2 * sizeof(void*) * D, s));
  std::vector<const void*> ptrs(2 * D);
  for (int64_t d = 0; d < D; ++d) {
    ptrs[d] = A[d];
    ptrs[D + d] = A8[d];
  }
  TSK_CUDA(h, cudaMemcpyAsync(dp, ptrs.data(), 2 * sizeof(void*) * D, cudaMemcpyHostToDevice, s));
  TSK_CUDA(h, launch_quantize_e4m3((int)prec, (const void* const*)dp, D, m, n, lda,
                                   (unsigned char* const*)dp + D, ld8, scales, vec, s));
  TSK_CUDA(h, cudaFreeAsync(dp, s));
  TSK_CUDA(h, cudaStreamSynchronize(s));  // the host pointer array must outlive the copy
  return TSK_OK;
}

extern "C" tsk_status tsk_gram_e4m3(tsk_handle h, const void* const* A8, const float* scales,
                                    int64_t D, int64_t m, int64_t n, int64_t ld8, double* G,
                                    int32_t accumulate, tsk_stream stream) {
  TSK_NVTX_RANGE("tsk_gram_e4m3");
  if (!h) return TSK_EINVAL;
  if (!A8 || !scales || !G || D < 1 || m < 1 || n < 1 || ld8 < n || ld8 % 16 != 0) {
    set_err(h, "tsk_gram_e4m3: need A8, scales, G non-NULL, D, m, n >= 1, ld8 >= n and a "
               "multiple of 16");
    return TSK_EINVAL;
  }
  for (int64_t d = 0; d < D; ++d)
    if (!A8[d] || ((uintptr_t)A8[d]) % 16 != 0) {
      set_err(h, "tsk_gram_e4m3: A8[%lld] is NULL or not 16-byte aligned", (long long)d);
      return TSK_EINVAL;
    }
  if (!tc_supported()) {
    set_err(h, "tsk_gram_e4m3: needs the tensor cores of a GB300");
    return TSK_EUNSUPPORTED;
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (!accumulate) TSK_CUDA(h, cudaMemsetAsync(G, 0, sizeof(double) * m * m, s));
  if (!h->gram_cache) h->gram_cache = gram_cache_create();
  const cudaError_t ge = launch_gram_tc(A8, D, m, n, ld8, 1, G, h->d_status, h->opts.spin_limit,
                                        h->gram_cache, true, s, scales);
  if (ge == cudaErrorNotSupported) {
    set_err(h, "tsk_gram_e4m3: tensor maps cannot be encoded for these shapes");
    return TSK_EUNSUPPORTED;
  }
  TSK_CUDA(h, ge);
  TSK_CUDA(h, cudaStreamSynchronize(s));
  return TSK_OK;
}
