// C ABI of libkm.so (declared in include/km.h): context, device buffers,
// launches of the assign and update kernels, and the loop drivers (one host
// round trip per step, or a CUDA graph of unrolled steps whose kernels stop
// themselves once the device-side stop flag is set).
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/km.h"

#include "km_internal.cuh"

using namespace km;

namespace km {
// allocations left before the injected failure (< 0: off)
static std::atomic<long long> g_alloc_countdown{-1};
bool inject_alloc_failure() {
  long long v = g_alloc_countdown.load();
  while (v >= 0) {
    if (g_alloc_countdown.compare_exchange_weak(v, v - 1)) return v == 0;
  }
  return false;
}
// The fused kernel's constant-bank screen table exists once per device (a
// module-level __constant__ array), so at most one context per device may use
// it at a time: the context that claims it at km_create keeps it until
// km_destroy; the others read their tables from shared memory.
static std::atomic<int> g_const_tab_owner[64];
static bool claim_const_tab(int dev) {
  if (dev < 0 || dev >= 64) return false;
  int expected = 0;
  return g_const_tab_owner[dev].compare_exchange_strong(expected, 1);
}
static void release_const_tab(int dev) {
  if (dev >= 0 && dev < 64) g_const_tab_owner[dev].store(0);
}
}  // namespace km

struct km_ctx {
  int64_t n = 0;
  int d = 0, k = 0;
  km_options opt{};
  cudaStream_t st = nullptr;
  bool own_stream = false;
  int dev = 0, sms = 0;
  bool fast = false;
  bool tcs = false;  // the fused step screens on the tensor cores (tcgen05 TF32; d <= 3, K <= 32)
  int kpad = 0;
  // points
  float* x_own = nullptr;
  const float* x = nullptr;
  int64_t ld = 0;
  bool have_points = false, have_init = false;
  // per-step buffers
  int32_t* labels = nullptr;
  uint8_t* labels8 = nullptr;  // labels as bytes (label_bytes = 1); labels is then not allocated
  double* mu = nullptr;
  long long* counts = nullptr;
  long long* partials = nullptr;
  int G = 0;
  long long* s128 = nullptr;
  int RB = 0;
  unsigned long long* tab2 = nullptr;
  float4* ctil4 = nullptr;
  float* ctil = nullptr;
  float* cnorm = nullptr;
  float* shift = nullptr;
  float* gen_bmax = nullptr;
  DataConst* dc = nullptr;
  IterConst* ic = nullptr;
  LoopState* ls = nullptr;
  float* scan = nullptr;  // [2d] min/max + [1] amax
  unsigned long long* scan_bad = nullptr;
  size_t fast_smem = 0;
  int nwin = 2;  // fused path: sum windows per warp
  bool const_tab = false;  // this context holds the device's constant-bank screen table
  int grid_ex = 0;         // fixed-point grid exponent: |x| < 2^(grid_ex - 1), G0 = grid_ex - 44
  int grid_ex_local = 0;   // the exponent this context's own points need
  long long* shard_out = nullptr;  // [k][d+1][2] column totals (host-memory requests)
  long long* shard_in = nullptr;   // [ranks][k][d+1][2] gathered totals (host-memory requests)
  int shard_in_ranks = 0;
  int path = 0;  // 1 fused (d <= 4, K <= 256), 2 generic, 3 tensor cores (d = 64, K <= 1024),
                 // 4 fused with the tcgen05 TF32 screen (d <= 3, K <= 32)
  // tensor-core path
  void* xb = nullptr;
  float* xa_pt = nullptr;
  float* xaos = nullptr;
  void* cbf = nullptr;
  float* nprime = nullptr;
  GemmConst* gc = nullptr;
  int32_t* rescue_list = nullptr;
  int4* tie_list = nullptr;
  unsigned* rescue_count = nullptr;  // [2]: rescue and near-tie list lengths
  // sorted mean calculation
  unsigned long long* ms_counts = nullptr;
  int64_t* ms_offsets = nullptr;
  int* ms_cfirst = nullptr;
  unsigned long long* ms_cursor = nullptr;
  int4* ms_chunks = nullptr;
  int* ms_nchunks = nullptr;
  long long* ms_chunk_sums = nullptr;
  int32_t* ms_perm = nullptr;
  double* ms_df2 = nullptr;
  double* bnorm = nullptr;
  int ms_max_chunks = 0;
  float A_max = 0.f;
  int tc_ex = 0;           // FP16 tensor-core operands: points scaled by 2^tc_ex
  int G0 = 0;
  // loop
  cudaGraphExec_t graph = nullptr;
  int graph_unroll = 16;
  LoopState host_ls{};
  std::string err;
};

namespace {

km_status fail(km_ctx* c, km_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

#define KM_CUDA(ctx, call)                                                                   \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return fail((ctx), e_ == cudaErrorMemoryAllocation ? KM_ENOMEM : KM_ECUDA,             \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                      \
  } while (0)

template <class T>
cudaError_t dalloc(T** p, size_t count) {
  if (inject_alloc_failure()) return cudaErrorMemoryAllocation;
  return cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T) + 16);
}

void free_all(km_ctx* c) {
  if (c->const_tab) release_const_tab(c->dev);
  c->const_tab = false;
  if (c->graph) cudaGraphExecDestroy(c->graph);
  c->graph = nullptr;
  void* bufs[] = {c->x_own, c->labels, c->labels8, c->mu, c->counts, c->partials, c->s128, c->tab2,
                  c->ctil4, c->ctil, c->cnorm, c->shift, c->gen_bmax, c->dc, c->ic, c->ls,
                  c->scan, c->scan_bad, c->xb, c->xa_pt, c->xaos, c->cbf, c->nprime, c->gc,
                  c->ms_counts, c->ms_offsets, c->ms_cfirst, c->ms_cursor, c->ms_chunks, c->ms_nchunks,
                  c->ms_chunk_sums, c->ms_perm, c->rescue_list, c->tie_list, c->rescue_count, c->ms_df2, c->bnorm,
                  c->shard_out, c->shard_in};
  for (void* b : bufs)
    if (b) cudaFree(b);
  if (c->own_stream && c->st) cudaStreamDestroy(c->st);
}

UpdateArgs update_args(km_ctx* c) {
  UpdateArgs u{};
  u.partials = c->partials; u.G = c->G; u.k = c->k; u.d = c->d;
  u.s128 = c->s128; u.RB = c->RB;
  u.mu = c->mu; u.counts = c->counts;
  u.dc = c->dc; u.ic = c->ic; u.ls = c->ls;
  u.tab2 = c->tab2; u.ctil4 = c->ctil4; u.ctil = c->ctil; u.cnorm = c->cnorm;
  u.shift = c->shift; u.kpad = c->kpad; u.fast = c->fast ? 1 : 0;
  u.tie_rel = c->opt.tie_rel; u.A_max = c->A_max; u.gen_bmax = c->gen_bmax;
  return u;
}

GemmPrepArgs gemm_prep_args(km_ctx* c) {
  GemmPrepArgs g{};
  g.mu = c->mu; g.shift = c->shift; g.k = c->k; g.kpad = c->kpad;
  g.cb = c->cbf; g.nprime = c->nprime; g.ctil = c->ctil; g.gc = c->gc;
  g.A_max = c->A_max; g.tie_rel = c->opt.tie_rel; g.ls = c->ls; g.bnorm = c->bnorm;
  g.f16 = c->opt.tc_operands == KM_TC_F16 ? 1 : 0; g.ex = c->tc_ex;
  return g;
}

MsortArgs msort_args(km_ctx* c) {
  MsortArgs m{};
  m.labels = c->labels; m.n = c->n; m.k = c->k; m.d = c->d; m.xa = c->xaos; m.dc = c->dc;
  m.counts_u = c->ms_counts; m.offsets = c->ms_offsets; m.cfirst = c->ms_cfirst; m.cursor = c->ms_cursor;
  m.chunks = c->ms_chunks; m.nchunks = c->ms_nchunks; m.max_chunks = c->ms_max_chunks;
  m.chunk_sums = c->ms_chunk_sums; m.perm = c->ms_perm; m.mu = c->mu; m.counts = c->counts; m.ls = c->ls;
  m.df2 = c->ms_df2;
  return m;
}

// Screen tables from the current centroids.
cudaError_t launch_tables(km_ctx* c) {
  if (c->path == 3) return launch_gemm_prepare(c->st, gemm_prep_args(c));
  return launch_prepare(c->st, update_args(c));
}

// Reassignment (+ per-block sums on paths 1 and 2), one kernel.
// labels_pass: the final-labels pass of the "final" label policy (writes the
// labels of the current centroids even after the stop flag; the per-block
// sums it also forms are not used).
cudaError_t launch_assign(km_ctx* c, bool labels_pass = false) {
  cudaError_t e;
  const int store = (c->opt.label_policy == KM_LABELS_EVERY_STEP || labels_pass) ? 1 : 0;
  if (c->path == 3) {
    GemmArgs g{};
    g.xb = c->xb; g.xa = c->xa_pt; g.xaos = c->xaos; g.cb = c->cbf; g.nprime = c->nprime; g.ctil = c->ctil;
    g.mu = c->mu; g.shift = c->shift; g.gc = c->gc; g.ls = c->ls; g.labels = c->labels;
    g.rescue_list = c->rescue_list; g.tie_list = c->tie_list;
    g.rescue_count = c->rescue_count; g.tie_count = c->rescue_count + 1;
    g.n = c->n; g.k = c->k; g.kpad = c->kpad; g.ntiles = (int)((c->n + 127) / 128);
    g.f16 = c->opt.tc_operands == KM_TC_F16 ? 1 : 0;
    return launch_gemm_assign(c->G, c->st, g);
  }
  if (c->fast) {
    FastArgs a{};
    a.x = c->x; a.ld = c->ld; a.n = c->n; a.k = c->k; a.kpad = c->kpad;
    if (c->tcs) {
      a.tab2 = c->tab2; a.ctil = c->ctil4; a.mu = c->mu; a.ic = c->ic; a.dc = c->dc;
      a.ls = c->ls; a.labels = c->labels; a.labels8 = c->labels8; a.partials = c->partials;
      a.store_labels = store;
      a.ignore_done = labels_pass ? 1 : 0;
      return launch_assign_tcs(c->d, c->G, c->st, a);
    }
    a.tab2 = c->tab2; a.ctil = c->ctil4; a.mu = c->mu; a.ic = c->ic; a.dc = c->dc;
    a.ls = c->ls; a.labels = c->labels; a.labels8 = c->labels8; a.partials = c->partials;
    a.ntiles = (c->n + kWarpTile - 1) / kWarpTile;
    a.nwin = c->nwin;
    a.store_labels = store;
    a.ignore_done = labels_pass ? 1 : 0;
    a.const_tab = c->const_tab ? 1 : 0;
    e = launch_assign_fast(c->d, c->G, c->fast_smem, c->st, a);
  } else {
    GenericArgs a{};
    a.x = c->x; a.ld = c->ld; a.n = c->n; a.d = c->d; a.k = c->k;
    a.ctil = c->ctil; a.cnorm = c->cnorm; a.mu = c->mu; a.shift = c->shift; a.dc = c->dc;
    a.ls = c->ls; a.labels = c->labels; a.labels8 = c->labels8; a.partials = c->partials;
    a.A_max = c->A_max; a.B_max_ptr = c->gen_bmax; a.tau = (float)(c->opt.tie_rel * (1.0 + 1e-4));
    a.store_labels = store;
    a.ignore_done = labels_pass ? 1 : 0;
    e = launch_assign_generic(c->G, 0, c->st, a);
  }
  return e;
}

// Mean calculation, error and next tables.
cudaError_t launch_update_all(km_ctx* c) {
  if (c->path == 3) {
    cudaError_t e = launch_msort_step(msort_args(c), c->st);
    if (e != cudaSuccess) return e;
    return launch_gemm_prepare(c->st, gemm_prep_args(c));
  }
  return launch_update(c->st, update_args(c));
}

// One step: assign (+ accumulate), then reduce + divide + error + next tables.
cudaError_t launch_step(km_ctx* c) {
  cudaError_t e = launch_assign(c);
  if (e != cudaSuccess) return e;
  return launch_update_all(c);
}

km_status write_control(km_ctx* c, int done, int max_iter_abs, double tol) {
  LoopControl lc{};
  lc.done = done;
  lc.max_iter = max_iter_abs;
  lc.e_mode = c->opt.e_mode;
  lc.converged = 0;
  lc.tol = tol;
  KM_CUDA(c, cudaMemcpyAsync(c->ls, &lc, sizeof(lc), cudaMemcpyHostToDevice, c->st));
  return KM_OK;
}

km_status read_state(km_ctx* c) {
  KM_CUDA(c, cudaMemcpyAsync(&c->host_ls, c->ls, sizeof(LoopState), cudaMemcpyDeviceToHost, c->st));
  KM_CUDA(c, cudaStreamSynchronize(c->st));
  if (c->host_ls.error == 3)
    return fail(c, KM_ETIMEOUT, "a bounded device wait gave up (error word 3)");
  if (c->host_ls.error)
    return fail(c, KM_ECUDA, "device error word set (" + std::to_string(c->host_ls.error) + ")");
  return KM_OK;
}

km_status ready(km_ctx* c) {
  if (!c) return KM_EINVAL;
  if (!c->have_points || !c->have_init)
    return fail(c, KM_ESTATE, "km_set_points and km_set_init must come first");
  return KM_OK;
}

}  // namespace

extern "C" {

void km_default_options(km_options* opt) {
  if (!opt) return;
  opt->e_mode = KM_E_NORM;
  opt->use_graph = 1;
  opt->tie_rel = 1e-5;
  opt->stream = nullptr;
  opt->label_policy = KM_LABELS_EVERY_STEP;
  opt->dist_path = KM_DIST_AUTO;
  opt->tc_operands = KM_TC_BF16;
  opt->label_bytes = 4;
}

const char* km_version(void) { return "libkm 0.1 (sm_103a)"; }

void km_debug_fail_alloc_after(int64_t n) { g_alloc_countdown.store(n < 0 ? -1 : n); }

km_status km_selftest_bounded_wait(int32_t* gave_up, double* elapsed_ms) {
  if (!gave_up || !elapsed_ms) return KM_EINVAL;
  const auto t0 = std::chrono::steady_clock::now();
  int* d = nullptr;
  cudaStream_t st = nullptr;
  if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) return KM_ENOMEM;
  int h = -1;
  cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMemsetAsync(d, 0xFF, sizeof(int), st);
  if (e == cudaSuccess) e = launch_wait_selftest(d, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (st) cudaStreamDestroy(st);
  cudaFree(d);
  if (e != cudaSuccess) return KM_ECUDA;
  *gave_up = h;
  *elapsed_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return KM_OK;
}

km_status km_create(km_ctx** out, int64_t n, int32_t d, int32_t k, const km_options* opt) {
  if (!out) return KM_EINVAL;
  *out = nullptr;
  if (n < 1 || d < 1 || k < 1 || k > n || n > (int64_t(1) << 40) || d > 4096 || k > (1 << 20))
    return KM_EINVAL;
  km_ctx* c = new (std::nothrow) km_ctx();
  if (!c) return KM_ENOMEM;
  *out = c;
  c->n = n; c->d = d; c->k = k;
  km_default_options(&c->opt);
  if (opt) c->opt = *opt;
  if (!(c->opt.tie_rel >= 0.0 && c->opt.tie_rel < 0.5)) return fail(c, KM_EINVAL, "tie_rel out of range");
  if (c->opt.label_policy != KM_LABELS_EVERY_STEP && c->opt.label_policy != KM_LABELS_FINAL)
    return fail(c, KM_EINVAL, "label_policy out of range");
  if (c->opt.dist_path < KM_DIST_AUTO || c->opt.dist_path > KM_DIST_TENSOR)
    return fail(c, KM_EINVAL, "dist_path out of range");
  if (c->opt.tc_operands != KM_TC_BF16 && c->opt.tc_operands != KM_TC_F16)
    return fail(c, KM_EINVAL, "tc_operands out of range");
  if (c->opt.label_bytes != 4 && c->opt.label_bytes != 1) return fail(c, KM_EINVAL, "label_bytes must be 4 or 1");
  if (c->opt.label_bytes == 1 && k > 256) return fail(c, KM_EINVAL, "1-byte labels need K <= 256");
  if (c->opt.e_mode != KM_E_NORM && c->opt.e_mode != KM_E_SQUARED) return fail(c, KM_EINVAL, "bad e_mode");
  KM_CUDA(c, cudaGetDevice(&c->dev));
  cudaDeviceProp p{};
  KM_CUDA(c, cudaGetDeviceProperties(&p, c->dev));
  if (!(p.major == 10 && p.minor == 3))
    return fail(c, KM_ECUDA, std::string("libkm is built for sm_103a; device is ") + p.name);
  c->sms = p.multiProcessorCount;
  if (c->opt.stream) {
    c->st = static_cast<cudaStream_t>(c->opt.stream);
  } else {
    KM_CUDA(c, cudaStreamCreate(&c->st));  // blocking: ordered after legacy-stream work
    c->own_stream = true;
  }
  c->kpad = (k + 7) / 8 * 8;  // the screen works on pairs of groups of 4 centroids
  c->fast = d <= kMaxDFast && k <= kMaxKFast;
  const bool gemm = d == kGemmD && k <= kGemmMaxK && n < (int64_t(1) << 31) &&
                    gemm_smem_bytes((k + 255) / 256 * 256) <= (size_t)p.sharedMemPerBlockOptin;
  // the fused step with its screen on the tensor cores: d <= 3, K <= 32
  // (one 32-column accumulator per tile; the screen tables are built for
  // kpad = 32), N < 2^31 (32-bit queue entries)
  const bool tcs_ok = c->fast && d <= 3 && k <= 32 && n < (int64_t(1) << 31) &&
                      tcs_smem_bytes() <= (size_t)p.sharedMemPerBlockOptin;
  c->tcs = tcs_ok && c->opt.dist_path == KM_DIST_TENSOR;  // opt-in: the FFMA2 screen is faster here
  if (c->tcs) c->kpad = 32;
  if (c->fast && !c->tcs) {
    // one 32-bit sum window per half-warp (double-buffered points) when it
    // fits with as many resident blocks per SM as one window per warp
    // (single-buffered points) allows, else the smaller layout
    if (fast_has_const_table(d, c->kpad)) c->const_tab = claim_const_tab(c->dev);
    const size_t s4 = fast_smem_bytes(d, c->kpad, k, 4), s2 = fast_smem_bytes(d, c->kpad, k, 2),
                 s1 = fast_smem_bytes(d, c->kpad, k, 1);
    const size_t lim = (size_t)p.sharedMemPerBlockOptin;
    const bool ct = c->const_tab;
    const int b4 = s4 <= lim ? fast_blocks_per_sm(d, s4, c->kpad, ct) : 0,
              b2 = s2 <= lim ? fast_blocks_per_sm(d, s2, c->kpad, ct) : 0,
              b1 = s1 <= lim ? fast_blocks_per_sm(d, s1, c->kpad, ct) : 0;
    // four windows per warp (8 lanes each: fewer lanes adding to one bin in
    // one shared atomic, and half as many flushes per point) where they keep
    // as many resident blocks as two (at d = 3, K = 32: 0.873 -> 0.855 ms)
    c->nwin = (b4 > 0 && b4 >= b2 && b4 >= b1) ? 4 : (b2 > 0 && b2 >= b1) ? 2 : 1;
    c->fast_smem = c->nwin == 4 ? s4 : c->nwin == 2 ? s2 : s1;
    if (c->fast_smem > lim || (c->nwin == 4 ? b4 : c->nwin == 2 ? b2 : b1) == 0) c->fast = false;
    if (!c->fast && c->const_tab) {
      release_const_tab(c->dev);
      c->const_tab = false;
    }
  }
  const int64_t ntiles = (n + kWarpTile - 1) / kWarpTile;  // warp-tiles of 256 points
  if (c->opt.dist_path == KM_DIST_TENSOR && !gemm && !c->tcs)
    return fail(c, KM_EINVAL, "tensor-core distances need d <= 3 and K <= 32, or d = 64 and K <= 1024 (N < 2^31)");
  c->path = c->tcs ? 4
                   : c->opt.dist_path == KM_DIST_TENSOR ? 3
                                                        : (c->fast ? 1 : ((gemm && c->opt.dist_path == KM_DIST_AUTO) ? 3 : 2));
  if (c->path == 3 && c->opt.label_bytes == 1)
    return fail(c, KM_EINVAL, "1-byte labels are for the FP32 paths (the tensor-core path reads int32 labels)");
  if (c->path == 3) {
    c->kpad = (k + 255) / 256 * 256;
    c->G = (int)std::max<int64_t>(1, std::min<int64_t>((n + 127) / 128, c->sms));
  } else if (c->tcs) {
    // one CTA per SM (the whole TMEM); at most 4 x 1023 super-tiles of 256
    // points per CTA so that the int64 block totals stay in range
    const int64_t U = (n + 255) / 256;
    c->G = (int)std::max<int64_t>(tcs_grid(n, c->sms), (U + 4 * 1023 - 1) / (4 * 1023));
  } else if (c->fast) {
    // one resident wave; each warp strides over warp-tiles, and no block
    // takes more than 2^19 points (int64 per-block sums stay in range)
    const int bpsm = fast_blocks_per_sm(d, c->fast_smem, c->kpad, c->const_tab);
    int64_t g = std::min<int64_t>((ntiles + kWarps - 1) / kWarps, (int64_t)c->sms * bpsm);
    const int64_t tiles_per_block_max = kMaxPointsPerBlock / kWarpTile;
    g = std::max<int64_t>(g, (ntiles + tiles_per_block_max - 1) / tiles_per_block_max);
    c->G = (int)std::max<int64_t>(g, 1);
  } else {
    int64_t g = std::min<int64_t>((n + kThreads - 1) / kThreads, (int64_t)c->sms * 8);
    g = std::max<int64_t>(g, (n + kMaxPointsPerBlock - 1) / kMaxPointsPerBlock);
    c->G = (int)std::max<int64_t>(g, 1);
  }
  c->RB = (int)std::max<int64_t>(1, std::min<int64_t>(16, (c->G + kWarps * 4 - 1) / (kWarps * 4)));
  const size_t cols = (size_t)k * (d + 1);
  if (c->opt.label_bytes == 1) KM_CUDA(c, dalloc(&c->labels8, (size_t)n));
  else KM_CUDA(c, dalloc(&c->labels, (size_t)n));
  KM_CUDA(c, dalloc(&c->mu, (size_t)k * d));
  KM_CUDA(c, dalloc(&c->counts, (size_t)k));
  KM_CUDA(c, dalloc(&c->partials, (size_t)c->G * cols));
  KM_CUDA(c, dalloc(&c->s128, (size_t)c->RB * cols * 2));
  KM_CUDA(c, dalloc(&c->tab2, (size_t)c->kpad * (d + 1)));
  KM_CUDA(c, dalloc(&c->ctil4, (size_t)k));
  KM_CUDA(c, dalloc(&c->ctil, (size_t)k * d));
  KM_CUDA(c, dalloc(&c->cnorm, (size_t)k));
  KM_CUDA(c, dalloc(&c->shift, (size_t)d));
  KM_CUDA(c, dalloc(&c->gen_bmax, 1));
  KM_CUDA(c, dalloc(&c->dc, 1));
  KM_CUDA(c, dalloc(&c->ic, 1));
  KM_CUDA(c, dalloc(&c->ls, 1));
  KM_CUDA(c, dalloc(&c->scan, (size_t)2 * d + 1));
  KM_CUDA(c, dalloc(&c->scan_bad, 1));
  if (c->path == 3) {
    KM_CUDA(c, dalloc(reinterpret_cast<uint16_t**>(&c->xb), (size_t)gemm_xb_rows(n) * kGemmD));
    KM_CUDA(c, dalloc(&c->xa_pt, (size_t)n));
    KM_CUDA(c, dalloc(&c->xaos, (size_t)n * kGemmD));
    KM_CUDA(c, dalloc(reinterpret_cast<uint16_t**>(&c->cbf), (size_t)c->kpad * kGemmD));
    KM_CUDA(c, dalloc(&c->nprime, (size_t)c->kpad));
    KM_CUDA(c, dalloc(&c->gc, 1));
    KM_CUDA(c, dalloc(&c->rescue_list, (size_t)n));
    KM_CUDA(c, dalloc(&c->tie_list, (size_t)gemm_tie_entries(n, c->G) * 3));
    KM_CUDA(c, dalloc(&c->rescue_count, 2));
    c->ms_max_chunks = (int)msort_max_chunks(n, k);
    KM_CUDA(c, dalloc(&c->ms_counts, (size_t)k));
    KM_CUDA(c, dalloc(&c->ms_offsets, (size_t)k));
    KM_CUDA(c, dalloc(&c->ms_cfirst, (size_t)k));
    KM_CUDA(c, dalloc(&c->ms_cursor, (size_t)k));
    KM_CUDA(c, dalloc(&c->ms_chunks, (size_t)c->ms_max_chunks));
    KM_CUDA(c, dalloc(&c->ms_nchunks, 1));
    KM_CUDA(c, dalloc(&c->ms_chunk_sums, (size_t)c->ms_max_chunks * d));
    KM_CUDA(c, dalloc(&c->ms_perm, (size_t)n));
    KM_CUDA(c, dalloc(&c->ms_df2, (size_t)k * d));
    KM_CUDA(c, dalloc(&c->bnorm, (size_t)c->kpad));
  }
  KM_CUDA(c, cudaMemsetAsync(c->ls, 0, sizeof(LoopState), c->st));
  KM_CUDA(c, cudaMemsetAsync(c->counts, 0, sizeof(long long) * k, c->st));
  if (c->labels8) KM_CUDA(c, cudaMemsetAsync(c->labels8, 0, (size_t)n, c->st));
  else KM_CUDA(c, cudaMemsetAsync(c->labels, 0, sizeof(int32_t) * n, c->st));
  KM_CUDA(c, cudaStreamSynchronize(c->st));
  return KM_OK;
}

km_status km_set_points(km_ctx* c, const float* x, int64_t ld, int32_t layout, int32_t mem) {
  if (!c) return KM_EINVAL;
  if (!x) return fail(c, KM_EINVAL, "null points");
  if (layout != KM_SOA_DxN && layout != KM_AOS_NxD) return fail(c, KM_EINVAL, "bad layout");
  if (mem != KM_HOST && mem != KM_DEVICE_COPY && mem != KM_DEVICE_BORROW)
    return fail(c, KM_EINVAL, "bad memory kind");
  if (layout == KM_SOA_DxN && ld < c->n) return fail(c, KM_EINVAL, "ld < N for the d x N layout");
  if (layout == KM_AOS_NxD && ld < c->d) return fail(c, KM_EINVAL, "ld < d for the N x d layout");
  if (layout == KM_AOS_NxD && mem == KM_DEVICE_BORROW)
    return fail(c, KM_EINVAL, "only the d x N layout can be borrowed");
  c->have_points = false;
  if (c->graph) { cudaGraphExecDestroy(c->graph); c->graph = nullptr; }
  const int d = c->d;
  const int64_t n = c->n;
  bool borrow = mem == KM_DEVICE_BORROW && (reinterpret_cast<uintptr_t>(x) % 16 == 0) && (ld % 4 == 0);
  if (borrow) {
    c->x = x;
    c->ld = ld;
  } else {
    const int64_t ldo = (n + 63) / 64 * 64;
    if (!c->x_own) KM_CUDA(c, dalloc(&c->x_own, (size_t)d * ldo));
    c->ld = ldo;
    c->x = c->x_own;
    if (layout == KM_SOA_DxN) {
      KM_CUDA(c, cudaMemcpy2DAsync(c->x_own, ldo * 4, x, ld * 4, n * 4, d,
                                   mem == KM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                                   c->st));
    } else {
      const float* src = x;
      float* tmp = nullptr;
      if (mem == KM_HOST) {
        KM_CUDA(c, dalloc(&tmp, (size_t)n * ld));
        KM_CUDA(c, cudaMemcpyAsync(tmp, x, sizeof(float) * n * ld, cudaMemcpyHostToDevice, c->st));
        src = tmp;
      }
      cudaError_t e = launch_aos_to_soa(src, ld, n, d, c->x_own, ldo, c->st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
      if (tmp) cudaFree(tmp);
      KM_CUDA(c, e);
    }
  }
  // Range scan: shift, fixed-point grid, non-finite values.
  float* mn = c->scan;
  float* mx = c->scan + d;
  KM_CUDA(c, launch_scan_range(c->x, c->ld, n, d, mn, mx, c->scan_bad, c->st));
  std::vector<uint32_t> hmn(d), hmx(d);
  unsigned long long bad = 0;
  KM_CUDA(c, cudaMemcpyAsync(hmn.data(), mn, 4 * d, cudaMemcpyDeviceToHost, c->st));
  KM_CUDA(c, cudaMemcpyAsync(hmx.data(), mx, 4 * d, cudaMemcpyDeviceToHost, c->st));
  KM_CUDA(c, cudaMemcpyAsync(&bad, c->scan_bad, 8, cudaMemcpyDeviceToHost, c->st));
  KM_CUDA(c, cudaStreamSynchronize(c->st));
  if (bad) return fail(c, KM_ENUMERIC, std::to_string(bad) + " non-finite coordinate(s) in the points");
  auto decode = [](uint32_t o) {
    uint32_t b = (o & 0x80000000u) ? (o & 0x7fffffffu) : ~o;
    float f;
    std::memcpy(&f, &b, 4);
    return f;
  };
  std::vector<float> shift(d);
  double absmax = 0.0;
  for (int j = 0; j < d; ++j) {
    const double lo = decode(hmn[j]), hi = decode(hmx[j]);
    shift[j] = (float)(0.5 * (lo + hi));
    absmax = std::max(absmax, std::max(std::fabs(lo), std::fabs(hi)));
  }
  int ex = absmax > 0.0 ? (int)std::floor(std::log2(absmax)) + 2 : -104;
  if (absmax > 0.0 && std::ldexp(1.0, ex - 1) <= absmax) ++ex;  // guard log2 rounding
  // C_lo = 1.5 * 2^(ex - 21) must stay a normal float: ex >= -104 (data
  // below 2^-106 in magnitude is summed on the 2^-148 grid)
  ex = std::max(ex, -104);
  if (ex > 100) return fail(c, KM_ENUMERIC, "coordinates too large for the fixed-point sums (|x| >= 2^99)");
  DataConst hdc{};
  for (int j = 0; j < kMaxDFast; ++j) hdc.s[j] = j < d ? shift[j] : 0.f;
  hdc.G0 = ex - 44;
  hdc.C_hi = std::ldexp(1.5f, ex + 1);
  hdc.C_lo = std::ldexp(1.5f, ex - 21);
  std::memcpy(&hdc.bits_C_hi, &hdc.C_hi, 4);
  std::memcpy(&hdc.bits_C_lo, &hdc.C_lo, 4);
  KM_CUDA(c, cudaMemcpyAsync(c->shift, shift.data(), 4 * d, cudaMemcpyHostToDevice, c->st));
  float* amax = c->scan + 2 * d;
  KM_CUDA(c, launch_scan_amax(c->x, c->ld, n, d, c->shift, amax, c->st));
  float ha = 0.f;
  KM_CUDA(c, cudaMemcpyAsync(&ha, amax, 4, cudaMemcpyDeviceToHost, c->st));
  KM_CUDA(c, cudaStreamSynchronize(c->st));
  hdc.A_max = ha;
  c->A_max = ha;
  c->G0 = hdc.G0;
  c->grid_ex = c->grid_ex_local = ex;
  KM_CUDA(c, cudaMemcpyAsync(c->dc, &hdc, sizeof(hdc), cudaMemcpyHostToDevice, c->st));
  KM_CUDA(c, cudaStreamSynchronize(c->st));
  if (c->path == 3) {
    // FP16 operands: |fl(x_j - s_j)| <= sqrt(A_max) scaled to at most 2^14
    c->tc_ex = 0;
    if (c->opt.tc_operands == KM_TC_F16 && ha > 0.f) {
      const double xm = std::sqrt((double)ha) * 1.001;
      int e = (int)std::floor(std::log2(16384.0 / xm));
      while (e > -200 && std::ldexp(xm, e) > 16384.0) --e;
      c->tc_ex = std::max(-100, std::min(100, e));
    }
    KM_CUDA(c, launch_gemm_prep_points(c->x, c->ld, n, c->shift, c->xb, c->xa_pt, c->xaos,
                                       c->opt.tc_operands == KM_TC_F16 ? 1 : 0, c->tc_ex, c->st));
    KM_CUDA(c, cudaStreamSynchronize(c->st));
  }
  c->have_points = true;
  if (c->have_init) {  // tables depend on the shift and A_max
    KM_CUDA(c, launch_tables(c));
    KM_CUDA(c, cudaStreamSynchronize(c->st));
  }
  return KM_OK;
}

km_status km_set_init(km_ctx* c, const double* mu0) {
  if (!c) return KM_EINVAL;
  if (!mu0) return fail(c, KM_EINVAL, "null centroids");
  const size_t kd = (size_t)c->k * c->d;
  for (size_t q = 0; q < kd; ++q)
    if (!std::isfinite(mu0[q])) return fail(c, KM_ENUMERIC, "non-finite starting centroid");
  KM_CUDA(c, cudaMemcpyAsync(c->mu, mu0, sizeof(double) * kd, cudaMemcpyHostToDevice, c->st));
  KM_CUDA(c, cudaMemsetAsync(c->ls, 0, sizeof(LoopState), c->st));
  c->have_init = true;
  if (c->have_points) KM_CUDA(c, launch_tables(c));
  KM_CUDA(c, cudaStreamSynchronize(c->st));
  std::memset(&c->host_ls, 0, sizeof(c->host_ls));
  return KM_OK;
}

km_status km_init_kmeanspp(km_ctx* c, const double* u, double* mu_out, int64_t* idx_out) {
  if (!c) return KM_EINVAL;
  if (!u) return fail(c, KM_EINVAL, "null uniforms");
  if (!c->have_points) return fail(c, KM_ESTATE, "km_init_kmeanspp before km_set_points");
  if (c->d > kMaxKppD) return fail(c, KM_EINVAL, "d > 256 for k-means++");
  for (int q = 0; q < c->k; ++q)
    if (!(u[q] >= 0.0 && u[q] < 1.0)) return fail(c, KM_EINVAL, "uniforms must lie in [0, 1)");
  const int64_t n = c->n;
  const int64_t nch = kpp_chunks(n);
  double *du = nullptr, *dmu = nullptr, *d2 = nullptr, *cs = nullptr, *sc = nullptr;
  int64_t* didx = nullptr;
  auto release = [&]() {
    void* b[] = {du, dmu, d2, cs, sc, didx};
    for (void* p : b)
      if (p) cudaFree(p);
  };
  cudaError_t e = cudaSuccess;
  if ((e = dalloc(&du, (size_t)c->k)) != cudaSuccess || (e = dalloc(&dmu, (size_t)c->k * c->d)) != cudaSuccess ||
      (e = dalloc(&d2, (size_t)n)) != cudaSuccess || (e = dalloc(&cs, (size_t)nch)) != cudaSuccess ||
      (e = dalloc(&sc, (size_t)4096)) != cudaSuccess || (e = dalloc(&didx, (size_t)c->k)) != cudaSuccess) {
    release();
    return fail(c, KM_ENOMEM, std::string("k-means++ buffers: ") + cudaGetErrorString(e));
  }
  std::vector<double> hmu((size_t)c->k * c->d);
  std::vector<int64_t> hidx((size_t)c->k);
  e = cudaMemcpyAsync(du, u, sizeof(double) * c->k, cudaMemcpyHostToDevice, c->st);
  if (e == cudaSuccess) e = launch_kmeanspp(c->x, c->ld, n, c->d, c->k, du, dmu, didx, d2, cs, sc, c->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hmu.data(), dmu, sizeof(double) * hmu.size(), cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hidx.data(), didx, sizeof(int64_t) * hidx.size(), cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  release();
  if (e != cudaSuccess) return fail(c, KM_ECUDA, std::string("k-means++: ") + cudaGetErrorString(e));
  if (mu_out) std::memcpy(mu_out, hmu.data(), sizeof(double) * hmu.size());
  if (idx_out) std::memcpy(idx_out, hidx.data(), sizeof(int64_t) * hidx.size());
  return km_set_init(c, hmu.data());
}

km_status km_init_learned(km_ctx* c, km_setnet* net, int32_t sample_n, uint64_t seed, double* mu_out) {
  if (!c) return KM_EINVAL;
  if (!net) return fail(c, KM_EINVAL, "null network");
  if (!c->have_points) return fail(c, KM_ESTATE, "km_init_learned before km_set_points");
  int32_t nk = 0;
  const int32_t nd = km_setnet_dims(net, &nk);
  if (nd != c->d || nk != c->k) return fail(c, KM_EINVAL, "network d or K differs from the context's");
  if (sample_n < 64 || sample_n % 64) return fail(c, KM_EINVAL, "sample_n must be a positive multiple of 64");
  float* buf = nullptr;
  cudaError_t e = dalloc(&buf, (size_t)sample_n * c->d);
  if (e != cudaSuccess) return fail(c, KM_ENOMEM, std::string("sample buffer: ") + cudaGetErrorString(e));
  e = launch_setnet_sample(c->x, c->ld, c->n, c->d, sample_n, (unsigned long long)seed, buf, c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);  // the network runs on its own stream
  if (e != cudaSuccess) {
    cudaFree(buf);
    return fail(c, KM_ECUDA, std::string("sample: ") + cudaGetErrorString(e));
  }
  std::vector<double> mu((size_t)c->k * c->d);
  const km_status s = km_setnet_predict(net, buf, 1, sample_n, KM_DEVICE_BORROW, mu.data());
  cudaFree(buf);
  if (s != KM_OK) return fail(c, s, std::string("network: ") + km_setnet_last_error(net));
  if (mu_out) std::memcpy(mu_out, mu.data(), sizeof(double) * mu.size());
  return km_set_init(c, mu.data());
}

km_status km_objective(km_ctx* c, double* obj_out) {
  km_status s = ready(c);
  if (s != KM_OK) return s;
  if (!obj_out) return fail(c, KM_EINVAL, "null output");
  double* part = nullptr;
  const int64_t nch = objective_chunks(c->n);
  cudaError_t e = dalloc(&part, (size_t)nch + 1);
  if (e != cudaSuccess) return fail(c, KM_ENOMEM, std::string("objective buffer: ") + cudaGetErrorString(e));
  e = launch_objective(c->x, c->ld, c->n, c->d, c->mu, c->labels, c->labels8, part, part + nch, c->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(obj_out, part + nch, sizeof(double), cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  cudaFree(part);
  if (e != cudaSuccess) return fail(c, KM_ECUDA, std::string("objective: ") + cudaGetErrorString(e));
  return KM_OK;
}

// int32 labels to out (host or device), widening byte labels on the device
// first (into a temporary buffer for a host destination).  Queued only.
static km_status copy_labels_i32(km_ctx* c, int32_t* out, int32_t mem) {
  if (!c->labels8) {
    KM_CUDA(c, cudaMemcpyAsync(out, c->labels, sizeof(int32_t) * c->n,
                               mem == KM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, c->st));
    return KM_OK;
  }
  if (mem == KM_DEVICE_COPY) {
    KM_CUDA(c, launch_widen_labels(c->labels8, out, c->n, c->st));
    return KM_OK;
  }
  int32_t* tmp = nullptr;
  KM_CUDA(c, dalloc(&tmp, (size_t)c->n));
  cudaError_t e = launch_widen_labels(c->labels8, tmp, c->n, c->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, tmp, sizeof(int32_t) * c->n, cudaMemcpyDeviceToHost, c->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
  cudaFree(tmp);
  if (e != cudaSuccess) return fail(c, KM_ECUDA, std::string("labels: ") + cudaGetErrorString(e));
  return KM_OK;
}

km_status km_write_labels(km_ctx* c) {
  km_status s = ready(c);
  if (s != KM_OK) return s;
  if (c->path == 3) return KM_OK;  // the tensor-core path writes labels every step
  KM_CUDA(c, launch_assign(c, true));
  // the pass's re-check counters are not a step's: clear them
  KM_CUDA(c, cudaMemsetAsync(&c->ls->flagged, 0, 2 * sizeof(unsigned long long), c->st));
  return KM_OK;
}

km_status km_step(km_ctx* c, double* e_out, double* e2_out) {
  km_status s = ready(c);
  if (s != KM_OK) return s;
  s = write_control(c, 0, 0x7fffffff, -1.0);
  if (s != KM_OK) return s;
  KM_CUDA(c, launch_step(c));
  s = read_state(c);
  if (s != KM_OK) return s;
  if (e_out) *e_out = c->host_ls.E;
  if (e2_out) *e2_out = c->host_ls.E2;
  return KM_OK;
}

km_status km_run(km_ctx* c, int32_t max_iter, double tol, int32_t* labels_out,
                 double* centroids_out, int32_t* iters_out, double* e_out) {
  km_status s = ready(c);
  if (s != KM_OK) return s;
  if (max_iter < 0) return fail(c, KM_EINVAL, "max_iter < 0");
  s = read_state(c);
  if (s != KM_OK) return s;
  const int start = c->host_ls.iter;
  if (max_iter > 0) {
    s = write_control(c, 0, start + max_iter, tol);
    if (s != KM_OK) return s;
    if (c->opt.use_graph) {
      if (!c->graph) {
        cudaGraph_t g = nullptr;
        KM_CUDA(c, cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = cudaSuccess;
        for (int u = 0; u < c->graph_unroll && e == cudaSuccess; ++u) e = launch_step(c);
        cudaError_t e2 = cudaStreamEndCapture(c->st, &g);
        KM_CUDA(c, e);
        KM_CUDA(c, e2);
        e = cudaGraphInstantiate(&c->graph, g, 0);
        cudaGraphDestroy(g);
        KM_CUDA(c, e);
      }
      while (true) {
        KM_CUDA(c, cudaGraphLaunch(c->graph, c->st));
        s = read_state(c);
        if (s != KM_OK) return s;
        if (c->host_ls.done) break;
      }
    } else {
      while (true) {
        KM_CUDA(c, launch_step(c));
        s = read_state(c);
        if (s != KM_OK) return s;
        if (c->host_ls.done) break;
      }
    }
  }
  if (c->opt.label_policy == KM_LABELS_FINAL) {
    s = km_write_labels(c);
    if (s != KM_OK) return s;
  }
  if (labels_out) {
    s = copy_labels_i32(c, labels_out, KM_HOST);
    if (s != KM_OK) return s;
  }
  if (centroids_out)
    KM_CUDA(c, cudaMemcpyAsync(centroids_out, c->mu, sizeof(double) * c->k * c->d, cudaMemcpyDeviceToHost, c->st));
  KM_CUDA(c, cudaStreamSynchronize(c->st));
  if (iters_out) *iters_out = c->host_ls.iter - start;
  if (e_out) *e_out = c->host_ls.E;
  return c->host_ls.converged ? KM_OK : KM_NOT_CONVERGED;
}

km_status km_begin(km_ctx* c, int32_t max_iter, double tol) {
  km_status s = ready(c);
  if (s != KM_OK) return s;
  if (max_iter < 0) return fail(c, KM_EINVAL, "max_iter < 0");
  s = read_state(c);
  if (s != KM_OK) return s;
  return write_control(c, 0, c->host_ls.iter + max_iter, tol);
}

km_status km_assign_async(km_ctx* c) {
  km_status s = ready(c);
  if (s != KM_OK) return s;
  KM_CUDA(c, launch_assign(c));
  return KM_OK;
}

km_status km_update_async(km_ctx* c) {
  km_status s = ready(c);
  if (s != KM_OK) return s;
  KM_CUDA(c, launch_update_all(c));
  return KM_OK;
}

km_status km_grid_exponent(km_ctx* c, int32_t* ex_out) {
  if (!c || !ex_out) return KM_EINVAL;
  if (!c->have_points) return fail(c, KM_ESTATE, "km_set_points must come first");
  *ex_out = c->grid_ex;
  return KM_OK;
}

km_status km_set_grid_exponent(km_ctx* c, int32_t ex) {
  if (!c) return KM_EINVAL;
  if (!c->have_points) return fail(c, KM_ESTATE, "km_set_points must come first");
  if (ex < c->grid_ex_local)
    return fail(c, KM_EINVAL, "grid exponent below the one this context's points need (" +
                                  std::to_string(c->grid_ex_local) + ")");
  if (ex > 100) return fail(c, KM_EINVAL, "grid exponent above 100 (|x| >= 2^99)");
  DataConst hdc{};
  KM_CUDA(c, cudaMemcpyAsync(&hdc, c->dc, sizeof(hdc), cudaMemcpyDeviceToHost, c->st));
  KM_CUDA(c, cudaStreamSynchronize(c->st));
  hdc.G0 = ex - 44;
  hdc.C_hi = std::ldexp(1.5f, ex + 1);
  hdc.C_lo = std::ldexp(1.5f, ex - 21);
  std::memcpy(&hdc.bits_C_hi, &hdc.C_hi, 4);
  std::memcpy(&hdc.bits_C_lo, &hdc.C_lo, 4);
  KM_CUDA(c, cudaMemcpyAsync(c->dc, &hdc, sizeof(hdc), cudaMemcpyHostToDevice, c->st));
  KM_CUDA(c, cudaStreamSynchronize(c->st));
  c->G0 = hdc.G0;
  c->grid_ex = ex;
  return KM_OK;
}

km_status km_shard_totals(km_ctx* c, int64_t* out, int32_t mem) {
  km_status s = ready(c);
  if (s != KM_OK) return s;
  if (!out || (mem != KM_HOST && mem != KM_DEVICE_COPY)) return fail(c, KM_EINVAL, "bad output");
  const size_t words = (size_t)c->k * (c->d + 1) * 2;
  long long* dst = reinterpret_cast<long long*>(out);
  if (mem == KM_HOST) {
    if (!c->shard_out) KM_CUDA(c, dalloc(&c->shard_out, words));
    dst = c->shard_out;
  }
  // the tensor-core path sums by the sorted mean calculation; the FP32 paths
  // add their per-block partials
  KM_CUDA(c, c->path == 3 ? launch_msort_shard_totals(msort_args(c), dst, c->st)
                          : launch_shard_totals(c->st, update_args(c), dst));
  if (mem == KM_HOST) {
    KM_CUDA(c, cudaMemcpyAsync(out, dst, words * sizeof(long long), cudaMemcpyDeviceToHost, c->st));
    KM_CUDA(c, cudaStreamSynchronize(c->st));
  }
  return KM_OK;
}

km_status km_shard_update(km_ctx* c, const int64_t* tables, int32_t ranks, int32_t mem) {
  km_status s = ready(c);
  if (s != KM_OK) return s;
  if (!tables || ranks < 1 || (mem != KM_HOST && mem != KM_DEVICE_COPY)) return fail(c, KM_EINVAL, "bad tables");
  const size_t words = (size_t)c->k * (c->d + 1) * 2;
  const long long* src = reinterpret_cast<const long long*>(tables);
  if (mem == KM_HOST) {
    if (ranks > c->shard_in_ranks) {
      if (c->shard_in) cudaFree(c->shard_in);
      c->shard_in = nullptr;
      c->shard_in_ranks = 0;
      KM_CUDA(c, dalloc(&c->shard_in, words * ranks));
      c->shard_in_ranks = ranks;
    }
    KM_CUDA(c, cudaMemcpyAsync(c->shard_in, tables, words * ranks * sizeof(long long), cudaMemcpyHostToDevice, c->st));
    src = c->shard_in;
  }
  if (c->path == 3) {
    KM_CUDA(c, launch_msort_shard_update(msort_args(c), src, ranks, c->st));
    KM_CUDA(c, launch_gemm_prepare(c->st, gemm_prep_args(c)));  // the next step's tables
  } else {
    KM_CUDA(c, launch_shard_update(c->st, update_args(c), src, ranks));
  }
  if (mem == KM_HOST) KM_CUDA(c, cudaStreamSynchronize(c->st));  // the host tables may be reused at once
  return KM_OK;
}

km_status km_sync(km_ctx* c, int32_t* iters_out, double* e_out, int32_t* done_out) {
  if (!c) return KM_EINVAL;
  km_status s = read_state(c);
  if (s != KM_OK) return s;
  if (iters_out) *iters_out = c->host_ls.iter;
  if (e_out) *e_out = c->host_ls.E;
  if (done_out) *done_out = c->host_ls.done;
  return KM_OK;
}

void* km_stream(km_ctx* c) { return c ? (void*)c->st : nullptr; }

km_status km_get_labels(km_ctx* c, int32_t* out, int32_t mem) {
  if (!c) return KM_EINVAL;
  if (!out || (mem != KM_HOST && mem != KM_DEVICE_COPY)) return fail(c, KM_EINVAL, "bad output");
  km_status s = copy_labels_i32(c, out, mem);
  if (s != KM_OK) return s;
  KM_CUDA(c, cudaStreamSynchronize(c->st));
  return KM_OK;
}

km_status km_get_labels_u8(km_ctx* c, uint8_t* out, int32_t mem) {
  if (!c) return KM_EINVAL;
  if (!out || (mem != KM_HOST && mem != KM_DEVICE_COPY)) return fail(c, KM_EINVAL, "bad output");
  if (!c->labels8) return fail(c, KM_EINVAL, "labels are stored as int32 (label_bytes = 4)");
  KM_CUDA(c, cudaMemcpyAsync(out, c->labels8, (size_t)c->n,
                             mem == KM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, c->st));
  KM_CUDA(c, cudaStreamSynchronize(c->st));
  return KM_OK;
}

km_status km_get_centroids(km_ctx* c, double* out, int32_t mem) {
  if (!c) return KM_EINVAL;
  if (!out || (mem != KM_HOST && mem != KM_DEVICE_COPY)) return fail(c, KM_EINVAL, "bad output");
  KM_CUDA(c, cudaMemcpyAsync(out, c->mu, sizeof(double) * c->k * c->d,
                             mem == KM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, c->st));
  KM_CUDA(c, cudaStreamSynchronize(c->st));
  return KM_OK;
}

km_status km_get_counts(km_ctx* c, int64_t* out) {
  if (!c) return KM_EINVAL;
  if (!out) return fail(c, KM_EINVAL, "null output");
  KM_CUDA(c, cudaMemcpyAsync(out, c->counts, sizeof(int64_t) * c->k, cudaMemcpyDeviceToHost, c->st));
  KM_CUDA(c, cudaStreamSynchronize(c->st));
  return KM_OK;
}

km_status km_get_stats(km_ctx* c, km_stats* out) {
  if (!c) return KM_EINVAL;
  if (!out) return fail(c, KM_EINVAL, "null output");
  km_status s = read_state(c);
  if (s != KM_OK) return s;
  out->iters = c->host_ls.iter;
  out->converged = c->host_ls.converged;
  out->e = c->host_ls.E;
  out->e2 = c->host_ls.E2;
  out->flagged = (int64_t)c->host_ls.last_flagged;
  out->fp64_decided = (int64_t)c->host_ls.last_fp64;
  out->empty_clusters = c->host_ls.empty;
  out->overflowed = (int64_t)c->host_ls.last_overflowed;
  out->path = c->path;
  return KM_OK;
}

km_status km_device_buffers(km_ctx* c, const float** points, int64_t* ld_out, int32_t** labels,
                            double** centroids) {
  if (!c) return KM_EINVAL;
  if (points) *points = c->x;
  if (ld_out) *ld_out = c->ld;
  if (labels) *labels = c->labels;
  if (centroids) *centroids = c->mu;
  return KM_OK;
}

const char* km_last_error(const km_ctx* c) { return c ? c->err.c_str() : "null context"; }

void km_destroy(km_ctx* c) {
  if (!c) return;
  if (c->st) cudaStreamSynchronize(c->st);
  free_all(c);
  delete c;
}

}  // extern "C"
