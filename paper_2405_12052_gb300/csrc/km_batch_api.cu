// C ABI of the batched form: many independent Lloyd instances (d <= 3,
// K <= 64) advanced by shared launches.  The step (assign + accumulate over
// every active instance's tiles, then one update block per instance) is
// captured U times in a CUDA graph that is replayed until no instance is
// active; the tile size and block size of the assign kernel are picked by
// timing the candidates on the batch itself.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/km.h"
#include "km_internal.cuh"

using namespace km;

struct km_batch {
  int count = 0;
  std::vector<BatchInst> hinst;
  std::vector<BatchState> hstate;
  int64_t total_n = 0, total_x = 0, total_kd = 0, total_k = 0;
  km_options opt{};
  cudaStream_t st = nullptr;
  bool own_stream = false;
  int sms = 0;
  // device buffers
  float* x = nullptr;
  int32_t* labels = nullptr;
  double* mu = nullptr;
  float* ctil = nullptr;
  long long* counts = nullptr;
  BatchInst* inst = nullptr;
  BatchState* state = nullptr;
  int4* tiles = nullptr;
  int64_t* tile_poff = nullptr;
  long long* partials = nullptr;
  unsigned long long* stats = nullptr;  // [0] flagged, [1] fp64, [2] non-finite
  unsigned long long* tab2 = nullptr;   // fused kernel: per-instance screen tables
  float4* ctil4 = nullptr;
  IterConst* ic = nullptr;
  int64_t total_tab = 0;
  int kind = 0;                         // assign kernel: 0 the batch kernel, 1 the fused kernel's tiles
  int* active = nullptr;
  int64_t max_tiles = 0, max_partials = 0;
  // launch shape
  int ntiles = 0, tile_pts = 0, threads = 0, grid = 0;
  bool tuned = false, have_points = false, have_init = false;
  std::vector<float> tune_ms;  // per candidate, in candidate order
  cudaGraphExec_t graph = nullptr;
  int graph_steps = 0;
  double graph_tol = -1.0;  // the tolerance captured in the graph
  std::string err;
};

namespace {

constexpr int kTileCand[2] = {512, 1024};
constexpr int kThreadCand[3] = {128, 256, 512};
// the fused kernel's tiles (a multiple of its 256-point warp-tiles; 256 threads)
constexpr int kFastTileCand[2] = {8192, 32768};
constexpr int kGraphSteps = 4;

km_status bfail(km_batch* b, km_status s, const std::string& m) {
  b->err = m;
  return s;
}
#define KB_CUDA(b, call)                                                                           \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess)                                                                         \
      return bfail(b, e_ == cudaErrorMemoryAllocation ? KM_ENOMEM : KM_ECUDA,                      \
                   std::string(#call) + ": " + cudaGetErrorString(e_));                            \
  } while (0)

template <typename T>
cudaError_t balloc(T** p, size_t n) {
  if (inject_alloc_failure()) return cudaErrorMemoryAllocation;
  return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * (n > 0 ? n : 1));
}

BatchArgs bargs(km_batch* b) {
  BatchArgs a{};
  a.x = b->x; a.inst = b->inst; a.state = b->state; a.tiles = b->tiles; a.tile_poff = b->tile_poff;
  a.ntiles = b->ntiles; a.partials = b->partials; a.labels = b->labels; a.mu = b->mu; a.ctil = b->ctil;
  a.counts = b->counts; a.flagged = b->stats; a.fp64 = b->stats + 1; a.active = b->active;
  a.tau = (float)(b->opt.tie_rel * (1.0 + 1e-4)); a.e_mode = b->opt.e_mode; a.tol = 0.0;
  a.tab2 = b->tab2; a.ctil4 = b->ctil4; a.ic = b->ic; a.tie_rel = b->opt.tie_rel;
  return a;
}

// Tile list for a tile size (instance-major) and the instances' tile ranges.
km_status build_tiles(km_batch* b, int tile_pts) {
  std::vector<int4> tl;
  std::vector<int64_t> poff;
  int64_t off = 0;
  for (int i = 0; i < b->count; ++i) {
    BatchInst& bi = b->hinst[i];
    bi.tile0 = (int32_t)tl.size();
    for (int64_t s = 0; s < bi.n; s += tile_pts) {
      tl.push_back(make_int4(i, (int)s, (int)std::min<int64_t>(tile_pts, bi.n - s), 0));
      poff.push_back(off);
      off += (int64_t)bi.k * (bi.d + 1);
    }
    bi.ntiles = (int32_t)tl.size() - bi.tile0;
  }
  if ((int64_t)tl.size() > b->max_tiles || off > b->max_partials)
    return bfail(b, KM_EINVAL, "tile list larger than allocated");
  b->ntiles = (int)tl.size();
  b->tile_pts = tile_pts;
  // only the tile fields of the device instance table change
  std::vector<BatchInst> dev(b->count);
  KB_CUDA(b, cudaMemcpyAsync(dev.data(), b->inst, sizeof(BatchInst) * b->count, cudaMemcpyDeviceToHost, b->st));
  KB_CUDA(b, cudaStreamSynchronize(b->st));
  for (int i = 0; i < b->count; ++i) {
    dev[i].tile0 = b->hinst[i].tile0;
    dev[i].ntiles = b->hinst[i].ntiles;
  }
  KB_CUDA(b, cudaMemcpyAsync(b->inst, dev.data(), sizeof(BatchInst) * b->count, cudaMemcpyHostToDevice, b->st));
  KB_CUDA(b, cudaMemcpyAsync(b->tiles, tl.data(), sizeof(int4) * tl.size(), cudaMemcpyHostToDevice, b->st));
  KB_CUDA(b, cudaMemcpyAsync(b->tile_poff, poff.data(), sizeof(int64_t) * poff.size(), cudaMemcpyHostToDevice, b->st));
  KB_CUDA(b, cudaStreamSynchronize(b->st));
  return KM_OK;
}

void drop_graph(km_batch* b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
}

int grid_for(km_batch* b, int threads) {
  const int per_sm = b->kind == 1 ? batch_fast_blocks_per_sm() : batch_blocks_per_sm(threads);
  const int64_t g = std::min<int64_t>(b->ntiles, (int64_t)b->sms * per_sm);
  return (int)std::max<int64_t>(1, g);
}

cudaError_t launch_assign_kind(km_batch* b, const BatchArgs& a) {
  return b->kind == 1 ? launch_batch_fast(a, b->grid, b->st) : launch_batch_assign(a, b->grid, b->threads, b->st);
}

}  // namespace

extern "C" {

km_status km_batch_create(km_batch** out, int32_t count, const int64_t* n, const int32_t* d, const int32_t* k,
                          const km_options* opt) {
  if (!out) return KM_EINVAL;
  *out = nullptr;
  km_batch* b = new (std::nothrow) km_batch();
  if (!b) return KM_ENOMEM;
  *out = b;
  if (count <= 0 || !n || !d || !k) return bfail(b, KM_EINVAL, "count <= 0 or a null size array");
  km_default_options(&b->opt);
  if (opt) b->opt = *opt;
  b->count = count;
  b->hinst.resize(count);
  b->hstate.assign(count, BatchState{});
  int64_t xo = 0, lo = 0, mo = 0, ko = 0, tiles_max = 0, part_max = 0;
  for (int i = 0; i < count; ++i) {
    if (d[i] < 1 || d[i] > kBatchMaxD) return bfail(b, KM_EINVAL, "instance " + std::to_string(i) + ": d not in 1..3");
    if (k[i] < 1 || k[i] > kBatchMaxK) return bfail(b, KM_EINVAL, "instance " + std::to_string(i) + ": K not in 1..64");
    if (n[i] < k[i] || n[i] >= (int64_t(1) << 31)) return bfail(b, KM_EINVAL, "instance " + std::to_string(i) + ": K > N or N too large");
    BatchInst& bi = b->hinst[i];
    std::memset(&bi, 0, sizeof(bi));
    bi.n = n[i]; bi.d = d[i]; bi.k = k[i];
    bi.x_off = xo; bi.lab_off = lo; bi.mu_off = (int32_t)mo; bi.k_off = (int32_t)ko;
    bi.kpad = (k[i] + 7) / 8 * 8;
    bi.tab_off = (int32_t)b->total_tab;
    b->total_tab += (int64_t)bi.kpad * (d[i] + 1);
    xo += n[i] * d[i]; lo += n[i]; mo += (int64_t)k[i] * d[i]; ko += k[i];
    const int64_t nt = (n[i] + kTileCand[0] - 1) / kTileCand[0];
    tiles_max += nt;
    part_max += nt * k[i] * (d[i] + 1);
  }
  b->total_x = xo; b->total_n = lo; b->total_kd = mo; b->total_k = ko;
  b->max_tiles = tiles_max; b->max_partials = part_max;
  int dev = 0;
  KB_CUDA(b, cudaGetDevice(&dev));
  KB_CUDA(b, cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev));
  if (b->opt.stream) {
    b->st = static_cast<cudaStream_t>(b->opt.stream);
  } else {
    KB_CUDA(b, cudaStreamCreate(&b->st));
    b->own_stream = true;
  }
  KB_CUDA(b, balloc(&b->x, (size_t)xo));
  KB_CUDA(b, balloc(&b->labels, (size_t)lo));
  KB_CUDA(b, balloc(&b->mu, (size_t)mo));
  KB_CUDA(b, balloc(&b->ctil, (size_t)mo));
  KB_CUDA(b, balloc(&b->counts, (size_t)ko));
  KB_CUDA(b, balloc(&b->inst, (size_t)count));
  KB_CUDA(b, balloc(&b->state, (size_t)count));
  KB_CUDA(b, balloc(&b->tiles, (size_t)tiles_max));
  KB_CUDA(b, balloc(&b->tile_poff, (size_t)tiles_max));
  KB_CUDA(b, balloc(&b->partials, (size_t)part_max));
  KB_CUDA(b, balloc(&b->stats, 3));
  KB_CUDA(b, balloc(&b->tab2, (size_t)b->total_tab));
  KB_CUDA(b, balloc(&b->ctil4, (size_t)ko));
  KB_CUDA(b, balloc(&b->ic, (size_t)count));
  KB_CUDA(b, balloc(&b->active, 1));
  KB_CUDA(b, cudaMemcpyAsync(b->inst, b->hinst.data(), sizeof(BatchInst) * count, cudaMemcpyHostToDevice, b->st));
  KB_CUDA(b, cudaMemsetAsync(b->state, 0, sizeof(BatchState) * count, b->st));
  KB_CUDA(b, cudaMemsetAsync(b->labels, 0, sizeof(int32_t) * (size_t)lo, b->st));
  KB_CUDA(b, cudaMemsetAsync(b->stats, 0, sizeof(unsigned long long) * 3, b->st));
  KB_CUDA(b, cudaStreamSynchronize(b->st));
  km_status s = build_tiles(b, kTileCand[1]);
  if (s != KM_OK) return s;
  b->threads = 256;
  b->grid = grid_for(b, b->threads);
  return KM_OK;
}

km_status km_batch_set_points(km_batch* b, const float* x, int32_t mem) {
  if (!b) return KM_EINVAL;
  if (!x) return bfail(b, KM_EINVAL, "null points");
  if (mem != KM_HOST && mem != KM_DEVICE_COPY) return bfail(b, KM_EINVAL, "mem must be KM_HOST or KM_DEVICE_COPY");
  KB_CUDA(b, cudaMemcpyAsync(b->x, x, sizeof(float) * (size_t)b->total_x,
                             mem == KM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, b->st));
  KB_CUDA(b, cudaMemsetAsync(b->stats + 2, 0, sizeof(unsigned long long), b->st));
  KB_CUDA(b, launch_batch_scan(b->x, b->inst, b->count, b->stats + 2, b->st));
  unsigned long long bad = 0;
  KB_CUDA(b, cudaMemcpyAsync(&bad, b->stats + 2, 8, cudaMemcpyDeviceToHost, b->st));
  KB_CUDA(b, cudaStreamSynchronize(b->st));
  if (bad) return bfail(b, KM_ENUMERIC, "non-finite or too large coordinates in the points");
  b->have_points = true;
  b->tuned = false;
  drop_graph(b);
  if (b->have_init) {
    KB_CUDA(b, launch_batch_tables(bargs(b), b->count, b->st));  // tables depend on the shift
    KB_CUDA(b, cudaStreamSynchronize(b->st));
  }
  return KM_OK;
}

km_status km_batch_set_init(km_batch* b, const double* mu0) {
  if (!b) return KM_EINVAL;
  if (!mu0) return bfail(b, KM_EINVAL, "null init");
  for (int64_t q = 0; q < b->total_kd; ++q)
    if (!std::isfinite(mu0[q])) return bfail(b, KM_ENUMERIC, "non-finite initial centroid");
  KB_CUDA(b, cudaMemcpyAsync(b->mu, mu0, sizeof(double) * (size_t)b->total_kd, cudaMemcpyHostToDevice, b->st));
  b->hstate.assign(b->count, BatchState{});
  KB_CUDA(b, cudaMemcpyAsync(b->state, b->hstate.data(), sizeof(BatchState) * b->count, cudaMemcpyHostToDevice, b->st));
  KB_CUDA(b, cudaMemsetAsync(b->counts, 0, sizeof(long long) * (size_t)b->total_k, b->st));
  b->have_init = true;
  if (b->have_points) KB_CUDA(b, launch_batch_tables(bargs(b), b->count, b->st));
  KB_CUDA(b, cudaStreamSynchronize(b->st));
  return KM_OK;
}

km_status km_batch_tune(km_batch* b, int32_t* tile_out, int32_t* threads_out) {
  if (!b) return KM_EINVAL;
  if (!b->have_points || !b->have_init) return bfail(b, KM_ESTATE, "set_points and set_init first");
  cudaEvent_t e0, e1;
  KB_CUDA(b, cudaEventCreate(&e0));
  KB_CUDA(b, cudaEventCreate(&e1));
  float best = 3.0e38f;
  int bt = kTileCand[1], bth = 256, bkind = 0;
  b->tune_ms.clear();
  // the assign kernel writes labels, partials and counters only: timing it
  // leaves the centroids and the loop state untouched.  Candidates: the
  // batch kernel's tiles x block sizes, then the fused kernel's tiles.
  auto time_shape = [&](int kind, int tp, int th) -> km_status {
    km_status s = build_tiles(b, tp);
    if (s != KM_OK) return s;
    b->kind = kind;
    b->threads = th;
    b->grid = grid_for(b, th);
    BatchArgs a = bargs(b);
    KB_CUDA(b, launch_assign_kind(b, a));  // warm-up
    KB_CUDA(b, cudaEventRecord(e0, b->st));
    for (int r = 0; r < 3; ++r) KB_CUDA(b, launch_assign_kind(b, a));
    KB_CUDA(b, cudaEventRecord(e1, b->st));
    KB_CUDA(b, cudaEventSynchronize(e1));
    float ms = 0.f;
    KB_CUDA(b, cudaEventElapsedTime(&ms, e0, e1));
    b->tune_ms.push_back(ms / 3.f);
    if (ms < best) { best = ms; bt = tp; bth = th; bkind = kind; }
    return KM_OK;
  };
  for (int tp : kTileCand)
    for (int th : kThreadCand) {
      km_status s = time_shape(0, tp, th);
      if (s != KM_OK) return s;
    }
  for (int tp : kFastTileCand) {
    km_status s = time_shape(1, tp, 256);
    if (s != KM_OK) return s;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  km_status s = build_tiles(b, bt);
  if (s != KM_OK) return s;
  b->kind = bkind;
  b->threads = bth;
  b->grid = grid_for(b, bth);
  KB_CUDA(b, cudaMemsetAsync(b->stats, 0, sizeof(unsigned long long) * 2, b->st));
  KB_CUDA(b, cudaStreamSynchronize(b->st));
  b->tuned = true;
  drop_graph(b);
  if (tile_out) *tile_out = bt;
  if (threads_out) *threads_out = bth;
  return KM_OK;
}

km_status km_batch_set_shape(km_batch* b, int32_t tile_points, int32_t threads) {
  if (!b) return KM_EINVAL;
  if (!b->have_points) return bfail(b, KM_ESTATE, "set_points first");
  bool ok_t = false, ok_th = false, fast = false;
  for (int tp : kTileCand) ok_t = ok_t || tp == tile_points;
  for (int th : kThreadCand) ok_th = ok_th || th == threads;
  for (int tp : kFastTileCand) fast = fast || (tp == tile_points && threads == 256);
  if (!fast && (!ok_t || !ok_th)) return bfail(b, KM_EINVAL, "tile_points or threads is not one the tuner times");
  km_status s = build_tiles(b, tile_points);
  if (s != KM_OK) return s;
  b->kind = fast ? 1 : 0;
  b->threads = threads;
  b->grid = grid_for(b, threads);
  b->tune_ms.clear();
  b->tuned = true;
  drop_graph(b);
  return KM_OK;
}

km_status km_batch_run(km_batch* b, int32_t max_iter, double tol, int32_t* labels_out, double* centroids_out,
                       int32_t* iters_out, double* e_out, int32_t* converged_out) {
  if (!b) return KM_EINVAL;
  if (!b->have_points || !b->have_init) return bfail(b, KM_ESTATE, "set_points and set_init first");
  if (max_iter < 0) return bfail(b, KM_EINVAL, "max_iter < 0");
  if (!(tol >= 0.0)) return bfail(b, KM_EINVAL, "tol must be >= 0");
  if (!b->tuned) {
    km_status s = km_batch_tune(b, nullptr, nullptr);
    if (s != KM_OK) return s;
  }
  // every instance runs up to max_iter more steps from its current centres
  KB_CUDA(b, cudaMemcpyAsync(b->hstate.data(), b->state, sizeof(BatchState) * b->count, cudaMemcpyDeviceToHost, b->st));
  KB_CUDA(b, cudaStreamSynchronize(b->st));
  int act = 0;
  for (auto& s : b->hstate) {
    s.max_iter = s.iter + max_iter;
    s.converged = 0;
    s.done = max_iter == 0 ? 1 : 0;
    act += !s.done;
  }
  KB_CUDA(b, cudaMemcpyAsync(b->state, b->hstate.data(), sizeof(BatchState) * b->count, cudaMemcpyHostToDevice, b->st));
  KB_CUDA(b, cudaMemcpyAsync(b->active, &act, sizeof(int), cudaMemcpyHostToDevice, b->st));
  BatchArgs a = bargs(b);
  a.tol = tol;
  // the tolerance is a kernel argument: the graph is rebuilt when it changes
  if (b->graph && b->graph_tol != tol) drop_graph(b);
  if (b->opt.use_graph && !b->graph) {
    cudaGraph_t g = nullptr;
    KB_CUDA(b, cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
    for (int r = 0; r < kGraphSteps; ++r) {
      launch_assign_kind(b, a);
      launch_batch_update(a, b->count, b->st);
    }
    cudaError_t ce = cudaStreamEndCapture(b->st, &g);
    if (ce != cudaSuccess) return bfail(b, KM_ECUDA, std::string("capture: ") + cudaGetErrorString(ce));
    ce = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) return bfail(b, KM_ECUDA, std::string("instantiate: ") + cudaGetErrorString(ce));
    b->graph_tol = tol;
    b->graph_steps = kGraphSteps;
  }
  int remaining = act;
  for (int done_steps = 0; remaining > 0 && done_steps < max_iter;) {
    if (b->graph) {
      KB_CUDA(b, cudaGraphLaunch(b->graph, b->st));
      done_steps += b->graph_steps;
    } else {
      KB_CUDA(b, launch_assign_kind(b, a));
      KB_CUDA(b, launch_batch_update(a, b->count, b->st));
      done_steps += 1;
    }
    KB_CUDA(b, cudaMemcpyAsync(&remaining, b->active, sizeof(int), cudaMemcpyDeviceToHost, b->st));
    KB_CUDA(b, cudaStreamSynchronize(b->st));
  }
  KB_CUDA(b, cudaMemcpyAsync(b->hstate.data(), b->state, sizeof(BatchState) * b->count, cudaMemcpyDeviceToHost, b->st));
  if (labels_out)
    KB_CUDA(b, cudaMemcpyAsync(labels_out, b->labels, sizeof(int32_t) * (size_t)b->total_n, cudaMemcpyDefault, b->st));
  if (centroids_out)
    KB_CUDA(b, cudaMemcpyAsync(centroids_out, b->mu, sizeof(double) * (size_t)b->total_kd, cudaMemcpyDefault, b->st));
  KB_CUDA(b, cudaStreamSynchronize(b->st));
  bool all_conv = true;
  for (int i = 0; i < b->count; ++i) {
    const BatchState& s = b->hstate[i];
    if (iters_out) iters_out[i] = s.iter;
    if (e_out) e_out[i] = b->opt.e_mode == 1 ? s.E2 : s.E;
    if (converged_out) converged_out[i] = s.converged;
    all_conv = all_conv && s.converged;
  }
  return all_conv ? KM_OK : KM_NOT_CONVERGED;
}

km_status km_batch_get_counts(km_batch* b, int64_t* counts_out) {
  if (!b || !counts_out) return KM_EINVAL;
  KB_CUDA(b, cudaMemcpyAsync(counts_out, b->counts, sizeof(long long) * (size_t)b->total_k, cudaMemcpyDefault, b->st));
  KB_CUDA(b, cudaStreamSynchronize(b->st));
  return KM_OK;
}

km_status km_batch_objective(km_batch* b, double* out) {
  if (!b || !out) return KM_EINVAL;
  if (!b->have_points || !b->have_init) return bfail(b, KM_ESTATE, "set_points and set_init first");
  double* d = nullptr;
  KB_CUDA(b, balloc(&d, (size_t)b->count));
  cudaError_t e = launch_batch_objective(b->x, b->inst, b->labels, b->mu, d, b->count, b->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, d, sizeof(double) * b->count, cudaMemcpyDeviceToHost, b->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
  cudaFree(d);
  if (e != cudaSuccess) return bfail(b, KM_ECUDA, std::string("objective: ") + cudaGetErrorString(e));
  return KM_OK;
}

km_status km_batch_get_info(km_batch* b, km_batch_info* out) {
  if (!b || !out) return KM_EINVAL;
  std::memset(out, 0, sizeof(*out));
  unsigned long long st[2] = {0, 0};
  KB_CUDA(b, cudaMemcpyAsync(st, b->stats, sizeof(st), cudaMemcpyDeviceToHost, b->st));
  KB_CUDA(b, cudaStreamSynchronize(b->st));
  out->flagged = st[0];
  out->fp64_decided = st[1];
  out->tile_points = b->tile_pts;
  out->threads = b->threads;
  out->grid = b->grid;
  out->tiles = b->ntiles;
  out->tuned = b->tuned ? 1 : 0;
  const int nc = (int)std::min<size_t>(b->tune_ms.size(), sizeof(out->tune_ms) / sizeof(out->tune_ms[0]));
  for (int q = 0; q < nc; ++q) out->tune_ms[q] = b->tune_ms[q];
  out->tune_candidates = nc;
  return KM_OK;
}

const char* km_batch_last_error(const km_batch* b) { return b ? b->err.c_str() : "null batch"; }

void km_batch_destroy(km_batch* b) {
  if (!b) return;
  drop_graph(b);
  void* bufs[] = {b->x, b->labels, b->mu, b->ctil, b->counts, b->inst, b->state, b->tiles,
                  b->tile_poff, b->partials, b->stats, b->active, b->tab2, b->ctil4, b->ic};
  for (void* p : bufs)
    if (p) cudaFree(p);
  if (b->own_stream && b->st) cudaStreamDestroy(b->st);
  delete b;
}

}  // extern "C"
