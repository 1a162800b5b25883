/*
 * km.h -- C ABI of the GB300 (sm_103a) Lloyd's K-means library (libkm.so).
 *
 * The library runs the data-parallel hot path of Lloyd's algorithm as stated
 * in "Parallelization of the K-Means Algorithm with Applications to Big Data
 * Clustering" (arXiv 2405.12052):
 *   - reassignment  z_i = argmin_k ||x_i - mu_k||_2^2
 *                   (section "The Lloyd's algorithm", step 2);
 *   - mean update   mu_k = sum_i 1(z_i = k) x_i / sum_i 1(z_i = k)
 *                   (same section, step 3);
 *   - error         E^2 = sum_k ||mu_k^{t+1} - mu_k^t||_2^2, loop until the
 *                   error is below a tolerance (section "Serial Lloyd's
 *                   algorithm").
 * The inputs the paper names for its serial program are the dataset, the
 * number of clusters and the number of points (same section); the outputs
 * are the final cluster indicators and means.
 *
 * Conventions shared by every entry point
 *   - Points are float32 in the paper's layout X in R^{d x N}: coordinate j of
 *     point i is at x[j * ld + i] (KM_SOA_DxN), or row-major N x d
 *     (KM_AOS_NxD, copied into the SoA layout on entry).
 *   - Centroids are double, K x d, row-major.  Labels are int32 in 0..K-1
 *     (the paper numbers clusters 1..K); a context may keep them as bytes
 *     (km_options.label_bytes = 1, K <= 256).
 *   - Labels are exact: every point's label equals the argmin of the
 *     double-precision squared distances sum_j (x_ij - mu_kj)^2 accumulated
 *     over j in order, ties to the lowest k.  Points whose two nearest FP32
 *     distances are within a rigorous error bound, or within 1e-5 relative,
 *     are re-decided in double precision on the GPU.
 *   - Per-cluster sums are exact integer (fixed-point) sums; centroids are
 *     one rounding of sum / count.  An empty cluster keeps its centre.
 *   - Every call returns a km_status.  A status < 0 leaves the context
 *     usable only for km_last_error and km_destroy.  km_last_error returns a
 *     message owned by the context, valid until the next call on it.
 *   - Calls on one context are not thread-safe; distinct contexts are
 *     independent.  Work is queued on the stream given in km_options (NULL:
 *     a blocking stream the context creates, which orders itself after work
 *     on the legacy default stream); calls that return host data synchronize
 *     it.
 *   - There is no CPU fallback: if no sm_103a device is present, km_create
 *     returns KM_ECUDA.
 */
#ifndef KM_H
#define KM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct km_ctx km_ctx; /* opaque; owns every device buffer it allocates */

typedef enum {
  KM_OK = 0,
  KM_NOT_CONVERGED = 1, /* km_run reached max_iter; outputs are still valid */
  KM_EINVAL = -1,       /* bad argument (null pointer, size, layout, K > N) */
  KM_ENOMEM = -2,       /* device or host allocation failed */
  KM_ECUDA = -3,        /* a CUDA call failed, or no usable device */
  KM_ESTATE = -4,       /* step/run before km_set_points and km_set_init */
  KM_ETIMEOUT = -5,     /* a bounded device wait gave up (error word 3) */
  KM_ENUMERIC = -6      /* NaN/Inf in the points or centroids, or data out of range */
} km_status;

enum { KM_SOA_DxN = 0, KM_AOS_NxD = 1 };                       /* point layouts */
enum { KM_HOST = 0, KM_DEVICE_COPY = 1, KM_DEVICE_BORROW = 2 }; /* where a buffer lives */
enum { KM_E_NORM = 0, KM_E_SQUARED = 1 };                      /* which error km_run tests */
enum { KM_LABELS_EVERY_STEP = 0, KM_LABELS_FINAL = 1 };         /* label write policy */
enum { KM_DIST_AUTO = 0, KM_DIST_SIMT = 1, KM_DIST_TENSOR = 2 }; /* distance path */
enum { KM_TC_BF16 = 0, KM_TC_F16 = 1 };                         /* tensor-core operand type */

typedef struct km_options {
  int32_t e_mode;  /* KM_E_NORM (default): stop when sqrt(E^2) < tol;
                      KM_E_SQUARED: the paper's E^2 = sum ||dmu||^2 < tol */
  int32_t use_graph; /* 1 (default): km_run drives the loop from one CUDA graph
                        with a device-side stop; 0: one host round trip per step */
  double tie_rel;  /* relative near-tie threshold re-decided in FP64 (default 1e-5) */
  void* stream;    /* cudaStream_t for all work (NULL: the context creates one) */
  int32_t label_policy; /* KM_LABELS_EVERY_STEP (default): every step writes its labels
                           (the "final cluster indicators" are the last step's);
                           KM_LABELS_FINAL: steps skip the N label writes and
                           km_run ends with one assignment pass against the returned
                           centroids (km_write_labels); ignored by the tensor-core
                           path, whose next step reads the labels */
  int32_t dist_path;    /* KM_DIST_AUTO (default): tensor cores for d = 64 and K <= 1024,
                           else FP32 SIMT; KM_DIST_SIMT: FP32 SIMT kernels always;
                           KM_DIST_TENSOR: a tcgen05 path -- the BF16 GEMM form (d = 64,
                           K <= 1024) or, for d <= 3 and K <= 32, the fused step with
                           its screen on TF32 tensor cores (same labels and sums;
                           slower than the FFMA2 screen at these sizes) -- or KM_EINVAL */
  int32_t tc_operands;  /* operands of the tcgen05 distances: KM_TC_BF16 (default; 8
                           significand bits) or KM_TC_F16 (11 bits, same tensor rate;
                           points and centres scaled by powers of two into FP16's
                           range), so a candidate window 8x narrower; the labels are
                           exact either way */
  int32_t label_bytes;  /* 4 (default): int32 labels; 1: labels kept as bytes (K <= 256,
                           FP32 paths only, else KM_EINVAL): a quarter of the label
                           traffic; read them with km_get_labels_u8 (km_get_labels and
                           km_run's labels_out still give int32, widened on the device) */
} km_options;

/* Fill *opt with the defaults above. */
void km_default_options(km_options* opt);

/* Create a context for N points of dimension d and K clusters on the current
 * CUDA device.  opt may be NULL (defaults).  Allocates the per-context device
 * buffers (labels, centroids, per-block partial sums).
 * Errors: KM_EINVAL (out == NULL, n < 1, d < 1, k < 1, k > n),
 *         KM_ECUDA (no sm_103a device), KM_ENOMEM. */
km_status km_create(km_ctx** out, int64_t n, int32_t d, int32_t k, const km_options* opt);

/* Give the context its points X (section "The Lloyd's algorithm": X in
 * R^{d x N}).  layout: KM_SOA_DxN (ld = elements between coordinate rows,
 * >= N) or KM_AOS_NxD (ld = elements between points, >= d).  mem: KM_HOST
 * (host pointer; copied to the device), KM_DEVICE_COPY (device pointer;
 * copied), KM_DEVICE_BORROW (device SoA pointer kept as is: it must stay
 * valid and unchanged until km_destroy or the next km_set_points; a pointer
 * that is not 16-byte aligned, or an ld that is not a multiple of 4, is
 * copied instead).  Scans the points once for their range; any NaN/Inf gives
 * KM_ENUMERIC.  Synchronizes the stream. */
km_status km_set_points(km_ctx* ctx, const float* x, int64_t ld, int32_t layout, int32_t mem);

/* Set the starting centroids mu^0 (section "The Lloyd's algorithm", step 1),
 * K x d row-major doubles in host memory, and reset the iteration count.
 * Resuming from km_get_centroids output continues a run bit-identically.
 * Errors: KM_EINVAL (null), KM_ENUMERIC (non-finite). */
km_status km_set_init(km_ctx* ctx, const double* mu0);

/* k-means++ seeding (D^2 sampling, Arthur and Vassilvitskii 2007) on the
 * context's points, then km_set_init with the result.  u: K uniforms in
 * [0, 1) (host), the only randomness: the first centre is point
 * floor(u[0] N); centre c is the first point whose running sum of D^2
 * (squared FP64 distance to the nearest centre chosen so far, coordinates in
 * order) exceeds u[c] times the total, the last point if none does.  The
 * sums run over 4096-point chunks in a fixed order, so the picks equal a
 * sequential scan's except when a target lies within FP64 rounding of a
 * running-sum boundary.  Outputs (host, may be NULL): mu_out K x d doubles,
 * idx_out K point indices.  Needs km_set_points first; d <= 256; allocates
 * N + N/4096 + 4096 doubles of scratch for the call.
 * Errors: KM_ESTATE, KM_EINVAL (u outside [0, 1)), KM_ENOMEM, KM_ECUDA. */
km_status km_init_kmeanspp(km_ctx* ctx, const double* u, double* mu_out, int64_t* idx_out);

/* One Lloyd step from the current centroids: reassignment, mean update and
 * error.  Writes E (sqrt of E^2) and E^2 to the non-NULL outputs and
 * synchronizes the stream.  Errors: KM_ESTATE, KM_ECUDA. */
km_status km_step(km_ctx* ctx, double* e_out, double* e2_out);

/* Run steps until the selected error (km_options.e_mode) is < tol or max_iter
 * steps have run (section "Serial Lloyd's algorithm").  Outputs (each may be
 * NULL): labels_out (N int32, host memory) from the last step, centroids_out
 * (K x d doubles, host), iters_out (steps run, including the one that met the
 * tolerance), e_out (E of the last step).  Returns KM_OK when converged,
 * KM_NOT_CONVERGED when max_iter was reached.  The iteration count restarts
 * at km_set_init; a second km_run continues from the current centroids. */
km_status km_run(km_ctx* ctx, int32_t max_iter, double tol, int32_t* labels_out,
                 double* centroids_out, int32_t* iters_out, double* e_out);

/* Asynchronous pieces of a step, for callers that drive (or capture into a
 * CUDA graph) their own loop on the context's stream.  None of them
 * synchronizes.  km_begin sets the stop rule for the steps that follow
 * (max_iter counted from the current iteration, tol as in km_run); then each
 * step is km_assign_async (reassignment and per-block sums, one kernel)
 * followed by km_update_async (fixed-order reduction, divide, error and next
 * screen tables, one kernel).  Once the stop rule has fired, further kernels
 * return immediately.  km_sync reads the step count and error back.
 * Errors: KM_ESTATE before points and centroids are set, KM_ECUDA. */
km_status km_begin(km_ctx* ctx, int32_t max_iter, double tol);
km_status km_assign_async(km_ctx* ctx);
km_status km_update_async(km_ctx* ctx);
km_status km_sync(km_ctx* ctx, int32_t* iters_out, double* e_out, int32_t* done_out);

/* Sharded steps: the points split over R contexts (one per process or GPU,
 * each holding a contiguous or any other disjoint part), with the caller
 * exchanging a small table per step -- the paper's OpenMP scheme, where each
 * thread's local sums are merged before the master thread divides (section
 * "Parallel Lloyd's algorithm", "Using OpenMP"), with an all-gather in place
 * of the critical section.
 *
 * Set-up: after km_set_points on every shard, read each shard's fixed-point
 * grid exponent with km_grid_exponent, take the maximum over the shards and
 * give it to every shard with km_set_grid_exponent (the exponent of a single
 * context over all points is that maximum).  Then km_set_init with the same
 * centroids on every shard, and km_begin as for the asynchronous pieces.
 *
 * Each step on each shard: km_assign_async; km_shard_totals writes this
 * shard's column totals -- for every centre k and column j (0..d-1 the
 * coordinate sums on the fixed-point grid, d the count) one exact int128 as
 * two int64 words, low word first: K * (d+1) * 2 int64 in total, row-major
 * [k][j][word]; the caller all-gathers the R tables in rank order
 * (R * K * (d+1) * 2 int64) and passes them to km_shard_update, which adds
 * them in rank order (exact integers), divides, forms E, applies the stop
 * rule and prepares the next step.  Because every sum is an exact integer
 * and the labels are exact, every shard's centroids, counts (global) and E
 * are bit-identical to one context over all points, and each shard's labels
 * are that context's labels of its points.
 *
 * mem: KM_HOST (host arrays; the call synchronizes) or KM_DEVICE_COPY
 * (device arrays of the context's device, used on the context's stream
 * without synchronizing).  Every path: on the tensor-core GEMM path the
 * totals come from its sorted mean calculation (each cluster's chunk sums
 * added in order), with the same table layout.  km_set_grid_exponent
 * returns KM_EINVAL below the
 * exponent the shard's own points need or above 100, KM_ESTATE before
 * km_set_points. */
km_status km_grid_exponent(km_ctx* ctx, int32_t* ex_out);
km_status km_set_grid_exponent(km_ctx* ctx, int32_t ex);
km_status km_shard_totals(km_ctx* ctx, int64_t* totals_out, int32_t mem);
km_status km_shard_update(km_ctx* ctx, const int64_t* tables, int32_t ranks, int32_t mem);

/* The stream the context queues its work on (a cudaStream_t). */
void* km_stream(km_ctx* ctx);

/* Labels of the current centroids: one assignment pass (its sums are not
 * used; the stop flag does not stop it) writing the N labels, for the
 * KM_LABELS_FINAL policy (km_run calls it at the end).  Queued on the stream;
 * km_get_labels synchronizes.  No-op on the tensor-core path (its steps
 * always write labels).  Errors: KM_ESTATE, KM_ECUDA. */
km_status km_write_labels(km_ctx* ctx);

/* The objective sum_i ||x_i - mu_{z_i}||^2 of the current labels (last step)
 * and centroids, in FP64 with the oracle's order: per point coordinates in
 * order, points in index order within 65536-point chunks, then the chunks
 * in order.  Synchronizes.  Errors: KM_ESTATE, KM_ENOMEM, KM_ECUDA. */
km_status km_objective(km_ctx* ctx, double* obj_out);

/* Copy results of the last step.  mem: KM_HOST or KM_DEVICE_COPY (device
 * pointer of the caller).  Sizes: labels N int32, centroids K x d doubles,
 * counts K int64.  Synchronize the stream. */
km_status km_get_labels(km_ctx* ctx, int32_t* labels_out, int32_t mem);
/* The labels as N bytes (contexts created with label_bytes = 1; else
 * KM_EINVAL).  mem as for km_get_labels.  Synchronizes. */
km_status km_get_labels_u8(km_ctx* ctx, uint8_t* labels_out, int32_t mem);
km_status km_get_centroids(km_ctx* ctx, double* centroids_out, int32_t mem);
km_status km_get_counts(km_ctx* ctx, int64_t* counts_out);

/* Diagnostics of the last step. */
typedef struct km_stats {
  int32_t iters;          /* steps since km_set_init */
  int32_t converged;      /* 1 once the tolerance was met in km_run */
  double e, e2;           /* error of the last step */
  int64_t flagged;        /* points re-checked past the FP32 screen in the last step */
  int64_t fp64_decided;   /* of those, points decided in FP64 */
  int32_t empty_clusters; /* clusters with no points in the last step */
  int64_t overflowed;     /* tensor-core path: points whose candidate list overflowed (all K re-ranked) */
  int32_t path;           /* 1: fused FFMA2 kernel (d <= 4, K <= 256); 2: generic kernel;
                             3: tcgen05 BF16 GEMM-form kernel (d = 64, K <= 1024);
                             4: fused kernel with the tcgen05 TF32 screen (d <= 3, K <= 32) */
} km_stats;
km_status km_get_stats(km_ctx* ctx, km_stats* out);

/* Device pointers owned by the context, for callers that keep data on the
 * GPU (valid until km_destroy).  Points are the SoA copy (or the borrowed
 * pointer) with row stride *ld_out; *labels is NULL when the context keeps
 * 1-byte labels. */
km_status km_device_buffers(km_ctx* ctx, const float** points, int64_t* ld_out,
                            int32_t** labels, double** centroids);

/* One Lloyd step that allocates no memory (the paper has no counterpart; this
 * entry point exists for callers that cannot call cudaMalloc, for example
 * code running under an allocator that must not be entered after start-up, a
 * real-time loop that forbids allocation, or a host framework that owns every
 * device allocation).  Everything is caller-owned device memory: x (d x N SoA,
 * row stride ld >= N, finite float32 with |x| < 2^99), mu_in (K x d doubles),
 * and the outputs
 * labels (N int32), mu_out (K x d doubles, may not alias mu_in), counts
 * (K int64) and e2_out (one double: E^2 against mu_in).  Same results as
 * km_step: exact labels (FP64 re-decision of near ties, ties to the lowest k),
 * exact fixed-point sums, an empty cluster keeps its centre.
 *
 * Limits of the fixed scratch (a ~0.6 MB file-scope __device__ array that
 * every device loading the library holds until exit): K*(d+1) <= 256 and
 * N <= 304 * 2^19.  Larger sizes return KM_EINVAL with a message in errbuf
 * (errbuf may be NULL; errlen is its size in bytes).  The call returns before
 * the data is read, so data outside the range above (a NaN, an infinity or
 * |x| >= 2^99) cannot be reported by the status: the step then marks its
 * outputs invalid instead -- every mu_out entry and *e2_out are NaN and every
 * count is -1 (labels are in 0..K-1 but meaningless).
 *
 * The work is queued on `stream` (a cudaStream_t, NULL = legacy default
 * stream) and the call returns without synchronizing.  The first call on a
 * device looks up the scratch array's device address (once per device, with
 * that device current, and once more after the device's context has been
 * destroyed and re-created, e.g. by cudaDeviceReset); make that first call
 * before any stream capture.  All
 * calls share the one scratch array, which keeps the last call's contents:
 * calls that overlap on the GPU (different streams, or devices sharing the
 * same context) race and give wrong results; serialize them. */
km_status km_lloyd_step_noalloc(const float* x, int64_t ld, int64_t n, int32_t d, int32_t k,
                                const double* mu_in, int32_t* labels, double* mu_out,
                                int64_t* counts, double* e2_out, void* stream, char* errbuf,
                                int32_t errlen);

const char* km_last_error(const km_ctx* ctx);
void km_destroy(km_ctx* ctx);

/* ---- Batched instances ------------------------------------------------
 * Many independent clustering problems (instance i: N_i points of dimension
 * d_i in 1..3, K_i in 1..64 clusters) run by shared launches: each step is
 * one persistent assign kernel over the tiles of every active instance and
 * one update kernel with a block per instance (section "The Lloyd's
 * algorithm", steps 2-3, per instance; every instance keeps its own stop
 * test).  Results per instance are those of km_run on that instance alone:
 * exact labels, exact fixed-point sums, the same E.
 *
 * Layouts (all concatenated in instance order):
 *   points     instance i is d_i x N_i SoA (row stride N_i) at element
 *              offset sum_{j<i} d_j N_j;
 *   labels     N_i int32 at offset sum_{j<i} N_j;
 *   centroids  K_i x d_i row-major doubles at offset sum_{j<i} K_j d_j;
 *   counts     K_i int64 at offset sum_{j<i} K_j. */
typedef struct km_batch km_batch;

/* count instances with sizes n[i], d[i], k[i] (host arrays).  opt may be
 * NULL; e_mode, tie_rel, use_graph and stream apply.  On a non-OK status
 * *out may still hold a batch that only km_batch_last_error and
 * km_batch_destroy accept.
 * Errors: KM_EINVAL (count < 1, d not in 1..3, K not in 1..64, K > N,
 *         N >= 2^31), KM_ECUDA. */
km_status km_batch_create(km_batch** out, int32_t count, const int64_t* n, const int32_t* d, const int32_t* k,
                          const km_options* opt);

/* Copy all instances' points (layout above; mem KM_HOST or KM_DEVICE_COPY),
 * then per instance on the GPU: coordinate range, FP32 shift, fixed-point
 * grid.  Errors: KM_ENUMERIC (NaN/Inf or |x| >= 2^99). */
km_status km_batch_set_points(km_batch* b, const float* x, int32_t mem);

/* Starting centroids of every instance (host doubles, layout above); resets
 * every instance's iteration count.  Errors: KM_ENUMERIC (non-finite). */
km_status km_batch_set_init(km_batch* b, const double* mu0);

/* Time the launch shapes on this batch and keep the fastest (the first
 * km_batch_run does this when it was not called): the batch kernel's tile
 * sizes (512, 1024 points) x block sizes (128, 256, 512 threads), then the
 * fused kernel's tile machinery (8 points per lane, 256 threads) on tiles of
 * 8192 and 32768 points.  Every shape gives the same results.  Leaves
 * centroids and iteration counts unchanged.  Outputs may be NULL. */
km_status km_batch_tune(km_batch* b, int32_t* tile_out, int32_t* threads_out);

/* Use a launch shape without timing (one the tuner times: tile_points 512 or
 * 1024 with threads 128, 256 or 512, or tile_points 8192 or 32768 with 256
 * threads for the fused kernel), e.g. a shape a previous km_batch_tune chose
 * for the same instances, kept in a cache.  Errors: KM_EINVAL (another
 * shape), KM_ESTATE (no points). */
km_status km_batch_set_shape(km_batch* b, int32_t tile_points, int32_t threads);

/* Per instance the objective sum_i ||x_i - mu_{z_i}||^2 of its current
 * labels (last step) and centroids, in FP64 (host out[count]; a fixed
 * summation order, so repeatable).  Synchronizes.  Errors: KM_EINVAL,
 * KM_ESTATE, KM_ENOMEM, KM_ECUDA. */
km_status km_batch_objective(km_batch* b, double* out);

/* Run every instance until its selected error is < tol or max_iter more
 * steps have run; the steps are replayed from a captured CUDA graph (4 steps
 * per launch; stopped instances do no work) until no instance is active.
 * Outputs (host or device pointers, each may be NULL): labels_out (sum N_i),
 * centroids_out (sum K_i d_i), and per instance iters_out (steps since
 * km_batch_set_init), e_out (E, or E^2 when e_mode = 1), converged_out.
 * Returns KM_OK when every instance converged, else KM_NOT_CONVERGED. */
km_status km_batch_run(km_batch* b, int32_t max_iter, double tol, int32_t* labels_out, double* centroids_out,
                       int32_t* iters_out, double* e_out, int32_t* converged_out);

/* Cluster sizes of the last step (sum K_i int64, host or device). */
km_status km_batch_get_counts(km_batch* b, int64_t* counts_out);

typedef struct km_batch_info {
  int64_t flagged;        /* points re-checked past the FP32 screen, all steps so far */
  int64_t fp64_decided;   /* of those, decided in FP64 */
  int32_t tile_points;    /* launch shape in use */
  int32_t threads;
  int32_t grid;
  int32_t tiles;
  int32_t tuned;          /* 1 once km_batch_tune ran */
  int32_t tune_candidates;
  float tune_ms[8];       /* per candidate: 512 x {128,256,512}, 1024 x {...}, then 8192 and 32768 (fused) */
} km_batch_info;
km_status km_batch_get_info(km_batch* b, km_batch_info* out);

const char* km_batch_last_error(const km_batch* b);
void km_batch_destroy(km_batch* b);

/* ---- Learned initialiser ------------------------------------------------
 * A set network that predicts K starting centres from a sample of S points
 * (the paper notes how the result depends on the initial centres, section
 * "The Lloyd's algorithm"): per point h1 = relu(W1 x' + b1) and
 * h2 = relu(W2 h1 + b2) (128 wide) on x' = (x - m) / s, the sample's
 * per-coordinate mean m and population std s (1 where 0); g = the mean of h2
 * over the points; a3 = relu(W3 g + b3); p = W4 a3 + b4 (K x d); centres
 * c = p * s + m.  Training minimises the mean over sets of the symmetric
 * Chamfer distance between p and the standardised target centres.
 * Parameters are one float32 vector in the order W1 (128 x d), b1, W2
 * (128 x 128), b2, W3 (128 x 128), b3, W4 (K d x 128), b4 (row-major).
 * Inputs: x is [B][S][d] float32 (set b, point i, coordinate j at
 * (b S + i) d + j), targets [B][K][d]; S a positive multiple of 64; mem
 * KM_HOST (copied) or a device kind (the pointer is read in place).  FP32
 * kernels, every sum in a fixed order: a step is deterministic. */
typedef struct km_setnet km_setnet;

/* d in 1..3, K in 1..64; parameters start at zero (set them).  stream may be
 * NULL (the network creates one). */
km_status km_setnet_create(km_setnet** out, int32_t d, int32_t k, void* stream);
int64_t km_setnet_param_count(const km_setnet* net);
int32_t km_setnet_dims(const km_setnet* net, int32_t* k_out); /* returns d */
void* km_setnet_stream(const km_setnet* net);
/* Host copies of the parameters; setting them also clears Adam's moments. */
km_status km_setnet_set_params(km_setnet* net, const float* params);
km_status km_setnet_get_params(km_setnet* net, float* params_out);
/* Forward, loss and backward on a batch of B sets; the gradients stay on the
 * device (km_setnet_get_grads copies them).  loss_out (host) may be NULL
 * (then nothing synchronizes). */
km_status km_setnet_loss_grad(km_setnet* net, const float* x, const float* targets, int32_t B, int32_t S,
                              int32_t mem, float* loss_out);
km_status km_setnet_get_grads(km_setnet* net, float* grads_out);
/* One Adam step (Kingma and Ba 2015, bias-corrected) with the last gradients. */
km_status km_setnet_adam(km_setnet* net, float lr, float beta1, float beta2, float eps);
/* loss_grad + Adam (beta1 0.9, beta2 0.999, eps 1e-8). */
km_status km_setnet_train_step(km_setnet* net, const float* x, const float* targets, int32_t B, int32_t S,
                               int32_t mem, float lr, float* loss_out);
/* Centres for each of B sets: centroids_out [B][K][d] doubles (host or device). */
km_status km_setnet_predict(km_setnet* net, const float* x, int32_t B, int32_t S, int32_t mem,
                            double* centroids_out);
const char* km_setnet_last_error(const km_setnet* net);
void km_setnet_destroy(km_setnet* net);

/* Starting centroids of a context from the network: a sample of sample_n
 * points (a positive multiple of 64) of the context's points, point
 * floor(u_j N) for u_j the j-th SplitMix64 output from seed (53 bits), then
 * km_setnet_predict and km_set_init.  mu_out (host K x d) may be NULL.
 * Errors: KM_ESTATE (no points), KM_EINVAL (d or K differ from the
 * network's), KM_ENOMEM, KM_ECUDA. */
km_status km_init_learned(km_ctx* ctx, km_setnet* net, int32_t sample_n, uint64_t seed, double* mu_out);

/* Set transforms used around the network (test-time rotations of the
 * sample, rotations of training sets): the network's error depends on the
 * orientation of its input, so predictions for several rotated copies of
 * one sample can be compared (section "The Lloyd's algorithm": the result
 * depends on the initial centres).  All pointers are device memory of the
 * current device; the work is queued on `stream` without synchronizing.
 *   km_sets_mean: means_out[b][j] = the FP64 mean over s of x[b][s][j], for
 *     B sets of S points of dimension d (1..3), set b at x + b * set_stride
 *     (floats; 0 repeats one set), point s at offset s * d.
 *   km_sets_rotate_f32 / _f64: out[b][s] = R_b (x[b][s] - c_b) + c_b, or
 *     with R_b^T when transpose is non-zero; R is B x d x d row-major
 *     doubles (the rotations are inputs: random numbers the caller draws),
 *     c_b = center + b * center_stride (NULL: the origin); out is B x S x d
 *     contiguous; arithmetic in FP64, one rounding to the output type.
 * Errors: KM_EINVAL (null pointer, d outside 1..3, negative sizes),
 *         KM_ECUDA. */
km_status km_sets_mean(const float* x, int64_t set_stride, int32_t B, int32_t S, int32_t d, double* means_out,
                       void* stream);
km_status km_sets_rotate_f32(const float* x, int64_t set_stride, int32_t B, int32_t S, int32_t d, const double* R,
                             const double* center, int64_t center_stride, int32_t transpose, float* out, void* stream);
km_status km_sets_rotate_f64(const double* x, int64_t set_stride, int32_t B, int32_t S, int32_t d, const double* R,
                             const double* center, int64_t center_stride, int32_t transpose, double* out,
                             void* stream);

/* Library version string and the sm architecture it was built for. */
const char* km_version(void);

/* Self-test of the bounded device waits that every kernel waiting on an
 * mbarrier uses (the tensor-core path's producer and epilogue): one block
 * waits on an mbarrier that nothing arrives on, gives up after its limit
 * (about one second of GPU time) and records that, as a real wait would by
 * setting the device error word (which the host then reports as
 * KM_ETIMEOUT).  Sets *gave_up to 1 when the wait ended by its limit and
 * *elapsed_ms to the wall time of the call; the device stays usable.
 * Errors: KM_EINVAL (null output), KM_ENOMEM, KM_ECUDA. */
km_status km_selftest_bounded_wait(int32_t* gave_up, double* elapsed_ms);

/* Testing hook (allocation-failure injection, process-wide): after n more
 * successful device allocations by the library, the next one fails as if
 * the device were out of memory, and the call making it returns KM_ENOMEM
 * (the context then only accepts km_destroy, which frees what was
 * allocated).  n < 0 turns the injection off (the default). */
void km_debug_fail_alloc_after(int64_t n);

#ifdef __cplusplus
}
#endif
#endif /* KM_H */
