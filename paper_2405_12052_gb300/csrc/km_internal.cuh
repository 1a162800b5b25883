// Internal definitions shared by the kernels and the C ABI of libkm.so.
//
// Numerical scheme of one Lloyd step (reassignment, mean update, error; the
// paper's section "The Lloyd's algorithm" and section "Serial Lloyd's
// algorithm"):
//
// Screen (FP32).  With a per-dataset shift s, x~ = fl(x - s) and
// c~_k = fl32(mu_k - s), the kernel ranks W_k = ||c~_k||^2 - 2 x~.c~_k, which
// differs from D_ik = ||x_i - mu_k||^2 by a per-point constant.  The value is
// evaluated as r = M + 2^sigma W_k by an FMA chain whose every intermediate
// lies in one binade [2^eM, 2^(eM+1)) (M and sigma are chosen each step from
// bounds on ||x~||^2 and ||c~||^2), so every rounding is at most half an ulp
// of that binade.  The bits of r shifted left by L, plus k, form a positive
// float whose order is (r, k): top-2 tracking then needs only FMNMX.
//
// Flag.  A point is re-checked unless the gap between its two smallest r
// exceeds a rigorous bound on every error (input roundings, chain roundings,
// the oracle's own FP64 roundings) plus tie_rel * D2.  Flagged points go to a
// per-block queue and are decided by an FP32 direct-form pass with its own
// bound, and if that is not conclusive (or the two nearest are within
// tie_rel), by FP64 in the exact expression order sum_j (x_j - mu_kj)^2.
//
// Sums.  Each coordinate is split exactly into two integers on fixed grids
// (x = hi 2^G1 + lo 2^G0 up to a quantisation below 2^(G0-1), G1 = G0 + 22)
// with FP32 magic-number additions; the biased bit patterns are added with
// 32-bit shared-memory atomics (integer, so order-independent) into per-warp
// windows that are flushed into int64 per-warp totals.  Per-block int64
// partials are reduced in a fixed order in int128 and converted once.
#pragma once
#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>

namespace km {

constexpr int kMaxDFast = 4;        // fused FFMA2 kernel: d <= 4
constexpr int kMaxKFast = 256;      // and K <= 256 (index in <= 8 low bits)
constexpr int kThreads = 256;       // threads per block of the assign kernels
constexpr int kWarps = kThreads / 32;
#ifndef KM_PTS
#define KM_PTS 8
#endif
constexpr int kPts = KM_PTS;        // points per lane per warp-tile (fused kernel): 4 or 8
constexpr int kNG = kPts / 4;       // groups of 4 consecutive points per lane
constexpr int kGS = 128;            // points between a lane's groups (32 lanes x 4)
constexpr int kWarpTile = 32 * kPts;  // points per warp-tile
static_assert(kPts == 4 || kPts == 8, "points per lane");
#ifndef KM_MINB
#define KM_MINB 2                   // resident blocks per SM the fused kernel is compiled for
#endif
constexpr int kWarpQueue = 320;     // flagged points queued per warp (drained above 64)
constexpr int64_t kMaxPointsPerBlock = int64_t(1) << 19;
constexpr int kConstTabWords = 64 * 5;  // constant-bank screen table: kpad <= 64, d + 1 <= 5 packed pairs

// Per-dataset constants, fixed by km_set_points.
struct DataConst {
  float s[kMaxDFast];   // shift used by the screen (fused kernel)
  float A_max;          // max_i fl32 ||fl(x_i - s)||^2 with the kernel's expression
  int G0;               // fixed-point grid exponent of the low limb
  float C_hi, C_lo;     // 1.5 * 2^(G0+45), 1.5 * 2^(G0+23)
  uint32_t bits_C_hi, bits_C_lo;
};

// Per-step constants of the screen, written by the update kernel.
struct IterConst {
  float M;              // bias, 2^eM * (1.5 | 1.25 | 1.375)
  uint32_t bitsM_low;   // bits(M) with the top L bits cleared
  uint32_t mul;         // 2^L
  int L;                // index bits
  float thr_c0;         // flag threshold, constant part (ulps of the binade)
  float thr_cA;         // per unit of ||x~||^2 (ulps)
  float tau;            // tie_rel * (1 + 1e-4)
  float G;              // 2^(sigma - eM + 23): unscaled -> ulps
  float B_max;          // max_k ||c~_k||^2 (FP32, rounded up)
  float pad[3];
};

// Loop state on the device.  The first 24 bytes are control fields written
// by the host before a run or a step; the rest is written by the kernels.
struct LoopState {
  int32_t done;         // 1: the stop test passed or max_iter reached
  int32_t max_iter;     // absolute iteration count at which to stop
  int32_t e_mode;       // 0: test sqrt(E^2); 1: test E^2
  int32_t converged;    // set by the update kernel when the test passes
  double tol;
  int32_t iter;         // steps done since set_init
  int32_t empty;        // empty clusters in the last step
  double E, E2;         // error of the last step
  unsigned long long flagged;       // accumulating during a step
  unsigned long long fp64_decided;  // accumulating during a step
  unsigned long long last_flagged;  // of the last completed step
  unsigned long long last_fp64;
  unsigned long long overflowed;    // tensor-core path: candidate lists that overflowed (this step)
  unsigned long long last_overflowed;
  unsigned int ticket;              // last-block counter of the reduction
  int32_t error;                    // sticky device error word (0 = none)
};
struct LoopControl {
  int32_t done, max_iter, e_mode, converged;
  double tol;
};
static_assert(sizeof(LoopControl) == 24, "control block layout");

struct FastArgs {
  const float* x; int64_t ld; int64_t n; int k; int kpad;
  const unsigned long long* tab2;  // [kpad][D+1] packed (a, a) float pairs
  const float4* ctil;              // [k] (c~_0.., B_k) fp32 table for the re-check
  const double* mu;                // [k][D] current centroids (FP64)
  const IterConst* ic;
  const DataConst* dc;
  LoopState* ls;
  int32_t* labels;
  long long* partials;             // [gridDim.x][k][D+1]
  int64_t ntiles;
  int nwin;                        // 32-bit sum windows per warp: 4 (one per 8 lanes), 2 (one per half-warp) or 1 (large K)
  int store_labels;                // 0: labels are not written (label policy "final")
  uint8_t* labels8;                // non-null: labels are written here as bytes (K <= 256), not to labels
  int ignore_done;                 // 1: run even after the stop flag (the final labels pass)
  int const_tab;                   // 1: the screen reads the table from the constant bank (copied at launch)
  int labels_unaligned;            // 1: labels + i may not be 16-byte aligned (store them one by one)
};

struct GenericArgs {
  const float* x; int64_t ld; int64_t n; int d; int k;
  const float* ctil;               // [k][d] fp32 (mu - s)
  const float* cnorm;              // [k] ||c~||^2 fp32 (unused by the direct form)
  const double* mu;                // [k][d]
  const float* shift;              // [d]
  const DataConst* dc;
  LoopState* ls;
  int32_t* labels;
  long long* partials;             // [gridDim.x][k][d+1]
  float A_max;
  const float* B_max_ptr;          // max_k ||c~_k||^2, written by the update kernel
  float tau;
  int store_labels;                // as in FastArgs
  uint8_t* labels8;                // as in FastArgs
  int ignore_done;
};

// ---- tensor-core path (d = 64) and sorted mean calculation ----
constexpr int kGemmD = 64;          // dimension of the tcgen05 path (one 128-byte BF16 row)
constexpr int kGemmMaxK = 1024;     // centroid rows resident in shared memory
constexpr int kChunk = 2048;        // points per chunk of the sorted mean calculation

struct GemmConst {
  float scale;   // -2^(sigma+1)
  float M;       // 1.5: r = M + 2^sigma (h - 2 S) lies in [1, 2)
  float c0, c1, cA;  // candidate window Delta(x) = c0 + ||x~|| c1 + ||x~||^2 cA (units of r)
  float cest;    // extra window of the start estimate per unit ||x~||
  float B_max;   // max_k ||mu_k - s||^2 (rounded up)
  float tau;     // tie_rel * (1 + 1e-4)
  float pad0, pad1;
};

struct GemmArgs {
  const void* xb;        // [ceil(N/128)*128][64] BF16 (or scaled FP16) rows of fl(x - s), 128-byte swizzled
  const float* xa;       // [N] ||fl(x - s)||^2, rounded up
  const float* xaos;     // [N][64] FP32 points
  const void* cb;        // [kpad][64] BF16 rows of fl(mu - s), 128-byte swizzled
  const float* nprime;   // [kpad] n'_k = fl(M + 2^sigma ||mu_k - s||^2)
  const float* ctil;     // [k][64] fl32(mu - s)
  const double* mu;      // [k][64]
  const float* shift;    // [64]
  const GemmConst* gc;
  LoopState* ls;
  int32_t* labels;       // out: labels
  int32_t* rescue_list;  // [N] points resolved over all K by the rescue kernel
  int4* tie_list;        // [gemm_tie_entries][3] near ties: point, count (0: unused), up to 20 16-bit candidates
  unsigned* rescue_count;  // [0] rescue entries, [1] near-tie entries
  unsigned* tie_count;     // = rescue_count + 1
  int64_t n;
  int k, kpad, ntiles;
  int f16;               // operands are FP16 (scaled by powers of two), else BF16
};

struct GemmPrepArgs {
  const double* mu; const float* shift; int k, kpad;
  void* cb; float* nprime; float* ctil; GemmConst* gc;
  double* bnorm;                   // [kpad] ||mu_k - s||^2
  float A_max; double tie_rel;
  int f16;                         // FP16 operands: cb written by the consts kernel, scaled by 2^ec
  int ex;                          // FP16: the points were scaled by 2^ex
  const LoopState* ls;
};

struct MsortArgs {
  const int32_t* labels; int64_t n; int k; int d;
  const float* xa;                 // [N][d] FP32 points
  const DataConst* dc;
  unsigned long long* counts_u;    // [k]
  int64_t* offsets;                // [k]
  int* cfirst;                     // [k] first chunk of each cluster
  unsigned long long* cursor;      // [k]
  int4* chunks; int* nchunks; int max_chunks;
  long long* chunk_sums;           // [max_chunks][d]
  int32_t* perm;                   // [N]
  double* df2;                     // [k][d] squared centroid moves
  double* mu; long long* counts;   // out
  LoopState* ls;
};

cudaError_t launch_gemm_assign(int grid, cudaStream_t st, const GemmArgs& a);
cudaError_t launch_gemm_prep_points(const float* x, int64_t ld, int64_t n, const float* shift, void* xb, float* xa,
                                    float* xaos, int f16, int ex, cudaStream_t st);
cudaError_t launch_gemm_prepare(cudaStream_t st, const GemmPrepArgs& a);
cudaError_t launch_wait_selftest(int* out, cudaStream_t st);
// Allocation-failure injection (testing): true when this device allocation
// is to fail as if the device were out of memory.
bool inject_alloc_failure();
size_t gemm_smem_bytes(int kpad);
int64_t gemm_xb_rows(int64_t n);
// fused step with the tcgen05 TF32 screen (d <= 3, K <= 32; the screen tables built for kpad = 32)
size_t tcs_smem_bytes();
int tcs_grid(int64_t n, int sms);
cudaError_t launch_assign_tcs(int d, int grid, cudaStream_t st, const FastArgs& a);
int64_t gemm_tie_entries(int64_t n, int grid);  // near-tie list capacity (entries of 3 int4)
int64_t msort_max_chunks(int64_t n, int k);
cudaError_t launch_msort_step(const MsortArgs& a, cudaStream_t st);
// sharded steps on the tensor-core path: the context's int128 column totals
// ([k][d+1] of low, high word), and the update from the ranks' tables
cudaError_t launch_msort_shard_totals(const MsortArgs& a, long long* out, cudaStream_t st);
cudaError_t launch_msort_shard_update(const MsortArgs& a, const long long* tables, int ranks, cudaStream_t st);

// ---- batched instances (d <= 3, K <= 64) ----
constexpr int kBatchMaxK = 64;
constexpr int kBatchMaxD = 3;
constexpr int kBatchMaxTile = 1024;  // points per tile: keeps every limb sum in int32
constexpr int kBatchMaxThreads = 512;  // assign block size limit (per-warp windows in shared memory)

struct BatchInst {        // per instance, written at set_points (scan kernel) and create
  int64_t n, x_off, lab_off;       // points; element offset of row 0 (rows of n); label offset
  int32_t d, k, mu_off, k_off;     // mu/ctil offset (K*d), counts offset (K)
  int32_t tile0, ntiles;           // the instance's tiles (contiguous in the tile list)
  int32_t kpad, tab_off;           // fused-kernel screen table: kpad = K rounded up to 8, offset in tab2
  float s[3];                      // shift (FP32 midrange)
  float A_max;                     // max fl32 ||x - s||^2
  int32_t G0;                      // fixed-point grid exponent
  float C_hi, C_lo;
  uint32_t bits_C_hi, bits_C_lo;
};

struct BatchState {       // per instance, advanced on the device
  int32_t done, iter, converged, empty;
  int32_t max_iter, pad;
  double E, E2;
  float B_max, pad2;
};

struct BatchArgs {
  const float* x;
  const BatchInst* inst;
  BatchState* state;
  const int4* tiles;              // {instance, first point, points, 0}
  const int64_t* tile_poff;       // partial row offset of each tile (K_i (d_i + 1) entries)
  int ntiles;
  long long* partials;
  int32_t* labels;
  double* mu;
  float* ctil;
  long long* counts;
  unsigned long long* flagged;
  unsigned long long* fp64;
  int* active;                    // instances not yet stopped
  float tau;
  int e_mode;
  double tol;
  // the fused kernel's per-instance screen tables (written by the update)
  unsigned long long* tab2;       // [sum kpad_i (d_i + 1)] packed pairs
  float4* ctil4;                  // [sum K_i] fl32(mu - s)
  IterConst* ic;                  // [count] screen constants
  double tie_rel;
};

cudaError_t launch_batch_scan(const float* x, BatchInst* inst, int count, unsigned long long* bad, cudaStream_t st);
cudaError_t launch_batch_tables(const BatchArgs& a, int count, cudaStream_t st);
cudaError_t launch_batch_assign(const BatchArgs& a, int grid, int threads, cudaStream_t st);
// The batch through the fused kernel's tile machinery (256 threads per block;
// tiles of a multiple of 256 points).
cudaError_t launch_batch_fast(const BatchArgs& a, int grid, cudaStream_t st);
int batch_fast_blocks_per_sm();
cudaError_t launch_batch_update(const BatchArgs& a, int count, cudaStream_t st);
int batch_blocks_per_sm(int threads);
cudaError_t launch_batch_objective(const float* x, const BatchInst* inst, const int32_t* labels, const double* mu,
                                   double* out, int count, cudaStream_t st);

// ---- k-means++ seeding ----
constexpr int kMaxKppD = 256;
int64_t kpp_chunks(int64_t n);
cudaError_t launch_kmeanspp(const float* x, int64_t ld, int64_t n, int d, int k, const double* u, double* mu,
                            int64_t* idx, double* d2, double* chunk_sum, double* scan, cudaStream_t st);

// ---- learned initialiser: set network (d <= 3, K <= 64, H = 128) ----
constexpr int kSetH = 128;
struct SetNetArgs {
  const float* x;     // [B][S][d] points
  const float* t;     // [B][K][d] targets (training)
  int B, S, d, k;
  const float* prm;   // flat parameters
  float* grads;
  float* xs; float* ts; float* ms;   // standardised points, targets; [B][2d] mean, std
  float* w2t; float* h1; float* h2; float* tile_pool; float* G; float* P; float* dG; float* loss;
  float* dz2; float* dz1; float* part;
};
int setnet_param_count(int d, int k);
size_t setnet_point_smem();
int64_t setnet_part_floats(int64_t P, int d);
cudaError_t launch_setnet_forward(const SetNetArgs& a, bool train, cudaStream_t st);
cudaError_t launch_setnet_backward(const SetNetArgs& a, cudaStream_t st);
cudaError_t launch_setnet_adam(float* prm, const float* grads, float* m, float* v, int n, float lr, float b1,
                               float b2, float eps, float c1, float c2, cudaStream_t st);
cudaError_t launch_setnet_sample(const float* x, int64_t ld, int64_t n, int d, int S, unsigned long long seed,
                                 float* out, cudaStream_t st);
// Set transforms of the learned initialiser: per-set FP64 means, and
// out = R (x - c) + c per set (R^T with transpose), in FP64.
cudaError_t launch_sets_mean(const float* x, int64_t set_stride, int B, int S, int d, double* means, cudaStream_t st);
template <typename T>
cudaError_t launch_sets_rotate(const T* x, int64_t set_stride, int B, int S, int d, const double* R,
                               const double* c, int64_t center_stride, int transpose, T* out, cudaStream_t st);
cudaError_t launch_setnet_destandardize(const float* P, const float* ms, int B, int d, int k, double* out,
                                        cudaStream_t st);

// ---- objective ----
int64_t objective_chunks(int64_t n);
cudaError_t launch_widen_labels(const uint8_t* z8, int32_t* z, int64_t n, cudaStream_t st);
cudaError_t launch_objective(const float* x, int64_t ld, int64_t n, int d, const double* mu, const int32_t* z,
                             const uint8_t* z8, double* part, double* out, cudaStream_t st);

// Host-side launchers (defined in the .cu files).
cudaError_t launch_assign_fast(int d, int grid, size_t smem, cudaStream_t st, const FastArgs& a);
size_t fast_smem_bytes(int d, int kpad, int k, int nwin);
int fast_blocks_per_sm(int d, size_t smem, int kpad, bool ct);
// The fused kernel has a constant-bank screen table for this shape.
bool fast_has_const_table(int d, int kpad);
cudaError_t launch_assign_generic(int grid, size_t smem, cudaStream_t st, const GenericArgs& a);
size_t generic_smem_bytes(int d, int k);

struct UpdateArgs {
  const long long* partials; int G; int k; int d;
  long long* s128;                 // [RB][k][d+1][2] per-row-block int128 partial sums
  int RB;
  double* mu;                      // [k][d] in/out
  long long* counts;               // [k]
  const DataConst* dc;
  IterConst* ic;
  LoopState* ls;
  unsigned long long* tab2;        // out: next step's screen table [kpad][d+1]
  float4* ctil4;                   // out (d <= 4)
  float* ctil;                     // out (generic) [k][d]
  float* cnorm;                    // out (generic) [k]
  const float* shift;              // [d] generic shift
  int kpad;
  int fast;                        // 1: fused kernel tables
  double tie_rel;
  float A_max;
  float* gen_bmax;                 // out (generic)
};
cudaError_t launch_update(cudaStream_t st, const UpdateArgs& a);
cudaError_t launch_prepare(cudaStream_t st, const UpdateArgs& a);  // tables from mu, no step
// Sharded steps: this context's int128 column totals ([k][d+1][2] int64), and
// the update from the totals of R shards gathered in rank order.
cudaError_t launch_shard_totals(cudaStream_t st, const UpdateArgs& a, long long* out);
cudaError_t launch_shard_update(cudaStream_t st, const UpdateArgs& a, const long long* tables, int ranks);

// Data scan: per-coordinate min/max, absmax, non-finite count.
cudaError_t launch_scan_range(const float* x, int64_t ld, int64_t n, int d, float* mn, float* mx,
                              unsigned long long* nonfinite, cudaStream_t st);
cudaError_t launch_scan_amax(const float* x, int64_t ld, int64_t n, int d, const float* shift,
                             float* amax, cudaStream_t st);
cudaError_t launch_aos_to_soa(const float* src, int64_t lds, int64_t n, int d, float* dst,
                              int64_t ldd, cudaStream_t st);

}  // namespace km
