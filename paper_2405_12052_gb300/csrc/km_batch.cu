// Batched Lloyd iterations: thousands of independent instances of uneven
// N, d (<= 3) and K (<= 64) advanced together (paper, section "The Lloyd's
// algorithm": every instance runs steps 2-3 and the convergence test of its
// own; the batch only shares launches).
//
// Points of all instances are cut into tiles of at most 1024 points listed
// instance-major.  Per step:
//  * batch_assign_kernel (persistent: CTAs stride over the tile list): per
//    tile, the instance's screen table in shared memory; per pair of points
//    the FP32 expanded-form values ||c~||^2 - 2 x~.c~ to all K centres on
//    coordinates shifted by the instance's shift (paired FMA chains, minima
//    of groups of four centres, the winning group evaluated again), the
//    argmin and runner-up, and the rigorous bound that sends an unresolved
//    point to FP64 in the oracle's order (lowest index on ties); then exact
//    fixed-point sums: each coordinate split into
//    two 32-bit limbs added with 32-bit shared atomics (a tile of <= 1024
//    points keeps every limb sum inside int32), written as one int64 partial
//    row per (tile, cluster) plus the count.
//  * batch_update_kernel (one block per instance): the instance's tile
//    partials added in tile order in int128, one conversion, the divide (an
//    empty cluster keeps its centre), E^2 by a fixed-order tree, the stop
//    test, and the FP32 tables of the next step.
// Stopped instances are skipped by both kernels, so a captured run of U
// steps can be replayed until no instance is active.
#include "km_internal.cuh"
#include "km_tables.cuh"

#include <algorithm>

namespace km {

namespace {

constexpr float kBU = 5.9604644775390625e-08f;            // 2^-24
constexpr float kBU64x = 1.1102230246251565e-16f * 4.1f;  // 4.1 * 2^-53

__device__ __forceinline__ double bd64(const float* xo, const double* mu_k, int d) {
  double acc = 0.0;
  for (int j = 0; j < d; ++j) {
    const double t = __dsub_rn((double)xo[j], mu_k[j]);
    acc = __dadd_rn(acc, __dmul_rn(t, t));
  }
  return acc;
}

__device__ __forceinline__ double i128_to_double(unsigned long long lo, long long hs) {
  unsigned long long hi = (unsigned long long)hs;
  const bool neg = hs < 0;
  if (neg) {
    lo = ~lo + 1ull;
    hi = ~hi + (lo == 0ull ? 1ull : 0ull);
  }
  double r;
  if (hi == 0ull) {
    r = __ull2double_rn(lo);
  } else {
    const int sh = 64 - __clzll((long long)hi);
    unsigned long long top = (hi << (64 - sh)) | (lo >> sh);
    if (lo << (64 - sh)) top |= 1ull;  // sticky bit: one rounding in the conversion
    r = ldexp(__ull2double_rn(top), sh);
  }
  return neg ? -r : r;
}

__device__ __forceinline__ unsigned long long bfma2(unsigned long long a, unsigned long long b,
                                                    unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ unsigned long long bpack(float lo, float hi) {
  unsigned long long p;
  asm("mov.b64 %0, {%1, %2};" : "=l"(p) : "f"(lo), "f"(hi));
  return p;
}
__device__ __forceinline__ void bunpack(unsigned long long p, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(p));
}
// running minimum and runner-up with the minimum's index (first index on
// equal values)
__device__ __forceinline__ void btop2(float& b, float& s, int& i, float v, int c) {
  const bool lt = v < b;
  s = lt ? b : fminf(s, v);
  i = lt ? c : i;
  b = lt ? v : b;
}

// The points of one tile (d = D), two per thread per round: screen values
// v_k = n'_k + sum_j x~_j (-2 c~_kj) (= ||c~_k||^2 - 2 x~.c~_k) by one paired
// FMA chain per centroid from the duplicated table w2 ({(-2c~_j, -2c~_j)},
// (n'_k, n'_k)); a point is decided when its two smallest values are apart by
// more than their rigorous error (FMA chains, n'_k's rounding, the rounding
// of x~ and c~, the oracle's FP64 error) plus 1e-5 D; otherwise in FP64 in
// the oracle's order.  Then labels and the fixed-point limb sums.
template <int D>
__device__ __forceinline__ void tile_points(const BatchArgs& a, const BatchInst& bi,
                                            const unsigned long long* __restrict__ w2,
                                            const float* __restrict__ rc, int* s_acc, int start,
                                            int count, float B_max, int& myflag, int& my64) {
  const int k = bi.k;
  constexpr int W = 2 * D + 1;
  const float sB = sqrtf(B_max);
  const int step = blockDim.x;
  // the next round's two points are loaded while this round's are screened
  auto load = [&](int pp, float (&dst)[2][D]) {
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const float* row = a.x + bi.x_off + (int64_t)j * bi.n + start;
      dst[0][j] = row[pp];
      dst[1][j] = pp + step < count ? row[pp + step] : dst[0][j];
    }
  };
  float nxt[2][D];
  if (threadIdx.x < count) load(threadIdx.x, nxt);
  for (int p = threadIdx.x; p < count; p += 2 * step) {
    const bool two = p + step < count;
    float xo[2][D], A[2] = {0.f, 0.f};
#pragma unroll
    for (int j = 0; j < D; ++j) {
      xo[0][j] = nxt[0][j];
      xo[1][j] = nxt[1][j];
    }
    if (p + 2 * step < count) load(p + 2 * step, nxt);
    unsigned long long X[D];
    float tt[2][D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const float t0 = __fsub_rn(xo[0][j], bi.s[j]), t1 = __fsub_rn(xo[1][j], bi.s[j]);
      A[0] = __fmaf_rn(t0, t0, A[0]);
      A[1] = __fmaf_rn(t1, t1, A[1]);
      X[j] = bpack(t0, t1);
      tt[0][j] = t0;
      tt[1][j] = t1;
    }
    // Groups of four centroids (the table is padded to a multiple of four
    // with values of 3e38): only each group's minimum enters the running
    // best / runner-up (with the group's first index)...
    float gb[2] = {3.0e38f, 3.0e38f}, gs[2] = {3.0e38f, 3.0e38f};
    int gi[2] = {0, 0};
    const int k4 = (k + 3) & ~3;
    for (int c = 0; c < k4; c += 4) {
      float v[4][2];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const ulonglong2 wa = *reinterpret_cast<const ulonglong2*>(w2 + 4 * (c + q));
        const ulonglong2 wb = *reinterpret_cast<const ulonglong2*>(w2 + 4 * (c + q) + 2);
        unsigned long long r = bfma2(X[0], wa.x, wb.y);
        if constexpr (D > 1) r = bfma2(X[1], wa.y, r);
        if constexpr (D > 2) r = bfma2(X[2], wb.x, r);
        bunpack(r, v[q][0], v[q][1]);
      }
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        float m;
        asm("min.f32 %0, %1, %2, %3;" : "=f"(m) : "f"(v[0][e]), "f"(v[1][e]), "f"(v[2][e]));
        btop2(gb[e], gs[e], gi[e], fminf(m, v[3][e]), c);
      }
    }
    // ...then the winning group is evaluated again with the same FMA chain
    // for the argmin (first index on equal values) and the group's own
    // runner-up: b = the minimum, sv = the second smallest value over all K.
    float b[2], sv[2];
    int ib[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      float best = 3.0e38f, sec = gs[e];
      int kb = gi[e];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int c = gi[e] + q;
        // the same coefficients, by coefficient (rc[j][c]): threads of a warp
        // read different centroids here, and this layout spreads them over banks
        float r = __fmaf_rn(tt[e][0], rc[c], rc[3 * kBatchMaxK + c]);
        if constexpr (D > 1) r = __fmaf_rn(tt[e][1], rc[kBatchMaxK + c], r);
        if constexpr (D > 2) r = __fmaf_rn(tt[e][2], rc[2 * kBatchMaxK + c], r);
        if (r < best) { sec = fminf(sec, best); best = r; kb = c; }
        else sec = fminf(sec, r);
      }
      b[e] = best;
      sv[e] = sec;
      ib[e] = kb;
    }
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      if (e == 1 && !two) break;
      const int64_t i = (int64_t)start + p + e * step;
      int kb = ib[e];
      if (k > 1) {
        const float Ae = A[e] * 1.0001f, sA = sqrtf(Ae);
        const float ev = 2.03f * (float)(D + 1) * kBU * (B_max + 2.f * sA * sB);  // one value's chain error
        const float thr = 2.f * ev + 4.001f * kBU * (Ae + 2.f * B_max) +
                          2.f * kBU64x * (float)(D + 1) * (Ae + B_max) + a.tau * (sv[e] + Ae + ev) + 1e-30f;
        if (!(sv[e] - b[e] > thr)) {
          ++myflag;
          ++my64;
          const double* mu = a.mu + bi.mu_off;
          double bd = bd64(xo[e], mu, D);
          kb = 0;
          for (int c = 1; c < k; ++c) {
            const double dd = bd64(xo[e], mu + c * D, D);
            if (dd < bd) { bd = dd; kb = c; }
          }
        }
      }
      a.labels[bi.lab_off + i] = kb;
      int* acc = s_acc + kb * W;
      atomicAdd(&acc[0], 1);
#pragma unroll
      for (int j = 0; j < D; ++j) {
        // exact split on the instance's fixed-point grid (unit 2^G0)
        const float tt = __fadd_rn(xo[e][j], bi.C_hi);
        const float h = __fsub_rn(tt, bi.C_hi);
        const float r = __fsub_rn(xo[e][j], h);
        const float t2 = __fadd_rn(r, bi.C_lo);
        atomicAdd(&acc[1 + j], (int)(__float_as_uint(tt) - bi.bits_C_hi));
        atomicAdd(&acc[1 + D + j], (int)(__float_as_uint(t2) - bi.bits_C_lo));
      }
    }
  }
}

__global__ void __launch_bounds__(kBatchMaxThreads) batch_assign_kernel(BatchArgs a) {
  // two sets of the per-tile shared arrays, alternating between the tiles a
  // block takes: a tile's table and sums are rebuilt only two tiles later,
  // after two block barriers, so no barrier is needed between tiles
  __shared__ __align__(16) unsigned long long s_w2b[2][kBatchMaxK * 4];  // duplicated screen table
  __shared__ float s_rcb[2][4 * kBatchMaxK];  // the same coefficients by coefficient: [j][c], n' at j = 3
  __shared__ int s_accb[2][kBatchMaxK * 7];   // per cluster: count, hi limbs, lo limbs
  __shared__ int s_nflag, s_n64;
  const int tid = threadIdx.x;
  int my64 = 0, myflag = 0;
  int par = 0;  // tiles this block has processed, mod 2 (block-uniform)
  for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
    const int4 tl = a.tiles[t];
    const int inst = tl.x;
    if (a.state[inst].done) continue;  // block-uniform
    const BatchInst bi = a.inst[inst];
    const int d = bi.d, k = bi.k, w = 2 * d + 1;
    unsigned long long* s_w2 = s_w2b[par];
    float* s_rc = s_rcb[par];
    int* s_acc = s_accb[par];
    par ^= 1;
    for (int c = tid; c < ((k + 3) & ~3); c += blockDim.x) {
      float n = 3.0e38f, m[3] = {0.f, 0.f, 0.f};  // padding centroids: value 3e38 for every point
      if (c < k) {
        n = 0.f;
        for (int j = 0; j < d; ++j) {
          const float cv = a.ctil[bi.mu_off + c * d + j];
          n = __fmaf_rn(cv, cv, n);
          m[j] = -2.f * cv;  // exact
        }
      }
      s_w2[4 * c + 0] = bpack(m[0], m[0]);
      s_w2[4 * c + 1] = bpack(m[1], m[1]);
      s_w2[4 * c + 2] = bpack(m[2], m[2]);
      s_w2[4 * c + 3] = bpack(n, n);
      s_rc[c] = m[0];
      s_rc[kBatchMaxK + c] = m[1];
      s_rc[2 * kBatchMaxK + c] = m[2];
      s_rc[3 * kBatchMaxK + c] = n;
    }
    for (int q = tid; q < k * w; q += blockDim.x) s_acc[q] = 0;
    __syncthreads();
    const float B_max = a.state[inst].B_max;
    if (d == 3) tile_points<3>(a, bi, s_w2, s_rc, s_acc, tl.y, tl.z, B_max, myflag, my64);
    else if (d == 2) tile_points<2>(a, bi, s_w2, s_rc, s_acc, tl.y, tl.z, B_max, myflag, my64);
    else tile_points<1>(a, bi, s_w2, s_rc, s_acc, tl.y, tl.z, B_max, myflag, my64);
    __syncthreads();
    long long* prow = a.partials + a.tile_poff[t];
    for (int q = tid; q < k * (d + 1); q += blockDim.x) {
      const int c = q / (d + 1), j = q - c * (d + 1);
      const int* acc = s_acc + c * w;
      prow[q] = j == d ? (long long)acc[0] : ((long long)acc[1 + j] << 22) + (long long)acc[1 + d + j];
    }
  }
  if (tid == 0) { s_nflag = 0; s_n64 = 0; }
  __syncthreads();
  if (myflag) atomicAdd(&s_nflag, myflag);
  if (my64) atomicAdd(&s_n64, my64);
  __syncthreads();
  if (tid == 0) {
    if (s_nflag) atomicAdd(a.flagged, (unsigned long long)s_nflag);
    if (s_n64) atomicAdd(a.fp64, (unsigned long long)s_n64);
  }
}

// One block (256 threads) per instance.
__global__ void __launch_bounds__(256) batch_update_kernel(BatchArgs a) {
  __shared__ double s_red[256];
  __shared__ double s_bmax[256];
  __shared__ int s_empty;
  const int inst = blockIdx.x, tid = threadIdx.x;
  BatchState* st = a.state + inst;
  if (st->done) return;
  const BatchInst bi = a.inst[inst];
  const int d = bi.d, k = bi.k, dp = d + 1;
  if (tid == 0) s_empty = 0;
  __syncthreads();
  double* mu = a.mu + bi.mu_off;
  double e2p = 0.0;
  int empty = 0;
  for (int q = tid; q < k * d; q += blockDim.x) {
    const int c = q / d, j = q - c * d;
    unsigned long long lo = 0ull;
    long long hi = 0ll, cnt = 0;
    for (int t = 0; t < bi.ntiles; ++t) {
      const long long* prow = a.partials + a.tile_poff[bi.tile0 + t] + (size_t)c * dp;
      const long long v = prow[j];
      const unsigned long long nl = lo + (unsigned long long)v;
      hi += (v < 0 ? -1ll : 0ll) + (nl < lo ? 1ll : 0ll);
      lo = nl;
      cnt += prow[d];
    }
    const double old = mu[q];
    double nw = old;
    if (cnt > 0) nw = __ddiv_rn(ldexp(i128_to_double(lo, hi), bi.G0), (double)cnt);
    const double df = __dsub_rn(nw, old);
    e2p = __dadd_rn(e2p, __dmul_rn(df, df));
    mu[q] = nw;
    if (j == 0) {
      a.counts[bi.k_off + c] = cnt;
      empty += cnt == 0;
    }
  }
  s_red[tid] = e2p;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (tid < w) s_red[tid] = __dadd_rn(s_red[tid], s_red[tid + w]);
    __syncthreads();
  }
  if (empty) atomicAdd(&s_empty, empty);
  // next step's FP32 table c~ = fl32(mu - s) and max ||mu - s||^2
  double bm = 0.0;
  for (int c = tid; c < k; c += blockDim.x) {
    double B = 0.0;
    for (int j = 0; j < d; ++j) {
      const double t = __dsub_rn(mu[c * d + j], (double)bi.s[j]);
      a.ctil[bi.mu_off + c * d + j] = __double2float_rn(t);
      B = __dadd_rn(B, __dmul_rn(t, t));
    }
    bm = fmax(bm, B);
  }
  s_bmax[tid] = bm;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (tid < w) s_bmax[tid] = fmax(s_bmax[tid], s_bmax[tid + w]);
    __syncthreads();
  }
  // the fused kernel's screen tables of the new centres
  __shared__ double s_fB[kBatchMaxK];
  fast_screen_tables(mu, bi.s, bi.A_max, k, d, bi.kpad, a.tie_rel, a.ctil4 + bi.k_off, a.ic + inst,
                     a.tab2 + bi.tab_off, s_fB);
  if (tid == 0) {
    const double E2 = s_red[0], E = sqrt(E2);
    st->E2 = E2;
    st->E = E;
    st->iter += 1;
    st->empty = s_empty;
    st->B_max = (float)(s_bmax[0] * (1.0 + 1e-6));
    const double esel = a.e_mode == 1 ? E2 : E;
    if (esel < a.tol) st->converged = 1;
    if (st->converged || st->iter >= st->max_iter) {
      st->done = 1;
      atomicSub(a.active, 1);
    }
  }
}

// Tables of the first step from mu0 (one block per instance).
__global__ void __launch_bounds__(256) batch_tables_kernel(BatchArgs a) {
  __shared__ double s_bmax[256];
  const int inst = blockIdx.x, tid = threadIdx.x;
  const BatchInst bi = a.inst[inst];
  const int d = bi.d, k = bi.k;
  double bm = 0.0;
  for (int c = tid; c < k; c += blockDim.x) {
    double B = 0.0;
    for (int j = 0; j < d; ++j) {
      const double t = __dsub_rn(a.mu[bi.mu_off + c * d + j], (double)bi.s[j]);
      a.ctil[bi.mu_off + c * d + j] = __double2float_rn(t);
      B = __dadd_rn(B, __dmul_rn(t, t));
    }
    bm = fmax(bm, B);
  }
  s_bmax[tid] = bm;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (tid < w) s_bmax[tid] = fmax(s_bmax[tid], s_bmax[tid + w]);
    __syncthreads();
  }
  if (tid == 0) a.state[inst].B_max = (float)(s_bmax[0] * (1.0 + 1e-6));
  __shared__ double s_fB[kBatchMaxK];
  fast_screen_tables(a.mu + bi.mu_off, bi.s, bi.A_max, k, d, bi.kpad, a.tie_rel, a.ctil4 + bi.k_off, a.ic + inst,
                     a.tab2 + bi.tab_off, s_fB);
}

// Per instance (one block): coordinate ranges, non-finite values, the shift
// (midrange, FP32), the fixed-point grid and A_max = max fl32 ||x - s||^2.
__global__ void __launch_bounds__(256) batch_scan_kernel(const float* __restrict__ x, BatchInst* inst,
                                                        unsigned long long* bad) {
  __shared__ float s_lo[256 * 3], s_hi[256 * 3];
  __shared__ float s_a[256];
  __shared__ int s_bad;
  BatchInst& bi = inst[blockIdx.x];
  const int tid = threadIdx.x, d = bi.d;
  const int64_t n = bi.n;
  if (tid == 0) s_bad = 0;
  float lo[3] = {3.0e38f, 3.0e38f, 3.0e38f}, hi[3] = {-3.0e38f, -3.0e38f, -3.0e38f};
  int nb = 0;
  for (int j = 0; j < d; ++j)
    for (int64_t i = tid; i < n; i += blockDim.x) {
      const float v = x[bi.x_off + (int64_t)j * n + i];
      if (!isfinite(v)) { ++nb; continue; }
      lo[j] = fminf(lo[j], v);
      hi[j] = fmaxf(hi[j], v);
    }
  for (int j = 0; j < 3; ++j) { s_lo[j * 256 + tid] = lo[j]; s_hi[j * 256 + tid] = hi[j]; }
  __syncthreads();
  if (nb) atomicAdd(&s_bad, nb);
  for (int w = 128; w > 0; w >>= 1) {
    if (tid < w)
      for (int j = 0; j < 3; ++j) {
        s_lo[j * 256 + tid] = fminf(s_lo[j * 256 + tid], s_lo[j * 256 + tid + w]);
        s_hi[j * 256 + tid] = fmaxf(s_hi[j * 256 + tid], s_hi[j * 256 + tid + w]);
      }
    __syncthreads();
  }
  if (tid == 0) {
    if (s_bad) atomicAdd(bad, (unsigned long long)s_bad);
    double amax = 0.0;
    for (int j = 0; j < 3; ++j) {
      if (j < d) {
        const double l = s_lo[j * 256], h = s_hi[j * 256];
        bi.s[j] = (float)(0.5 * (l + h));
        amax = fmax(amax, fmax(fabs(l), fabs(h)));
      } else {
        bi.s[j] = 0.f;
      }
    }
    int ex = amax > 0.0 ? ilogb(amax) + 2 : -104;
    if (amax > 0.0 && ldexp(1.0, ex - 1) <= amax) ++ex;
    ex = max(ex, -104);  // C_lo = 1.5 * 2^(ex - 21) stays a normal float
    bi.G0 = ex - 44;
    bi.C_hi = ldexpf(1.5f, ex + 1);
    bi.C_lo = ldexpf(1.5f, ex - 21);
    bi.bits_C_hi = __float_as_uint(bi.C_hi);
    bi.bits_C_lo = __float_as_uint(bi.C_lo);
    if (ex > 100) atomicAdd(bad, 1ull);  // too large for the fixed-point sums
  }
  __syncthreads();
  float am = 0.f;
  for (int64_t i = tid; i < n; i += blockDim.x) {
    float A = 0.f;
    for (int j = 0; j < d; ++j) {
      const float t = __fsub_rn(x[bi.x_off + (int64_t)j * n + i], bi.s[j]);
      A = __fmaf_rn(t, t, A);
    }
    am = fmaxf(am, A);
  }
  s_a[tid] = am;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (tid < w) s_a[tid] = fmaxf(s_a[tid], s_a[tid + w]);
    __syncthreads();
  }
  if (tid == 0) bi.A_max = s_a[0];
}

}  // namespace

cudaError_t launch_batch_scan(const float* x, BatchInst* inst, int count, unsigned long long* bad, cudaStream_t st) {
  batch_scan_kernel<<<count, 256, 0, st>>>(x, inst, bad);
  return cudaGetLastError();
}

cudaError_t launch_batch_tables(const BatchArgs& a, int count, cudaStream_t st) {
  batch_tables_kernel<<<count, 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_batch_assign(const BatchArgs& a, int grid, int threads, cudaStream_t st) {
  batch_assign_kernel<<<grid, threads, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_batch_update(const BatchArgs& a, int count, cudaStream_t st) {
  batch_update_kernel<<<count, 256, 0, st>>>(a);
  return cudaGetLastError();
}

// Per instance sum_i ||x_i - mu_{z_i}||^2 (current labels and centroids),
// FP64 without fused multiply-add, one block per instance: thread t takes
// points t, t + 256, ..., then a fixed-order tree (deterministic).
__global__ void __launch_bounds__(256) batch_objective_kernel(const float* __restrict__ x,
                                                              const BatchInst* __restrict__ inst,
                                                              const int32_t* __restrict__ labels,
                                                              const double* __restrict__ mu, double* out) {
  __shared__ double s_red[256];
  const BatchInst in = inst[blockIdx.x];
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < in.n; i += blockDim.x) {
    const int z = labels[in.lab_off + i];
    double dd = 0.0;
    for (int j = 0; j < in.d; ++j) {
      const double t = __dsub_rn((double)x[in.x_off + (int64_t)j * in.n + i], mu[in.mu_off + z * in.d + j]);
      dd = __dadd_rn(dd, __dmul_rn(t, t));
    }
    acc = __dadd_rn(acc, dd);
  }
  s_red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) s_red[threadIdx.x] = __dadd_rn(s_red[threadIdx.x], s_red[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = s_red[0];
}

cudaError_t launch_batch_objective(const float* x, const BatchInst* inst, const int32_t* labels, const double* mu,
                                   double* out, int count, cudaStream_t st) {
  batch_objective_kernel<<<count, 256, 0, st>>>(x, inst, labels, mu, out);
  return cudaGetLastError();
}

int batch_blocks_per_sm(int threads) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_assign_kernel, threads, 0) != cudaSuccess) return 1;
  return nb > 0 ? nb : 1;
}

}  // namespace km
