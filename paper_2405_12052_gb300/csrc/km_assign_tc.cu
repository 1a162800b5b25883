// Reassignment + per-block accumulation with the screen's dot products on the
// tensor cores: the expectation step and the first half of the mean
// calculation of Lloyd's algorithm (paper, section "The Lloyd's algorithm",
// steps 2 and 3) for d <= 3 and K <= 32, fused in one pass over the points.
//
// The screen values are those of the FFMA2 kernel, r_k = n_k + sum_j x~_j a_kj
// (n_k = fl32(M + 2^sigma ||c~_k||^2), a_kj = -2^(sigma+1) c~_kj, one binade
// [2^eM, 2^(eM+1))), formed by tcgen05.mma kind::tf32 with every operand
// split into TF32 pieces (x~ = xh + xl exactly, a = ah + al + tiny, n = nh +
// nm + nl exactly):
//   A row (per point)      [xh_0..2, xl_0..2, 1, 1]
//   B row 1 (per centroid) [ah_0..2, ah_0..2, nh, nm]  -> xh.ah + xl.ah + nh + nm
//   B row 2 (per centroid) [al_0..2,  0 0 0,  nl, 0]   -> xh.al + nl
// two K = 8 MMAs into one FP32 accumulator of 32 columns per 128-point tile.
// The products the tensor core forms are exact (11 x 11 significand bits).
// The error against the FP32-chain screen value is bounded by
//   16 * 2^-23 * (sum of the terms' magnitudes)      accumulation, any order,
//                                                    truncation allowed
//   + 3 * 2^-20 * sum_j |x~_j a_kj|                  a's tail cut, xl cut to
//                                                    TF32 by the hardware,
//                                                    xl.al omitted
// with sum_j |x~_j a_kj| <= 2^sigma (||x~||^2 + B_max) and |n| < 2^(eM+1):
// 32 ulps of the binade plus 40.2 2^-23 G (A + B_max) ulps, added to the flag
// threshold (constant part and per unit of A = ||x~||^2).  Everything after
// the screen -- group minima packed with the group index, running top-2,
// exact FP32-chain recompute of the winning group, flag test in units of the
// binade, per-warp queue and FP32 / FP64 re-check, exact integer sums -- is
// the FFMA2 kernel's.
//
// CTA: 16 warps in 4 quads; a quad (warps 4q .. 4q+3, TMEM lane quarters
// 0..3) owns 256-point super-tiles (two MMA tiles of 128 points), two stages
// deep: it writes the A rows of super-tile m, one thread issues its MMAs and
// commits them to an mbarrier, and the quad then runs the epilogue of
// super-tile m - 1 while the tensor core works.  Quads never wait for one
// another; every mbarrier wait is bounded.
#include "km_internal.cuh"
#include "km_fast_common.cuh"
#include "km_tcgen05.cuh"

namespace km {

namespace {

constexpr int kTcsWarps = 16;
constexpr int kTcsThreads = kTcsWarps * 32;
constexpr int kTcsK = 32;                  // MMA N = columns per tile (kpad)
constexpr int kTcsQueue = 256;             // flagged points per warp (drained above kTcsQueue - 64)
constexpr int kTcsWin = (kTcsK + 1) * 7;   // 32-bit window words per warp (D <= 3)
// shared-memory layout (bytes from the 1024-aligned base)
constexpr int kTcsOffA = 0;                                   // [4 quads][128 rows][128 B], 128-byte swizzle
constexpr int kTcsOffB = kTcsOffA + 4 * 128 * 128;            // [32 rows][128 B]
constexpr int kTcsOffG = kTcsOffB + kTcsK * 128;              // [8 groups][5] float4 group table
constexpr int kTcsOffC = kTcsOffG + 8 * 5 * 16;               // [32] float4 re-check centroids
constexpr int kTcsOffAcc = kTcsOffC + kTcsK * 16;             // [32][4] int64 block totals
constexpr int kTcsOffWin = kTcsOffAcc + kTcsK * 4 * 8;        // [16][kTcsWin] u32 windows
constexpr int kTcsOffQ = kTcsOffWin + kTcsWarps * kTcsWin * 4;  // [16][kTcsQueue] u32 queues
constexpr int kTcsOffBar = kTcsOffQ + kTcsWarps * kTcsQueue * 4;  // [4][2] mbarriers
constexpr int kTcsOffMisc = kTcsOffBar + 8 * 8;               // TMEM base, counters
constexpr int kTcsSmem = kTcsOffMisc + 16 + 1024;             // + alignment slack

// D(128 x 32, f32) (+)= A(128 x 8, TF32, K-major) x B(32 x 8, TF32, K-major)^T:
// D type F32 (bit 4), A and B type TF32 (2 at bits 7 and 10), N >> 3 at bit
// 17, M >> 4 at bit 24.
constexpr uint32_t kIdescTf32 = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(kTcsK >> 3) << 17) |
                                ((uint32_t)(128 >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t acc) {
  asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
               ::"r"(tmem), "l"(ad), "l"(bd), "r"(kIdescTf32), "r"(acc));
}
// Barrier of one quad (named barrier 1 + q, 128 threads) that also ORs a flag.
__device__ __forceinline__ bool quad_sync_or(int q, bool v) {
  uint32_t r;
  asm volatile("{\n.reg .pred p, t;\nsetp.ne.u32 p, %1, 0;\nbar.red.or.pred t, %2, 128, p;\nselp.u32 %0, 1, 0, t;\n}"
               : "=r"(r) : "r"((uint32_t)v), "r"(1 + q) : "memory");
  return r != 0;
}
// Byte offset of 32-bit element e of row r in a 128-byte-swizzled K-major
// tile (16-byte chunk e / 4 of row r sits at chunk (e / 4) ^ (r % 8)).
__device__ __forceinline__ uint32_t swz32(int r, int e) {
  return (uint32_t)(r * 128 + ((((e >> 2) ^ (r & 7)) & 7) << 4) + ((e & 3) << 2));
}
// TF32 head of an FP32 value (the 13 low significand bits cleared) -- an
// exact TF32 number, so the tensor core sees it unchanged.
__device__ __forceinline__ float tf32_head(float v) { return __uint_as_float(__float_as_uint(v) & 0xFFFFE000u); }


template <int D>
__global__ void __launch_bounds__(kTcsThreads, 1) assign_tcs_kernel(FastArgs a) {
  constexpr int DP = D + 1, WIN = 2 * D + 1, GS = (DP & 1) ? DP : DP + 1;
  static_assert(D >= 1 && D <= 3 && WIN * (kTcsK + 1) <= kTcsWin, "d <= 3");
  constexpr int LB = 5;  // index bits of the packed screen values (kpad = 32)
  extern __shared__ __align__(16) unsigned char raw[];
  if (a.ls->done && !a.ignore_done) return;
  unsigned char* sm = raw + ((1024u - ((uint32_t)__cvta_generic_to_shared(raw) & 1023u)) & 1023u);
  unsigned char* sA = sm + kTcsOffA;
  unsigned char* sB = sm + kTcsOffB;
  float4* gtab = reinterpret_cast<float4*>(sm + kTcsOffG);
  float4* sctil = reinterpret_cast<float4*>(sm + kTcsOffC);
  long long* acc = reinterpret_cast<long long*>(sm + kTcsOffAcc);
  uint32_t* win = reinterpret_cast<uint32_t*>(sm + kTcsOffWin);
  uint32_t* queue = reinterpret_cast<uint32_t*>(sm + kTcsOffQ);
  unsigned long long* s_bar = reinterpret_cast<unsigned long long*>(sm + kTcsOffBar);
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(sm + kTcsOffMisc);
  int* s_cnt = reinterpret_cast<int*>(sm + kTcsOffMisc + 4);  // [2]: flagged, fp64-decided
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, q = warp >> 2, wq = warp & 3;
  const int k = a.k;
  auto bar_addr = [&](int st) { return (uint32_t)__cvta_generic_to_shared(&s_bar[q * 2 + st]); };

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(s_tmem)), "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid < 8) bar_init((uint32_t)__cvta_generic_to_shared(&s_bar[tid]), 1);
  if (tid == 0) { s_cnt[0] = 0; s_cnt[1] = 0; }
  // B rows (TF32 head / tail of the screen coefficients) and the group table
  // of the FP32 recompute, from the packed screen table (kpad = 32 rows)
  for (int c = tid; c < kTcsK; c += kTcsThreads) {
    float av[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int j = 0; j < D; ++j) av[j] = __uint_as_float((uint32_t)a.tab2[c * DP + j]);
    const float nv = __uint_as_float((uint32_t)a.tab2[c * DP + D]);
    float ah[3], al[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      ah[j] = tf32_head(av[j]);
      al[j] = tf32_head(__fsub_rn(av[j], ah[j]));
    }
    const float nh = tf32_head(nv), nr = __fsub_rn(nv, nh), nm = tf32_head(nr), nl = __fsub_rn(nr, nm);  // exact
    const float r1[8] = {ah[0], ah[1], ah[2], ah[0], ah[1], ah[2], nh, nm};
    const float r2[8] = {al[0], al[1], al[2], 0.f, 0.f, 0.f, nl, 0.f};
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      *reinterpret_cast<float*>(sB + swz32(c, e)) = r1[e];
      *reinterpret_cast<float*>(sB + swz32(c, 8 + e)) = r2[e];
    }
#pragma unroll
    for (int j = 0; j <= D; ++j) reinterpret_cast<float*>(gtab + (c >> 2) * GS + j)[c & 3] = j < D ? av[j] : nv;
  }
  for (int c = tid; c < k; c += kTcsThreads) sctil[c] = a.ctil[c];
  for (int i = tid; i < k * DP; i += kTcsThreads) acc[i] = 0;
  for (int i = tid; i < kTcsWarps * kTcsWin; i += kTcsThreads) win[i] = 0u;
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // B rows -> the tensor core's view
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *s_tmem;

  const IterConst ic = *a.ic;
  const DataConst dc = *a.dc;
  float s[D];
#pragma unroll
  for (int j = 0; j < D; ++j) s[j] = dc.s[j];
  const uint32_t ehi = __float_as_uint(ic.M) >> (32 - LB);
  const float M = ic.M, tau = ic.tau;
  float c0, cA;
  {
    // flag threshold in units of r: the FFMA2 kernel's, plus the tensor
    // core's error bound (see the top of this file) in ulps of the binade
    const float ulp = __uint_as_float(__float_as_uint(ic.M) & 0x7f800000u) * 0x1p-23f;
    const float etcA = 40.25f * 0x1p-23f * ic.G, etc0 = 32.5f + etcA * ic.B_max;
    c0 = (ic.thr_c0 + etc0) * ulp;
    cA = (ic.thr_cA + ic.tau * ic.G + etcA) * ulp;
  }
  const int64_t n = a.n;
  const int64_t U = (n + 255) >> 8;  // 256-point super-tiles
  const int64_t qstride = (int64_t)gridDim.x * 4;
  uint32_t* wmine = win + warp * kTcsWin;
  uint32_t* qw = queue + warp * kTcsQueue;
  int qn = 0, nflag = 0, n64 = 0, since_flush = 0;
  bool aborted = false;
  const int row = wq * 32 + lane;  // this lane's row (TMEM lane) in each 128-point tile
  unsigned char* aq = sA + q * (128 * 128);
  const uint32_t aq_addr = (uint32_t)__cvta_generic_to_shared(aq), b_addr = (uint32_t)__cvta_generic_to_shared(sB);
  auto col = [&](int st, int h) { return (uint32_t)(((q * 2 + st) * 2 + h) * kTcsK); };
  auto load_x = [&](int64_t u, float (&xv)[2][D]) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int64_t i = u * 256 + h * 128 + row;
#pragma unroll
      for (int j = 0; j < D; ++j) xv[h][j] = (u < U && i < n) ? __ldg(a.x + (int64_t)j * a.ld + i) : 0.f;
    }
  };
  // Re-decide the warp's queued points (FP32 direct form, then FP64 when
  // open) and add them to the window; the window is flushed every 16 rounds
  // (32 lanes x 16 <= 512 additions per bin).
  auto drain = [&]() {
    flush_windows<D>(wmine, acc, k, 1, lane, dc.bits_C_hi, dc.bits_C_lo);
    for (int r = 0, b = 0; b < qn; ++r, b += 32) {
      const int e = b + lane;
      if (e < qn) {
        const int64_t i = qw[e];
        float xo[D];
#pragma unroll
        for (int j = 0; j < D; ++j) xo[j] = a.x[(int64_t)j * a.ld + i];
        bool used64;
        const int kk = recheck_fast<D>(xo, s, sctil, a.mu, k, ic.B_max, ic.tau, used64);
        n64 += used64 ? 1 : 0;
        if (a.store_labels) {
          if (a.labels8) a.labels8[i] = (uint8_t)kk;
          else a.labels[i] = kk;
        }
        accumulate_point<D>(wmine, kk, xo, dc.C_hi, dc.C_lo);
      }
      if ((r & 15) == 15) flush_windows<D>(wmine, acc, k, 1, lane, dc.bits_C_hi, dc.bits_C_lo);
    }
    flush_windows<D>(wmine, acc, k, 1, lane, dc.bits_C_hi, dc.bits_C_lo);
    nflag += qn;
    qn = 0;
    since_flush = 0;
  };
  // Epilogue of the quad's local super-tile me (points of super-tile ue, x
  // values xe): wait for its MMAs, screen the 32 values of each of the lane's
  // two points, recompute the winning group exactly, flag, label, sums.
  auto epilogue = [&](int me, int64_t ue, const float (&xe)[2][D]) {
    const int st = me & 1;
    bool ok = wait_bar(bar_addr(st), (uint32_t)(me >> 1) & 1u);
    ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld below needs the whole warp
    if (!ok) {
      aborted = true;
      a.ls->error = 3;
      return;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    float m1[2], m2[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      unsigned long long u[16];
      tmem_ld32(tmem + ((uint32_t)(wq * 32) << 16) + col(st, h), u);
      float g[8];
#pragma unroll
      for (int gi = 0; gi < 8; ++gi) {
        float v0, v1, v2, v3;
        unpack2(u[2 * gi], v0, v1);
        unpack2(u[2 * gi + 1], v2, v3);
        g[gi] = __uint_as_float((__float_as_uint(fminf(fmin3(v0, v1, v2), v3)) << LB) + 4u * gi);
      }
      float lo = fminf(g[0], g[1]);
      m1[h] = lo;
      m2[h] = fmaxf(g[0], g[1]);
#pragma unroll
      for (int gp = 1; gp < 4; ++gp) {
        lo = fminf(g[2 * gp], g[2 * gp + 1]);
        const float hi = fmaxf(g[2 * gp], g[2 * gp + 1]);
        m2[h] = fmin3(m2[h], hi, fmaxf(m1[h], lo));
        m1[h] = fminf(m1[h], lo);
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");  // the accumulators may be rewritten
    const int64_t ib = ue * 256 + row;
    const bool full = ue * 256 + 256 <= n;
    int lab[2];
    bool flg[2], disc[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float xt[D];
#pragma unroll
      for (int j = 0; j < D; ++j) xt[j] = __fsub_rn(xe[h][j], s[j]);
      // A = ||x~||^2 exactly as the data scan that bounds it: x0*x0, then FMAs
      float A = __fmul_rn(xt[0], xt[0]);
#pragma unroll
      for (int j = 1; j < D; ++j) A = __fmaf_rn(xt[j], xt[j], A);
      const uint32_t gsel = __float_as_uint(m1[h]) & 31u;  // the winning group's first index
      const ulonglong2* gt = reinterpret_cast<const ulonglong2*>(gtab + (gsel >> 2) * GS);
      const ulonglong2 nv = gt[D];
      unsigned long long rA = nv.x, rB = nv.y;
#pragma unroll
      for (int j = 0; j < D; ++j) {
        const unsigned long long xx = dup2(xt[j]);
        const ulonglong2 cv = gt[j];
        rA = ffma2(xx, cv.x, rA);
        rB = ffma2(xx, cv.y, rB);
      }
      float r0, r1, r2, r3;
      unpack2(rA, r0, r1);
      unpack2(rB, r2, r3);
      const float w0 = __uint_as_float(__float_as_uint(r0) << LB), w1 = __uint_as_float((__float_as_uint(r1) << LB) + 1u);
      const float w2 = __uint_as_float((__float_as_uint(r2) << LB) + 2u), w3 = __uint_as_float((__float_as_uint(r3) << LB) + 3u);
      const float lo01 = fminf(w0, w1), hi01 = fmaxf(w0, w1), lo23 = fminf(w2, w3), hi23 = fmaxf(w2, w3);
      const float best = fminf(lo01, lo23);
      const float sec = fmin3(fmaxf(lo01, lo23), fminf(hi01, hi23), m2[h]);
      lab[h] = (int)(gsel | (__float_as_uint(best) & 3u));
      const float v1 = __uint_as_float(__funnelshift_r(__float_as_uint(best), ehi, LB));
      const float v2 = __uint_as_float(__funnelshift_r(__float_as_uint(sec), ehi, LB));
      const float T = fmaf(tau, v2 - M, fmaf(A, cA, c0));
      bool f = !(v2 - v1 > T);
      if (k < kTcsK) f = f || lab[h] >= k;  // a padding column never decides a label
      const int64_t i = ib + h * 128;
      const bool valid = full || i < n;
      flg[h] = f && valid;
      disc[h] = f || !valid;
      if (valid && a.store_labels) {
        if (a.labels8) a.labels8[i] = (uint8_t)lab[h];
        else a.labels[i] = lab[h];
      }
    }
    // flagged points to the warp's queue (their labels are rewritten by the re-check)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const unsigned bq = __ballot_sync(0xffffffffu, flg[h]);
      if (flg[h]) qw[qn + __popc(bq & ((1u << lane) - 1u))] = (uint32_t)(ib + h * 128);
      qn += __popc(bq);
    }
    // exact sums; flagged and padding points go to the discard bin k
#pragma unroll
    for (int h = 0; h < 2; ++h) accumulate_point<D>(wmine, disc[h] ? k : lab[h], xe[h], dc.C_hi, dc.C_lo);
    if (++since_flush == 8) {  // 32 lanes x 2 points x 8 <= 512 additions per bin
      flush_windows<D>(wmine, acc, k, 1, lane, dc.bits_C_hi, dc.bits_C_lo);
      since_flush = 0;
    }
    if (qn > kTcsQueue - 64) {
      __syncwarp();
      drain();
    }
  };

  // Main loop: A rows of super-tile m, its MMAs, then the epilogue of m - 1
  // (the points of m + 1 are loaded into registers meanwhile).
  float xn[2][D], xc[2][D], xp[2][D];
  int64_t u = (int64_t)blockIdx.x * 4 + q, up = -1;
  int m = 0;
  load_x(u, xn);
  for (; u < U; u += qstride, ++m) {
    const int st = m & 1;
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int j = 0; j < D; ++j) xc[h][j] = xn[h][j];
    load_x(u + qstride, xn);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float hd[3] = {0.f, 0.f, 0.f}, tl[3] = {0.f, 0.f, 0.f};
#pragma unroll
      for (int j = 0; j < D; ++j) {
        const float xt = __fsub_rn(xc[h][j], s[j]);
        hd[j] = tf32_head(xt);
        tl[j] = __fsub_rn(xt, hd[j]);  // exact
      }
      const int e0 = (2 * st + h) * 8;  // this tile's K-slice of the row
      *reinterpret_cast<float4*>(aq + swz32(row, e0)) = make_float4(hd[0], hd[1], hd[2], tl[0]);
      *reinterpret_cast<float4*>(aq + swz32(row, e0 + 4)) = make_float4(tl[1], tl[2], 1.f, 1.f);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // A rows -> the tensor core's view
    aborted = quad_sync_or(q, aborted);
    if (aborted) break;
    if (wq == 0 && lane == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const uint64_t ad = sm_desc(aq_addr + (uint32_t)((2 * st + h) * 32));
        mma_tf32(tmem + col(st, h), ad, sm_desc(b_addr), 0u);
        mma_tf32(tmem + col(st, h), ad, sm_desc(b_addr + 32), 1u);
      }
      mma_commit(bar_addr(st));
    }
    __syncwarp();
    if (m > 0) epilogue(m - 1, up, xp);
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int j = 0; j < D; ++j) xp[h][j] = xc[h][j];
    up = u;
  }
  if (m > 0) {
    if (!aborted) {
      epilogue(m - 1, up, xp);
    } else {
      // the last MMAs issued may still run: wait (bounded) before TMEM is released
      wait_bar(bar_addr((m - 1) & 1), (uint32_t)((m - 1) >> 1) & 1u);
    }
  }
  __syncwarp();
  if (qn > 0) drain();
  else flush_windows<D>(wmine, acc, k, 1, lane, dc.bits_C_hi, dc.bits_C_lo);
  if (lane == 0 && nflag) atomicAdd(&s_cnt[0], nflag);
  if (n64) atomicAdd(&s_cnt[1], n64);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  long long* out = a.partials + (size_t)blockIdx.x * k * DP;
  for (int i = tid; i < k * DP; i += kTcsThreads) out[i] = acc[i];
  if (tid == 0) {
    if (s_cnt[0]) atomicAdd(&a.ls->flagged, (unsigned long long)s_cnt[0]);
    if (s_cnt[1]) atomicAdd(&a.ls->fp64_decided, (unsigned long long)s_cnt[1]);
  }
}
}  // namespace

size_t tcs_smem_bytes() { return (size_t)kTcsSmem; }

int tcs_grid(int64_t n, int sms) {
  const int64_t quads = ((n + 255) >> 8);
  return (int)std::max<int64_t>(1, std::min<int64_t>((quads + 3) / 4, sms));
}

cudaError_t launch_assign_tcs(int d, int grid, cudaStream_t st, const FastArgs& a) {
  const size_t smem = tcs_smem_bytes();
  cudaError_t e;
  switch (d) {
    case 1:
      e = cudaFuncSetAttribute(assign_tcs_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess) assign_tcs_kernel<1><<<grid, kTcsThreads, smem, st>>>(a);
      break;
    case 2:
      e = cudaFuncSetAttribute(assign_tcs_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess) assign_tcs_kernel<2><<<grid, kTcsThreads, smem, st>>>(a);
      break;
    case 3:
      e = cudaFuncSetAttribute(assign_tcs_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess) assign_tcs_kernel<3><<<grid, kTcsThreads, smem, st>>>(a);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

}  // namespace km
