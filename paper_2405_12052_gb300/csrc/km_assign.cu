// Reassignment + per-block accumulation: the expectation step and the first
// half of the mean calculation of Lloyd's algorithm (paper, section "The
// Lloyd's algorithm", steps 2 and 3), fused in one pass over the points.
//
// assign_fast_kernel<D, KG, CT> (d <= 4, K <= 256) is the hot kernel: SoA
// point tiles staged by 16-byte cp.async copies; an FP32 screen on FFMA2
// chains over groups of 4 centroids, the group minima packed with the group
// index and a running top-2 updated two groups at a time; the winning group
// recomputed for the label and the runner-up; a flag test in units of the
// screen's binade; per-warp queues of flagged points re-decided in batches;
// exact integer sums in per-warp (or per-half-warp) shared windows flushed
// into the block's int64 totals.  KG > 0 fixes the number of groups at
// compile time (shift packing, unrolled screen); CT reads the screen table
// from the constant bank instead of shared memory (no vector registers and
// no shared-memory loads for the table; one context per device holds it).
// assign_generic_kernel handles any d and K with a direct-form FP32 screen,
// the same re-check rules and 64-bit atomics into the block's own partial row.
#include "km_internal.cuh"
#include "km_fast_common.cuh"

namespace km {

namespace {

constexpr int kGpUnroll = 1;  // the shared-memory-table screen keeps its group-pair loop rolled

// Shared memory of the fused kernel.  The windows, point buffers and queues
// are private to one warp; the int64 totals are the block's (windows are
// flushed into them with 64-bit shared atomics).  With one window per warp
// (large K) the points are single-buffered, so that two blocks fit on an SM.
template <int D>
struct FastSmem {
  static constexpr int DP = D + 1, WIN = 2 * D + 1;
  static constexpr int GS = (DP & 1) ? DP : DP + 1;  // float4 slots per group (odd: no bank conflicts)
  unsigned long long* tab;  // [kpad][DP] screen table, packed (a, a) pairs (block)
  long long* acc;           // [k][DP] int64 totals (block)
  float4* gtab;             // [kpad/4][GS] screen table by group: slot j = coefficient j of the 4 centroids
  float4* ctil;             // [k] fp32 centroids for the re-check (block; two-window layout only, else global)
  float* xbuf;              // [kWarps][nbuf][D][kWarpTile] points (double-buffered when nbuf = 2)
  uint32_t* queue;          // [kWarps][kWarpQueue] flagged points
  uint32_t* win;            // [kWarps][nwin][k+1][WIN] 32-bit windows (per 8 lanes when nwin = 4, per half-warp when 2); bin k discards
  int* cnt;                 // [2]: flagged, fp64-decided (block totals)
  FastSmem() = default;
  __device__ FastSmem(unsigned char* sm, int kpad, int k, int nwin, int nbuf) {
    tab = reinterpret_cast<unsigned long long*>(sm);
    acc = reinterpret_cast<long long*>(tab + (size_t)kpad * DP);
    gtab = reinterpret_cast<float4*>(acc + (size_t)k * DP + (k * DP & 1));
    ctil = nbuf == 2 ? gtab + (size_t)(kpad / 4) * GS : nullptr;
    xbuf = reinterpret_cast<float*>(gtab + (size_t)(kpad / 4) * GS + (nbuf == 2 ? k : 0));
    queue = reinterpret_cast<uint32_t*>(xbuf + (size_t)kWarps * nbuf * D * kWarpTile);
    win = queue + (size_t)kWarps * kWarpQueue;
    cnt = reinterpret_cast<int*>(win + (size_t)kWarps * nwin * (k + 1) * WIN);
  }
};

// Asynchronous copy of this lane's two 16-byte chunks of each coordinate row
// of warp-tile `base` (points base+4*lane.. and base+128+4*lane..) into a
// warp buffer; chunks past N are zero-filled and read nothing past N.
template <int D>
__device__ __forceinline__ void prefetch_tile(const FastArgs& a, float* xb, int64_t base, int lane) {
  if (base + kWarpTile <= a.n) {  // a full tile: no bounds logic
#pragma unroll
    for (int g = 0; g < kNG; ++g) {
      const int off = g * kGS + 4 * lane;
#pragma unroll
      for (int j = 0; j < D; ++j) {
        const float* src = a.x + (int64_t)j * a.ld + base + off;
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(xb + j * kWarpTile + off);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src));
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
    return;
  }
#pragma unroll
  for (int g = 0; g < kNG; ++g) {
    const int off = g * kGS + 4 * lane;
    const int64_t i0 = base + off;
    const int64_t rem = a.n - i0;
    const int bytes = rem >= 4 ? 16 : (rem > 0 ? (int)rem * 4 : 0);
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const float* src = a.x + (int64_t)j * a.ld + (bytes ? i0 : 0);
      const uint32_t dst = (uint32_t)__cvta_generic_to_shared(xb + j * kWarpTile + off);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes));
    }
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

// Re-decide the points in this warp's queue (warp-level: lanes take
// entries; windows are flushed every 64 rounds with four windows per warp,
// 32 with two, 16 with one: <= 512 additions per bin).
template <int D>
__device__ void drain_warp_queue(const FastArgs& a, FastSmem<D>& sm, uint32_t* q, int qn, int wid,
                                 int wtot, uint32_t* wwarp, uint32_t* wmine, long long* acc, int lane,
                                 const float* s, const DataConst& dc, float B_max, float tau, int& n64) {
  flush_windows<D>(wwarp, acc, a.k, a.nwin, lane, dc.bits_C_hi, dc.bits_C_lo);
  const int rmask = a.nwin == 4 ? 63 : a.nwin == 2 ? 31 : 15;
  for (int r = 0, b = 0; b < qn; ++r, b += 32) {
    const int e = b + lane;
    if (e < qn) {
      const uint32_t loc = q[e];
      const int64_t tile = (int64_t)wid + (int64_t)(loc >> 8) * wtot;
      const int64_t i = tile * kWarpTile + (loc & 255u);
      float xo[D];
#pragma unroll
      for (int j = 0; j < D; ++j) xo[j] = a.x[(int64_t)j * a.ld + i];
      bool used64;
      const int kk = recheck_fast<D>(xo, s, sm.ctil ? sm.ctil : a.ctil, a.mu, a.k, B_max, tau, used64);
      n64 += used64 ? 1 : 0;
      if (a.store_labels) {
        if (a.labels8) a.labels8[i] = (uint8_t)kk;
        else a.labels[i] = kk;
      }
      accumulate_point<D>(wmine, kk, xo, dc.C_hi, dc.C_lo);
    }
    if ((r & rmask) == rmask) flush_windows<D>(wwarp, acc, a.k, a.nwin, lane, dc.bits_C_hi, dc.bits_C_lo);
  }
  flush_windows<D>(wwarp, acc, a.k, a.nwin, lane, dc.bits_C_hi, dc.bits_C_lo);
}

// Per-launch constants of the fused kernel, in registers.  The flag test is
// evaluated in units of r: a point is accepted when
//   r2 - r1 > c0 + A cA + tau (r2 - M),
// r1 <= r2 its two smallest screen values, A = ||x~||^2.  r2 - r1 and r2 - M
// are exact (one binade); c0 and cA are the ulp-unit constants of the update
// kernel times the binade's ulp (a power of two).
struct FastCtx {
  uint32_t mul, L, kmask, ehi;  // ehi: the top L bits shared by every r's bit pattern
  float M, c0, cA, tau;
  unsigned long long chi2, clo2;
  int k, kpad;
};

// bits(v) * 2^L + idx: the screen value with an index in its low L bits.
// With a compile-time L this is a shift and an add (integer ALU pipe).
template <int LB>
__device__ __forceinline__ float pack_idx(float v, const FastCtx& cx, uint32_t idx) {
  if constexpr (LB > 0) return __uint_as_float((__float_as_uint(v) << LB) + idx);
  else return __uint_as_float(imad(__float_as_uint(v), cx.mul, idx));
}
// The screen value r back from a packed value (one funnel shift).
template <int LB>
__device__ __forceinline__ float unpack_val(float w, const FastCtx& cx) {
  return __uint_as_float(__funnelshift_r(__float_as_uint(w), cx.ehi, LB > 0 ? LB : cx.L));
}

// Screen of one group of 4 centroids (table rows tr) for this lane's 8
// points: r = n_k + sum_j x~_j a_kj by one FFMA2 chain per pair of points,
// the group minimum by FMNMX3 + FMNMX, packed with the group's first index.
template <int D, int LB>
__device__ __forceinline__ void screen_group(const unsigned long long* tr, const unsigned long long (&X)[D][kPts / 2],
                                             uint32_t g4, const FastCtx& cx, float (&gm)[kPts]) {
  constexpr int DP = D + 1;
  unsigned long long T[4][DP];
  if constexpr (D <= 3) {
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int j = 0; j < DP; ++j) T[c][j] = tr[c * DP + j];
  }
#pragma unroll
  for (int pp = 0; pp < kPts / 2; ++pp) {
    if constexpr (D > 3) {  // reloaded per pair of points: fewer live registers
#pragma unroll
      for (int c = 0; c < 4; ++c)
#pragma unroll
        for (int j = 0; j < DP; ++j) T[c][j] = tr[c * DP + j];
    }
    float v0[4], v1[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      unsigned long long r = T[c][D];
#pragma unroll
      for (int j = 0; j < D; ++j) r = ffma2(X[j][pp], T[c][j], r);
      unpack2(r, v0[c], v1[c]);
    }
    gm[2 * pp] = pack_idx<LB>(fminf(fmin3(v0[0], v0[1], v0[2]), v0[3]), cx, g4);
    gm[2 * pp + 1] = pack_idx<LB>(fminf(fmin3(v1[0], v1[1], v1[2]), v1[3]), cx, g4);
  }
}

// Screen table in the constant bank (one process-wide copy per device,
// kpad <= 64): the compile-time-unrolled screen reads its coefficients as
// uniform operands, so they take no vector registers and no shared-memory
// loads.  Written by a device-to-device copy before each launch that uses it.
__constant__ union {
  unsigned long long u[kConstTabWords];  // packed (a, a) pairs, as in the global table
  float f[2 * kConstTabWords];           // f[2 i] = the coefficient of pair i
} c_screen_tab;

// Running top-2 over groups, two groups at a time: with lo <= hi the pair's
// packed minima, m1' = min(m1, lo) and m2' = min(m2, hi, max(m1, lo)).
template <bool FIRST>
__device__ __forceinline__ void top2_pair(float (&m1)[kPts], float (&m2)[kPts], const float (&ga)[kPts],
                                          const float (&gb)[kPts]) {
#pragma unroll
  for (int p = 0; p < kPts; ++p) {
    const float lo = fminf(ga[p], gb[p]), hi = fmaxf(ga[p], gb[p]);
    if constexpr (FIRST) {
      m1[p] = lo;
      m2[p] = hi;
    } else {
      m2[p] = fmin3(m2[p], hi, fmaxf(m1[p], lo));
      m1[p] = fminf(m1[p], lo);
    }
  }
}

// Screen of groups G0/4 and G0/4 + 1 (centroids G0 .. G0 + 7) from the
// constant-bank table, one pair of points at a time: 8 FFMA2 chains, the two
// group minima per point, and the running top-2 update.  G0 is a
// compile-time constant after unrolling, so every table operand has a fixed
// offset.
template <int D, int LB, bool FIRST>
__device__ __forceinline__ void screen_pair_ct(int G0, const unsigned long long (&X)[D][kPts / 2], const FastCtx& cx,
                                               float (&m1)[kPts], float (&m2)[kPts]) {
  constexpr int DP = D + 1;
#pragma unroll
  for (int pp = 0; pp < kPts / 2; ++pp) {
    float a0[4], a1[4], b0[4], b1[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      unsigned long long ra = c_screen_tab.u[(G0 + c) * DP + D], rb = c_screen_tab.u[(G0 + 4 + c) * DP + D];
#pragma unroll
      for (int j = 0; j < D; ++j) {
        ra = ffma2(X[j][pp], c_screen_tab.u[(G0 + c) * DP + j], ra);
        rb = ffma2(X[j][pp], c_screen_tab.u[(G0 + 4 + c) * DP + j], rb);
      }
      unpack2(ra, a0[c], a1[c]);
      unpack2(rb, b0[c], b1[c]);
    }
    const float ga[2] = {pack_idx<LB>(fminf(fmin3(a0[0], a0[1], a0[2]), a0[3]), cx, (uint32_t)G0),
                         pack_idx<LB>(fminf(fmin3(a1[0], a1[1], a1[2]), a1[3]), cx, (uint32_t)G0)};
    const float gb[2] = {pack_idx<LB>(fminf(fmin3(b0[0], b0[1], b0[2]), b0[3]), cx, (uint32_t)G0 + 4u),
                         pack_idx<LB>(fminf(fmin3(b1[0], b1[1], b1[2]), b1[3]), cx, (uint32_t)G0 + 4u)};
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int p = 2 * pp + e;
      const float lo = fminf(ga[e], gb[e]), hi = fmaxf(ga[e], gb[e]);
      if constexpr (FIRST) {
        m1[p] = lo;
        m2[p] = hi;
      } else {
        m2[p] = fmin3(m2[p], hi, fmaxf(m1[p], lo));
        m1[p] = fminf(m1[p], lo);
      }
    }
  }
}

// One warp-tile: grouped screen, exact recompute of the winning group, flags,
// labels and exact sums.  FULL: all 256 points exist (no bounds checks).
// KG: groups of 4 centroids (kpad / 4) when fixed at compile time, else 0.
template <int D, int KG, bool CT, bool FULL>
__device__ __forceinline__ void process_tile(const FastArgs& a, FastSmem<D>& sm, const FastCtx& cx,
                                             const unsigned long long* s2, const float* xcur, int64_t base,
                                             int m, int lane, uint32_t* wmine, uint32_t* q, int& qn) {
  constexpr int DP = D + 1, WIN = 2 * D + 1, GS = FastSmem<D>::GS;
  constexpr int LB = KG == 2 ? 3 : KG == 4 ? 4 : KG == 8 ? 5 : KG == 16 ? 6 : KG == 32 ? 7 : KG == 64 ? 8 : 0;
  static_assert(KG == 0 || LB > 0, "compile-time group counts: 2, 4, 8, 16, 32, 64");
  // this lane's points: base + g*128 + 4*lane + q, g in {0,1}, q in 0..3;
  // pair pp holds points 2pp, 2pp+1.  X = x~ = fl(x - s) per pair.
  unsigned long long X[D][kPts / 2];
#pragma unroll
  for (int g = 0; g < kNG; ++g)
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const ulonglong2 v = *reinterpret_cast<const ulonglong2*>(xcur + j * kWarpTile + g * kGS + 4 * lane);
      X[j][2 * g] = fsub2(v.x, s2[j]);
      X[j][2 * g + 1] = fsub2(v.y, s2[j]);
    }
  // Grouped screen over pairs of groups (kpad is a multiple of 8).
  float m1[kPts], m2[kPts];
  if constexpr (CT) {
    static_assert(KG > 0, "the constant-bank screen needs a compile-time group count");
    screen_pair_ct<D, LB, true>(0, X, cx, m1, m2);
#pragma unroll
    for (int gp = 1; gp < KG / 2; ++gp) screen_pair_ct<D, LB, false>(8 * gp, X, cx, m1, m2);
  } else {
    {
      float ga[kPts], gb[kPts];
      screen_group<D, LB>(sm.tab, X, 0u, cx, ga);
      screen_group<D, LB>(sm.tab + 4 * DP, X, 4u, cx, gb);
      top2_pair<true>(m1, m2, ga, gb);
    }
  }
  if constexpr (CT) {
  } else if constexpr (KG > 0) {
#pragma unroll kGpUnroll
    for (int gp = 1; gp < KG / 2; ++gp) {
      float ga[kPts], gb[kPts];
      screen_group<D, LB>(sm.tab + (size_t)(8 * gp) * DP, X, 8u * gp, cx, ga);
      screen_group<D, LB>(sm.tab + (size_t)(8 * gp + 4) * DP, X, 8u * gp + 4u, cx, gb);
      top2_pair<false>(m1, m2, ga, gb);
    }
  } else {
#pragma unroll 1
    for (int g8 = 8; g8 < cx.kpad; g8 += 8) {
      float ga[kPts], gb[kPts];
      screen_group<D, 0>(sm.tab + (size_t)g8 * DP, X, (uint32_t)g8, cx, ga);
      screen_group<D, 0>(sm.tab + (size_t)(g8 + 4) * DP, X, (uint32_t)g8 + 4u, cx, gb);
      top2_pair<false>(m1, m2, ga, gb);
    }
  }

  // Epilogue: the winning group is recomputed exactly (the same FMA chain,
  // two centroids per FFMA2), its values packed with the index within the
  // group; the label, the runner-up and the flag follow.
  // bin[p]: the label, or k (the discard bin of the sums) for a flagged or
  // padding point; a flagged point's label is written by the re-check.
  int lab[kPts];
  uint32_t fbits = 0u, dbits = 0u;  // flagged; not accumulated here
  float Ap[2];
#pragma unroll
  for (int p = 0; p < kPts; ++p) {
    if ((p & 1) == 0) {
      // A = ||x~||^2 exactly as the data scan that bounds it: x0*x0, then FMAs.
      unsigned long long a2 = ffma2(X[0][p >> 1], X[0][p >> 1], 0ull);
#pragma unroll
      for (int j = 1; j < D; ++j) a2 = ffma2(X[j][p >> 1], X[j][p >> 1], a2);
      unpack2(a2, Ap[0], Ap[1]);
    }
    const uint32_t gsel = __float_as_uint(m1[p]) & cx.kmask;  // the group's first index
    const ulonglong2* gt = reinterpret_cast<const ulonglong2*>(sm.gtab + (size_t)(gsel >> 2) * GS);
    float r0, r1, r2, r3;
    {
      const ulonglong2 nv = gt[D];
      unsigned long long rA = nv.x, rB = nv.y;
#pragma unroll
      for (int j = 0; j < D; ++j) {
        float lo, hi;
        unpack2(X[j][p >> 1], lo, hi);
        const unsigned long long xx = dup2((p & 1) ? hi : lo);
        const ulonglong2 cv = gt[j];
        rA = ffma2(xx, cv.x, rA);
        rB = ffma2(xx, cv.y, rB);
      }
      unpack2(rA, r0, r1);
      unpack2(rB, r2, r3);
    }
    const float w0 = pack_idx<LB>(r0, cx, 0u), w1 = pack_idx<LB>(r1, cx, 1u);
    const float w2 = pack_idx<LB>(r2, cx, 2u), w3 = pack_idx<LB>(r3, cx, 3u);
    const float lo01 = fminf(w0, w1), hi01 = fmaxf(w0, w1);
    const float lo23 = fminf(w2, w3), hi23 = fmaxf(w2, w3);
    const float best = fminf(lo01, lo23);
    const float sec = fmin3(fmaxf(lo01, lo23), fminf(hi01, hi23), m2[p]);
    lab[p] = (int)(gsel | (__float_as_uint(best) & 3u));
    const float v1 = unpack_val<LB>(best, cx), v2 = unpack_val<LB>(sec, cx);
    const float T = fmaf(cx.tau, v2 - cx.M, fmaf(Ap[p & 1], cx.cA, cx.c0));
    bool f = !(v2 - v1 > T);
    // a label outside 0..K-1 (only a padding centroid could give one) is
    // never trusted: the point goes to the re-check
    if (cx.k < cx.kpad) f = f || lab[p] >= cx.k;
    bool valid = true;
    if constexpr (!FULL) valid = base + (p >> 2) * kGS + 4 * lane + (p & 3) < a.n;
    fbits |= ((f && valid) ? 1u : 0u) << p;
    dbits |= ((f || !valid) ? 1u : 0u) << p;
  }
  if (__any_sync(0xffffffffu, fbits != 0u)) {
    const int nf = __popc(fbits);
    int incl = nf;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    int at = qn + incl - nf;
    for (uint32_t fb = fbits; fb; fb &= fb - 1u) {
      const int p = __ffs(fb) - 1;
      q[at++] = (uint32_t)(m << 8) | (uint32_t)((p >> 2) * kGS + 4 * lane + (p & 3));
    }
    qn += __shfl_sync(0xffffffffu, incl, 31);
  }
  // labels (flagged points are overwritten by the re-check)
  if (a.store_labels) {
#pragma unroll
    for (int g = 0; g < kNG; ++g) {
      const int64_t i0 = base + g * kGS + 4 * lane;
      if (a.labels8) {
        if constexpr (FULL) {
          const uint32_t w = __byte_perm(__byte_perm(lab[4 * g], lab[4 * g + 1], 0x0040),
                                         __byte_perm(lab[4 * g + 2], lab[4 * g + 3], 0x0040), 0x5410);
          *reinterpret_cast<uint32_t*>(a.labels8 + i0) = w;
        } else {
#pragma unroll
          for (int qq = 0; qq < 4; ++qq) if (i0 + qq < a.n) a.labels8[i0 + qq] = (uint8_t)lab[4 * g + qq];
        }
      } else if (FULL && !a.labels_unaligned) {
        *reinterpret_cast<int4*>(a.labels + i0) = make_int4(lab[4 * g], lab[4 * g + 1], lab[4 * g + 2], lab[4 * g + 3]);
      } else if constexpr (FULL) {
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) a.labels[i0 + qq] = lab[4 * g + qq];
      } else {
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) if (i0 + qq < a.n) a.labels[i0 + qq] = lab[4 * g + qq];
      }
    }
  }
  // Exact sums: limb splits on FADD2 pairs, then 32-bit shared atomics into
  // this half-warp's window; flagged and padding points go to the discard bin k.
#pragma unroll
  for (int g = 0; g < kNG; ++g)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int p0 = 4 * g + 2 * h;
      uint32_t bh[D][2], bl[D][2];
#pragma unroll
      for (int j = 0; j < D; ++j) {
        const unsigned long long xv =
            *reinterpret_cast<const unsigned long long*>(xcur + j * kWarpTile + g * kGS + 4 * lane + 2 * h);
        const unsigned long long t = fadd2(xv, cx.chi2);
        const unsigned long long hh = fsub2(t, cx.chi2);
        const unsigned long long r = fsub2(xv, hh);
        const unsigned long long t2 = fadd2(r, cx.clo2);
        asm("mov.b64 {%0, %1}, %2;" : "=r"(bh[j][0]), "=r"(bh[j][1]) : "l"(t));
        asm("mov.b64 {%0, %1}, %2;" : "=r"(bl[j][0]), "=r"(bl[j][1]) : "l"(t2));
      }
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int bn = ((dbits >> (p0 + e)) & 1u) ? cx.k : lab[p0 + e];
        uint32_t* wb = wmine + bn * WIN;
        atomicAdd(&wb[0], 1u);
#pragma unroll
        for (int j = 0; j < D; ++j) {
          atomicAdd(&wb[1 + j], bh[j][e]);
          atomicAdd(&wb[1 + D + j], bl[j][e]);
        }
      }
    }
}

template <int D, int KG, bool CT>
__global__ void __launch_bounds__(kThreads, KM_MINB) assign_fast_kernel(FastArgs a) {
  constexpr int DP = D + 1, WIN = 2 * D + 1, GS = FastSmem<D>::GS;
  extern __shared__ __align__(16) unsigned char smraw[];
  if (a.ls->done && !a.ignore_done) return;  // the loop already stopped (graph-driven runs)
  const int nbuf = a.nwin == 1 ? 1 : 2;
  FastSmem<D> sm(smraw, a.kpad, a.k, a.nwin, nbuf);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int k = a.k, kpad = KG > 0 ? 4 * KG : a.kpad;

  const IterConst ic = *a.ic;
  const DataConst dc = *a.dc;
  float s[D];
  unsigned long long s2[D];
#pragma unroll
  for (int j = 0; j < D; ++j) { s[j] = dc.s[j]; s2[j] = dup2(dc.s[j]); }

  const int nwin = a.nwin;
  uint32_t* wwarp = sm.win + (size_t)warp * nwin * (k + 1) * WIN;
  uint32_t* wmine = wwarp + (size_t)(nwin == 4 ? (lane >> 3) : nwin == 2 ? (lane >> 4) : 0) * (k + 1) * WIN;
  long long* acc = sm.acc;
  uint32_t* q = sm.queue + (size_t)warp * kWarpQueue;
  float* xb = sm.xbuf + (size_t)warp * nbuf * D * kWarpTile;
  const int wid = blockIdx.x * kWarps + warp;  // this warp's first tile
  const int wtot = gridDim.x * kWarps;         // tile stride
  const int ntiles = (int)a.ntiles;            // < 2^31 (N < 2^39)
  if (wid < ntiles) prefetch_tile<D>(a, xb, (int64_t)wid * kWarpTile, lane);

  for (int q2 = tid; q2 < kpad * DP; q2 += kThreads) {
    const unsigned long long v = a.tab2[q2];
    sm.tab[q2] = v;
    const int c = q2 / DP, j = q2 - c * DP;
    reinterpret_cast<float*>(sm.gtab + (size_t)(c >> 2) * GS + j)[c & 3] = __uint_as_float((uint32_t)v);
  }
  for (int q2 = tid; q2 < k * DP; q2 += kThreads) sm.acc[q2] = 0;
  if (sm.ctil)
    for (int q2 = tid; q2 < k; q2 += kThreads) sm.ctil[q2] = a.ctil[q2];
  for (int q2 = tid; q2 < kWarps * nwin * (k + 1) * WIN; q2 += kThreads) sm.win[q2] = 0u;
  if (tid < 2) sm.cnt[tid] = 0;
  __syncthreads();

  FastCtx cx;
  cx.L = (uint32_t)ic.L; cx.mul = ic.mul; cx.kmask = ic.mul - 1u;
  cx.ehi = __float_as_uint(ic.M) >> (32 - ic.L);
  cx.M = ic.M;
  {
    // ulp of the binade [2^eM, 2^(eM+1)) that holds every r: exact scaling
    const float ulp = __uint_as_float(__float_as_uint(ic.M) & 0x7f800000u) * 0x1p-23f;
    cx.c0 = ic.thr_c0 * ulp;
    cx.cA = (ic.thr_cA + ic.tau * ic.G) * ulp;
  }
  cx.tau = ic.tau;
  cx.chi2 = dup2(dc.C_hi); cx.clo2 = dup2(dc.C_lo);
  cx.k = k; cx.kpad = kpad;
  int qn = 0, nflag = 0, n64 = 0, since_flush = 0;
  int m = 0;  // this warp's local tile counter

  for (int tile = wid; tile < ntiles; tile += wtot, ++m) {
    const int64_t base = (int64_t)tile * kWarpTile;
    const float* xcur = xb + (nbuf == 2 ? (m & 1) : 0) * D * kWarpTile;
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    // each lane reads only the chunks it copied itself, so the next copy
    // needs no warp barrier
    if (nbuf == 2 && tile + wtot < ntiles)
      prefetch_tile<D>(a, xb + ((m + 1) & 1) * D * kWarpTile, (int64_t)(tile + wtot) * kWarpTile, lane);
    if (base + kWarpTile <= a.n)
      process_tile<D, KG, CT, true>(a, sm, cx, s2, xcur, base, m, lane, wmine, q, qn);
    else
      process_tile<D, KG, CT, false>(a, sm, cx, s2, xcur, base, m, lane, wmine, q, qn);
    if (nbuf == 1 && tile + wtot < ntiles) prefetch_tile<D>(a, xb, (int64_t)(tile + wtot) * kWarpTile, lane);
    // 8 lanes x 8 points x 8 tiles, 16 x 8 x 4 or 32 x 8 x 2: <= 512 additions per bin
    if (++since_flush == (nwin == 4 ? 8 : nwin == 2 ? 4 : 2)) {
      flush_windows<D>(wwarp, acc, k, nwin, lane, dc.bits_C_hi, dc.bits_C_lo);
      since_flush = 0;
    }
    if (qn > kWarpQueue - kWarpTile) {
      __syncwarp();
      drain_warp_queue<D>(a, sm, q, qn, wid, wtot, wwarp, wmine, acc, lane, s, dc, ic.B_max, ic.tau, n64);
      nflag += qn;
      qn = 0;
      since_flush = 0;
    }
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncwarp();
  if (qn > 0) {
    drain_warp_queue<D>(a, sm, q, qn, wid, wtot, wwarp, wmine, acc, lane, s, dc, ic.B_max, ic.tau, n64);
    nflag += qn;
  } else {
    flush_windows<D>(wwarp, acc, k, nwin, lane, dc.bits_C_hi, dc.bits_C_lo);
  }
  if (lane == 0 && nflag) atomicAdd(&sm.cnt[0], nflag);
  if (n64) atomicAdd(&sm.cnt[1], n64);
  __syncthreads();
  long long* out = a.partials + (size_t)blockIdx.x * k * DP;
  for (int q2 = tid; q2 < k * DP; q2 += kThreads) out[q2] = sm.acc[q2];
  if (tid == 0) {
    if (sm.cnt[0]) atomicAdd(&a.ls->flagged, (unsigned long long)sm.cnt[0]);
    if (sm.cnt[1]) atomicAdd(&a.ls->fp64_decided, (unsigned long long)sm.cnt[1]);
  }
}

// ---- Batched instances through the fused kernel's tile machinery ----
//
// Per tile (a run of one instance's points, a multiple of 256 long but the
// instance's last), the block loads the instance's screen table, group table
// and re-check centroids into shared memory; each warp then screens the
// tile's 256-point warp-tiles w, w + 8, ... exactly as the fused kernel
// does (same screen, flag test, re-check and exact sums), and the block
// writes its int64 totals as the tile's partial row.  The regions of shared
// memory have fixed bases (the layout of d = 3, K = 64), so instances of any
// d follow one another without clearing: windows are zero after every flush.

// Points of an instance are packed without padding, so the staging copies
// are 4 bytes each (rows need not be 16-byte aligned); past N, zero-filled.
template <int D>
__device__ __forceinline__ void prefetch_tile_any(const FastArgs& a, float* xb, int64_t base, int lane) {
#pragma unroll
  for (int g = 0; g < kNG; ++g)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int off = g * kGS + 4 * lane + e;
      const int64_t i = base + off;
      const int bytes = i < a.n ? 4 : 0;
#pragma unroll
      for (int j = 0; j < D; ++j) {
        const float* src = a.x + (int64_t)j * a.ld + (bytes ? i : 0);
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(xb + j * kWarpTile + off);
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(bytes));
      }
    }
  asm volatile("cp.async.commit_group;" ::: "memory");
}

constexpr int kBatchWinWords = 2 * (kBatchMaxK + 1) * 7;  // per warp: two windows of 65 bins of 7 words

template <int D>
__device__ __forceinline__ FastSmem<D> batch_smem(unsigned char* raw) {
  const FastSmem<3> f(raw, kBatchMaxK, kBatchMaxK, 2, 2);
  FastSmem<D> s;
  s.tab = f.tab;
  s.acc = f.acc;
  s.gtab = f.gtab;
  s.ctil = f.ctil;
  s.xbuf = f.xbuf;
  s.queue = f.queue;
  s.win = f.win;
  s.cnt = f.cnt;
  return s;
}

template <int D>
__device__ void batch_fast_tile(const BatchArgs& ba, int t, const int4& tl, unsigned char* raw, int tid, int lane,
                                int warp, int& nflag, int& n64) {
  constexpr int DP = D + 1, WIN = 2 * D + 1, GS = FastSmem<D>::GS;
  FastSmem<D> sm = batch_smem<D>(raw);
  const int inst = tl.x;
  const BatchInst bi = ba.inst[inst];
  const int k = bi.k, kpad = bi.kpad;
  const unsigned long long* tab2 = ba.tab2 + bi.tab_off;
  for (int q = tid; q < kpad * DP; q += kThreads) {
    const unsigned long long v = tab2[q];
    sm.tab[q] = v;
    const int c = q / DP, j = q - c * DP;
    reinterpret_cast<float*>(sm.gtab + (size_t)(c >> 2) * GS + j)[c & 3] = __uint_as_float((uint32_t)v);
  }
  for (int q = tid; q < k; q += kThreads) sm.ctil[q] = ba.ctil4[bi.k_off + q];
  __syncthreads();

  FastArgs a{};
  a.x = ba.x + bi.x_off; a.ld = bi.n; a.n = bi.n; a.k = k; a.kpad = kpad;
  a.ctil = ba.ctil4 + bi.k_off; a.mu = ba.mu + bi.mu_off;
  a.labels = ba.labels + bi.lab_off; a.labels8 = nullptr; a.store_labels = 1; a.nwin = 2;
  a.labels_unaligned = (bi.lab_off & 3) != 0;
  const IterConst ic = ba.ic[inst];
  DataConst dc{};
  for (int j = 0; j < kMaxDFast; ++j) dc.s[j] = j < 3 ? bi.s[j] : 0.f;
  dc.A_max = bi.A_max; dc.G0 = bi.G0; dc.C_hi = bi.C_hi; dc.C_lo = bi.C_lo;
  dc.bits_C_hi = bi.bits_C_hi; dc.bits_C_lo = bi.bits_C_lo;
  float s[D];
  unsigned long long s2[D];
#pragma unroll
  for (int j = 0; j < D; ++j) { s[j] = bi.s[j]; s2[j] = dup2(bi.s[j]); }
  FastCtx cx;
  cx.L = (uint32_t)ic.L; cx.mul = ic.mul; cx.kmask = ic.mul - 1u;
  cx.ehi = __float_as_uint(ic.M) >> (32 - ic.L);
  cx.M = ic.M;
  {
    const float ulp = __uint_as_float(__float_as_uint(ic.M) & 0x7f800000u) * 0x1p-23f;
    cx.c0 = ic.thr_c0 * ulp;
    cx.cA = (ic.thr_cA + ic.tau * ic.G) * ulp;
  }
  cx.tau = ic.tau;
  cx.chi2 = dup2(dc.C_hi); cx.clo2 = dup2(dc.C_lo);
  cx.k = k; cx.kpad = kpad;

  uint32_t* wwarp = sm.win + (size_t)warp * kBatchWinWords;
  uint32_t* wmine = wwarp + (size_t)(lane >> 4) * (k + 1) * WIN;
  uint32_t* q = sm.queue + (size_t)warp * kWarpQueue;
  float* xb = sm.xbuf + (size_t)warp * 2 * 3 * kWarpTile;
  const int64_t first = tl.y;
  const int nwt = (tl.z + kWarpTile - 1) / kWarpTile;  // warp-tiles of this tile
  const int wid0 = (int)(first / kWarpTile) + warp;  // this warp's first warp-tile (index within the instance)
  int qn = 0, m = 0, since_flush = 0;
  if (warp < nwt) prefetch_tile_any<D>(a, xb, first + (int64_t)warp * kWarpTile, lane);
  for (int wt = warp; wt < nwt; wt += kWarps, ++m) {
    const int64_t base = first + (int64_t)wt * kWarpTile;
    const float* xcur = xb + (m & 1) * D * kWarpTile;
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    if (wt + kWarps < nwt)
      prefetch_tile_any<D>(a, xb + ((m + 1) & 1) * D * kWarpTile, base + (int64_t)kWarps * kWarpTile, lane);
    if (base + kWarpTile <= bi.n)
      process_tile<D, 0, false, true>(a, sm, cx, s2, xcur, base, m, lane, wmine, q, qn);
    else
      process_tile<D, 0, false, false>(a, sm, cx, s2, xcur, base, m, lane, wmine, q, qn);
    // 16 lanes x 8 points x 4 warp-tiles: <= 512 additions per bin
    if (++since_flush == 4) {
      flush_windows<D>(wwarp, sm.acc, k, 2, lane, dc.bits_C_hi, dc.bits_C_lo);
      since_flush = 0;
    }
    if (qn > kWarpQueue - kWarpTile) {
      __syncwarp();
      drain_warp_queue<D>(a, sm, q, qn, wid0, kWarps, wwarp, wmine, sm.acc, lane, s, dc, ic.B_max, ic.tau, n64);
      nflag += qn;
      qn = 0;
      since_flush = 0;
    }
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncwarp();
  if (qn > 0) {
    drain_warp_queue<D>(a, sm, q, qn, wid0, kWarps, wwarp, wmine, sm.acc, lane, s, dc, ic.B_max, ic.tau, n64);
    nflag += qn;
  } else if (warp < nwt) {
    flush_windows<D>(wwarp, sm.acc, k, 2, lane, dc.bits_C_hi, dc.bits_C_lo);
  }
  __syncthreads();
  // the tile's partial row; the totals go back to zero for the next tile
  // (each thread its own entries; the next tile's flushes come after its
  // first barrier)
  long long* prow = ba.partials + ba.tile_poff[t];
  for (int q2 = tid; q2 < k * DP; q2 += kThreads) {
    prow[q2] = sm.acc[q2];
    sm.acc[q2] = 0;
  }
}

__global__ void __launch_bounds__(kThreads, KM_MINB) batch_fast_kernel(BatchArgs ba) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const FastSmem<3> base(smraw, kBatchMaxK, kBatchMaxK, 2, 2);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int q = tid; q < kWarps * kBatchWinWords; q += kThreads) base.win[q] = 0u;
  for (int q = tid; q < kBatchMaxK * 4; q += kThreads) base.acc[q] = 0;
  if (tid < 2) base.cnt[tid] = 0;
  __syncthreads();
  int nflag = 0, n64 = 0;
  for (int t = blockIdx.x; t < ba.ntiles; t += gridDim.x) {
    const int4 tl = ba.tiles[t];
    if (ba.state[tl.x].done) continue;  // block-uniform
    const int d = ba.inst[tl.x].d;
    if (d == 3) batch_fast_tile<3>(ba, t, tl, smraw, tid, lane, warp, nflag, n64);
    else if (d == 2) batch_fast_tile<2>(ba, t, tl, smraw, tid, lane, warp, nflag, n64);
    else batch_fast_tile<1>(ba, t, tl, smraw, tid, lane, warp, nflag, n64);
  }
  if (lane == 0 && nflag) atomicAdd(&base.cnt[0], nflag);
  if (n64) atomicAdd(&base.cnt[1], n64);
  __syncthreads();
  if (tid == 0) {
    if (base.cnt[0]) atomicAdd(ba.flagged, (unsigned long long)base.cnt[0]);
    if (base.cnt[1]) atomicAdd(ba.fp64, (unsigned long long)base.cnt[1]);
  }
}

// Generic path: any d, any K.  One point per thread per iteration of a
// grid-stride loop; FP32 direct-form screen with the same bound and FP64
// re-decision as the re-check of the fused kernel; exact integer sums with
// 64-bit atomics into this block's own partial row.
__global__ void __launch_bounds__(kThreads) assign_generic_kernel(GenericArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  if (a.ls->done && !a.ignore_done) return;
  const int d = a.d, k = a.k, dp = d + 1;
  unsigned long long* row = reinterpret_cast<unsigned long long*>(a.partials) + (size_t)blockIdx.x * k * dp;
  for (int q = threadIdx.x; q < k * dp; q += blockDim.x) row[q] = 0ull;
  __shared__ int n64s, nflag;
  if (threadIdx.x == 0) { n64s = 0; nflag = 0; }
  __syncthreads();
  const DataConst dc = *a.dc;
  const float B_max = *a.B_max_ptr;
  const float sB = sqrtf(B_max);
  int my64 = 0, myflag = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float A = 0.f;
    for (int j = 0; j < d; ++j) {
      float t = __fsub_rn(a.x[(int64_t)j * a.ld + i], a.shift[j]);
      A = __fmaf_rn(t, t, A);
    }
    A *= 1.0001f;
    float best = 3.0e38f, second = 3.0e38f;
    int kb = 0;
    for (int c = 0; c < k; ++c) {
      const float* cc = a.ctil + (size_t)c * d;
      float dv = 0.f;
      for (int j = 0; j < d; ++j) {
        float xt = __fsub_rn(a.x[(int64_t)j * a.ld + i], a.shift[j]);
        float t = __fsub_rn(xt, __ldg(cc + j));
        dv = __fmaf_rn(t, t, dv);
      }
      if (dv < best) { second = best; best = dv; kb = c; }
      else if (dv < second) { second = dv; }
    }
    if (k > 1) {
      float sA = sqrtf(A), AB = A + B_max;
      float e1 = direct_bound(best, sA, sB, AB, d), e2 = direct_bound(second, sA, sB, AB, d);
      float lo2 = second - e2, hi1 = best + e1;
      bool clear = (lo2 > hi1) && (lo2 - hi1 > a.tau * (second + e2));
      if (!clear) {
        ++myflag;
        ++my64;
        double bd = d64_dyn(a.x, a.ld, i, d, a.mu);
        kb = 0;
        for (int c = 1; c < k; ++c) {
          double dd = d64_dyn(a.x, a.ld, i, d, a.mu + (size_t)c * d);
          if (dd < bd) { bd = dd; kb = c; }
        }
      }
    }
    if (a.store_labels) {
      if (a.labels8) a.labels8[i] = (uint8_t)kb;
      else a.labels[i] = kb;
    }
    unsigned long long* r = row + (size_t)kb * dp;
    for (int j = 0; j < d; ++j) {
      uint32_t bh, bl;
      split_limbs(a.x[(int64_t)j * a.ld + i], dc.C_hi, dc.C_lo, bh, bl);
      long long hi = (long long)(int)(bh - dc.bits_C_hi), lo = (long long)(int)(bl - dc.bits_C_lo);
      atomicAdd(r + j, (unsigned long long)((hi << 22) + lo));
    }
    atomicAdd(r + d, 1ull);
  }
  if (my64) atomicAdd(&n64s, my64);
  if (myflag) atomicAdd(&nflag, myflag);
  __syncthreads();
  if (threadIdx.x == 0) {
    if (nflag) atomicAdd(&a.ls->flagged, (unsigned long long)nflag);
    if (n64s) atomicAdd(&a.ls->fp64_decided, (unsigned long long)n64s);
  }
}

}  // namespace

size_t fast_smem_bytes(int d, int kpad, int k, int nwin) {
  const int dp = d + 1, win = 2 * d + 1, gs = (dp & 1) ? dp : dp + 1;
  const int nbuf = nwin == 1 ? 1 : 2;
  size_t b = (size_t)kpad * dp * 8 + (size_t)(k * dp + (k * dp & 1)) * 8 + (size_t)(kpad / 4) * gs * 16 +
             (nbuf == 2 ? (size_t)k * 16 : 0) +
             (size_t)kWarps * nbuf * d * kWarpTile * 4 + (size_t)kWarps * kWarpQueue * 4 +
             (size_t)kWarps * nwin * (k + 1) * win * 4 + 16;
  return (b + 15) & ~size_t(15);
}

template <int D, int KG, bool CT>
static cudaError_t launch_fast_dk(int grid, size_t smem, cudaStream_t st, const FastArgs& a) {
  auto fn = assign_fast_kernel<D, KG, CT>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if constexpr (CT) {
    e = cudaMemcpyToSymbolAsync(c_screen_tab, a.tab2, (size_t)a.kpad * (D + 1) * sizeof(unsigned long long), 0,
                                cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
  }
  fn<<<grid, kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

template <int D, int KG, bool CT>
static int blocks_dk(size_t smem) {
  int nb = 0;
  cudaFuncSetAttribute(assign_fast_kernel<D, KG, CT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, assign_fast_kernel<D, KG, CT>, kThreads, smem) !=
      cudaSuccess)
    return 1;
  return nb > 0 ? nb : 1;
}

// Instantiations: the constant-bank screen (compile-time group count, fully
// unrolled, shift packing) for 3-D data with K <= 32 in groups of 8; for 3-D
// data with kpad = 256, the shared-memory table with a compile-time group
// count (index packing by shifts, 1.5 % faster than the run-time count); a
// runtime loop over the shared-memory table otherwise.
#define KM_FAST_DISPATCH(FN, D, CT_OK, ...)                           \
  do {                                                                \
    if constexpr (D == 3) {                                           \
      if (kpad == 32) {                                               \
        if (CT_OK) return FN<D, 8, true>(__VA_ARGS__);                \
        return FN<D, 8, false>(__VA_ARGS__);                          \
      }                                                               \
      if (kpad == 256) return FN<D, 64, false>(__VA_ARGS__);          \
    }                                                                 \
    return FN<D, 0, false>(__VA_ARGS__);                              \
  } while (0)

template <int D>
static int blocks_d(size_t smem, int kpad, bool ct) {
  KM_FAST_DISPATCH(blocks_dk, D, ct, smem);
}

template <int D>
static cudaError_t launch_fast_d(int grid, size_t smem, cudaStream_t st, const FastArgs& a) {
  const int kpad = a.kpad;
  KM_FAST_DISPATCH(launch_fast_dk, D, a.const_tab != 0, grid, smem, st, a);
}

bool fast_has_const_table(int d, int kpad) { return d == 3 && kpad == 32; }

int fast_blocks_per_sm(int d, size_t smem, int kpad, bool ct) {
  switch (d) {
    case 1: return blocks_d<1>(smem, kpad, ct);
    case 2: return blocks_d<2>(smem, kpad, ct);
    case 3: return blocks_d<3>(smem, kpad, ct);
    default: return blocks_d<4>(smem, kpad, ct);
  }
}

cudaError_t launch_assign_fast(int d, int grid, size_t smem, cudaStream_t st, const FastArgs& a) {
  switch (d) {
    case 1: return launch_fast_d<1>(grid, smem, st, a);
    case 2: return launch_fast_d<2>(grid, smem, st, a);
    case 3: return launch_fast_d<3>(grid, smem, st, a);
    case 4: return launch_fast_d<4>(grid, smem, st, a);
    default: return cudaErrorInvalidValue;
  }
}

static size_t batch_fast_smem() { return fast_smem_bytes(3, kBatchMaxK, kBatchMaxK, 2); }

cudaError_t launch_batch_fast(const BatchArgs& a, int grid, cudaStream_t st) {
  const size_t smem = batch_fast_smem();
  cudaError_t e = cudaFuncSetAttribute(batch_fast_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  batch_fast_kernel<<<grid, kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

int batch_fast_blocks_per_sm() {
  const size_t smem = batch_fast_smem();
  int nb = 0;
  cudaFuncSetAttribute(batch_fast_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, batch_fast_kernel, kThreads, smem) != cudaSuccess) return 1;
  return nb > 0 ? nb : 1;
}

size_t generic_smem_bytes(int, int) { return 0; }

cudaError_t launch_assign_generic(int grid, size_t smem, cudaStream_t st, const GenericArgs& a) {
  assign_generic_kernel<<<grid, kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace km
