// Reassignment + per-block accumulation: the expectation step and the first
// half of the mean calculation of Lloyd's algorithm (paper, section "The
// Lloyd's algorithm", steps 2 and 3), fused in one pass over the points.
//
// assign_fast_kernel<D> (d <= 4, K <= 256) is the hot kernel: SoA float4
// streaming loads, FP32 screen on FFMA2 with the index packed by IMAD and
// top-2 by FMNMX, a per-block queue of flagged points re-decided at the end
// of the block's work, and exact integer sums in per-warp shared windows.
// assign_generic_kernel handles any d and K with a direct-form FP32 screen,
// the same re-check rules and 64-bit atomics into the block's own partial row.
#include "km_internal.cuh"

namespace km {

namespace {

__device__ __forceinline__ unsigned long long pack2(float a, float b) {
  unsigned long long p;
  asm("mov.b64 %0, {%1, %2};" : "=l"(p) : "f"(a), "f"(b));
  return p;
}
__device__ __forceinline__ void unpack2(unsigned long long p, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(p));
}
// d = a * b + c on two float lanes (one FFMA2 instruction).
__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b,
                                                    unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ float fmin3(float a, float b, float c) {
  float d;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}
// a * b + c on the FMA pipe (keeps the index packing off the ALU pipe).
__device__ __forceinline__ uint32_t imad(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
__device__ __forceinline__ float4 ld_stream4(const float* p) {
  float4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
  return v;
}

// Top-2 of packed (value, index) floats, two new candidates at a time:
// m1' = min(m1, a, b); m2' = min(m2, max(a, b), max(m1, min(a, b))).
__device__ __forceinline__ void top2_pair(float& m1, float& m2, float a, float b) {
  float lo = fminf(a, b), hi = fmaxf(a, b);
  float t = fmaxf(m1, lo);
  m2 = fmin3(m2, hi, t);
  m1 = fminf(m1, lo);
}

// Exact split of x into the two fixed-point limbs (biased bit patterns).
__device__ __forceinline__ void split_limbs(float x, float C_hi, float C_lo, uint32_t& bhi,
                                            uint32_t& blo) {
  float t = __fadd_rn(x, C_hi);   // rounds x to the 2^G1 grid; bits(t) - bits(C_hi) = hi
  float h = __fsub_rn(t, C_hi);   // exact
  float r = __fsub_rn(x, h);      // exact remainder, |r| <= 2^(G1-1)
  float t2 = __fadd_rn(r, C_lo);  // rounds r to the 2^G0 grid
  bhi = __float_as_uint(t);
  blo = __float_as_uint(t2);
}

// FP64 squared distance in the oracle's order: sum over j of (x_j - mu_j)^2,
// no fused multiply-add.
template <int D>
__device__ __forceinline__ double d64_fixed(const float* xo, const double* mu_k) {
  double acc = 0.0;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    double t = __dsub_rn((double)xo[j], mu_k[j]);
    acc = __dadd_rn(acc, __dmul_rn(t, t));
  }
  return acc;
}
__device__ __forceinline__ double d64_dyn(const float* x, int64_t ld, int64_t i, int d,
                                          const double* mu_k) {
  double acc = 0.0;
  for (int j = 0; j < d; ++j) {
    double t = __dsub_rn((double)x[(int64_t)j * ld + i], mu_k[j]);
    acc = __dadd_rn(acc, __dmul_rn(t, t));
  }
  return acc;
}

constexpr float kU = 5.9604644775390625e-08f;        // 2^-24
constexpr float kU64x = 1.1102230246251565e-16f * 4.1f;  // 4.1 * 2^-53

// Error bound of the FP32 direct form sum_j fl(x~_j - c~_j)^2 against the
// exact D = ||x - mu||^2, plus the FP64 rounding the oracle itself makes.
__device__ __forceinline__ float direct_bound(float dv, float sqrtA, float sqrtB, float AB,
                                              int d) {
  float sd = sqrtf(fmaxf(dv, 0.f));
  return 1.01f * kU * ((float)(d + 2) * dv + 2.f * sd * (sqrtA + sqrtB)) +
         kU64x * (float)(d + 1) * AB + 1e-30f;
}

// Re-decide one flagged point: FP32 direct form with a rigorous bound, and
// FP64 in the oracle's order when the bound (or the tie_rel rule) leaves it
// open.  Returns the label; sets used64.
template <int D>
__device__ int recheck_fast(const float* xo, const float* s, const float4* ctil, const double* mu,
                            int k, float B_max, float tau, bool& used64) {
  float xt[D];
  float A = 0.f;
#pragma unroll
  for (int j = 0; j < D; ++j) {
    xt[j] = __fsub_rn(xo[j], s[j]);
    A = __fmaf_rn(xt[j], xt[j], A);
  }
  A *= 1.0001f;
  float best = 3.0e38f, second = 3.0e38f;
  int kb = 0;
  for (int c = 0; c < k; ++c) {
    float4 cc = ctil[c];
    float cv[4] = {cc.x, cc.y, cc.z, cc.w};
    float dv = 0.f;
#pragma unroll
    for (int j = 0; j < D; ++j) {
      float t = __fsub_rn(xt[j], cv[j]);
      dv = __fmaf_rn(t, t, dv);
    }
    if (dv < best) { second = best; best = dv; kb = c; }
    else if (dv < second) { second = dv; }
  }
  used64 = false;
  if (k > 1) {
    float sA = sqrtf(A), sB = sqrtf(B_max), AB = A + B_max;
    float e1 = direct_bound(best, sA, sB, AB, D);
    float e2 = direct_bound(second, sA, sB, AB, D);
    float lo2 = second - e2, hi1 = best + e1;
    bool clear = (lo2 > hi1) && (lo2 - hi1 > tau * (second + e2));
    if (!clear) {
      used64 = true;
      double bd = d64_fixed<D>(xo, mu);
      kb = 0;
      for (int c = 1; c < k; ++c) {
        double dd = d64_fixed<D>(xo, mu + (int64_t)c * D);
        if (dd < bd) { bd = dd; kb = c; }
      }
    }
  }
  return kb;
}

template <int D>
struct FastSmem {
  static constexpr int DP = D + 1, WIN = 2 * D + 1;
  unsigned long long* tab;  // [kpad][DP]
  long long* acc;           // [kWarps][k][DP]
  uint32_t* queue;          // [kQueueCap]
  float4* ctil;             // [k]
  uint32_t* win;            // [kWarps][k][WIN]
  int* qn;                  // [4]: queue count, flagged, fp64
  __device__ FastSmem(unsigned char* sm, int kpad, int k) {
    tab = reinterpret_cast<unsigned long long*>(sm);
    acc = reinterpret_cast<long long*>(tab + (size_t)kpad * DP);
    queue = reinterpret_cast<uint32_t*>(acc + (size_t)kWarps * k * DP);
    ctil = reinterpret_cast<float4*>(queue + kQueueCap);
    win = reinterpret_cast<uint32_t*>(ctil + k);
    qn = reinterpret_cast<int*>(win + (size_t)kWarps * k * WIN);
  }
};

template <int D>
__device__ __forceinline__ void flush_window(uint32_t* win, long long* acc, int k, int lane,
                                             uint32_t bias_hi, uint32_t bias_lo) {
  constexpr int DP = D + 1, WIN = 2 * D + 1;
  __syncwarp();
  // acc columns per centroid: 0..D-1 coordinate sums, D the count (the
  // layout of the per-block partials); window slots: 0 the count, 1..D the
  // high limbs, D+1..2D the low limbs.
  for (int s = lane; s < k * DP; s += 32) {
    int kk = s / DP, j = s - kk * DP;
    const uint32_t* w = win + kk * WIN;
    uint32_t c = w[0];
    long long v;
    if (j == D) {
      v = (long long)c;
    } else {
      int hi = (int)(w[1 + j] - c * bias_hi);       // exact: |sum| < 2^30
      int lo = (int)(w[1 + D + j] - c * bias_lo);
      v = ((long long)hi << 22) + (long long)lo;
    }
    acc[s] += v;
  }
  __syncwarp();
  for (int s = lane; s < k * WIN; s += 32) win[s] = 0u;
  __syncwarp();
}

template <int D>
__device__ __forceinline__ void accumulate_point(uint32_t* win, int kk, const float* xo,
                                                 float C_hi, float C_lo) {
  constexpr int WIN = 2 * D + 1;
  uint32_t* w = win + kk * WIN;
  atomicAdd(&w[0], 1u);
#pragma unroll
  for (int j = 0; j < D; ++j) {
    uint32_t bh, bl;
    split_limbs(xo[j], C_hi, C_lo, bh, bl);
    atomicAdd(&w[1 + j], bh);
    atomicAdd(&w[1 + D + j], bl);
  }
}

// Drain the block's queue of flagged points.  Must be called by the whole
// block, after a barrier that follows the last push.
template <int D>
__device__ void drain_queue(const FastArgs& a, FastSmem<D>& sm, const float* s, float C_hi,
                            float C_lo, uint32_t bias_hi, uint32_t bias_lo, float B_max, float tau) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint32_t* win = sm.win + (size_t)warp * a.k * (2 * D + 1);
  long long* acc = sm.acc + (size_t)warp * a.k * (D + 1);
  flush_window<D>(win, acc, a.k, lane, bias_hi, bias_lo);
  const int qn = min(sm.qn[0], kQueueCap);
  int n64 = 0;
  // Rounds of one entry per thread; the window is flushed every 16 rounds so
  // that no bin receives more than 512 additions between flushes.
  for (int r = 0, base = 0; base < qn; ++r, base += kThreads) {
    const int q = base + tid;
    if (q < qn) {
      uint32_t loc = sm.queue[q];
      int64_t tile = (int64_t)blockIdx.x + (int64_t)(loc >> 11) * gridDim.x;
      int64_t i = tile * kTile + (loc & 2047u);
      float xo[D];
#pragma unroll
      for (int j = 0; j < D; ++j) xo[j] = a.x[(int64_t)j * a.ld + i];
      bool used64;
      int kk = recheck_fast<D>(xo, s, sm.ctil, a.mu, a.k, B_max, tau, used64);
      n64 += used64 ? 1 : 0;
      a.labels[i] = kk;
      accumulate_point<D>(win, kk, xo, C_hi, C_lo);
    }
    if ((r & 15) == 15) flush_window<D>(win, acc, a.k, lane, bias_hi, bias_lo);
  }
  flush_window<D>(win, acc, a.k, lane, bias_hi, bias_lo);
  if (n64) atomicAdd(&sm.qn[2], n64);
  __syncthreads();
  if (tid == 0) { sm.qn[1] += qn; sm.qn[0] = 0; }
  __syncthreads();
}

template <int D>
__global__ void __launch_bounds__(kThreads, 2) assign_fast_kernel(FastArgs a) {
  constexpr int DP = D + 1;
  extern __shared__ __align__(16) unsigned char smraw[];
  if (a.ls->done) return;  // the loop already stopped (graph-driven runs)
  FastSmem<D> sm(smraw, a.kpad, a.k);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int k = a.k, kpad = a.kpad;

  const IterConst ic = *a.ic;
  const DataConst dc = *a.dc;
  float s[D];
#pragma unroll
  for (int j = 0; j < D; ++j) s[j] = dc.s[j];

  for (int q = tid; q < kpad * DP; q += kThreads) sm.tab[q] = a.tab2[q];
  for (int q = tid; q < k; q += kThreads) sm.ctil[q] = a.ctil[q];
  for (int q = tid; q < kWarps * k * DP; q += kThreads) sm.acc[q] = 0;
  for (int q = tid; q < kWarps * k * (2 * D + 1); q += kThreads) sm.win[q] = 0u;
  if (tid < 4) sm.qn[tid] = 0;
  __syncthreads();

  uint32_t* win = sm.win + (size_t)warp * k * (2 * D + 1);
  long long* acc = sm.acc + (size_t)warp * k * DP;
  const uint32_t mul = ic.mul, L = (uint32_t)ic.L, kmask = mul - 1u;
  int since_flush = 0;
  int64_t local_tile = 0;

  for (int64_t tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x, ++local_tile) {
    const int64_t base = tile * kTile;
    const bool full = base + kTile <= a.n;
    float xo[D][kPts];
#pragma unroll
    for (int g = 0; g < 2; ++g) {
      const int64_t i0 = base + g * (kTile / 2) + 4 * tid;
      if (full) {
#pragma unroll
        for (int j = 0; j < D; ++j) {
          float4 v = ld_stream4(a.x + (int64_t)j * a.ld + i0);
          xo[j][4 * g + 0] = v.x; xo[j][4 * g + 1] = v.y;
          xo[j][4 * g + 2] = v.z; xo[j][4 * g + 3] = v.w;
        }
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int64_t i = i0 + q;
#pragma unroll
          for (int j = 0; j < D; ++j) xo[j][4 * g + q] = (i < a.n) ? a.x[(int64_t)j * a.ld + i] : s[j];
        }
      }
    }
    // Shifted coordinates (x~ = fl(x - s)) and A = ||x~||^2 in the same
    // expression as the data scan that bounds it.
    float Ap[kPts];
    unsigned long long X[D][kPts / 2];
#pragma unroll
    for (int p = 0; p < kPts; p += 2) {
      float t0[D], t1[D];
#pragma unroll
      for (int j = 0; j < D; ++j) {
        t0[j] = __fsub_rn(xo[j][p], s[j]);
        t1[j] = __fsub_rn(xo[j][p + 1], s[j]);
        X[j][p / 2] = pack2(t0[j], t1[j]);
      }
      float a0 = __fmul_rn(t0[0], t0[0]), a1 = __fmul_rn(t1[0], t1[0]);
#pragma unroll
      for (int j = 1; j < D; ++j) { a0 = __fmaf_rn(t0[j], t0[j], a0); a1 = __fmaf_rn(t1[j], t1[j], a1); }
      Ap[p] = a0; Ap[p + 1] = a1;
    }
    // Screen: top-2 of packed (r, k) over all centroids.
    float m1[kPts], m2[kPts];
#pragma unroll
    for (int p = 0; p < kPts; ++p) { m1[p] = 3.0e38f; m2[p] = 3.0e38f; }
#pragma unroll 2
    for (int kp = 0; kp < kpad; kp += 2) {
      unsigned long long ta[DP], tb[DP];
      const unsigned long long* ra = sm.tab + (size_t)kp * DP;
#pragma unroll
      for (int j = 0; j < DP; ++j) { ta[j] = ra[j]; tb[j] = ra[DP + j]; }
#pragma unroll
      for (int pp = 0; pp < kPts / 2; ++pp) {
        unsigned long long rA = ta[D], rB = tb[D];
#pragma unroll
        for (int j = 0; j < D; ++j) { rA = ffma2(X[j][pp], ta[j], rA); rB = ffma2(X[j][pp], tb[j], rB); }
        float a0, a1, b0, b1;
        unpack2(rA, a0, a1);
        unpack2(rB, b0, b1);
        const float pa0 = __uint_as_float(imad(__float_as_uint(a0), mul, (uint32_t)kp));
        const float pa1 = __uint_as_float(imad(__float_as_uint(a1), mul, (uint32_t)kp));
        const float pb0 = __uint_as_float(imad(__float_as_uint(b0), mul, (uint32_t)kp + 1u));
        const float pb1 = __uint_as_float(imad(__float_as_uint(b1), mul, (uint32_t)kp + 1u));
        top2_pair(m1[2 * pp], m2[2 * pp], pa0, pb0);
        top2_pair(m1[2 * pp + 1], m2[2 * pp + 1], pa1, pb1);
      }
    }
    // Epilogue: labels, flags, accumulation.
    int lab[kPts];
    bool flg[kPts];
#pragma unroll
    for (int p = 0; p < kPts; ++p) {
      const int64_t i = base + (p >> 2) * (kTile / 2) + 4 * tid + (p & 3);
      const bool valid = full || i < a.n;
      const uint32_t u1 = __float_as_uint(m1[p]), u2 = __float_as_uint(m2[p]);
      lab[p] = (int)(u1 & kmask);
      const uint32_t b1 = u1 >> L, b2 = u2 >> L;
      const float gap = (float)(b2 - b1);
      const float w2u = (float)(int)(b2 - ic.bitsM_low);
      const float T = ic.thr_c0 + Ap[p] * ic.thr_cA + ic.tau * fmaxf(0.f, w2u + Ap[p] * ic.G);
      // a label outside 0..K-1 (only the padding centroid could give one) is
      // never trusted: the point goes to the re-check
      flg[p] = valid && (!(gap > T) || lab[p] >= k);
      if (flg[p]) {
        const int q = atomicAdd(&sm.qn[0], 1);
        if (q < kQueueCap)
          sm.queue[q] = (uint32_t)(local_tile << 11) | (uint32_t)((p >> 2) * (kTile / 2) + 4 * tid + (p & 3));
        else
          a.ls->error = 1;  // cannot happen: the queue is drained above kQueueCap - kTile
      }
    }
#pragma unroll
    for (int g = 0; g < 2; ++g) {
      const int64_t i0 = base + g * (kTile / 2) + 4 * tid;
      if (full) {
        *reinterpret_cast<int4*>(a.labels + i0) =
            make_int4(lab[4 * g], lab[4 * g + 1], lab[4 * g + 2], lab[4 * g + 3]);
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) if (i0 + q < a.n) a.labels[i0 + q] = lab[4 * g + q];
      }
    }
#pragma unroll
    for (int p = 0; p < kPts; ++p) {
      const int64_t i = base + (p >> 2) * (kTile / 2) + 4 * tid + (p & 3);
      if ((full || i < a.n) && !flg[p]) {
        float xp[D];
#pragma unroll
        for (int j = 0; j < D; ++j) xp[j] = xo[j][p];
        accumulate_point<D>(win, lab[p], xp, dc.C_hi, dc.C_lo);
      }
    }
    if (++since_flush == 2) {
      flush_window<D>(win, acc, k, lane, dc.bits_C_hi, dc.bits_C_lo);
      since_flush = 0;
    }
    __syncthreads();
    if (sm.qn[0] > kQueueCap - kTile) {
      drain_queue<D>(a, sm, s, dc.C_hi, dc.C_lo, dc.bits_C_hi, dc.bits_C_lo, ic.B_max, ic.tau);
    }
  }
  flush_window<D>(win, acc, k, lane, dc.bits_C_hi, dc.bits_C_lo);
  __syncthreads();
  if (sm.qn[0] > 0) drain_queue<D>(a, sm, s, dc.C_hi, dc.C_lo, dc.bits_C_hi, dc.bits_C_lo, ic.B_max, ic.tau);
  __syncthreads();
  long long* out = a.partials + (size_t)blockIdx.x * k * DP;
  for (int q = tid; q < k * DP; q += kThreads) {
    long long v = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) v += sm.acc[(size_t)w * k * DP + q];
    out[q] = v;
  }
  if (tid == 0) {
    if (sm.qn[1]) atomicAdd(&a.ls->flagged, (unsigned long long)sm.qn[1]);
    if (sm.qn[2]) atomicAdd(&a.ls->fp64_decided, (unsigned long long)sm.qn[2]);
  }
}

// Generic path: any d, any K.  One point per thread per iteration of a
// grid-stride loop; FP32 direct-form screen with the same bound and FP64
// re-decision as the re-check of the fused kernel; exact integer sums with
// 64-bit atomics into this block's own partial row.
__global__ void __launch_bounds__(kThreads) assign_generic_kernel(GenericArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  if (a.ls->done) return;
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
    a.labels[i] = kb;
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

size_t fast_smem_bytes(int d, int kpad, int k) {
  const int dp = d + 1, win = 2 * d + 1;
  size_t b = (size_t)kpad * dp * 8 + (size_t)kWarps * k * dp * 8 + (size_t)kQueueCap * 4 +
             (size_t)k * 16 + (size_t)kWarps * k * win * 4 + 16;
  return (b + 15) & ~size_t(15);
}

template <int D>
static cudaError_t launch_fast_d(int grid, size_t smem, cudaStream_t st, const FastArgs& a) {
  auto fn = assign_fast_kernel<D>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  fn<<<grid, kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

template <int D>
static int blocks_d(size_t smem) {
  int nb = 0;
  cudaFuncSetAttribute(assign_fast_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, assign_fast_kernel<D>, kThreads, smem) != cudaSuccess)
    return 1;
  return nb > 0 ? nb : 1;
}

int fast_blocks_per_sm(int d, size_t smem) {
  switch (d) {
    case 1: return blocks_d<1>(smem);
    case 2: return blocks_d<2>(smem);
    case 3: return blocks_d<3>(smem);
    default: return blocks_d<4>(smem);
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

size_t generic_smem_bytes(int, int) { return 0; }

cudaError_t launch_assign_generic(int grid, size_t smem, cudaStream_t st, const GenericArgs& a) {
  assign_generic_kernel<<<grid, kThreads, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace km
