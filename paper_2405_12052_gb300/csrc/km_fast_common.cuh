// Device helpers of the FP32 fused assignment kernels (the FFMA2 screen and
// the tcgen05 TF32 screen): paired FP32 arithmetic, the exact fixed-point limb
// split of a coordinate, the FP32 direct-form re-check with its rigorous
// bound and FP64 fallback in the oracle's order, and the 32-bit sum windows.
#pragma once
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

__device__ __forceinline__ unsigned long long fadd2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long fsub2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ unsigned long long dup2(float v) { return pack2(v, v); }

// Flush the warp's windows (nwin of them) into the block's int64 totals.  acc
// columns per centroid: 0..D-1 coordinate sums, D the count (the layout of
// the per-block partials); window slots: 0 the count, 1..D the high limbs,
// D+1..2D the low limbs.
template <int D>
__device__ __forceinline__ void flush_windows(uint32_t* wwarp, long long* acc, int k, int nwin, int lane,
                                              uint32_t bias_hi, uint32_t bias_lo) {
  constexpr int DP = D + 1, WIN = 2 * D + 1;
  const int half = (k + 1) * WIN;
  __syncwarp();
  for (int s = lane; s < k * DP; s += 32) {
    const int kk = s / DP, j = s - kk * DP;
    long long v = 0;
    for (int h = 0; h < nwin; ++h) {
      const uint32_t* w = wwarp + h * half + kk * WIN;
      const uint32_t c = w[0];
      if (j == D) {
        v += (long long)c;
      } else {
        const int hi = (int)(w[1 + j] - c * bias_hi);  // exact: |sum| < 2^30
        const int lo = (int)(w[1 + D + j] - c * bias_lo);
        v += ((long long)hi << 22) + (long long)lo;
      }
    }
    if (v) atomicAdd(reinterpret_cast<unsigned long long*>(&acc[s]), (unsigned long long)v);
  }
  __syncwarp();
  for (int s = lane; s < nwin * half; s += 32) wwarp[s] = 0u;
  __syncwarp();
}

}  // namespace
}  // namespace km
