// Screen tables of the fused assignment kernel from the current centroids,
// shared by the single-context update and the batched update (one block;
// every thread of the block calls it).
//
// For centroids mu (k x d, FP64), the data shift s and A_max >= max_i
// fl32 ||fl(x_i - s)||^2: c~_k = fl32(mu_k - s) (ctil4), B_k = ||c~_k||^2 in
// FP64, and the screen r_k = M + 2^sigma (||c~_k||^2 - 2 x~.c~_k) in one
// binade [2^eM, 2^(eM+1)) chosen so that an index of L = ceil(log2 kpad) bits
// packed below the value keeps positive floats in value order; the flag
// constants bound every rounding of the chain, of x~ and c~, and the
// oracle's own FP64 rounding (see the fused kernel).  tab2 holds, per
// centroid, d packed pairs (a_kj, a_kj) with a_kj = -2^(sigma+1) c~_kj and the
// pair (n_k, n_k), n_k = fl32(M + 2^sigma B_k); padding centroids k..kpad-1
// get zero coefficients and the largest value of the binade.
#pragma once
#include "km_internal.cuh"

namespace km {

static __device__ void fast_screen_tables(const double* mu, const float* shift, float A_max, int k, int d, int kpad,
                                          double tie_rel, float4* ctil4, IterConst* ic_out,
                                          unsigned long long* tab2, double* sB) {
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int nth = blockDim.x * blockDim.y;
  __shared__ int sh_sigma;
  __shared__ double sh_M, sh_dummy;
  for (int c = tid; c < k; c += nth) {
    float cv[4] = {0.f, 0.f, 0.f, 0.f};
    double B = 0.0;
    for (int j = 0; j < d; ++j) {
      cv[j] = __double2float_rn(__dsub_rn(mu[(size_t)c * d + j], (double)shift[j]));
      B = __dadd_rn(B, __dmul_rn((double)cv[j], (double)cv[j]));
    }
    ctil4[c] = make_float4(cv[0], cv[1], cv[2], cv[3]);
    sB[c] = B;
  }
  __syncthreads();
  if (tid == 0) {
    double bmax = 0.0;
    for (int c = 0; c < k; ++c) bmax = fmax(bmax, sB[c]);
        int L = 1;
    while ((1 << L) < kpad) ++L;
    int E;
    double frac, hw;
    if (L <= 6) {
      const int base = 1 << (7 - L), step = 1 << (9 - L);
      E = base + ((127 - base) / step) * step;
      frac = 1.5; hw = 0.5;
    } else if (L == 7) {
      E = 125; frac = 1.25; hw = 0.25;
    } else {
      E = 126; frac = 1.375; hw = 0.125;
    }
    const int eM = E - 127;
    const double M = ldexp(frac, eM);
    const double top = ldexp(hw, eM);
    const double P = (A_max * (1.0 + 0x1p-20) + 2.0 * bmax) * (1.0 + 0x1p-10) + 1e-300;
    int sigma = ilogb(top / P);
    if (ldexp(P, sigma) >= top) sigma -= 1;
    sigma = max(-120, min(120, sigma));
    const double G = ldexp(1.0, sigma - eM + 23);
    const double u = 0x1p-24, u64x = 4.1 * 0x1p-53;
    IterConst ic;
    ic.M = (float)M;
    ic.L = L;
    ic.mul = 1u << L;
    ic.bitsM_low = __float_as_uint(ic.M) & ((1u << (32 - L)) - 1u);
    ic.G = (float)G;
    ic.thr_c0 = __double2float_ru(((double)(d + 1) + 2.0 + (8.002 * u + u64x * (d + 1)) * bmax * G) *
                                  (1.0 + 1e-4));
    ic.thr_cA = __double2float_ru((4.001 * u + u64x * (d + 1)) * G * (1.0 + 1e-4) * (1.0 + 1e-5));
    ic.tau = __double2float_ru(tie_rel * (1.0 + 1e-4));
    ic.B_max = __double2float_ru(bmax);
    ic.pad[0] = ic.pad[1] = ic.pad[2] = 0.f;
    *ic_out = ic;
    sh_sigma = sigma;
    sh_M = M;
    sh_dummy = (L <= 6 ? ldexp(2.0 - 0x1p-23, eM) : ldexp(1.5 - 0x1p-23, eM));
  }
  __syncthreads();
  const int sigma = sh_sigma, dp = d + 1;
  const float scale = -ldexpf(1.0f, sigma + 1);
  for (int c = tid; c < kpad; c += nth) {
    unsigned long long* row = tab2 + (size_t)c * dp;
    if (c < k) {
      const float4 cv4 = ctil4[c];
      const float cv[4] = {cv4.x, cv4.y, cv4.z, cv4.w};
      for (int j = 0; j < d; ++j) {
        const uint32_t b = __float_as_uint(__fmul_rn(cv[j], scale));
        row[j] = ((unsigned long long)b << 32) | b;
      }
      const uint32_t nb = __float_as_uint(__double2float_rn(sh_M + ldexp(sB[c], sigma)));
      row[d] = ((unsigned long long)nb << 32) | nb;
    } else {
      for (int j = 0; j < d; ++j) row[j] = 0ull;
      const uint32_t nb = __float_as_uint((float)sh_dummy);
      row[d] = ((unsigned long long)nb << 32) | nb;
    }
  }
}

}  // namespace km
