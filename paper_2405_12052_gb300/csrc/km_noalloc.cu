// km_lloyd_step_noalloc: one Lloyd step on caller-owned device buffers that
// allocates no memory at all.
//
// Some callers cannot call cudaMalloc: code that runs where the process's
// allocator must not be entered (inside a region whose memory budget was
// fixed up front, in a real-time loop that forbids allocation after start-up,
// or inside another framework that owns every device allocation).  For them
// this entry point keeps its only scratch -- the per-block partial sums of the
// assignment kernel and a range word -- in a file-scope __device__ array of
// fixed size, which every GPU that loads the library holds until the process
// exits.  The caller passes the points, the starting centroids and every
// output buffer.
//
// The step is a variant of the generic assignment kernel: FP32 direct-form
// distances with a rigorous error bound, FP64 re-decision (in the order
// sum_j (x_j - mu_kj)^2, ties to the lowest k) of every point the bound leaves
// open or whose two nearest are within 1e-5 relative, exact fixed-point
// per-block sums, then a fixed-order int128 reduction, the divide and E^2.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/km.h"

namespace {

constexpr int kNaMaxBlocks = 304;   // blocks of the assignment variant
constexpr int kNaMaxCols = 256;     // K * (d + 1)
constexpr int kNaThreads = 256;
constexpr long long kNaMaxPointsPerBlock = 1ll << 19;
constexpr int kNaMaxDevices = 64;

struct NaScratch {
  unsigned int absmax_bits;  // max |x| as float bits (bit order = value order for |x|)
  unsigned int pad[63];
  long long partials[kNaMaxBlocks * kNaMaxCols];  // [block][k][d+1]: coordinate sums, count
};

// The scratch: about 0.6 MB per device, shared by every call on that device.
static __device__ __align__(256) NaScratch g_na_scratch;

constexpr float kNaU = 5.9604644775390625e-08f;  // 2^-24

__global__ void na_absmax_kernel(const float* __restrict__ x, int64_t ld, int64_t n, int d,
                                 NaScratch* sc) {
  unsigned int best = 0u;
  for (int j = 0; j < d; ++j)
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
      best = max(best, __float_as_uint(fabsf(x[(int64_t)j * ld + i])));
  for (int off = 16; off > 0; off >>= 1) best = max(best, __shfl_down_sync(0xffffffffu, best, off));
  if ((threadIdx.x & 31) == 0) atomicMax(&sc->absmax_bits, best);
}

// Fixed-point grid from max |x|: x = hi 2^(G0+22) + lo 2^G0, |hi| <= 2^21.
__device__ __forceinline__ int na_grid_ex(unsigned int absmax_bits) {
  const float amax = __uint_as_float(absmax_bits);
  if (!(amax > 0.f)) return -104;
  int e;
  frexpf(amax, &e);  // amax = m 2^e, m in [0.5, 1)
  int ex = e + 1;    // |x| < 2^(ex - 1)
  return max(-104, min(ex, 100));  // C_lo = 1.5 * 2^(ex - 21) stays a normal float
}

__global__ void __launch_bounds__(kNaThreads) na_assign_kernel(
    const float* __restrict__ x, int64_t ld, int64_t n, int d, int k, const double* __restrict__ mu,
    int32_t* __restrict__ labels, NaScratch* sc, float tau) {
  extern __shared__ float s_c[];  // [k][d] fp32 centroids, then B_max
  const int dp = d + 1;
  unsigned long long* row = reinterpret_cast<unsigned long long*>(sc->partials) + (size_t)blockIdx.x * k * dp;
  for (int q = threadIdx.x; q < k * dp; q += blockDim.x) row[q] = 0ull;  // this block's row starts at zero
  __shared__ unsigned int s_bmax;
  if (threadIdx.x == 0) s_bmax = 0u;
  __syncthreads();
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    float b = 0.f;
    for (int j = 0; j < d; ++j) {
      const float v = __double2float_rn(mu[(size_t)c * d + j]);
      s_c[c * d + j] = v;
      b = __fmaf_ru(v, v, b);
    }
    atomicMax(&s_bmax, __float_as_uint(b * 1.0001f));
  }
  __syncthreads();
  const float B_max = __uint_as_float(s_bmax), sB = sqrtf(B_max);
  const int ex = na_grid_ex(sc->absmax_bits);
  const float C_hi = ldexpf(1.5f, ex + 1), C_lo = ldexpf(1.5f, ex - 21);
  const unsigned int bC_hi = __float_as_uint(C_hi), bC_lo = __float_as_uint(C_lo);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float A = 0.f;
    for (int j = 0; j < d; ++j) {
      const float v = x[(int64_t)j * ld + i];
      A = __fmaf_ru(v, v, A);
    }
    float best = 3.0e38f, second = 3.0e38f;
    int kb = 0;
    for (int c = 0; c < k; ++c) {
      float dv = 0.f;
      for (int j = 0; j < d; ++j) {
        const float t = __fsub_rn(x[(int64_t)j * ld + i], s_c[c * d + j]);
        dv = __fmaf_rn(t, t, dv);
      }
      if (dv < best) { second = best; best = dv; kb = c; }
      else if (dv < second) { second = dv; }
    }
    if (k > 1) {
      // |fp32 direct form - exact D| <= 1.01 u [(d+2) D + 2 sqrt(D)(||x|| + ||c||)],
      // plus the FP64 rounding of the oracle-order sum
      const float sA = sqrtf(A), AB = A + B_max;
      const float g64 = 4.6e-16f * (float)(d + 1) * AB + 1e-30f;
      const float e1 = 1.01f * kNaU * ((float)(d + 2) * best + 2.f * sqrtf(best) * (sA + sB)) + g64;
      const float e2 = 1.01f * kNaU * ((float)(d + 2) * second + 2.f * sqrtf(second) * (sA + sB)) + g64;
      const float lo2 = second - e2, hi1 = best + e1;
      if (!((lo2 > hi1) && (lo2 - hi1 > tau * (second + e2)))) {
        double bd = 0.0;
        kb = 0;
        for (int c = 0; c < k; ++c) {
          double acc = 0.0;
          for (int j = 0; j < d; ++j) {
            const double t = __dsub_rn((double)x[(int64_t)j * ld + i], mu[(size_t)c * d + j]);
            acc = __dadd_rn(acc, __dmul_rn(t, t));
          }
          if (c == 0 || acc < bd) { bd = acc; kb = c; }
        }
      }
    }
    labels[i] = kb;
    unsigned long long* r = row + (size_t)kb * dp;
    for (int j = 0; j < d; ++j) {
      const float v = x[(int64_t)j * ld + i];
      const float t = __fadd_rn(v, C_hi);
      const float h = __fsub_rn(t, C_hi);
      const float rr = __fsub_rn(v, h);
      const float t2 = __fadd_rn(rr, C_lo);
      const long long hi = (long long)(int)(__float_as_uint(t) - bC_hi);
      const long long lo = (long long)(int)(__float_as_uint(t2) - bC_lo);
      atomicAdd(r + j, (unsigned long long)((hi << 22) + lo));
    }
    atomicAdd(r + d, 1ull);
  }
}

__device__ __forceinline__ double na_i128_to_double(unsigned long long lo, long long hs) {
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
    if (lo << (64 - sh)) top |= 1ull;
    r = ldexp(__ull2double_rn(top), sh);
  }
  return neg ? -r : r;
}

// One block: per column, the G block rows summed in index order in int128;
// then counts, mu_k = S_k / n_k (an empty cluster keeps mu_k) and
// E^2 = sum_k ||mu_k - mu_in_k||^2 by a fixed-order tree.
__global__ void __launch_bounds__(kNaThreads) na_reduce_kernel(const NaScratch* sc, int G, int d, int k,
                                                                const double* __restrict__ mu_in,
                                                                double* __restrict__ mu_out,
                                                                int64_t* __restrict__ counts, double* e2_out) {
  __shared__ long long s_cnt[kNaMaxCols];
  __shared__ double s_red[kNaThreads];
  const int dp = d + 1, cols = k * dp, tid = threadIdx.x;
  // Data the fixed-point grid cannot hold (a NaN, an infinity or |x| >= 2^99;
  // 0x71000000 is the bit pattern of 2^99): every output is marked invalid.
  if (!(sc->absmax_bits < 0x71000000u)) {
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    for (int q = tid; q < k * d; q += blockDim.x) mu_out[q] = nan;
    for (int c = tid; c < k; c += blockDim.x) counts[c] = -1;
    if (tid == 0) *e2_out = nan;
    return;
  }
  for (int c = tid; c < k; c += blockDim.x) {
    long long nsum = 0;
    for (int g = 0; g < G; ++g) nsum += sc->partials[(size_t)g * cols + (size_t)c * dp + d];
    s_cnt[c] = nsum;
    counts[c] = nsum;
  }
  __syncthreads();
  const int G0 = na_grid_ex(sc->absmax_bits) - 44;
  double e2p = 0.0;
  for (int q = tid; q < k * d; q += blockDim.x) {
    const int c = q / d, j = q - c * d;
    unsigned long long lo = 0ull;
    long long hi = 0ll;
    for (int g = 0; g < G; ++g) {
      const long long v = sc->partials[(size_t)g * cols + (size_t)c * dp + j];
      const unsigned long long nl = lo + (unsigned long long)v;
      hi += (v < 0 ? -1ll : 0ll) + (nl < lo ? 1ll : 0ll);
      lo = nl;
    }
    const double old = mu_in[q];
    double nw = old;
    if (s_cnt[c] > 0) nw = __ddiv_rn(ldexp(na_i128_to_double(lo, hi), G0), (double)s_cnt[c]);
    mu_out[q] = nw;
    const double df = __dsub_rn(nw, old);
    e2p = __dadd_rn(e2p, __dmul_rn(df, df));
  }
  s_red[tid] = e2p;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (tid < w) s_red[tid] = __dadd_rn(s_red[tid], s_red[tid + w]);
    __syncthreads();
  }
  if (tid == 0) *e2_out = s_red[0];
}

std::mutex g_na_mutex;
void* g_na_ptr[kNaMaxDevices] = {};
void* g_na_ctx[kNaMaxDevices] = {};  // the context the cached address belongs to

// The calling thread's current CUDA context (a driver handle), looked up
// through the runtime's driver entry point so that libcuda is not linked.
void* na_current_context() {
  using GetCurrent = int (*)(void**);
  static GetCurrent fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      f = nullptr;
    return reinterpret_cast<GetCurrent>(f);
  }();
  void* ctx = nullptr;
  if (!fn || fn(&ctx) != 0) return nullptr;
  return ctx;
}

km_status na_fail(char* errbuf, int32_t errlen, km_status s, const char* msg) {
  if (errbuf && errlen > 0) std::snprintf(errbuf, (size_t)errlen, "%s", msg);
  return s;
}

}  // namespace

extern "C" km_status km_lloyd_step_noalloc(const float* x, int64_t ld, int64_t n, int32_t d, int32_t k,
                                           const double* mu_in, int32_t* labels, double* mu_out,
                                           int64_t* counts, double* e2_out, void* stream, char* errbuf,
                                           int32_t errlen) {
  if (errbuf && errlen > 0) errbuf[0] = '\0';
  if (!x || !mu_in || !labels || !mu_out || !counts || !e2_out)
    return na_fail(errbuf, errlen, KM_EINVAL, "km_lloyd_step_noalloc: null pointer argument");
  if (n < 1 || d < 1 || k < 1 || k > n || ld < n)
    return na_fail(errbuf, errlen, KM_EINVAL, "km_lloyd_step_noalloc: need n >= k >= 1, d >= 1, ld >= n");
  if ((int64_t)k * (d + 1) > kNaMaxCols)
    return na_fail(errbuf, errlen, KM_EINVAL,
                   "km_lloyd_step_noalloc: K*(d+1) exceeds the fixed scratch limit of 256 columns");
  int64_t G = (n + kNaThreads - 1) / kNaThreads;
  if (G > kNaMaxBlocks) G = kNaMaxBlocks;
  if (n > G * kNaMaxPointsPerBlock)
    return na_fail(errbuf, errlen, KM_EINVAL,
                   "km_lloyd_step_noalloc: N exceeds the fixed scratch limit of 304 * 2^19 points");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return na_fail(errbuf, errlen, KM_ECUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kNaMaxDevices)
    return na_fail(errbuf, errlen, KM_ECUDA, "km_lloyd_step_noalloc: device ordinal out of range");
  NaScratch* sc = nullptr;
  {
    // Set-up, once per device (and again after the device's context was
    // destroyed and re-created, e.g. by cudaDeviceReset, which reloads the
    // module), with that device current: the host-side name of the array is
    // only a stand-in, so its device address is looked up.
    // (No context yet, or no way to ask: the address is looked up every time.)
    void* ctx = na_current_context();
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev] || ctx != g_na_ctx[dev] || !ctx) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_na_scratch);
      if (e != cudaSuccess || !p)
        return na_fail(errbuf, errlen, KM_ECUDA, "km_lloyd_step_noalloc: cudaGetSymbolAddress failed");
      g_na_ptr[dev] = p;
      g_na_ctx[dev] = ctx;
    }
    sc = static_cast<NaScratch*>(g_na_ptr[dev]);
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  e = cudaMemsetAsync(&sc->absmax_bits, 0, sizeof(unsigned int), st);  // must start at zero
  if (e == cudaSuccess) {
    const int64_t gb = std::min<int64_t>((n + 255) / 256, 1216);
    na_absmax_kernel<<<(unsigned)gb, 256, 0, st>>>(x, ld, n, d, sc);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    const size_t smem = sizeof(float) * (size_t)k * d;
    na_assign_kernel<<<(unsigned)G, kNaThreads, smem, st>>>(x, ld, n, d, k, mu_in, labels, sc,
                                                            (float)(1e-5 * (1.0 + 1e-4)));
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    na_reduce_kernel<<<1, kNaThreads, 0, st>>>(sc, (int)G, d, k, mu_in, mu_out, counts, e2_out);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return na_fail(errbuf, errlen, KM_ECUDA, cudaGetErrorString(e));
  return KM_OK;
}
