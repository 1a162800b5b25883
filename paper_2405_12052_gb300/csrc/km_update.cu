// Mean calculation and convergence error of Lloyd's algorithm (paper,
// section "The Lloyd's algorithm", step 3, and section "Serial Lloyd's
// algorithm"), plus the per-dataset scans that size the FP32 screen and the
// fixed-point grid.
//
// reduce_update_kernel: every block sums its slice of the per-block int64
// partials in int128 (rows in a fixed order), the last block to finish
// (integer ticket) adds the row-block sums in a fixed order, divides
// mu_k = S_k / n_k (an empty cluster keeps mu_k), forms E^2 with a fixed-order
// tree, tests the stop rule, and writes the next step's screen tables.
#include "km_internal.cuh"
#include "km_tables.cuh"

namespace km {

namespace {

__device__ __forceinline__ double i128_to_double(long long lo_s, long long hi_s) {
  // value = hi * 2^64 + (unsigned)lo, two's complement; correctly rounded.
  unsigned long long lo = (unsigned long long)lo_s, hi = (unsigned long long)hi_s;
  bool neg = (long long)hi < 0;
  if (neg) {  // negate the 128-bit value
    lo = ~lo + 1ull;
    hi = ~hi + (lo == 0ull ? 1ull : 0ull);
  }
  double r;
  if (hi == 0ull) {
    r = __ull2double_rn(lo);
  } else {
    int sh = 64 - __clzll((long long)hi);  // bits used in hi
    unsigned long long top = (hi << (64 - sh)) | (lo >> sh);
    unsigned long long rest = lo << (64 - sh);
    if (rest) top |= 1ull;  // sticky bit, 11 places below the rounding point
    r = ldexp(__ull2double_rn(top), sh);
  }
  return neg ? -r : r;
}

__device__ __forceinline__ void add128(unsigned long long& lo, long long& hi, long long v) {
  unsigned long long nl = lo + (unsigned long long)v;
  hi += (v < 0 ? -1ll : 0ll) + (nl < lo ? 1ll : 0ll);
  lo = nl;
}
__device__ __forceinline__ void add128p(unsigned long long& lo, long long& hi, unsigned long long vl,
                                        long long vh) {
  unsigned long long nl = lo + vl;
  hi += vh + (nl < lo ? 1ll : 0ll);
  lo = nl;
}

__device__ __forceinline__ uint32_t ordered(float f) {
  uint32_t b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// Screen tables for the next step from mu (one block).  Fused path: the
// tables of fast_screen_tables (km_tables.cuh); generic path: c~ and B_max
// only.
__device__ void prepare_tables(const UpdateArgs& a, double* sB) {
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int nth = blockDim.x * blockDim.y;
  const int k = a.k, d = a.d;
  if (a.fast) {
    fast_screen_tables(a.mu, a.dc->s, a.dc->A_max, k, d, a.kpad, a.tie_rel, a.ctil4, a.ic, a.tab2, sB);
  } else {
    __shared__ unsigned int sh_bmax_bits;
    if (tid == 0) sh_bmax_bits = 0u;
    __syncthreads();
    for (int c = tid; c < k; c += nth) {
      double B = 0.0;
      for (int j = 0; j < d; ++j) {
        const float cvj = __double2float_rn(__dsub_rn(a.mu[(size_t)c * d + j], (double)a.shift[j]));
        a.ctil[(size_t)c * d + j] = cvj;
        B = __dadd_rn(B, __dmul_rn((double)cvj, (double)cvj));
      }
      const float Bf = __double2float_ru(B);
      a.cnorm[c] = Bf;
      atomicMax(&sh_bmax_bits, __float_as_uint(Bf));  // B >= 0: bit order is value order
    }
    __syncthreads();
    if (tid == 0) *a.gen_bmax = __uint_as_float(sh_bmax_bits);
  }
  __syncthreads();
}

constexpr int kRedCols = 32, kRedRows = 8;

// The last step of the update, given the int128 column totals of RB row
// groups (the reduction's row blocks, or the shards of a sharded step) in
// s128 [RB][k][d+1][2]: totals added in row-group order, one conversion to
// FP64, the divide (an empty cluster keeps its centre), E^2 by a fixed-order
// tree, the stop test and the next step's screen tables.
__device__ void finish_update(const UpdateArgs& a, const long long* s128, int RB, double* sB, double* s_red,
                              int tid) {
  const int k = a.k, d = a.d, dp = d + 1, cols = k * dp;
  const int nth = kRedCols * kRedRows;
  int empty = 0;
  for (int c = tid; c < k; c += nth) {
    long long n = 0;
    for (int rb = 0; rb < RB; ++rb) n += s128[((size_t)rb * cols + (size_t)c * dp + d) * 2];
    a.counts[c] = n;
    empty += (n == 0);
  }
  __syncthreads();
  const int G0 = a.dc->G0;
  double e2p = 0.0;
  for (int q = tid; q < k * d; q += nth) {
    const int c = q / d, j = q - c * d;
    unsigned long long tl = 0ull;
    long long th = 0ll;
    for (int rb = 0; rb < RB; ++rb) {
      const long long* v = s128 + ((size_t)rb * cols + (size_t)c * dp + j) * 2;
      add128p(tl, th, (unsigned long long)v[0], v[1]);
    }
    const long long n = a.counts[c];
    const double old = a.mu[q];
    double nw = old;
    if (n > 0) nw = __ddiv_rn(ldexp(i128_to_double((long long)tl, th), G0), (double)n);
    const double df = __dsub_rn(nw, old);
    e2p = __dadd_rn(e2p, __dmul_rn(df, df));
    a.mu[q] = nw;
  }
  // fixed-order tree over threads
  s_red[tid] = e2p;
  __syncthreads();
  for (int w = nth / 2; w > 0; w >>= 1) {
    if (tid < w) s_red[tid] = __dadd_rn(s_red[tid], s_red[tid + w]);
    __syncthreads();
  }
  __shared__ int s_empty;
  if (tid == 0) s_empty = 0;
  __syncthreads();
  if (empty) atomicAdd(&s_empty, empty);
  __syncthreads();
  if (tid == 0) {
    LoopState* ls = a.ls;
    const double E2 = s_red[0];
    const double E = sqrt(E2);
    ls->E2 = E2;
    ls->E = E;
    ls->iter += 1;
    ls->empty = s_empty;
    const double esel = ls->e_mode == 1 ? E2 : E;
    if (esel < ls->tol) { ls->converged = 1; ls->done = 1; }
    if (ls->iter >= ls->max_iter) ls->done = 1;
    ls->last_flagged = ls->flagged;
    ls->last_fp64 = ls->fp64_decided;
    ls->last_overflowed = ls->overflowed;
    ls->flagged = 0ull;
    ls->fp64_decided = 0ull;
    ls->overflowed = 0ull;
    ls->ticket = 0u;
  }
  __syncthreads();
  prepare_tables(a, sB);
}


__global__ void __launch_bounds__(kRedCols * kRedRows) reduce_update_kernel(UpdateArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  double* sB = reinterpret_cast<double*>(smraw);  // [k] for the fused-path tables
  __shared__ unsigned long long s_lo[kRedRows][kRedCols];
  __shared__ long long s_hi[kRedRows][kRedCols];
  __shared__ bool s_last;
  __shared__ double s_red[kRedCols * kRedRows];
  if (a.ls->done) return;
  const int cols = a.k * (a.d + 1);
  const int col = blockIdx.x * kRedCols + threadIdx.x;
  const int tid = threadIdx.y * kRedCols + threadIdx.x;
  {
    unsigned long long lo = 0ull;
    long long hi = 0ll;
    if (col < cols) {
      for (int g = blockIdx.y * kRedRows + threadIdx.y; g < a.G; g += gridDim.y * kRedRows)
        add128(lo, hi, a.partials[(size_t)g * cols + col]);
    }
    s_lo[threadIdx.y][threadIdx.x] = lo;
    s_hi[threadIdx.y][threadIdx.x] = hi;
    __syncthreads();
    if (threadIdx.y == 0 && col < cols) {
      unsigned long long tl = 0ull;
      long long th = 0ll;
      for (int r = 0; r < kRedRows; ++r) add128p(tl, th, s_lo[r][threadIdx.x], s_hi[r][threadIdx.x]);
      long long* out = a.s128 + ((size_t)blockIdx.y * cols + col) * 2;
      out[0] = (long long)tl;
      out[1] = th;
    }
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) {
    const unsigned int t = atomicAdd(&a.ls->ticket, 1u);
    s_last = (t == gridDim.x * gridDim.y - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();

  finish_update(a, a.s128, (int)gridDim.y, sB, s_red, tid);
}

// One block of kRedCols x kRedRows threads: the mean calculation from the
// gathered column totals of R shards (rank order), as the last block above.
__global__ void __launch_bounds__(kRedCols * kRedRows) shard_update_kernel(UpdateArgs a, const long long* tables,
                                                                            int ranks) {
  extern __shared__ __align__(16) unsigned char smraw[];
  double* sB = reinterpret_cast<double*>(smraw);
  __shared__ double s_red[kRedCols * kRedRows];
  if (a.ls->done) return;
  finish_update(a, tables, ranks, sB, s_red, threadIdx.y * kRedCols + threadIdx.x);
}

// Column totals of this context's per-block partials: one int128 (two int64
// words, low word first) per column of [k][d+1]; integer sums, so exact.
__global__ void __launch_bounds__(kRedCols * kRedRows) shard_totals_kernel(UpdateArgs a, long long* out) {
  __shared__ unsigned long long s_lo[kRedRows][kRedCols];
  __shared__ long long s_hi[kRedRows][kRedCols];
  const int cols = a.k * (a.d + 1);
  const int col = blockIdx.x * kRedCols + threadIdx.x;
  unsigned long long lo = 0ull;
  long long hi = 0ll;
  if (col < cols)
    for (int g = threadIdx.y; g < a.G; g += kRedRows) add128(lo, hi, a.partials[(size_t)g * cols + col]);
  s_lo[threadIdx.y][threadIdx.x] = lo;
  s_hi[threadIdx.y][threadIdx.x] = hi;
  __syncthreads();
  if (threadIdx.y == 0 && col < cols) {
    unsigned long long tl = 0ull;
    long long th = 0ll;
    for (int r = 0; r < kRedRows; ++r) add128p(tl, th, s_lo[r][threadIdx.x], s_hi[r][threadIdx.x]);
    out[(size_t)col * 2] = (long long)tl;
    out[(size_t)col * 2 + 1] = th;
  }
}

__global__ void __launch_bounds__(256) prepare_kernel(UpdateArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  prepare_tables(a, reinterpret_cast<double*>(smraw));
}

__global__ void scan_range_kernel(const float* __restrict__ x, int64_t ld, int64_t n, int d,
                                  unsigned int* mn_ord, unsigned int* mx_ord,
                                  unsigned long long* nonfinite) {
  const int j = blockIdx.y;
  const float* row = x + (int64_t)j * ld;
  uint32_t lo = 0xffffffffu, hi = 0u;
  unsigned long long bad = 0;
  auto take = [&](float v) {
    if (!isfinite(v)) { ++bad; return; }
    const uint32_t o = ordered(v);
    lo = min(lo, o);
    hi = max(hi, o);
  };
  // four loads in flight per thread (min and max do not depend on the order)
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + 3 * stride < n; i += 4 * stride) {
    const float v0 = row[i], v1 = row[i + stride], v2 = row[i + 2 * stride], v3 = row[i + 3 * stride];
    take(v0);
    take(v1);
    take(v2);
    take(v3);
  }
  for (; i < n; i += stride) take(row[i]);
  for (int off = 16; off > 0; off >>= 1) {
    lo = min(lo, __shfl_down_sync(0xffffffffu, lo, off));
    hi = max(hi, __shfl_down_sync(0xffffffffu, hi, off));
    bad += __shfl_down_sync(0xffffffffu, bad, off);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMin(mn_ord + j, lo);
    atomicMax(mx_ord + j, hi);
    if (bad) atomicAdd(nonfinite, bad);
  }
}

// max_i of ||fl(x_i - s)||^2 evaluated exactly as the fused kernel does
// (first term a product, then fused multiply-adds in coordinate order).
__global__ void scan_amax_kernel(const float* __restrict__ x, int64_t ld, int64_t n, int d,
                                 const float* __restrict__ shift, unsigned int* amax_bits) {
  uint32_t best = 0u;
  // two points per thread and round, their coordinate loads issued together
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + stride < n; i += 2 * stride) {
    const int64_t i1 = i + stride;
    float t = __fsub_rn(x[i], shift[0]), u = __fsub_rn(x[i1], shift[0]);
    float A = __fmul_rn(t, t), B = __fmul_rn(u, u);
#pragma unroll 4
    for (int j = 1; j < d; ++j) {
      t = __fsub_rn(x[(int64_t)j * ld + i], shift[j]);
      u = __fsub_rn(x[(int64_t)j * ld + i1], shift[j]);
      A = __fmaf_rn(t, t, A);
      B = __fmaf_rn(u, u, B);
    }
    best = max(best, max(__float_as_uint(A), __float_as_uint(B)));
  }
  for (; i < n; i += stride) {
    float t = __fsub_rn(x[i], shift[0]);
    float A = __fmul_rn(t, t);
    for (int j = 1; j < d; ++j) {
      t = __fsub_rn(x[(int64_t)j * ld + i], shift[j]);
      A = __fmaf_rn(t, t, A);
    }
    best = max(best, __float_as_uint(A));
  }
  for (int off = 16; off > 0; off >>= 1) best = max(best, __shfl_down_sync(0xffffffffu, best, off));
  if ((threadIdx.x & 31) == 0) atomicMax(amax_bits, best);
}

__global__ void aos_to_soa_kernel(const float* __restrict__ src, int64_t lds, int64_t n, int d,
                                  float* __restrict__ dst, int64_t ldd) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    for (int j = 0; j < d; ++j) dst[(int64_t)j * ldd + i] = src[i * lds + j];
  }
}

}  // namespace

cudaError_t launch_update(cudaStream_t st, const UpdateArgs& a) {
  const int cols = a.k * (a.d + 1);
  dim3 grid((cols + kRedCols - 1) / kRedCols, a.RB), block(kRedCols, kRedRows);
  const size_t smem = (size_t)(a.fast ? a.k : 0) * sizeof(double);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(reduce_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  reduce_update_kernel<<<grid, block, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_shard_totals(cudaStream_t st, const UpdateArgs& a, long long* out) {
  const int cols = a.k * (a.d + 1);
  shard_totals_kernel<<<(cols + kRedCols - 1) / kRedCols, dim3(kRedCols, kRedRows), 0, st>>>(a, out);
  return cudaGetLastError();
}

cudaError_t launch_shard_update(cudaStream_t st, const UpdateArgs& a, const long long* tables, int ranks) {
  const size_t smem = (size_t)(a.fast ? a.k : 0) * sizeof(double);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(shard_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  shard_update_kernel<<<1, dim3(kRedCols, kRedRows), smem, st>>>(a, tables, ranks);
  return cudaGetLastError();
}

cudaError_t launch_prepare(cudaStream_t st, const UpdateArgs& a) {
  const size_t smem = (size_t)(a.fast ? a.k : 0) * sizeof(double);
  prepare_kernel<<<1, 256, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_scan_range(const float* x, int64_t ld, int64_t n, int d, float* mn, float* mx,
                              unsigned long long* nonfinite, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(mn, 0xff, sizeof(float) * d, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(mx, 0x00, sizeof(float) * d, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(nonfinite, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 1216);
  dim3 grid((unsigned)std::max<int64_t>(blocks, 1), d);
  scan_range_kernel<<<grid, 256, 0, st>>>(x, ld, n, d, reinterpret_cast<unsigned int*>(mn),
                                          reinterpret_cast<unsigned int*>(mx), nonfinite);
  return cudaGetLastError();
}

cudaError_t launch_scan_amax(const float* x, int64_t ld, int64_t n, int d, const float* shift,
                             float* amax, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(amax, 0, sizeof(float), st);
  if (e != cudaSuccess) return e;
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 1216);
  scan_amax_kernel<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, st>>>(
      x, ld, n, d, shift, reinterpret_cast<unsigned int*>(amax));
  return cudaGetLastError();
}

cudaError_t launch_aos_to_soa(const float* src, int64_t lds, int64_t n, int d, float* dst,
                              int64_t ldd, cudaStream_t st) {
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);
  aos_to_soa_kernel<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, st>>>(src, lds, n, d, dst, ldd);
  return cudaGetLastError();
}

}  // namespace km
