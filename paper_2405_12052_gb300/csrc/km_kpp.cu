// k-means++ seeding on the GPU (D^2 sampling, Arthur and Vassilvitskii
// 2007), the initialisation the configurations name for the start of
// Lloyd's algorithm (paper, section "The Lloyd's algorithm", step 1: initial
// centres).  The K uniforms are inputs, so a run is reproducible and the
// oracle can take the same ones.
//
// Pick 0 is floor(u_0 N).  Pick c >= 1: D^2_i = min over chosen centres
// of sum_j (x_ij - m_j)^2 in FP64 (coordinates in order, no fused
// multiply-add: the oracle's expression), total = sum_i D^2_i, target =
// u_c * total, and the pick is the first i whose running sum exceeds the
// target (the last point if none does).  The sums are taken over chunks of
// kKppChunk points (fixed-order tree per chunk), then over the chunk sums in
// order; so the pick equals a sequential scan's except when the target lies
// within FP64 rounding of a running-sum boundary.
#include "km_internal.cuh"

namespace km {

namespace {

constexpr int kKppChunk = 4096;
constexpr int kKppThreads = 256;

__device__ __forceinline__ double kpp_d2(const float* x, int64_t ld, int64_t i, int d, const double* m) {
  double acc = 0.0;
  for (int j = 0; j < d; ++j) {
    const double t = __dsub_rn((double)x[(int64_t)j * ld + i], m[j]);
    acc = __dadd_rn(acc, __dmul_rn(t, t));
  }
  return acc;
}

// D^2 against centre c (the minimum with the previous D^2 for c > 0) and
// the chunk sums.  One block per chunk; thread t takes points t, t + 256, ...
// of the chunk, then a fixed-order tree.
__global__ void __launch_bounds__(kKppThreads) kpp_d2_kernel(const float* __restrict__ x, int64_t ld, int64_t n,
                                                             int d, const double* __restrict__ mu, int c,
                                                             double* d2, double* chunk_sum) {
  __shared__ double s_red[kKppThreads];
  __shared__ double s_m[kMaxKppD];
  if (threadIdx.x < d) s_m[threadIdx.x] = mu[(size_t)c * d + threadIdx.x];
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kKppChunk;
  double acc = 0.0;
  for (int q = threadIdx.x; q < kKppChunk; q += kKppThreads) {
    const int64_t i = base + q;
    if (i >= n) break;
    double v = kpp_d2(x, ld, i, d, s_m);
    if (c > 0) v = fmin(v, d2[i]);
    d2[i] = v;
    acc = __dadd_rn(acc, v);
  }
  s_red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = kKppThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) s_red[threadIdx.x] = __dadd_rn(s_red[threadIdx.x], s_red[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) chunk_sum[blockIdx.x] = s_red[0];
}

// Inclusive scan of v[0..m) in place by one block (Hillis-Steele per
// 1024-wide pass plus the running carry): a fixed order.
__device__ void block_scan(double* v, int m, double* s_tmp) {
  __shared__ double carry;
  if (threadIdx.x == 0) carry = 0.0;
  __syncthreads();
  for (int base = 0; base < m; base += blockDim.x) {
    const int q = base + threadIdx.x;
    s_tmp[threadIdx.x] = q < m ? v[q] : 0.0;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
      const double a = threadIdx.x >= (unsigned)off ? s_tmp[threadIdx.x - off] : 0.0;
      __syncthreads();
      s_tmp[threadIdx.x] = __dadd_rn(s_tmp[threadIdx.x], a);
      __syncthreads();
    }
    if (q < m) v[q] = __dadd_rn(carry, s_tmp[threadIdx.x]);
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = __dadd_rn(carry, s_tmp[threadIdx.x]);
    __syncthreads();
  }
}

// One block (1024 threads): the pick of round c and its coordinates.
__global__ void __launch_bounds__(1024) kpp_pick_kernel(const float* __restrict__ x, int64_t ld, int64_t n, int d,
                                                        const double* __restrict__ u, int c, double* chunk_sum,
                                                        int nchunks, const double* d2, double* mu, int64_t* idx,
                                                        double* scan) {
  __shared__ double s_tmp[1024];
  __shared__ int64_t s_pick;
  __shared__ int s_chunk;
  if (c == 0) {
    if (threadIdx.x == 0) {
      int64_t f = (int64_t)floor(u[0] * (double)n);
      if (f >= n) f = n - 1;
      if (f < 0) f = 0;
      s_pick = f;
    }
  } else {
    block_scan(chunk_sum, nchunks, s_tmp);  // inclusive prefix of the chunk sums
    const double total = chunk_sum[nchunks - 1];
    const double target = __dmul_rn(u[c], total);
    if (threadIdx.x == 0) s_chunk = nchunks;
    __syncthreads();
    for (int b = threadIdx.x; b < nchunks; b += blockDim.x)
      if (chunk_sum[b] > target) atomicMin(&s_chunk, b);
    __syncthreads();
    const int b = s_chunk;
    if (b == nchunks) {
      if (threadIdx.x == 0) s_pick = n - 1;  // no running sum exceeds the target
    } else {
      const double before = b > 0 ? chunk_sum[b - 1] : 0.0;
      const int64_t i0 = (int64_t)b * kKppChunk;
      const int m = (int)min((int64_t)kKppChunk, n - i0);
      for (int q = threadIdx.x; q < m; q += blockDim.x) scan[q] = d2[i0 + q];
      __syncthreads();
      block_scan(scan, m, s_tmp);
      if (threadIdx.x == 0) s_pick = i0 + m - 1;  // when rounding leaves none in the chunk
      __syncthreads();
      __shared__ unsigned long long s_first;
      if (threadIdx.x == 0) s_first = (unsigned long long)m;
      __syncthreads();
      for (int q = threadIdx.x; q < m; q += blockDim.x)
        if (__dadd_rn(before, scan[q]) > target) atomicMin(&s_first, (unsigned long long)q);
      __syncthreads();
      if (threadIdx.x == 0 && s_first < (unsigned long long)m) s_pick = i0 + (int64_t)s_first;
    }
  }
  __syncthreads();
  const int64_t pick = s_pick;
  if (threadIdx.x < d) mu[(size_t)c * d + threadIdx.x] = (double)x[(int64_t)threadIdx.x * ld + pick];
  if (threadIdx.x == 0) idx[c] = pick;
}

}  // namespace

int64_t kpp_chunks(int64_t n) { return (n + kKppChunk - 1) / kKppChunk; }

cudaError_t launch_kmeanspp(const float* x, int64_t ld, int64_t n, int d, int k, const double* u, double* mu,
                            int64_t* idx, double* d2, double* chunk_sum, double* scan, cudaStream_t st) {
  const int nch = (int)kpp_chunks(n);
  for (int c = 0; c < k; ++c) {
    if (c > 0) {
      kpp_d2_kernel<<<nch, kKppThreads, 0, st>>>(x, ld, n, d, mu, c - 1, d2, chunk_sum);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
    kpp_pick_kernel<<<1, 1024, 0, st>>>(x, ld, n, d, u, c, chunk_sum, nch, d2, mu, idx, scan);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace km
