// The k-means objective sum_i ||x_i - mu_{z_i}||^2 (the quantity Lloyd's
// iteration decreases; paper, section "The Lloyd's algorithm") of the
// current labels and centroids, in FP64: per point the squared distance with
// coordinates in order (no fused multiply-add), summed in index order within
// chunks of 65536 points, the chunk sums then added in chunk order.
#include <algorithm>

#include "km_internal.cuh"

namespace km {

namespace {

constexpr int kObjChunk = 65536;

// One warp per chunk: lanes form 32 distances at a time, lane 0 adds them in
// index order.
template <typename L>
__global__ void __launch_bounds__(256) objective_kernel(const float* __restrict__ x, int64_t ld, int64_t n, int d,
                                                        const double* __restrict__ mu,
                                                        const L* __restrict__ z, double* part,
                                                        int nchunks) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (w >= nchunks) return;
  const int64_t lo = (int64_t)w * kObjChunk, hi = min(lo + kObjChunk, n);
  double s = 0.0;
  for (int64_t b = lo; b < hi; b += 32) {
    const int64_t i = b + lane;
    double dv = 0.0;
    if (i < hi) {
      const double* m = mu + (size_t)z[i] * d;
      for (int j = 0; j < d; ++j) {
        const double t = __dsub_rn((double)x[(int64_t)j * ld + i], m[j]);
        dv = __dadd_rn(dv, __dmul_rn(t, t));
      }
    }
    const int cnt = (int)min((int64_t)32, hi - b);
    for (int q = 0; q < cnt; ++q) {
      const double v = __shfl_sync(0xffffffffu, dv, q);
      if (lane == 0) s = __dadd_rn(s, v);
    }
  }
  if (lane == 0) part[w] = s;
}

__global__ void objective_sum_kernel(const double* part, int nchunks, double* out) {
  double s = 0.0;
  for (int c = 0; c < nchunks; ++c) s = __dadd_rn(s, part[c]);
  *out = s;
}

__global__ void widen_labels_kernel(const uint8_t* __restrict__ z8, int32_t* __restrict__ z, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    z[i] = z8[i];
}

}  // namespace

cudaError_t launch_widen_labels(const uint8_t* z8, int32_t* z, int64_t n, cudaStream_t st) {
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 8192));
  widen_labels_kernel<<<(unsigned)blocks, 256, 0, st>>>(z8, z, n);
  return cudaGetLastError();
}

int64_t objective_chunks(int64_t n) { return (n + kObjChunk - 1) / kObjChunk; }

cudaError_t launch_objective(const float* x, int64_t ld, int64_t n, int d, const double* mu, const int32_t* z,
                             const uint8_t* z8, double* part, double* out, cudaStream_t st) {
  const int nch = (int)objective_chunks(n);
  if (z8)
    objective_kernel<uint8_t><<<(nch * 32 + 255) / 256, 256, 0, st>>>(x, ld, n, d, mu, z8, part, nch);
  else
    objective_kernel<int32_t><<<(nch * 32 + 255) / 256, 256, 0, st>>>(x, ld, n, d, mu, z, part, nch);
  objective_sum_kernel<<<1, 1, 0, st>>>(part, nch, out);
  return cudaGetLastError();
}

}  // namespace km
