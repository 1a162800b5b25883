// Mean calculation from labels by sorting (paper, section "The Lloyd's
// algorithm", step 3: mu_k = sum_i 1(z_i = k) x_i / sum_i 1(z_i = k)), for
// shapes whose per-cluster sums do not fit in shared memory (d > 4 or large
// K).  Points are grouped by label with a counting sort (histogram, scan,
// scatter of point indices), each cluster's list is cut into chunks of at
// most kChunk points, every chunk is summed exactly in fixed point by one
// block reading whole rows of the N x d copy of the points (coalesced), and
// the finalize kernel adds each cluster's chunk sums in order in int128,
// divides and keeps empty centres; a one-block kernel forms E^2 by a
// fixed-order tree.  The scatter order inside a cluster is not
// deterministic, but integer sums do not depend on it.
#include "km_internal.cuh"

namespace km {

namespace {

__global__ void ms_hist_kernel(const int32_t* __restrict__ labels, int64_t n, int k,
                               unsigned long long* counts) {
  extern __shared__ unsigned int sh[];
  const bool use_sh = k <= 8192;
  if (use_sh)
    for (int c = threadIdx.x; c < k; c += blockDim.x) sh[c] = 0u;
  __syncthreads();
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int z = labels[i];
    if (use_sh) atomicAdd(&sh[z], 1u);
    else atomicAdd(&counts[z], 1ull);
  }
  __syncthreads();
  if (use_sh)
    for (int c = threadIdx.x; c < k; c += blockDim.x)
      if (sh[c]) atomicAdd(&counts[c], (unsigned long long)sh[c]);
}

// One block: exclusive scans of the counts (point offsets) and of the
// per-cluster chunk counts; chunk table entries (cluster, start, length).
__global__ void ms_scan_kernel(const unsigned long long* counts, int k, int64_t* offsets, int* cfirst,
                               unsigned long long* cursor, int4* chunks, int* nchunks, int max_chunks) {
  __shared__ long long s_pt[1024];
  __shared__ int s_ch[1024];
  __shared__ long long carry_pt;
  __shared__ int carry_ch;
  if (threadIdx.x == 0) { carry_pt = 0; carry_ch = 0; }
  __syncthreads();
  for (int base = 0; base < k; base += 1024) {
    const int c = base + threadIdx.x;
    const long long cnt = c < k ? (long long)counts[c] : 0;
    const int nch = (int)((cnt + kChunk - 1) / kChunk);
    s_pt[threadIdx.x] = cnt;
    s_ch[threadIdx.x] = nch;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {  // inclusive Hillis-Steele scans
      const long long vp = threadIdx.x >= off ? s_pt[threadIdx.x - off] : 0;
      const int vc = threadIdx.x >= off ? s_ch[threadIdx.x - off] : 0;
      __syncthreads();
      s_pt[threadIdx.x] += vp;
      s_ch[threadIdx.x] += vc;
      __syncthreads();
    }
    if (c < k) {
      const long long start = carry_pt + s_pt[threadIdx.x] - cnt;
      const int cstart = carry_ch + s_ch[threadIdx.x] - nch;
      offsets[c] = start;
      cfirst[c] = cstart;
      cursor[c] = 0ull;
      for (int q = 0; q < nch && cstart + q < max_chunks; ++q) {
        const long long a = (long long)q * kChunk;
        chunks[cstart + q] = make_int4(c, (int)(start + a), (int)min((long long)kChunk, cnt - a), 0);
      }
    }
    __syncthreads();
    if (threadIdx.x == 1023) { carry_pt += s_pt[1023]; carry_ch += s_ch[1023]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) *nchunks = min(carry_ch, max_chunks);
}

__global__ void ms_scatter_kernel(const int32_t* __restrict__ labels, int64_t n, const int64_t* offsets,
                                  unsigned long long* cursor, int32_t* perm) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int z = labels[i];
    const unsigned long long pos = atomicAdd(&cursor[z], 1ull);
    perm[offsets[z] + (int64_t)pos] = (int32_t)i;
  }
}

// The same scatter with one global reservation per (block, label): a block
// takes kScatterPts consecutive points, counts their labels in shared
// memory, reserves each label's run with one atomic on the cluster's cursor
// and places its points by shared-memory ranks (K <= kScatterMaxK).
constexpr int kScatterPts = 4096;
constexpr int kScatterMaxK = 4096;
__global__ void __launch_bounds__(256) ms_scatter_block_kernel(const int32_t* __restrict__ labels, int64_t n, int k,
                                                               const int64_t* __restrict__ offsets,
                                                               unsigned long long* cursor, int32_t* perm) {
  extern __shared__ unsigned long long s_base[];  // [k] run starts, then [k] u32 counts / ranks
  unsigned int* s_cnt = reinterpret_cast<unsigned int*>(s_base + k);
  const int64_t i0 = (int64_t)blockIdx.x * kScatterPts;
  const int64_t i1 = min(n, i0 + kScatterPts);
  for (int c = threadIdx.x; c < k; c += blockDim.x) s_cnt[c] = 0u;
  __syncthreads();
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) atomicAdd(&s_cnt[labels[i]], 1u);
  __syncthreads();
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    const unsigned m = s_cnt[c];
    if (m) s_base[c] = (unsigned long long)offsets[c] + atomicAdd(&cursor[c], (unsigned long long)m);
    s_cnt[c] = 0u;
  }
  __syncthreads();
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
    const int z = labels[i];
    const unsigned r = atomicAdd(&s_cnt[z], 1u);
    perm[s_base[z] + r] = (int32_t)i;
  }
}

// Chunk sums with 16-byte loads (d a multiple of 4): threads (r, q) =
// (threadIdx.x / (d/4), threadIdx.x % (d/4)) sum coordinates 4q..4q+3 of
// points r, r + R, ... of the chunk, four rows in flight, in int64 fixed
// point as below.
__global__ void __launch_bounds__(256) ms_chunk_sum4_kernel(const float4* __restrict__ xa4, int d,
                                                            const int32_t* __restrict__ perm,
                                                            const int4* __restrict__ chunks, const int* nchunks,
                                                            const DataConst* dcp, long long* chunk_sums) {
  extern __shared__ long long s_part4[];  // [R][d]
  const int ch = blockIdx.x;
  if (ch >= *nchunks) return;
  const int4 cd = chunks[ch];
  const int d4 = d >> 2;
  const int R = blockDim.x / d4;
  const int r = threadIdx.x / d4, q = threadIdx.x - r * d4;
  const DataConst dc = *dcp;
  auto fixed = [&](float v) {  // v in grid units of 2^G0, exactly (two FP32 limbs)
    const float t = __fadd_rn(v, dc.C_hi);
    const float h = __fsub_rn(t, dc.C_hi);
    const float rr = __fsub_rn(v, h);
    const float t2 = __fadd_rn(rr, dc.C_lo);
    const long long hi = (long long)(int)(__float_as_uint(t) - dc.bits_C_hi);
    const long long lo = (long long)(int)(__float_as_uint(t2) - dc.bits_C_lo);
    return (hi << 22) + lo;
  };
  long long a0 = 0, a1 = 0, a2 = 0, a3 = 0;
  auto add = [&](const float4 v) {
    a0 += fixed(v.x);
    a1 += fixed(v.y);
    a2 += fixed(v.z);
    a3 += fixed(v.w);
  };
  if (r < R) {
    int p = r;
    for (; p + 3 * R < cd.z; p += 4 * R) {
      const int i0 = perm[cd.y + p], i1 = perm[cd.y + p + R], i2 = perm[cd.y + p + 2 * R], i3 = perm[cd.y + p + 3 * R];
      const float4 v0 = xa4[(int64_t)i0 * d4 + q], v1 = xa4[(int64_t)i1 * d4 + q];
      const float4 v2 = xa4[(int64_t)i2 * d4 + q], v3 = xa4[(int64_t)i3 * d4 + q];
      add(v0);
      add(v1);
      add(v2);
      add(v3);
    }
    for (; p < cd.z; p += R) add(xa4[(int64_t)perm[cd.y + p] * d4 + q]);
    long long* o = s_part4 + (size_t)r * d + 4 * q;
    o[0] = a0;
    o[1] = a1;
    o[2] = a2;
    o[3] = a3;
  }
  __syncthreads();
  for (int jj = threadIdx.x; jj < d; jj += blockDim.x) {
    long long sum = 0;
    for (int w = 0; w < R; ++w) sum += s_part4[(size_t)w * d + jj];
    chunk_sums[(size_t)ch * d + jj] = sum;
  }
}

// One block per chunk: threads (r, j) = (threadIdx.x / d, threadIdx.x % d)
// sum coordinate j of points r, r + R, ... of the chunk in int64 fixed point
// (<= kChunk points of |x| < 2^43 grid units each: no overflow); rows are
// added in order r = 0..R-1.
__global__ void ms_chunk_sum_kernel(const float* __restrict__ xa, int d, const int32_t* __restrict__ perm,
                                    const int4* __restrict__ chunks, const int* nchunks, const DataConst* dcp,
                                    long long* chunk_sums /* [max_chunks][d] */) {
  extern __shared__ long long s_part[];  // [R][d]
  const int ch = blockIdx.x;
  if (ch >= *nchunks) return;
  const int4 cd = chunks[ch];
  const int R = blockDim.x / d;
  const int r = threadIdx.x / d, j = threadIdx.x - r * d;
  const DataConst dc = *dcp;
  long long acc = 0;
  if (r < R) {
    auto fixed = [&](float v) {  // v in grid units of 2^G0, exactly (two FP32 limbs)
      const float t = __fadd_rn(v, dc.C_hi);
      const float h = __fsub_rn(t, dc.C_hi);
      const float rr = __fsub_rn(v, h);
      const float t2 = __fadd_rn(rr, dc.C_lo);
      const long long hi = (long long)(int)(__float_as_uint(t) - dc.bits_C_hi);
      const long long lo = (long long)(int)(__float_as_uint(t2) - dc.bits_C_lo);
      return (hi << 22) + lo;
    };
    // four rows in flight per thread (integer sums do not depend on order)
    int p = r;
    for (; p + 3 * R < cd.z; p += 4 * R) {
      const int i0 = perm[cd.y + p], i1 = perm[cd.y + p + R], i2 = perm[cd.y + p + 2 * R], i3 = perm[cd.y + p + 3 * R];
      const float v0 = xa[(int64_t)i0 * d + j], v1 = xa[(int64_t)i1 * d + j];
      const float v2 = xa[(int64_t)i2 * d + j], v3 = xa[(int64_t)i3 * d + j];
      acc += fixed(v0) + fixed(v1) + fixed(v2) + fixed(v3);
    }
    for (; p < cd.z; p += R) acc += fixed(xa[(int64_t)perm[cd.y + p] * d + j]);
    s_part[r * d + j] = acc;
  }
  __syncthreads();
  for (int jj = threadIdx.x; jj < d; jj += blockDim.x) {
    long long s = 0;
    for (int q = 0; q < R; ++q) s += s_part[q * d + jj];
    chunk_sums[(size_t)ch * d + jj] = s;
  }
}

__device__ __forceinline__ double ms_i128_to_double(unsigned long long lo, long long hs) {
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

// One thread per (cluster, coordinate): the cluster's chunk sums added in
// chunk order in int128, one conversion, the divide (an empty cluster keeps
// its centre) and the squared move.  Centroid tables for the next step are
// written by the path's own prepare kernels afterwards.
__global__ void __launch_bounds__(256) ms_finalize_kernel(const unsigned long long* counts, const int* cfirst,
                                                          const long long* chunk_sums, int k, int d,
                                                          const DataConst* dcp, double* mu, long long* counts_out,
                                                          double* df2, const LoopState* ls) {
  if (ls->done) return;  // the loop already stopped (graph-driven runs)
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= k * d) return;
  const int c = q / d, j = q - c * d;
  const long long cnt = (long long)counts[c];
  const long long first = cfirst[c];  // index of the cluster's first chunk (from the scan)
  const int nch = (int)((cnt + kChunk - 1) / kChunk);
  unsigned long long lo = 0ull;
  long long hi = 0ll;
  for (int t = 0; t < nch; ++t) {
    const long long v = chunk_sums[(size_t)(first + t) * d + j];
    const unsigned long long nl = lo + (unsigned long long)v;
    hi += (v < 0 ? -1ll : 0ll) + (nl < lo ? 1ll : 0ll);
    lo = nl;
  }
  const double old = mu[q];
  double nw = old;
  if (cnt > 0) nw = __ddiv_rn(ldexp(ms_i128_to_double(lo, hi), dcp->G0), (double)cnt);
  const double df = __dsub_rn(nw, old);
  df2[q] = __dmul_rn(df, df);
  mu[q] = nw;
  if (j == 0) counts_out[c] = cnt;
}

// One block: E^2 = sum of the squared moves by a fixed-order tree (thread t
// adds entries t, t + 1024, ... in order), the empty-cluster count, the stop
// test and the per-step statistics.
__global__ void __launch_bounds__(1024) ms_close_kernel(const double* df2, int kd, const long long* counts, int k,
                                                        LoopState* ls) {
  __shared__ double s_red[1024];
  __shared__ int s_empty;
  if (ls->done) return;
  const int tid = threadIdx.x;
  if (tid == 0) s_empty = 0;
  double e2p = 0.0;
  for (int q = tid; q < kd; q += blockDim.x) e2p = __dadd_rn(e2p, df2[q]);
  int empty = 0;
  for (int c = tid; c < k; c += blockDim.x) empty += counts[c] == 0;
  s_red[tid] = e2p;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (tid < w) s_red[tid] = __dadd_rn(s_red[tid], s_red[tid + w]);
    __syncthreads();
  }
  if (empty) atomicAdd(&s_empty, empty);
  __syncthreads();
  if (tid == 0) {
    const double E2 = s_red[0], E = sqrt(E2);
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
  }
}

// Sharded steps: the cluster's exact int128 coordinate totals (its chunk
// sums added in chunk order, as the finalize kernel does) and its count, in
// the sharded-step table layout [k][d+1] of (low word, high word).
__global__ void __launch_bounds__(256) ms_shard_totals_kernel(const unsigned long long* counts, const int* cfirst,
                                                              const long long* chunk_sums, int k, int d,
                                                              long long* out) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= k * (d + 1)) return;
  const int c = q / (d + 1), j = q - c * (d + 1);
  const long long cnt = (long long)counts[c];
  unsigned long long lo = 0ull;
  long long hi = 0ll;
  if (j == d) {
    lo = (unsigned long long)cnt;
  } else {
    const long long first = cfirst[c];
    const int nch = (int)((cnt + kChunk - 1) / kChunk);
    for (int t = 0; t < nch; ++t) {
      const long long v = chunk_sums[(size_t)(first + t) * d + j];
      const unsigned long long nl = lo + (unsigned long long)v;
      hi += (v < 0 ? -1ll : 0ll) + (nl < lo ? 1ll : 0ll);
      lo = nl;
    }
  }
  out[(size_t)q * 2] = (long long)lo;
  out[(size_t)q * 2 + 1] = hi;
}

// Sharded steps: the ranks' tables added in rank order (int128), then the
// finalize kernel's conversion and divide -- the same integers as one
// context over all points, so the same centroids.
__global__ void __launch_bounds__(256) ms_shard_finalize_kernel(const long long* tables, int ranks, int k, int d,
                                                                const DataConst* dcp, double* mu,
                                                                long long* counts_out, double* df2,
                                                                const LoopState* ls) {
  if (ls->done) return;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= k * d) return;
  const int c = q / d, j = q - c * d;
  const size_t cols = (size_t)k * (d + 1);
  const size_t col = (size_t)c * (d + 1) + j, ccol = (size_t)c * (d + 1) + d;
  unsigned long long lo = 0ull, clo = 0ull;
  long long hi = 0ll, chi = 0ll;
  for (int r = 0; r < ranks; ++r) {
    const long long* t = tables + (size_t)r * cols * 2;
    const unsigned long long vl = (unsigned long long)t[col * 2];
    const unsigned long long nl = lo + vl;
    hi += t[col * 2 + 1] + (nl < lo ? 1ll : 0ll);
    lo = nl;
    const unsigned long long cl = (unsigned long long)t[ccol * 2];
    const unsigned long long ncl = clo + cl;
    chi += t[ccol * 2 + 1] + (ncl < clo ? 1ll : 0ll);
    clo = ncl;
  }
  const long long cnt = (long long)clo;  // counts fit in 64 bits
  const double old = mu[q];
  double nw = old;
  if (cnt > 0) nw = __ddiv_rn(ldexp(ms_i128_to_double(lo, hi), dcp->G0), (double)cnt);
  const double df = __dsub_rn(nw, old);
  df2[q] = __dmul_rn(df, df);
  mu[q] = nw;
  if (j == 0) counts_out[c] = cnt;
}

}  // namespace

int64_t msort_max_chunks(int64_t n, int k) { return n / kChunk + k + 1; }

static cudaError_t msort_sums(const MsortArgs& a, cudaStream_t st);

cudaError_t launch_msort_step(const MsortArgs& a, cudaStream_t st) {
  cudaError_t e = msort_sums(a, st);
  if (e != cudaSuccess) return e;
  ms_finalize_kernel<<<(a.k * a.d + 255) / 256, 256, 0, st>>>(a.counts_u, a.cfirst, a.chunk_sums, a.k, a.d, a.dc,
                                                              a.mu, a.counts, a.df2, a.ls);
  ms_close_kernel<<<1, 1024, 0, st>>>(a.df2, a.k * a.d, a.counts, a.k, a.ls);
  return cudaGetLastError();
}

cudaError_t launch_msort_shard_totals(const MsortArgs& a, long long* out, cudaStream_t st) {
  cudaError_t e = msort_sums(a, st);
  if (e != cudaSuccess) return e;
  ms_shard_totals_kernel<<<(a.k * (a.d + 1) + 255) / 256, 256, 0, st>>>(a.counts_u, a.cfirst, a.chunk_sums, a.k,
                                                                        a.d, out);
  return cudaGetLastError();
}

cudaError_t launch_msort_shard_update(const MsortArgs& a, const long long* tables, int ranks, cudaStream_t st) {
  ms_shard_finalize_kernel<<<(a.k * a.d + 255) / 256, 256, 0, st>>>(tables, ranks, a.k, a.d, a.dc, a.mu, a.counts,
                                                                    a.df2, a.ls);
  ms_close_kernel<<<1, 1024, 0, st>>>(a.df2, a.k * a.d, a.counts, a.k, a.ls);
  return cudaGetLastError();
}

// Histogram, scan, scatter and chunk sums of the sorted mean calculation.
static cudaError_t msort_sums(const MsortArgs& a, cudaStream_t st) {
  // callers skip the whole step once the loop has stopped: the flag is read
  // by the finalize kernel only, so the earlier kernels run unconditionally
  cudaError_t e = cudaMemsetAsync(a.counts_u, 0, sizeof(unsigned long long) * a.k, st);
  if (e != cudaSuccess) return e;
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((a.n + 255) / 256, 2048));
  const size_t hs = a.k <= 8192 ? sizeof(unsigned int) * a.k : 0;
  ms_hist_kernel<<<(unsigned)blocks, 256, hs, st>>>(a.labels, a.n, a.k, a.counts_u);
  ms_scan_kernel<<<1, 1024, 0, st>>>(a.counts_u, a.k, a.offsets, a.cfirst, a.cursor, a.chunks, a.nchunks, a.max_chunks);
  if (a.k <= kScatterMaxK) {
    const int64_t sb = (a.n + kScatterPts - 1) / kScatterPts;
    ms_scatter_block_kernel<<<(unsigned)std::max<int64_t>(1, sb), 256, (size_t)a.k * 12, st>>>(
        a.labels, a.n, a.k, a.offsets, a.cursor, a.perm);
  } else {
    ms_scatter_kernel<<<(unsigned)blocks, 256, 0, st>>>(a.labels, a.n, a.offsets, a.cursor, a.perm);
  }
  if (a.d % 4 == 0 && a.d <= 1024 &&
      (reinterpret_cast<uintptr_t>(a.xa) & 15u) == 0) {
    const int R = std::max(1, 256 / (a.d / 4));
    const int threads = R * (a.d / 4);
    ms_chunk_sum4_kernel<<<(unsigned)a.max_chunks, threads, sizeof(long long) * (size_t)R * a.d, st>>>(
        reinterpret_cast<const float4*>(a.xa), a.d, a.perm, a.chunks, a.nchunks, a.dc, a.chunk_sums);
  } else {
    const int R = std::max(1, 256 / a.d);
    const int threads = R * a.d <= 1024 ? R * a.d : a.d;
    ms_chunk_sum_kernel<<<(unsigned)a.max_chunks, threads, sizeof(long long) * (size_t)std::max(1, threads / a.d) * a.d,
                          st>>>(a.xa, a.d, a.perm, a.chunks, a.nchunks, a.dc, a.chunk_sums);
  }
  return cudaGetLastError();
}

}  // namespace km
