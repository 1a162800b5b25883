// Learned initialiser: a set network that predicts K starting centres for
// Lloyd's algorithm from a sample of S points (the paper notes the result's
// dependence on the initial centres, section "The Lloyd's algorithm").
//
//   standardise  x' = (x - m) / s   (per set: per-coordinate mean and
//                population std of its S points; s = 1 where it is 0)
//   per point    h1 = relu(W1 x' + b1), h2 = relu(W2 h1 + b2)    (H = 128)
//   pool         g = mean_i h2_i
//   head         a3 = relu(W3 g + b3), p = W4 a3 + b4  (K x d, standardised)
//   loss         mean over sets of the symmetric Chamfer distance to the
//                standardised targets (ties: lowest index)
//
// FP32 throughout; every reduction runs in a fixed order (no float
// atomics), so a step is deterministic.  Kernels:
//   sn_standardize   one block per set
//   sn_fwd_points    64 points per block: h1, h2 and the tile's pooled sum
//                    (W2 staged transposed in shared memory, 8x4 register
//                    tiles)
//   sn_pool          one block per set: tile sums in order / S
//   sn_head          one block: head forward, loss, head backward for every
//                    set in order (dW3, dW4, db3, db4, dg)
//   sn_bwd_points    64 points per block: dz2 = dg/S * [h2 > 0],
//                    dz1 = (dz2 W2) * [h1 > 0]
//   sn_wgrad         1024-point chunks: dW2 = sum dz2 h1^T, dW1, db1, db2
//                    partials; sn_wgrad_reduce adds the chunks in order
//   sn_adam          Adam with bias correction (Kingma and Ba 2015)
#include "km_internal.cuh"

#include <algorithm>

namespace km {

namespace {

constexpr int H = kSetH;
constexpr int kTileP = 64;     // points per block in the per-point kernels
constexpr int kChunkP = 1024;  // points per weight-gradient chunk
constexpr int kAT = 68;        // row stride of the transposed point tiles (16-byte rows, 4-way banks)

struct NetOff {  // offsets of the parameters in the flat vector
  int W1, b1, W2, b2, W3, b3, W4, b4, total;
};
__host__ __device__ inline NetOff net_off(int d, int k) {
  NetOff o;
  o.W1 = 0;
  o.b1 = o.W1 + H * d;
  o.W2 = o.b1 + H;
  o.b2 = o.W2 + H * H;
  o.W3 = o.b2 + H;
  o.b3 = o.W3 + H * H;
  o.W4 = o.b3 + H;
  o.b4 = o.W4 + k * d * H;
  o.total = o.b4 + k * d;
  return o;
}

__global__ void __launch_bounds__(256) sn_standardize(const float* __restrict__ x, const float* __restrict__ t,
                                                      int S, int d, int k, float* xs, float* ts, float* ms) {
  __shared__ float s_red[256];
  __shared__ float s_m[3], s_s[3];
  const int b = blockIdx.x, tid = threadIdx.x;
  const float* xb = x + (size_t)b * S * d;
  for (int j = 0; j < d; ++j) {
    float acc = 0.f;
    for (int i = tid; i < S; i += blockDim.x) acc += xb[(size_t)i * d + j];
    s_red[tid] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
      if (tid < w) s_red[tid] += s_red[tid + w];
      __syncthreads();
    }
    const float m = s_red[0] / (float)S;
    __syncthreads();
    acc = 0.f;
    for (int i = tid; i < S; i += blockDim.x) {
      const float u = xb[(size_t)i * d + j] - m;
      acc = fmaf(u, u, acc);
    }
    s_red[tid] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
      if (tid < w) s_red[tid] += s_red[tid + w];
      __syncthreads();
    }
    if (tid == 0) {
      const float sd = sqrtf(s_red[0] / (float)S);
      s_m[j] = m;
      s_s[j] = sd > 0.f ? sd : 1.f;
    }
    __syncthreads();
  }
  for (int q = tid; q < S * d; q += blockDim.x) {
    const int j = q % d;
    xs[(size_t)b * S * d + q] = (xb[q] - s_m[j]) / s_s[j];
  }
  if (t)
    for (int q = tid; q < k * d; q += blockDim.x) {
      const int j = q % d;
      ts[(size_t)b * k * d + q] = (t[(size_t)b * k * d + q] - s_m[j]) / s_s[j];
    }
  if (tid < d) {
    ms[b * 2 * d + tid] = s_m[tid];
    ms[b * 2 * d + d + tid] = s_s[tid];
  }
}

// 64 points x 128 outputs per block, 256 threads as 8 point-groups (8 points
// each) x 32 unit-groups (4 units each); A^T tile [128][64] and the weight
// matrix transposed [128][128] in shared memory.
__device__ __forceinline__ void tile_gemm_8x4(const float* __restrict__ aT, const float* __restrict__ wT, int ty,
                                              int tx, float acc[8][4]) {
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = 0.f;
#pragma unroll 4
  for (int q = 0; q < H; ++q) {
    const float4 a0 = *reinterpret_cast<const float4*>(aT + q * kAT + 8 * ty);
    const float4 a1 = *reinterpret_cast<const float4*>(aT + q * kAT + 8 * ty + 4);
    const float4 w = *reinterpret_cast<const float4*>(wT + q * H + 4 * tx);
    const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
    const float wv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(av[r], wv[c], acc[r][c]);
  }
}

__global__ void sn_transpose(const float* __restrict__ prm, int d, int k, float* w2t) {
  const NetOff o = net_off(d, k);
  const int q = blockIdx.x * blockDim.x + threadIdx.x;  // w2t[c][u] = W2[u][c]
  if (q < H * H) w2t[q] = prm[o.W2 + (q % H) * H + q / H];
}

__global__ void __launch_bounds__(256) sn_fwd_points(const float* __restrict__ xs, const float* __restrict__ prm,
                                                     const float* __restrict__ w2t, int d, int k, float* h1g,
                                                     float* h2g, float* tile_pool) {
  extern __shared__ __align__(16) float sm[];
  float* w2T = sm;                 // [128][128]: w2T[c][u] = W2[u][c]
  float* h1T = w2T + H * H;        // [128][kAT]: h1T[c][p]
  float* s_pool = h1T + H * kAT;   // [8][128]
  const NetOff o = net_off(d, k);
  const int tid = threadIdx.x, ty = tid >> 5, tx = tid & 31;
  const int64_t p0 = (int64_t)blockIdx.x * kTileP;
  for (int q = tid; q < H * H / 4; q += blockDim.x)
    reinterpret_cast<float4*>(w2T)[q] = reinterpret_cast<const float4*>(w2t)[q];
  for (int q = tid; q < kTileP * H; q += blockDim.x) {
    const int p = q / H, u = q % H;
    float z = prm[o.b1 + u];
    for (int j = 0; j < d; ++j) z = fmaf(prm[o.W1 + u * d + j], xs[(p0 + p) * d + j], z);
    const float h = fmaxf(z, 0.f);
    h1T[u * kAT + p] = h;
    h1g[(p0 + p) * H + u] = h;
  }
  __syncthreads();
  float acc[8][4];
  tile_gemm_8x4(h1T, w2T, ty, tx, acc);
  float ps[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int p = 8 * ty + r;
    float4 out;
    float* ov = reinterpret_cast<float*>(&out);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      ov[c] = fmaxf(acc[r][c] + prm[o.b2 + 4 * tx + c], 0.f);
      ps[c] += ov[c];
    }
    *reinterpret_cast<float4*>(h2g + (p0 + p) * H + 4 * tx) = out;
  }
#pragma unroll
  for (int c = 0; c < 4; ++c) s_pool[ty * H + 4 * tx + c] = ps[c];
  __syncthreads();
  if (tid < H) {
    float s = 0.f;
    for (int g = 0; g < 8; ++g) s += s_pool[g * H + tid];
    tile_pool[(size_t)blockIdx.x * H + tid] = s;
  }
}

__global__ void __launch_bounds__(H) sn_pool(const float* tile_pool, int tiles_per_set, int S, float* G) {
  const int b = blockIdx.x, u = threadIdx.x;
  float s = 0.f;
  for (int t = 0; t < tiles_per_set; ++t) s += tile_pool[((size_t)b * tiles_per_set + t) * H + u];
  G[b * H + u] = s / (float)S;
}

// Head for every set in order.  With targets: loss, head gradients (which
// it overwrites) and dg; without: the predictions only.
__global__ void __launch_bounds__(256) sn_head(const float* __restrict__ prm, const float* __restrict__ G, int B,
                                               int d, int k, const float* __restrict__ ts, float* P, float* grads,
                                               float* dG, float* loss) {
  __shared__ float s_g[H], s_z3[H], s_a3[H], s_dz3[H];
  __shared__ float s_p[kBatchMaxK * 3], s_dp[kBatchMaxK * 3], s_t[kBatchMaxK * 3];
  __shared__ float s_loss;
  const NetOff o = net_off(d, k);
  const int tid = threadIdx.x, KD = k * d;
  const bool train = ts != nullptr;
  if (train) {
    for (int q = tid; q < H * H; q += blockDim.x) grads[o.W3 + q] = 0.f;
    for (int q = tid; q < KD * H; q += blockDim.x) grads[o.W4 + q] = 0.f;
    for (int q = tid; q < H; q += blockDim.x) grads[o.b3 + q] = 0.f;
    for (int q = tid; q < KD; q += blockDim.x) grads[o.b4 + q] = 0.f;
  }
  if (tid == 0) s_loss = 0.f;
  __syncthreads();
  for (int b = 0; b < B; ++b) {
    if (tid < H) s_g[tid] = G[b * H + tid];
    __syncthreads();
    if (tid < H) {
      float z = prm[o.b3 + tid];
      for (int c = 0; c < H; ++c) z = fmaf(prm[o.W3 + tid * H + c], s_g[c], z);
      s_z3[tid] = z;
      s_a3[tid] = fmaxf(z, 0.f);
    }
    __syncthreads();
    for (int q = tid; q < KD; q += blockDim.x) {
      float z = prm[o.b4 + q];
      for (int u = 0; u < H; ++u) z = fmaf(prm[o.W4 + q * H + u], s_a3[u], z);
      s_p[q] = z;
      P[b * KD + q] = z;
      if (train) {
        s_t[q] = ts[b * KD + q];
        s_dp[q] = 0.f;
      }
    }
    __syncthreads();
    if (!train) continue;
    if (tid == 0) {
      // symmetric Chamfer distance; gradients scaled by 1 / (K B)
      const float sc = 2.f / ((float)k * (float)B);
      float l1 = 0.f, l2 = 0.f;
      for (int a = 0; a < k; ++a) {  // nearest target of each prediction
        int js = 0;
        float best = 3.0e38f;
        for (int j = 0; j < k; ++j) {
          float dd = 0.f;
          for (int c = 0; c < d; ++c) {
            const float u = s_p[a * d + c] - s_t[j * d + c];
            dd = fmaf(u, u, dd);
          }
          if (dd < best) { best = dd; js = j; }
        }
        l1 += best;
        for (int c = 0; c < d; ++c) s_dp[a * d + c] += sc * (s_p[a * d + c] - s_t[js * d + c]);
      }
      for (int j = 0; j < k; ++j) {  // nearest prediction of each target
        int as = 0;
        float best = 3.0e38f;
        for (int a = 0; a < k; ++a) {
          float dd = 0.f;
          for (int c = 0; c < d; ++c) {
            const float u = s_p[a * d + c] - s_t[j * d + c];
            dd = fmaf(u, u, dd);
          }
          if (dd < best) { best = dd; as = a; }
        }
        l2 += best;
        for (int c = 0; c < d; ++c) s_dp[as * d + c] += sc * (s_p[as * d + c] - s_t[j * d + c]);
      }
      s_loss += (l1 + l2) / (float)k / (float)B;
    }
    __syncthreads();
    for (int q = tid; q < KD * H; q += blockDim.x) grads[o.W4 + q] += s_dp[q / H] * s_a3[q % H];
    for (int q = tid; q < KD; q += blockDim.x) grads[o.b4 + q] += s_dp[q];
    if (tid < H) {
      float da = 0.f;
      for (int q = 0; q < KD; ++q) da = fmaf(prm[o.W4 + q * H + tid], s_dp[q], da);
      s_dz3[tid] = s_z3[tid] > 0.f ? da : 0.f;
    }
    __syncthreads();
    for (int q = tid; q < H * H; q += blockDim.x) grads[o.W3 + q] += s_dz3[q / H] * s_g[q % H];
    if (tid < H) {
      grads[o.b3 + tid] += s_dz3[tid];
      float dg = 0.f;
      for (int u = 0; u < H; ++u) dg = fmaf(prm[o.W3 + u * H + tid], s_dz3[u], dg);
      dG[b * H + tid] = dg;
    }
    __syncthreads();
  }
  if (tid == 0 && train) *loss = s_loss;
}

__global__ void __launch_bounds__(256) sn_bwd_points(const float* __restrict__ prm, int d, int k, int S,
                                                     const float* __restrict__ dG, const float* __restrict__ h1g,
                                                     const float* __restrict__ h2g, float* dz2g, float* dz1g) {
  extern __shared__ __align__(16) float sm[];
  float* w2 = sm;               // [128][128] = W2[u][c] (row u): the transposed use of W2
  float* dz2T = w2 + H * H;     // [128][kAT]: dz2T[u][p]
  const NetOff o = net_off(d, k);
  const int tid = threadIdx.x, ty = tid >> 5, tx = tid & 31;
  const int64_t p0 = (int64_t)blockIdx.x * kTileP;
  const int b = (int)(p0 / S);
  for (int q = tid; q < H * H / 4; q += blockDim.x)
    reinterpret_cast<float4*>(w2)[q] = reinterpret_cast<const float4*>(prm + o.W2)[q];
  for (int q = tid; q < kTileP * H; q += blockDim.x) {
    const int p = q / H, u = q % H;
    const float v = h2g[(p0 + p) * H + u] > 0.f ? dG[b * H + u] / (float)S : 0.f;
    dz2T[u * kAT + p] = v;
    dz2g[(p0 + p) * H + u] = v;
  }
  __syncthreads();
  float acc[8][4];  // dh1[p][c] = sum_u dz2[p][u] W2[u][c]
  tile_gemm_8x4(dz2T, w2, ty, tx, acc);
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int64_t p = p0 + 8 * ty + r;
    const float4 h = *reinterpret_cast<const float4*>(h1g + p * H + 4 * tx);
    float4 out;
    out.x = h.x > 0.f ? acc[r][0] : 0.f;
    out.y = h.y > 0.f ? acc[r][1] : 0.f;
    out.z = h.z > 0.f ? acc[r][2] : 0.f;
    out.w = h.w > 0.f ? acc[r][3] : 0.f;
    *reinterpret_cast<float4*>(dz1g + p * H + 4 * tx) = out;
  }
}

// Per 1024-point chunk: dW2 (8x8 outputs per thread over 32-point smem
// tiles), and dW1, db1, db2 (threads 0..127 by unit).
__global__ void __launch_bounds__(256) sn_wgrad(const float* __restrict__ dz2g, const float* __restrict__ h1g,
                                                const float* __restrict__ dz1g, const float* __restrict__ xs, int d,
                                                int64_t P, float* part) {
  __shared__ __align__(16) float s_a[32 * H], s_b[32 * H];
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const int64_t c0 = (int64_t)blockIdx.x * kChunkP;
  const int np = (int)min((int64_t)kChunkP, P - c0);
  float acc[8][8];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[r][c] = 0.f;
  for (int t0 = 0; t0 < np; t0 += 32) {
    const int m = min(32, np - t0);
    __syncthreads();
    for (int q = tid; q < 32 * H; q += blockDim.x) {
      const int p = q / H;
      s_a[q] = p < m ? dz2g[(c0 + t0 + p) * H + (q % H)] : 0.f;
      s_b[q] = p < m ? h1g[(c0 + t0 + p) * H + (q % H)] : 0.f;
    }
    __syncthreads();
    for (int p = 0; p < 32; ++p) {
      const float4 a0 = *reinterpret_cast<const float4*>(s_a + p * H + 8 * ty);
      const float4 a1 = *reinterpret_cast<const float4*>(s_a + p * H + 8 * ty + 4);
      const float4 b0 = *reinterpret_cast<const float4*>(s_b + p * H + 8 * tx);
      const float4 b1 = *reinterpret_cast<const float4*>(s_b + p * H + 8 * tx + 4);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[r][c] = fmaf(av[r], bv[c], acc[r][c]);
    }
  }
  const int stride = H * H + H * d + 2 * H;
  float* out = part + (size_t)blockIdx.x * stride;
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int c = 0; c < 8; ++c) out[(8 * ty + r) * H + 8 * tx + c] = acc[r][c];
  if (tid < H) {
    float w1[3] = {0.f, 0.f, 0.f}, g1 = 0.f, g2 = 0.f;
    for (int p = 0; p < np; ++p) {
      const float z1 = dz1g[(c0 + p) * H + tid];
      g1 += z1;
      g2 += dz2g[(c0 + p) * H + tid];
      for (int j = 0; j < d; ++j) w1[j] = fmaf(z1, xs[(c0 + p) * d + j], w1[j]);
    }
    for (int j = 0; j < d; ++j) out[H * H + tid * d + j] = w1[j];
    out[H * H + H * d + tid] = g1;
    out[H * H + H * d + H + tid] = g2;
  }
}

__global__ void sn_wgrad_reduce(const float* part, int nchunks, int d, int k, float* grads) {
  const NetOff o = net_off(d, k);
  const int stride = H * H + H * d + 2 * H;
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= stride) return;
  float s = 0.f;
  for (int c = 0; c < nchunks; ++c) s += part[(size_t)c * stride + q];
  int dst;
  if (q < H * H) dst = o.W2 + q;
  else if (q < H * H + H * d) dst = o.W1 + (q - H * H);
  else if (q < H * H + H * d + H) dst = o.b1 + (q - H * H - H * d);
  else dst = o.b2 + (q - H * H - H * d - H);
  grads[dst] = s;
}

__global__ void sn_adam(float* prm, const float* grads, float* m, float* v, int n, float lr, float b1, float b2,
                        float eps, float c1, float c2) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
  const float g = grads[q];
  const float mq = b1 * m[q] + (1.f - b1) * g;
  const float vq = b2 * v[q] + (1.f - b2) * g * g;
  m[q] = mq;
  v[q] = vq;
  prm[q] -= lr * (mq / c1) / (sqrtf(vq / c2) + eps);
}

// Sample of S points of a context: point floor(u_j N), u_j the j-th output
// of SplitMix64 (Vigna) from the seed, to 53 bits.
__global__ void sn_sample(const float* __restrict__ x, int64_t ld, int64_t n, int d, int S, unsigned long long seed,
                          float* out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= S) return;
  unsigned long long z = seed + (unsigned long long)(j + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  const double u = (double)(z >> 11) * 0x1p-53;
  int64_t i = (int64_t)(u * (double)n);
  if (i >= n) i = n - 1;
  for (int c = 0; c < d; ++c) out[(size_t)j * d + c] = x[(int64_t)c * ld + i];
}

// Centres in the points' coordinates: c = p * s + m (FP64 output).
__global__ void sn_destd(const float* P, const float* ms, int B, int d, int k, double* out) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= B * k * d) return;
  const int b = q / (k * d), j = q % d;
  out[q] = (double)P[q] * (double)ms[b * 2 * d + d + j] + (double)ms[b * 2 * d + j];
}

}  // namespace

int setnet_param_count(int d, int k) { return net_off(d, k).total; }

cudaError_t launch_setnet_destandardize(const float* P, const float* ms, int B, int d, int k, double* out,
                                        cudaStream_t st) {
  const int n = B * k * d;
  sn_destd<<<(n + 255) / 256, 256, 0, st>>>(P, ms, B, d, k, out);
  return cudaGetLastError();
}

size_t setnet_point_smem() { return sizeof(float) * (H * H + H * kAT + 8 * H); }

cudaError_t launch_setnet_forward(const SetNetArgs& a, bool train, cudaStream_t st) {
  const int64_t P = (int64_t)a.B * a.S;
  const int tiles = (int)(P / kTileP);
  sn_standardize<<<a.B, 256, 0, st>>>(a.x, train ? a.t : nullptr, a.S, a.d, a.k, a.xs, a.ts, a.ms);
  const size_t smem = setnet_point_smem();
  cudaError_t e = cudaFuncSetAttribute(sn_fwd_points, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  sn_transpose<<<H * H / 256, 256, 0, st>>>(a.prm, a.d, a.k, a.w2t);
  sn_fwd_points<<<tiles, 256, smem, st>>>(a.xs, a.prm, a.w2t, a.d, a.k, a.h1, a.h2, a.tile_pool);
  sn_pool<<<a.B, H, 0, st>>>(a.tile_pool, a.S / kTileP, a.S, a.G);
  sn_head<<<1, 256, 0, st>>>(a.prm, a.G, a.B, a.d, a.k, train ? a.ts : nullptr, a.P, a.grads, a.dG, a.loss);
  return cudaGetLastError();
}

cudaError_t launch_setnet_backward(const SetNetArgs& a, cudaStream_t st) {
  const int64_t P = (int64_t)a.B * a.S;
  const int tiles = (int)(P / kTileP);
  const size_t smem = sizeof(float) * (H * H + H * kAT);
  cudaError_t e = cudaFuncSetAttribute(sn_bwd_points, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  sn_bwd_points<<<tiles, 256, smem, st>>>(a.prm, a.d, a.k, a.S, a.dG, a.h1, a.h2, a.dz2, a.dz1);
  const int nch = (int)((P + kChunkP - 1) / kChunkP);
  sn_wgrad<<<nch, 256, 0, st>>>(a.dz2, a.h1, a.dz1, a.xs, a.d, P, a.part);
  const int stride = H * H + H * a.d + 2 * H;
  sn_wgrad_reduce<<<(stride + 255) / 256, 256, 0, st>>>(a.part, nch, a.d, a.k, a.grads);
  return cudaGetLastError();
}

int64_t setnet_part_floats(int64_t P, int d) {
  return ((P + kChunkP - 1) / kChunkP) * (int64_t)(H * H + H * d + 2 * H);
}

cudaError_t launch_setnet_adam(float* prm, const float* grads, float* m, float* v, int n, float lr, float b1,
                               float b2, float eps, float c1, float c2, cudaStream_t st) {
  sn_adam<<<(n + 255) / 256, 256, 0, st>>>(prm, grads, m, v, n, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

cudaError_t launch_setnet_sample(const float* x, int64_t ld, int64_t n, int d, int S, unsigned long long seed,
                                 float* out, cudaStream_t st) {
  sn_sample<<<(S + 255) / 256, 256, 0, st>>>(x, ld, n, d, S, seed, out);
  return cudaGetLastError();
}

namespace {

// Per-set mean of B sets of S points (d <= 3), FP64, one block per set:
// thread-strided partial sums combined by a fixed-order tree.
__global__ void __launch_bounds__(256) sets_mean_kernel(const float* __restrict__ x, int64_t set_stride, int S,
                                                        int d, double* __restrict__ means) {
  __shared__ double red[3][256];
  const int b = blockIdx.x, tid = threadIdx.x;
  const float* xs = x + (int64_t)b * set_stride;
  double acc[3] = {0.0, 0.0, 0.0};
  for (int s = tid; s < S; s += blockDim.x)
    for (int j = 0; j < d; ++j) acc[j] = __dadd_rn(acc[j], (double)xs[(int64_t)s * d + j]);
  for (int j = 0; j < 3; ++j) red[j][tid] = acc[j];
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (tid < w)
      for (int j = 0; j < 3; ++j) red[j][tid] = __dadd_rn(red[j][tid], red[j][tid + w]);
    __syncthreads();
  }
  if (tid < d) means[(int64_t)b * d + tid] = __ddiv_rn(red[tid][0], (double)S);
}

// out[b][s] = R_b (x[b][s] - c_b) + c_b (R_b^T with transpose), in FP64;
// R: B x d x d row-major, c: one centre per set (stride center_stride
// doubles; null = the origin).
template <typename T>
__global__ void sets_rotate_kernel(const T* __restrict__ x, int64_t set_stride, int B, int S, int d,
                                   const double* __restrict__ R, const double* __restrict__ c, int64_t center_stride,
                                   int transpose, T* __restrict__ out) {
  const int64_t total = (int64_t)B * S;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(q / S), s = (int)(q - (int64_t)b * S);
    const T* xp = x + (int64_t)b * set_stride + (int64_t)s * d;
    const double* Rb = R + (int64_t)b * d * d;
    double v[3], cc[3] = {0.0, 0.0, 0.0};
    for (int j = 0; j < d; ++j) {
      if (c) cc[j] = c[(int64_t)b * center_stride + j];
      v[j] = __dsub_rn((double)xp[j], cc[j]);
    }
    T* op = out + q * d;
    for (int i = 0; i < d; ++i) {
      double acc = 0.0;
      for (int j = 0; j < d; ++j)
        acc = __dadd_rn(acc, __dmul_rn(transpose ? Rb[j * d + i] : Rb[i * d + j], v[j]));
      op[i] = (T)__dadd_rn(acc, cc[i]);
    }
  }
}

}  // namespace

cudaError_t launch_sets_mean(const float* x, int64_t set_stride, int B, int S, int d, double* means, cudaStream_t st) {
  sets_mean_kernel<<<B, 256, 0, st>>>(x, set_stride, S, d, means);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sets_rotate(const T* x, int64_t set_stride, int B, int S, int d, const double* R,
                               const double* c, int64_t center_stride, int transpose, T* out, cudaStream_t st) {
  const int64_t total = (int64_t)B * S;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 4096));
  sets_rotate_kernel<T><<<grid, 256, 0, st>>>(x, set_stride, B, S, d, R, c, center_stride, transpose, out);
  return cudaGetLastError();
}
template cudaError_t launch_sets_rotate<float>(const float*, int64_t, int, int, int, const double*, const double*,
                                               int64_t, int, float*, cudaStream_t);
template cudaError_t launch_sets_rotate<double>(const double*, int64_t, int, int, int, const double*, const double*,
                                                int64_t, int, double*, cudaStream_t);

}  // namespace km
