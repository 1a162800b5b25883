// Reassignment for d = 64 in the GEMM form ||c||^2 - 2 x.c on the 5th-gen
// tensor cores (tcgen05, BF16 or FP16 operands, FP32 accumulation in TMEM), the
// expectation step of Lloyd's algorithm (paper, section "The Lloyd's
// algorithm", step 2) where d is large enough for a dense contraction.
//
// Persistent, warp-specialised CTA (one per SM, 17 warps):
//  * warp 16, one thread: bulk copies (cp.async.bulk, mbarrier tx counts) of
//    the whole BF16 centroid matrix once and of 128-point tiles into two
//    stages, both pre-swizzled in global memory to the 128-byte K-major
//    layout; and the MMAs: per tile, K/256 groups of M=128, N=256, K=4x16
//    into two TMEM accumulators of 256 columns (double-buffered against the
//    epilogue through full/empty mbarriers).
//  * warps 0-15, the epilogue: warp w reads TMEM lanes 32 (w % 4) (its 32
//    points) and 64 columns of each group, forms r_k = n'_k + scale S_k (one
//    binade [1, 2): r = M + 2^sigma (h - 2 S)) and the minimum of each half
//    of 16 columns.  A half whose minimum is within the point's threshold is
//    stored whole to shared memory (up to kSlots halves per point, 16 bits
//    per value: bits 8..23 of its FP32 pattern).  The threshold is the
//    best r seen so far plus the candidate window Delta(x), which bounds every
//    operand and FP32 rounding of the screen plus the oracle's FP64 error and
//    1e-5 D, so the kept set always holds the exact argmin and all near ties.
//    For the first group the epilogue takes two passes (minima, a barrier,
//    then the stores), so the threshold already covers 256 centroids.
//  * resolve, 4 threads per point: the stored values under the final
//    threshold are the candidates.  One candidate decides the label;
//    otherwise the candidates are re-ranked by the FP32 direct form with a
//    rigorous bound, then in FP64 in the oracle's order.  Points whose halves
//    did not fit go to a list that a second kernel resolves exactly over all
//    K (a fraction of a percent of points on split clusters).
// Labels only; the sums are formed by the sorted mean calculation.
// FP16 operands: the points are scaled by 2^ex (fixed with the points) and
// the centres by 2^ec (per step) so every coordinate is at most 2^14 in
// magnitude; the product is unscaled exactly in the epilogue's factor.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "km_internal.cuh"
#include "km_tcgen05.cuh"

namespace km {

namespace {

constexpr int kGM = 128;          // points per tile = TMEM lanes
constexpr int kGN = 256;          // centroids per MMA group = TMEM columns per accumulator
constexpr int kEpiWarps = 16;
constexpr int kEpiThreads = kEpiWarps * 32;
constexpr int kGThreads = kEpiThreads + 32;  // + the producer warp
constexpr int kSlots = 12;        // stored halves per point
constexpr int kHalf = 16;         // values per stored half
constexpr int kPtStride = kSlots * kHalf * 2 + 16;  // bytes per point (padding spreads banks)
constexpr int kTileBytes = kGM * kGemmD * 2;   // 16 KB of 16-bit operands per point tile
constexpr int kTieMax = 20;       // candidates per near-tie list entry (48 bytes)
constexpr int kTieChunk = 64;     // near-tie entries an epilogue warp reserves at a time
// shared-memory layout (bytes from the 1024-aligned base)
constexpr int kOffStore = 0;                                  // [128][kPtStride] bytes
constexpr int kOffSk = kOffStore + kGM * kPtStride;           // [128][kSlots] int16
constexpr int kOffThr = kOffSk + kGM * kSlots * 2;            // [2][128] u32
constexpr int kOffCnt = kOffThr + 2 * kGM * 4;                // [128] int
constexpr int kOffOver = kOffCnt + kGM * 4;                   // [128] int
constexpr int kOffStat = kOffOver + kGM * 4;                  // [4] int
constexpr int kOffBar = kOffStat + 16;                        // [10] mbarriers
constexpr int kOffTmem = kOffBar + 10 * 8;                    // TMEM base address
constexpr int kOffOperands = (kOffTmem + 4 + 1023) / 1024 * 1024;

// D(128 x 256, f32) += A(128 x 16, K-major) x B(256 x 16, K-major)^T with A
// and B both BF16 (A and B type fields 1) or both FP16 (fields 0)
constexpr uint32_t kIdescF16 = (1u << 4) | ((uint32_t)(kGN >> 3) << 17) | ((uint32_t)(kGM >> 4) << 24);
constexpr uint32_t kIdescBF16 = kIdescF16 | (1u << 7) | (1u << 10);

__device__ __forceinline__ void mma_16bit(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
               ::"r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ float fmin3g(float a, float b, float c) {
  float d;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}
// paired FP32 FMA, round to nearest: (a.lo, a.hi) * (b.lo, b.hi) + (c.lo, c.hi)
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b, unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ float lo_f(unsigned long long v) { return __uint_as_float((uint32_t)v); }
__device__ __forceinline__ float hi_f(unsigned long long v) { return __uint_as_float((uint32_t)(v >> 32)); }
// minimum of the 16 values in v[0..7] as a tree of depth 3 (eight
// three-input minima, the same count as a running chain of depth 8)
__device__ __forceinline__ float min16(const unsigned long long* v) {
  const float a = fmin3g(lo_f(v[0]), hi_f(v[0]), lo_f(v[1])), b = fmin3g(hi_f(v[1]), lo_f(v[2]), hi_f(v[2]));
  const float c = fmin3g(lo_f(v[3]), hi_f(v[3]), lo_f(v[4])), d = fmin3g(hi_f(v[4]), lo_f(v[5]), hi_f(v[5]));
  const float e = fmin3g(lo_f(v[6]), hi_f(v[6]), lo_f(v[7]));
  return fminf(fmin3g(a, b, c), fmin3g(d, e, hi_f(v[7])));
}
// Barrier of the 16 epilogue warps (named barrier 1) that also ORs a flag.
__device__ __forceinline__ bool epi_sync_or(bool v) {
  uint32_t r;
  asm volatile("{\n.reg .pred p, q;\nsetp.ne.u32 p, %1, 0;\nbar.red.or.pred q, 1, %2, p;\nselp.u32 %0, 1, 0, q;\n}"
               : "=r"(r) : "r"((uint32_t)v), "n"(kEpiThreads) : "memory");
  return r != 0;
}
// BF16 element index of (row, j) in the 128-byte-swizzled K-major layout
// (16-byte chunk j / 8 of row r sits at chunk (j / 8) ^ (r % 8))
__host__ __device__ __forceinline__ int64_t swz_index(int64_t row, int j) {
  return row * kGemmD + ((((j >> 3) ^ (int)(row & 7)) << 3) | (j & 7));
}

constexpr float kGU = 5.9604644775390625e-08f;  // 2^-24

// Bound on |FP32 direct form - FP64 oracle distance| (d = 64): the FP32
// rounding of sum_j (x~_j - c~_j)^2 against the exact D plus the oracle's own
// FP64 rounding.
__device__ __forceinline__ float bound64(float dv, float sA, float sB, float AB) {
  const float sd = sqrtf(fmaxf(dv, 0.f));
  return 1.01f * kGU * ((float)(kGemmD + 2) * dv + 2.f * sd * (sA + sB)) + 4.6e-16f * (float)(kGemmD + 1) * AB + 1e-30f;
}
// The oracle's distance: FP64, coordinates in order.
__device__ __forceinline__ double d64row(const float* __restrict__ xrow, const double* __restrict__ mrow) {
  double acc = 0.0;
  for (int j = 0; j < kGemmD; ++j) {
    const double t = __dsub_rn((double)xrow[j], mrow[j]);
    acc = __dadd_rn(acc, __dmul_rn(t, t));
  }
  return acc;
}

struct EpiSmem {
  unsigned char* store;  // [128][kPtStride]: per slot 16 values, 16 bits each (below)
  short* sk;        // [128][kSlots] first centroid of each stored half
  uint32_t* thr;    // [2][128] shared threshold (float bits), by tile parity
  int* cnt;         // [128] halves allocated
  int* over;        // [128] 1 if a half did not fit
};

// Keep the 16 values v[0..15] (columns k0..k0+15) of point p; past kSlots
// halves the point goes to the rescue list.  Each value is kept as bits 8..23
// of its FP32 pattern (one byte permute per pair): on the binade [1, 2) that
// holds the screen, q(r) = floor((r - 1) 2^15) + 2^15 is monotone in r, so a
// value r <= t tests q(r) <= q(t) and no value under the final threshold can
// be lost (values outside the binade only add candidates, resolved exactly).
__device__ __forceinline__ void store_half(const EpiSmem& s, int p, const unsigned long long* u, int k0) {
  const int slot = atomicAdd(&s.cnt[p], 1);
  if (slot < kSlots) {
    uint32_t w[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) w[q] = __byte_perm((uint32_t)u[q], (uint32_t)(u[q] >> 32), 0x6521);
    uint4* dst = reinterpret_cast<uint4*>(s.store + p * kPtStride + slot * kHalf * 2);
    dst[0] = make_uint4(w[0], w[1], w[2], w[3]);
    dst[1] = make_uint4(w[4], w[5], w[6], w[7]);
    s.sk[p * kSlots + slot] = (short)k0;
  } else {
    s.over[p] = 1;
  }
}

__global__ void __launch_bounds__(kGThreads, 1) gemm_assign_kernel(GemmArgs a) {
  extern __shared__ unsigned char raw[];
  if (a.ls->done) return;
  // 1024-byte-aligned base by pointer arithmetic on the shared array (keeps
  // the shared address space visible to the compiler)
  unsigned char* sm = raw + ((1024u - ((uint32_t)__cvta_generic_to_shared(raw) & 1023u)) & 1023u);
  const int kpad = a.kpad, NT = kpad / kGN;
  // fixed-offset per-point arrays first, then the 1024-aligned operand tiles
  EpiSmem es;
  es.store = sm + kOffStore;
  es.sk = reinterpret_cast<short*>(sm + kOffSk);
  es.thr = reinterpret_cast<uint32_t*>(sm + kOffThr);
  es.cnt = reinterpret_cast<int*>(sm + kOffCnt);
  es.over = reinterpret_cast<int*>(sm + kOffOver);
  int* s_stat = reinterpret_cast<int*>(sm + kOffStat);                                  // [4]
  unsigned long long* s_bar = reinterpret_cast<unsigned long long*>(sm + kOffBar);      // [10]
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(sm + kOffTmem);
  unsigned char* sC = sm + kOffOperands;                        // kpad x 128 B
  unsigned char* sA = sC + (size_t)kpad * 128;                  // 2 x 16 KB
  float* s_np = reinterpret_cast<float*>(sA + 2 * kTileBytes);  // [kpad] n'_k

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  auto bar_addr = [&](int q) { return (uint32_t)__cvta_generic_to_shared(&s_bar[q]); };
  // barriers: 0-1 a_full, 2-3 a_empty, 4-5 acc_full, 6-7 acc_empty, 8 centroids, 9 final
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(s_tmem)), "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    // a_empty completes on the MMAs' commit and on every epilogue warp
    // (the start estimate reads the point tile)
    for (int q = 0; q < 6; ++q) bar_init(bar_addr(q), (q == 2 || q == 3) ? 1 + kEpiWarps : 1);
    bar_init(bar_addr(6), kEpiWarps);
    bar_init(bar_addr(7), kEpiWarps);
    bar_init(bar_addr(8), 1);
    bar_init(bar_addr(9), 1);
  }
  if (tid < 4) s_stat[tid] = 0;
  for (int c = tid; c < kpad; c += kGThreads) s_np[c] = a.nprime[c];
  for (int q = tid; q < 2 * kGM; q += kGThreads) es.thr[q] = 0x7f800000u;  // +inf
  for (int q = tid; q < kGM; q += kGThreads) { es.cnt[q] = 0; es.over[q] = 0; }
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *s_tmem;
  const int ntiles = a.ntiles;
  const int nloc = (int)blockIdx.x < ntiles ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
  const GemmConst gc = *a.gc;
  bool aborted = false;

  if (warp == kEpiWarps) {
    // ---------------- producer: loads and MMAs (one thread) ----------------
    if (lane == 0) {
      const uint32_t sC_addr = (uint32_t)__cvta_generic_to_shared(sC);
      const uint32_t sA_addr = (uint32_t)__cvta_generic_to_shared(sA);
      const uint32_t idesc = a.f16 ? kIdescF16 : kIdescBF16;
      const unsigned char* xb = reinterpret_cast<const unsigned char*>(a.xb);
      auto load_tile = [&](int l) {
        const int s = l & 1;
        const int64_t tile = (int64_t)blockIdx.x + (int64_t)l * gridDim.x;
        bar_expect_tx(bar_addr(s), kTileBytes);
        bulk_load(sA_addr + s * kTileBytes, xb + tile * kTileBytes, kTileBytes, bar_addr(s));
      };
      int loads = 0;  // tiles whose load was issued
      if (nloc > 0) {
        bar_expect_tx(bar_addr(8), (uint32_t)kpad * 128u);
        bulk_load(sC_addr, a.cb, (uint32_t)kpad * 128u, bar_addr(8));
        for (; loads < min(2, nloc); ++loads) load_tile(loads);
        bool ok = wait_bar(bar_addr(8), 0);
        int gcount = 0, pending = -1;
        for (int l = 0; l < nloc && ok; ++l) {
          const int s = l & 1;
          ok = wait_bar(bar_addr(s), (uint32_t)(l >> 1) & 1u);
          for (int g = 0; g < NT && ok; ++g, ++gcount) {
            const int b = gcount & 1;
            if (gcount >= 2) ok = wait_bar(bar_addr(6 + b), ((uint32_t)(gcount >> 1) & 1u) ^ 1u);
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t d = tmem + (uint32_t)(b * kGN);
            const uint32_t abase = sA_addr + s * kTileBytes, bbase = sC_addr + (uint32_t)(g * kGN * 128);
#pragma unroll
            for (int kk = 0; kk < kGemmD / 16; ++kk)
              mma_16bit(d, sm_desc(abase + kk * 32), sm_desc(bbase + kk * 32), idesc, kk > 0 ? 1u : 0u);
            mma_commit(bar_addr(4 + b));
            if (g == 0 && pending >= 0) {
              // tile pending's MMAs were queued before this group: its stage
              // frees up while this group runs
              ok = wait_bar(bar_addr(2 + (pending & 1)), (uint32_t)(pending >> 1) & 1u);
              if (ok) { load_tile(pending + 2); ++loads; }
              pending = -1;
            }
          }
          if (!ok) break;
          mma_commit(bar_addr(2 + s));  // stage s is free once these MMAs complete
          if (l + 2 < nloc) pending = l;
        }
        if (!ok) a.ls->error = 3;  // a wait gave up
        // every MMA and copy issued must complete before TMEM and shared
        // memory are released
        mma_commit(bar_addr(9));
        wait_bar(bar_addr(9), 0);
        if (!ok)
          for (int l = max(0, loads - 2); l < loads; ++l) {
            // the last copy into each stage may still be in flight (earlier
            // ones were consumed before their stage was reloaded)
            wait_bar(bar_addr(l & 1), (uint32_t)(l >> 1) & 1u);
          }
      }
    }
  } else {
    // ---------------- epilogue warps ----------------
    const int quarter = warp & 3, cslice = warp >> 2;
    const int p = quarter * 32 + lane;  // TMEM lane = point within the tile
    const bool cold = a.ls->iter == 0;  // labels not yet from these centres' predecessors
    // the centroid matrix is resident (block-uniform decision: the named
    // barriers below need every epilogue warp)
    if (nloc > 0) {
      const bool ok8 = wait_bar(bar_addr(8), 0);
      __syncwarp();
      aborted = epi_sync_or(!ok8);
      if (aborted) a.ls->error = 3;
    }
    int gcount = 0;
    int nflag = 0, nresc = 0;
    // this warp's reserved near-tie entries [tnext, tend): one global atomic
    // per kTieChunk entries instead of one per warp and tile (every warp of
    // the grid adds to the same counter)
    unsigned tnext = 0, tend = 0;
    // per-point inputs of the next tile are loaded one tile ahead: z and
    // ||x~||^2 for the start estimate (4 threads per point, point tid / 4)
    // and ||x~||^2 for the window (point p)
    const int pp = tid >> 2, sub = tid & 3;
    int nz = 0;
    float nA4 = 0.f, nA = 0.f;
    auto prefetch = [&](int l) {
      if (l >= nloc) return;
      const int64_t t = (int64_t)blockIdx.x + (int64_t)l * gridDim.x;
      const int64_t i4 = t * kGM + pp, i1 = t * kGM + p;
      nz = i4 < a.n ? a.labels[i4] : 0;
      nA4 = i4 < a.n ? a.xa[i4] : 0.f;
      nA = i1 < a.n ? a.xa[i1] : 0.f;
    };
    // Start threshold of tile l from each point's previous label z (any
    // label in range bounds the minimum): r_z from the resident 16-bit
    // operands, 4 threads per point with 16 coordinates each, plus the window
    // and a bound on its difference from the tensor-core value of r_z.
    // Computed before the barrier that ends the previous tile, which
    // publishes it to the other warps.
    auto start_estimate = [&](int l, int z, float A4) {
      const int s = l & 1;
      const int64_t tile = (int64_t)blockIdx.x + (int64_t)l * gridDim.x;
      const bool okp = __all_sync(0xffffffffu, wait_bar(bar_addr(s), (uint32_t)(l >> 1) & 1u));
      const int64_t ii = tile * kGM + pp;
      float S = 0.f;
      z = (z >= 0 && z < a.k) ? z : 0;
      if (okp && ii < a.n) {
        const unsigned char* xr = sA + s * kTileBytes;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int c = 2 * sub + h;  // 16-byte chunk: coordinates 8c .. 8c+7
          const uint4 xv = *reinterpret_cast<const uint4*>(xr + pp * 128 + ((c ^ (pp & 7)) << 4));
          const uint4 cv = *reinterpret_cast<const uint4*>(sC + (size_t)z * 128 + ((c ^ (z & 7)) << 4));
          const uint32_t xw[4] = {xv.x, xv.y, xv.z, xv.w}, cw[4] = {cv.x, cv.y, cv.z, cv.w};
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            float2 xf, cf;
            if (a.f16) {
              xf = __half22float2(*reinterpret_cast<const __half2*>(&xw[q]));
              cf = __half22float2(*reinterpret_cast<const __half2*>(&cw[q]));
            } else {
              xf = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&xw[q]));
              cf = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&cw[q]));
            }
            S = __fmaf_rn(xf.x, cf.x, S);
            S = __fmaf_rn(xf.y, cf.y, S);
          }
        }
      }
      S = __fadd_rn(S, __shfl_xor_sync(0xffffffffu, S, 1));
      S = __fadd_rn(S, __shfl_xor_sync(0xffffffffu, S, 2));
      if (okp && ii < a.n && sub == 0) {
        const float nx = sqrtf(A4);
        const float t0 = __fmaf_rn(S, gc.scale, s_np[z]) + (gc.c0 + 4.8e-7f) + nx * (gc.c1 + gc.cest) + A4 * gc.cA;
        atomicMin(&es.thr[(l & 1) * kGM + pp], __float_as_uint(t0));
      }
      __syncwarp();
      if (lane == 0) bar_arrive(bar_addr(2 + s));  // done with the point tile
      if (!okp) a.ls->error = 3;
    };
    const unsigned long long sc2 = ((unsigned long long)__float_as_uint(gc.scale) << 32) | __float_as_uint(gc.scale);
    prefetch(0);
    if (nloc > 0 && !aborted) start_estimate(0, nz, nA4);
    float curA = nA;
    prefetch(1);
    __syncwarp();
    aborted = epi_sync_or(aborted);
    for (int l = 0; l < nloc && !aborted; ++l) {
      const int par = l & 1;
      const int64_t tile = (int64_t)blockIdx.x + (int64_t)l * gridDim.x;
      const int64_t i = tile * kGM + p;
      const bool valid = i < a.n;
      const float A = curA;
      const float delta = gc.c0 + sqrtf(A) * gc.c1 + A * gc.cA;
      uint32_t* thr_sh = es.thr + par * kGM;
      float thr = __uint_as_float(0x7f800000u);
      for (int g = 0; g < NT; ++g, ++gcount) {
        const int b = gcount & 1;
        bool ok = wait_bar(bar_addr(4 + b), (uint32_t)(gcount >> 1) & 1u);
        ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld below needs the whole warp
        if (!ok) a.ls->error = 3;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t ta = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * kGN + cslice * 64);
        const int kb = g * kGN + cslice * 64;
        // 32 columns: r values (16 pairs) and the minima of their two halves
        auto chunk = [&](int h2, unsigned long long* u, float& m0, float& m1) {
          tmem_ld32(ta + 32 * h2, u);
#pragma unroll
          for (int q = 0; q < 16; q += 2) {
            const ulonglong2 np = *reinterpret_cast<const ulonglong2*>(s_np + kb + 32 * h2 + 2 * q);
            u[q] = fma2(u[q], sc2, np.x);
            u[q + 1] = fma2(u[q + 1], sc2, np.y);
          }
          m0 = min16(u);
          m1 = min16(u + 8);
        };
        auto keep = [&](const unsigned long long* u, int kc, float m) {
          if (m <= thr) store_half(es, p, u, kc);
          thr = fminf(thr, m + delta);
        };
        auto release = [&]() {  // the accumulator may be overwritten
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          __syncwarp();
          if (lane == 0) bar_arrive(bar_addr(6 + b));
        };
        if (g == 0 && cold) {
          // first step after new centres (the labels give no start
          // threshold): minima of the first 256 columns first, then the
          // halves within the threshold are read again and stored
          float mn[4] = {0.f, 0.f, 0.f, 0.f};
          if (ok) {
            unsigned long long v[16];
            chunk(0, v, mn[0], mn[1]);
            chunk(1, v, mn[2], mn[3]);
            if (valid) atomicMin(&thr_sh[p], __float_as_uint(fminf(fminf(mn[0], mn[1]), fminf(mn[2], mn[3])) + delta));
          }
          __syncwarp();
          aborted = epi_sync_or(!ok);
          if (aborted) break;
          thr = __uint_as_float(thr_sh[p]);
#pragma unroll
          for (int h2 = 0; h2 < 2; ++h2) {
            const bool need = valid && (mn[2 * h2] <= thr || mn[2 * h2 + 1] <= thr);
            if (__any_sync(0xffffffffu, need)) {
              unsigned long long v[16];
              float m0, m1;
              chunk(h2, v, m0, m1);
              if (valid) {
                keep(v, kb + 32 * h2, mn[2 * h2]);
                keep(v + 8, kb + 32 * h2 + 16, mn[2 * h2 + 1]);
              }
            }
          }
          release();
        } else {
          aborted = !ok;  // warp-uniform; the end-of-tile barrier makes it block-wide
          if (aborted) break;
          thr = fminf(thr, __uint_as_float(thr_sh[p]));
          unsigned long long v[16];
          float m0, m1;
          chunk(0, v, m0, m1);
          if (valid) {
            keep(v, kb, m0);
            keep(v + 8, kb + 16, m1);
          }
          chunk(1, v, m0, m1);
          release();
          if (valid) {
            keep(v, kb + 32, m0);
            keep(v + 8, kb + 48, m1);
            atomicMin(&thr_sh[p], __float_as_uint(thr));
          }
        }
      }
      __syncwarp();
      aborted = epi_sync_or(aborted);  // all halves of the tile are stored
      if (aborted) break;

      // ---------------- resolve: 4 threads per point ----------------
      // The stored values under the final threshold are the candidates.  One
      // candidate is the label.  Up to kTieMax go to the near-tie list, more
      // (or a point whose halves did not fit) to the rescue list; both are
      // decided exactly by separate kernels.
      {
        const int64_t ii = tile * kGM + pp;
        const int nc = es.cnt[pp];
        const bool over = es.over[pp] != 0;
        const int ns = min(nc, kSlots);
        // the values (16-bit q, see store_half) under the final threshold t
        // are those with q <= q(t); t past the binade keeps every value
        const uint32_t tb = es.thr[par * kGM + pp];
        const uint32_t qt = tb >= 0x40000000u ? 0xFFFFu : tb < 0x3F800000u ? 0u : ((tb >> 8) & 0xFFFFu);
        const uint32_t qt2 = qt | (qt << 16);
        const unsigned char* srow = es.store + pp * kPtStride + sub * 8;
        auto slot_mask = [&](int j) {  // 4 bits: this thread's values of slot j under t
          const uint2 w = *reinterpret_cast<const uint2*>(srow + j * kHalf * 2);
          const uint32_t c0 = __vcmpleu2(w.x, qt2), c1 = __vcmpleu2(w.y, qt2);
          return (c0 & 1u) | ((c0 >> 15) & 2u) | ((c1 & 1u) << 2) | ((c1 >> 13) & 8u);
        };
        // this thread's 4-bit masks of the point's slots, kept for the
        // candidate pass below (kSlots x 4 bits fit in 64)
        unsigned long long masks = 0ull;
        int mine = 0;
        for (int j = 0; j < ns; ++j) {
          const uint32_t mm = slot_mask(j);
          masks |= (unsigned long long)mm << (4 * j);
          mine += __popc(mm);
        }
        const int n1 = __shfl_xor_sync(0xffffffffu, mine, 1);  // sub ^ 1
        const int n2 = __shfl_xor_sync(0xffffffffu, mine, 2);  // sub ^ 2
        const int n3 = __shfl_xor_sync(0xffffffffu, n1, 2);    // sub ^ 3
        const int tot = mine + n1 + n2 + n3;
        // candidates of the point's threads with a lower sub
        const int before = sub == 0 ? 0 : sub == 1 ? n1 : sub == 2 ? n2 + n3 : n1 + n2 + n3;
        const bool live = ii < a.n;
        // kind: 1 = decided here, 2 = near tie, 3 = rescue
        const int kind = !live ? 0 : (over || tot == 0 || tot > kTieMax) ? 3 : tot == 1 ? 1 : 2;
        // list slots: near ties from the warp's reserved entries (a new
        // chunk when they run out; the rest of the old one is used first),
        // rescues by one atomic per warp (rare)
        const bool lead = sub == 0;
        const unsigned btie = __ballot_sync(0xffffffffu, lead && kind == 2);
        const unsigned bres = __ballot_sync(0xffffffffu, lead && kind == 3);
        const unsigned ntie = (unsigned)__popc(btie), rem = tend - tnext, t0 = tnext;
        unsigned t1 = 0, base_r = 0;
        if (ntie > rem) {  // warp-uniform
          if (lane == 0) t1 = atomicAdd(a.tie_count, (unsigned)kTieChunk);
          t1 = __shfl_sync(0xffffffffu, t1, 0);
          tnext = t1 + (ntie - rem);
          tend = t1 + kTieChunk;
        } else {
          tnext += ntie;
        }
        if (bres) {
          if (lane == 0) base_r = atomicAdd(a.rescue_count, (unsigned)__popc(bres));
          base_r = __shfl_sync(0xffffffffu, base_r, 0);
        }
        const unsigned below = (1u << lane) - 1u;
        const unsigned jt = (unsigned)__popc(btie & ((1u << (lane & ~3)) - 1u));  // the point's rank
        const unsigned entry = jt < rem ? t0 + jt : t1 + (jt - rem);              // the point's entry
        if ((kind == 1 || kind == 2) && mine > 0) {
          // this thread's candidates: the label (one candidate in all) or
          // its part of the near-tie entry
          unsigned short* cl = reinterpret_cast<unsigned short*>(a.tie_list + 3 * (size_t)entry) + 4 + before;
          int q = 0;
          for (int j = 0; j < ns; ++j) {
            uint32_t mm = (uint32_t)(masks >> (4 * j)) & 0xFu;
            while (mm) {
              const int bb = __ffs((int)mm) - 1;
              mm &= mm - 1u;
              const int c = es.sk[pp * kSlots + j] + sub * 4 + bb;
              if (kind == 1) a.labels[ii] = c;
              else cl[q++] = (unsigned short)c;
            }
          }
        }
        if (lead && kind == 2) {
          *reinterpret_cast<int2*>(a.tie_list + 3 * (size_t)entry) = make_int2((int)ii, tot);
          ++nflag;
        }
        if (lead && kind == 3) {
          a.rescue_list[base_r + __popc(bres & below)] = (int32_t)ii;
          ++nresc;
        }
        // the 4 threads have read the point's slots; clear them for the next
        // tile (written again only after its first-group barrier)
        __syncwarp();
        if (lead) {
          es.cnt[pp] = 0;
          es.over[pp] = 0;
          es.thr[par * kGM + pp] = 0x7f800000u;  // next used by tile l + 2
        }
      }
      // the next tile's start threshold; the barrier publishes it and keeps
      // the next tile's stores behind every read of this tile's slots
      if (l + 1 < nloc) start_estimate(l + 1, nz, nA4);
      curA = nA;
      prefetch(l + 2);
      __syncwarp();
      aborted = epi_sync_or(aborted);
    }
    // unused reserved entries: marked empty (no candidates) for the tie kernel
    for (unsigned e = tnext + (unsigned)lane; e < tend; e += 32)
      *reinterpret_cast<int2*>(a.tie_list + 3 * (size_t)e) = make_int2(0, 0);
    if (nflag) atomicAdd(&s_stat[0], nflag);
    if (nresc) atomicAdd(&s_stat[2], nresc);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  if (tid == 0) {
    if (s_stat[0]) atomicAdd(&a.ls->flagged, (unsigned long long)s_stat[0]);
    if (s_stat[2]) {
      atomicAdd(&a.ls->overflowed, (unsigned long long)s_stat[2]);
      atomicAdd(&a.ls->flagged, (unsigned long long)s_stat[2]);
    }
  }
}

// Near ties listed by the assign kernel (2..kTieMax candidates under the
// final threshold): 4 threads per point (16 coordinates each) rank the
// candidates by the FP32 direct form with its rigorous bound; when that is
// not conclusive, the first thread decides in FP64 in the oracle's order
// (lowest index on ties).  Each group of 4 threads walks the list with a
// stride; the next entry is copied into shared memory (cp.async) while the
// current one is ranked, so the point's row and the first candidates' rows
// are requested as soon as an entry starts.
__global__ void __launch_bounds__(256, 4) gemm_tie_kernel(GemmArgs a) {
  __shared__ __align__(16) int4 s_ent[2][64][3];  // [stage][group] 48-byte entries
  if (a.ls->done) return;
  const unsigned cnt = *a.tie_count;
  const GemmConst gc = *a.gc;
  const int lane = threadIdx.x & 31, sub = lane & 3, grp = threadIdx.x >> 2;
  const unsigned gmask = 0xFu << (lane & ~3);
  const unsigned groups = gridDim.x * (blockDim.x / 4);
  const float sB = sqrtf(gc.B_max);
  auto fetch = [&](unsigned ee, int st) {  // threads 0..2 of the group copy 16 bytes each
    if (ee < cnt && sub < 3) {
      const uint32_t dst = (uint32_t)__cvta_generic_to_shared(&s_ent[st][grp][sub]);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(a.tie_list + 3 * (size_t)ee + sub));
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  int n64 = 0;
  unsigned e = (blockIdx.x * blockDim.x + threadIdx.x) / 4;
  fetch(e, 0);
  for (int st = 0; e < cnt; e += groups, st ^= 1) {
    fetch(e + groups, st ^ 1);
    asm volatile("cp.async.wait_group 1;" ::: "memory");
    __syncwarp(gmask);
    const int4 h = s_ent[st][grp][0];
    const int nc = h.y;
    if (nc != 0) {  // 0: an unused reserved entry (the same on the 4 threads)
      // candidate pairs as 32-bit words of the staged entry
      const uint32_t* cw = reinterpret_cast<const uint32_t*>(&s_ent[st][grp][0]) + 2;
      const int64_t ii = h.x;
      const float* xrow = a.xaos + (size_t)ii * kGemmD + sub * 16;
      const float A = a.xa[ii];
      float xt[16];
#pragma unroll
      for (int q = 0; q < 16; q += 4) {
        const float4 xv = *reinterpret_cast<const float4*>(xrow + q);
        const float4 sv = *reinterpret_cast<const float4*>(a.shift + sub * 16 + q);
        xt[q] = __fsub_rn(xv.x, sv.x);
        xt[q + 1] = __fsub_rn(xv.y, sv.y);
        xt[q + 2] = __fsub_rn(xv.z, sv.z);
        xt[q + 3] = __fsub_rn(xv.w, sv.w);
      }
      float best = 3.0e38f, second = 3.0e38f;
      int kbest = 0;
      auto partial = [&](const float4* cr) {  // this thread's 16 coordinates of sum (x~ - c~)^2
        float part = 0.f;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float4 cv = cr[j];
          float u = __fsub_rn(xt[4 * j], cv.x); part = __fmaf_rn(u, u, part);
          u = __fsub_rn(xt[4 * j + 1], cv.y); part = __fmaf_rn(u, u, part);
          u = __fsub_rn(xt[4 * j + 2], cv.z); part = __fmaf_rn(u, u, part);
          u = __fsub_rn(xt[4 * j + 3], cv.w); part = __fmaf_rn(u, u, part);
        }
        return part;
      };
      auto take = [&](int c, float part) {
        if (part < best || (part == best && c < kbest)) { second = best; best = part; kbest = c; }
        else if (part < second) second = part;
      };
      // two candidates per round (their loads in flight together), taken in
      // list order; padding columns (c >= K, the same on the 4 threads) skipped
#pragma unroll
      for (int q = 0; q < kTieMax; q += 2) {
        if (q >= nc) break;
        const int c0 = (int)(cw[q >> 1] & 0xFFFFu), c1 = q + 1 < nc ? (int)(cw[q >> 1] >> 16) : a.k;
        const bool v0 = c0 < a.k, v1 = c1 < a.k;
        float p0 = 0.f, p1 = 0.f;
        if (v0) p0 = partial(reinterpret_cast<const float4*>(a.ctil + (size_t)c0 * kGemmD + sub * 16));
        if (v1) p1 = partial(reinterpret_cast<const float4*>(a.ctil + (size_t)c1 * kGemmD + sub * 16));
        p0 = __fadd_rn(p0, __shfl_xor_sync(gmask, p0, 1));
        p1 = __fadd_rn(p1, __shfl_xor_sync(gmask, p1, 1));
        p0 = __fadd_rn(p0, __shfl_xor_sync(gmask, p0, 2));  // identical on the 4 threads
        p1 = __fadd_rn(p1, __shfl_xor_sync(gmask, p1, 2));
        if (v0) take(c0, p0);
        if (v1) take(c1, p1);
      }
      int lab = kbest;
      const float sA = sqrtf(A), AB = A + gc.B_max;
      const float e1 = bound64(best, sA, sB, AB), e2 = bound64(second, sA, sB, AB);
      const float lo2 = second - e2, hi1 = best + e1;
      const bool need64 = !((lo2 > hi1) && (lo2 - hi1 > gc.tau * (second + e2)));
      if (sub == 0) {
        if (need64) {
          // (rare) the candidates read again from the staged entry
          const unsigned short* cl = reinterpret_cast<const unsigned short*>(&s_ent[st][grp][0]) + 4;
          const float* xr = a.xaos + (size_t)ii * kGemmD;
          double bd = 0.0;
          int k64 = -1;
          for (int q = 0; q < nc; ++q) {
            const int c = cl[q];
            if (c >= a.k) continue;
            const double dd = d64row(xr, a.mu + (size_t)c * kGemmD);
            if (k64 < 0 || dd < bd || (dd == bd && c < k64)) { bd = dd; k64 = c; }
          }
          lab = k64;
          ++n64;
        }
        a.labels[ii] = lab;
      }
    }
    __syncwarp(gmask);  // stage st is refilled by the next iteration's copy
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  if (sub == 0 && n64) atomicAdd(&a.ls->fp64_decided, (unsigned long long)n64);
}

// Exact argmin over all K for the points listed by the assign kernel: one
// warp per point, lane l takes centroids l, l + 32, ...: FP32 direct form
// with its bound, then FP64 in the oracle's order over every centroid whose
// lower bound is not above the best upper bound (lowest index on ties).
__global__ void __launch_bounds__(256) gemm_rescue_kernel(GemmArgs a) {
  __shared__ float s_x[8][kGemmD];
  if (a.ls->done) return;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned cnt = *a.rescue_count;
  const GemmConst gc = *a.gc;
  int n64 = 0;
  for (unsigned e = blockIdx.x * 8u + w; e < cnt; e += gridDim.x * 8u) {
    const int64_t i = a.rescue_list[e];
    const float* xr = a.xaos + (size_t)i * kGemmD;
    s_x[w][lane] = __fsub_rn(xr[lane], a.shift[lane]);
    s_x[w][lane + 32] = __fsub_rn(xr[lane + 32], a.shift[lane + 32]);
    __syncwarp();
    const float A = a.xa[i];
    const float sA = sqrtf(A), sB = sqrtf(gc.B_max), AB = A + gc.B_max;
    float dv[kGemmMaxK / 32];
    float best = 3.0e38f;
#pragma unroll
    for (int t = 0; t < kGemmMaxK / 32; ++t) {
      const int c = lane + 32 * t;
      dv[t] = 3.0e38f;
      if (c < a.k) {
        const float* crow = a.ctil + (size_t)c * kGemmD;
        float acc = 0.f;
        for (int j = 0; j < kGemmD; j += 4) {
          const float4 cv = *reinterpret_cast<const float4*>(crow + j);
          float u = __fsub_rn(s_x[w][j], cv.x); acc = __fmaf_rn(u, u, acc);
          u = __fsub_rn(s_x[w][j + 1], cv.y); acc = __fmaf_rn(u, u, acc);
          u = __fsub_rn(s_x[w][j + 2], cv.z); acc = __fmaf_rn(u, u, acc);
          u = __fsub_rn(s_x[w][j + 3], cv.w); acc = __fmaf_rn(u, u, acc);
        }
        dv[t] = acc;
        best = fminf(best, acc);
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) best = fminf(best, __shfl_xor_sync(0xffffffffu, best, o));
    const float hi1 = best + bound64(best, sA, sB, AB);
    double bd = 0.0;
    int k64 = -1;
#pragma unroll
    for (int t = 0; t < kGemmMaxK / 32; ++t) {
      const int c = lane + 32 * t;
      if (c < a.k && dv[t] - bound64(dv[t], sA, sB, AB) <= hi1) {
        const double dd = d64row(xr, a.mu + (size_t)c * kGemmD);
        if (k64 < 0 || dd < bd || (dd == bd && c < k64)) { bd = dd; k64 = c; }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, bd, o);
      const int ok = __shfl_xor_sync(0xffffffffu, k64, o);
      if (ok >= 0 && (k64 < 0 || ob < bd || (ob == bd && ok < k64))) { bd = ob; k64 = ok; }
    }
    if (lane == 0) {
      a.labels[i] = k64;
      ++n64;
    }
    __syncwarp();
  }
  if (lane == 0 && n64) atomicAdd(&a.ls->fp64_decided, (unsigned long long)n64);
}

// Points -> 16-bit shifted rows in the swizzled tile layout (BF16, or FP16
// of 2^ex fl(x - s): an exact power-of-two scaling), ||x~||^2 (rounded up,
// coordinates in order) and an N x d FP32 copy.  One block of 128 threads
// per 128-point tile: the d x 128 block of points is staged in shared memory
// (coalesced reads of the d rows), then the AoS rows and the tile's 16 KB of
// swizzled 16-byte chunks are written coalesced.  Rows past N are left as
// they are (the caller zeroes the tile storage).
constexpr int kPrepPad = kGM + 1;
__global__ void __launch_bounds__(kGM) gemm_prep_points_kernel(const float* __restrict__ x, int64_t ld, int64_t n,
                                                             const float* __restrict__ shift, unsigned short* xb,
                                                             float* xa, float* xaos, int f16, float xscale) {
  __shared__ float s_x[kGemmD * kPrepPad];  // [j][row]
  const int tid = threadIdx.x;
  const int64_t base = (int64_t)blockIdx.x * kGM;
  const int rows = (int)min((int64_t)kGM, n - base);
  for (int j = 0; j < kGemmD; ++j) s_x[j * kPrepPad + tid] = tid < rows ? x[(int64_t)j * ld + base + tid] : 0.f;
  __syncthreads();
  if (tid < rows) {
    float A = 0.f;
    for (int j = 0; j < kGemmD; ++j) {
      const float t = __fsub_rn(s_x[j * kPrepPad + tid], shift[j]);
      A = __fmaf_ru(t, t, A);
    }
    xa[base + tid] = A;
  }
  for (int q = tid; q < rows * kGemmD; q += kGM) {
    const int r = q / kGemmD, j = q - r * kGemmD;
    xaos[(base + r) * kGemmD + j] = s_x[j * kPrepPad + r];
  }
  // 16-byte chunk p of row r holds coordinates 8 (p ^ (r & 7)) .. + 7
  for (int e = tid; e < rows * 8; e += kGM) {
    const int r = e >> 3, p = e & 7, c = p ^ (r & 7);
    uint32_t w[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const int j0 = 8 * c + 2 * h;
      const float t0 = __fsub_rn(s_x[j0 * kPrepPad + r], shift[j0]);
      const float t1 = __fsub_rn(s_x[(j0 + 1) * kPrepPad + r], shift[j0 + 1]);
      const uint32_t u0 = f16 ? __half_as_ushort(__float2half_rn(t0 * xscale)) : __bfloat16_as_ushort(__float2bfloat16_rn(t0));
      const uint32_t u1 = f16 ? __half_as_ushort(__float2half_rn(t1 * xscale)) : __bfloat16_as_ushort(__float2bfloat16_rn(t1));
      w[h] = u0 | (u1 << 16);
    }
    *reinterpret_cast<uint4*>(xb + (base + r) * kGemmD + p * 8) = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

// Tables of the next step from mu, one thread per centroid: BF16 rows in the
// swizzled layout (FP16 rows are written by the consts kernel, which knows
// their scale), FP32 c~ rows and B_k = ||mu_k - s||^2 (FP64, coordinates in
// order).
__global__ void __launch_bounds__(64) gemm_tables_kernel(GemmPrepArgs a) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= a.kpad) return;
  __nv_bfloat16* cb = reinterpret_cast<__nv_bfloat16*>(a.cb);
  double B = 0.0;
  for (int j = 0; j < kGemmD; ++j) {
    float cv = 0.f;
    if (c < a.k) {
      const double t = __dsub_rn(a.mu[(size_t)c * kGemmD + j], (double)a.shift[j]);
      cv = __double2float_rn(t);
      a.ctil[(size_t)c * kGemmD + j] = cv;
      B = __dadd_rn(B, __dmul_rn(t, t));
    }
    if (!a.f16) cb[swz_index(c, j)] = __float2bfloat16_rn(cv);
  }
  a.bnorm[c] = c < a.k ? B : 0.0;
}

// The scale and window constants from max_k B_k (one block), then n'_k and,
// for FP16 operands, the centre rows scaled by 2^ec.
__global__ void __launch_bounds__(256) gemm_consts_kernel(GemmPrepArgs a) {
  __shared__ double s_max[256];
  __shared__ int s_sigma, s_ec;
  const int k = a.k, kpad = a.kpad;
  double m = 0.0;
  for (int c = threadIdx.x; c < k; c += blockDim.x) m = fmax(m, a.bnorm[c]);
  s_max[threadIdx.x] = m;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) s_max[threadIdx.x] = fmax(s_max[threadIdx.x], s_max[threadIdx.x + w]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double bmax = s_max[0];
    const double P = 1.02 * ((double)a.A_max + 2.0 * bmax) + 1e-300;
    const double top = 0.5;  // binade [1, 2): M = 1.5, |2^sigma (h - 2S)| < 0.5
    int sigma = ilogb(top / P);
    if (ldexp(P, sigma) >= top) sigma -= 1;
    sigma = max(-120, min(120, sigma));
    s_sigma = sigma;
    const double u = 0x1p-24, tw = ldexp(1.0, sigma);
    const double sB = sqrt(bmax);
    // FP16: every |c~_kj| <= sqrt(B_max) is scaled to at most 2^14 (FP16
    // holds up to 65504), unless that would push the epilogue's factor
    // 2^(sigma + 1 - ex - ec) below FP32's normal range
    int ec = 0;
    double uop = 0x1p-8, ax = 0.0, ac = 0.0;
    if (a.f16) {
      const double cm = sB * 1.001 + 1e-300;
      ec = (int)floor(log2(0x1p14 / cm));
      while (ec > -200 && ldexp(cm, ec) > 0x1p14) --ec;
      ec = max(-100, min(ec, min(100, sigma + 126 - a.ex)));
      uop = 0x1p-11;
      ax = ldexp(0x1p-25, -a.ex);  // absolute rounding of a scaled value below 2^-14 (subnormal)
      ac = ldexp(0x1p-25, -ec);
    }
    s_ec = ec;
    // one operand: |fl16(fl32(t)) - t| <= (uop + 2^-24) |t| + a; a product of
    // two: (2 v + v^2) |x||c| + (1 + v)(a_c |x| + a_x |c|) + a_x a_c with
    // v = uop + 2^-24; summed over 64 coordinates (||.||_1 <= 8 ||.||) plus
    // the FP32 accumulation of 64 products in any order (<= 2^-16 sum |p|)
    const double v = uop + 0x1p-24;
    const double epsS = 2.0 * v + v * v + 0x1p-16;
    const double gam = 2.0 * 4.1 * (kGemmD + 1) * 0x1p-53;
    GemmConst g;
    g.scale = -(float)ldexp(1.0, sigma + 1 - (a.f16 ? a.ex + ec : 0));
    g.M = 1.5f;
    // Delta(x) = c0 + ||x~|| c1 + ||x~||^2 cA (units of r): two screen errors
    // 2 (epsS ||x~|| ||c~|| + 8 (1 + v)(a_c ||x~|| + a_x ||c~||) + 64 a_x a_c) + u h
    // each, the oracle's FP64 error, tie_rel * D2 with D2 <= (||x~|| + ||c~||)^2,
    // four ulps of the binade
    g.c0 = (float)((tw * (2.0 * u * bmax + gam * bmax + a.tie_rel * bmax + 4.0 * (8.0 * (1.0 + v) * ax * sB +
                                                                                64.0 * ax * ac)) +
                    8.0 * 0x1p-23) * (1.0 + 1e-3));
    g.c1 = (float)(tw * (4.0 * epsS * sB + 2.0 * a.tie_rel * sB + 4.0 * 8.0 * (1.0 + v) * ac) * (1.0 + 1e-3));
    g.cA = (float)(tw * (gam + a.tie_rel) * (1.0 + 1e-3));
    // start estimate: |r_est - r_tc| <= 2^(sigma+1) (2^-16 + 2^-18) ||x_b|| ||c_b|| (two FP32
    // sums of 64 products of 16-bit operands in different orders), taken as 2^-14 per unit ||x~||
    g.cest = (float)(2.0 * tw * 0x1p-14 * sB);
    g.B_max = (float)(bmax * (1.0 + 1e-6));
    g.tau = (float)(a.tie_rel * (1.0 + 1e-4));
    g.pad0 = g.pad1 = 0.f;
    *a.gc = g;
  }
  __syncthreads();
  const double tw = ldexp(1.0, s_sigma);
  // padding columns: r = 4, far above any real r < 2 plus the window
  for (int c = threadIdx.x; c < kpad; c += blockDim.x)
    a.nprime[c] = c < k ? __double2float_rn(1.5 + tw * a.bnorm[c]) : 4.0f;
  if (a.f16) {
    const float cs = ldexpf(1.f, s_ec);
    unsigned short* cb = reinterpret_cast<unsigned short*>(a.cb);
    for (int q = threadIdx.x; q < kpad * kGemmD; q += blockDim.x) {
      const int c = q / kGemmD, j = q - c * kGemmD;
      const float cv = c < k ? a.ctil[(size_t)c * kGemmD + j] : 0.f;
      cb[swz_index(c, j)] = __half_as_ushort(__float2half_rn(cv * cs));
    }
  }
}

// One thread waits on an mbarrier (expected count 1) that nothing arrives
// on: wait_bar gives up by its limit, and out[0] = 1 records it.
__global__ void wait_selftest_kernel(int* out) {
  __shared__ unsigned long long s_b;
  const uint32_t b = (uint32_t)__cvta_generic_to_shared(&s_b);
  bar_init(b, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  out[0] = wait_bar(b, 0) ? 0 : 1;
}

}  // namespace

cudaError_t launch_wait_selftest(int* out, cudaStream_t st) {
  wait_selftest_kernel<<<1, 1, 0, st>>>(out);
  return cudaGetLastError();
}

int64_t gemm_tie_entries(int64_t n, int grid) {
  // each point at most once, plus the reserved chunks' unused tails (at most
  // one chunk per epilogue warp)
  return n + (int64_t)grid * kEpiWarps * kTieChunk;
}

size_t gemm_smem_bytes(int kpad) {
  return 1024 + (size_t)kOffOperands + (size_t)kpad * 128 + 2 * kTileBytes + (size_t)kpad * 4;
}

int64_t gemm_xb_rows(int64_t n) { return (n + kGM - 1) / kGM * kGM; }

cudaError_t launch_gemm_assign(int grid, cudaStream_t st, const GemmArgs& a) {
  const size_t smem = gemm_smem_bytes(a.kpad);
  cudaError_t e = cudaFuncSetAttribute(gemm_assign_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // rescue_count and tie_count are adjacent: one memset clears both
  e = cudaMemsetAsync(a.rescue_count, 0, 2 * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  gemm_assign_kernel<<<grid, kGThreads, smem, st>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // one resident wave (4 blocks of 256 threads per SM at 64 registers); each
  // group of 4 threads strides over the list
  gemm_tie_kernel<<<grid * 4, 256, 0, st>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  gemm_rescue_kernel<<<grid * 4, 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_gemm_prep_points(const float* x, int64_t ld, int64_t n, const float* shift, void* xb, float* xa,
                                    float* xaos, int f16, int ex, cudaStream_t st) {
  // rows past N (to the next tile boundary) stay zero
  cudaError_t e = cudaMemsetAsync(xb, 0, (size_t)gemm_xb_rows(n) * kGemmD * 2, st);
  if (e != cudaSuccess) return e;
  const int64_t blocks = (n + kGM - 1) / kGM;  // < 2^24 (N < 2^31)
  gemm_prep_points_kernel<<<(unsigned)blocks, kGM, 0, st>>>(x, ld, n, shift, reinterpret_cast<unsigned short*>(xb),
                                                           xa, xaos, f16, std::ldexp(1.f, ex));
  return cudaGetLastError();
}

cudaError_t launch_gemm_prepare(cudaStream_t st, const GemmPrepArgs& a) {
  gemm_tables_kernel<<<(a.kpad + 63) / 64, 64, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  gemm_consts_kernel<<<1, 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace km
