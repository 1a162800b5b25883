// Reassignment for d = 64 in the GEMM form ||c||^2 - 2 x.c on the 5th-gen
// tensor cores (tcgen05, BF16 operands, FP32 accumulation in TMEM), the
// expectation step of Lloyd's algorithm (paper, section "The Lloyd's
// algorithm", step 2) where d is large enough for a dense contraction.
//
// Per CTA (one per SM, 512 threads): the whole centroid matrix stays in
// shared memory as BF16 rows of 128 bytes in the 128-byte-swizzled K-major
// layout; point tiles of 128 rows are double-buffered with cp.async.  One
// thread issues M=128, N=256, K=16 MMAs into two TMEM accumulators of 256
// columns (commit -> mbarrier, bounded waits).  16 warps read TMEM (4 per
// lane quarter, 64 columns each), form r_k = M + 2^sigma (h_k - 2 S_k) in one
// binade, and keep every centroid whose r is within the candidate window
// Delta(x) of the point's running minimum (the window bounds every BF16 and
// FP32 rounding plus 1e-5 * D: it always holds the exact argmin and all
// near ties).  The running minimum starts from the point's previous label,
// evaluated on the resident tiles.  A point with one candidate is decided;
// otherwise its candidates are re-ranked exactly (FP32 direct form with a
// rigorous bound, then FP64 in the oracle's order), over all K if the
// candidate list overflows.  Labels only; the sums are formed by the sorted
// mean calculation.
#include <cuda_bf16.h>

#include <algorithm>

#include "km_internal.cuh"

namespace km {

namespace {

constexpr int kGM = 128;        // points per tile = TMEM lanes
constexpr int kGN = 256;        // centroids per MMA group = TMEM columns per accumulator
constexpr int kGThreads = 512;  // 16 warps
constexpr int kGCand = 32;      // candidates kept per point
constexpr long kWaitLimit = 1L << 22;

__device__ __forceinline__ uint64_t sm_desc(uint32_t saddr) {
  // K-major, 128-byte swizzle: start address, LBO 16 B (unused), SBO 1024 B
  // (8 rows of 128 B), fixed 0b001 at bits 46-48, layout 2 at bits 61-63
  return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

// D(128 x 256, f32) += A(128 x 16, bf16, K-major) x B(256 x 16, bf16, K-major)^T
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kGN >> 3) << 17) |
                            ((uint32_t)(kGM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t acc) {
  asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
               ::"r"(tmem), "l"(ad), "l"(bd), "r"(kIdesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait on an mbarrier phase (at most ~1 s and kWaitLimit polls);
// returns false if it gave up.
__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity) {
  uint32_t ok = 0;
  const uint64_t t0 = gtimer();
  for (long it = 0; it < kWaitLimit && !ok; ++it) {
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                 : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    if (!ok && (it & 63) == 63 && gtimer() - t0 > 1000000000ull) break;
  }
  return ok != 0;
}
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                 "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
                 "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                 "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ float fmin3g(float a, float b, float c) {
  float d;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}
__device__ __forceinline__ void cp16(uint32_t dst, const void* src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(bytes));
}
// byte offset of 16-byte chunk c of row r in a 128B-swizzled K-major tile
__device__ __forceinline__ uint32_t swz(int r, int c) { return (uint32_t)(r * 128 + ((c ^ (r & 7)) << 4)); }

constexpr float kGU = 5.9604644775390625e-08f;  // 2^-24

// FP32 direct form sum_j (x~_j - c~_j)^2 and its bound against the exact D
// plus the oracle's FP64 rounding (d = 64).
__device__ __forceinline__ float direct64(const float* __restrict__ xrow, const float* __restrict__ s,
                                          const float* __restrict__ crow) {
  float dv = 0.f;
  for (int j = 0; j < kGemmD; ++j) {
    const float t = __fsub_rn(__fsub_rn(xrow[j], s[j]), crow[j]);
    dv = __fmaf_rn(t, t, dv);
  }
  return dv;
}
__device__ __forceinline__ float bound64(float dv, float sA, float sB, float AB) {
  const float sd = sqrtf(fmaxf(dv, 0.f));
  return 1.01f * kGU * ((float)(kGemmD + 2) * dv + 2.f * sd * (sA + sB)) + 4.6e-16f * (float)(kGemmD + 1) * AB + 1e-30f;
}
__device__ __forceinline__ double d64row(const float* __restrict__ xrow, const double* __restrict__ mrow) {
  double acc = 0.0;
  for (int j = 0; j < kGemmD; ++j) {
    const double t = __dsub_rn((double)xrow[j], mrow[j]);
    acc = __dadd_rn(acc, __dmul_rn(t, t));
  }
  return acc;
}

__global__ void __launch_bounds__(kGThreads, 1) gemm_assign_kernel(GemmArgs a) {
  extern __shared__ unsigned char raw[];
  if (a.ls->done) return;
  // 1024-byte-aligned base by pointer arithmetic on the shared array (keeps
  // the shared address space visible to the compiler)
  unsigned char* sm = raw + ((1024u - ((uint32_t)__cvta_generic_to_shared(raw) & 1023u)) & 1023u);
  const int kpad = a.kpad, NT = kpad / kGN;
  unsigned char* sC = sm;                                // kpad x 128 B
  unsigned char* sA = sC + (size_t)kpad * 128;           // 2 x 16 KB
  float* s_np = reinterpret_cast<float*>(sA + 2 * kGM * 128);  // [kpad] n'_k
  uint32_t* s_thr = reinterpret_cast<uint32_t*>(s_np + kpad);  // [128] float bits
  int* s_cnt = reinterpret_cast<int*>(s_thr + kGM);            // [128]
  uint32_t* s_cand = reinterpret_cast<uint32_t*>(s_cnt + kGM); // [128][kGCand]
  float* s_candr = reinterpret_cast<float*>(s_cand + kGM * kGCand);
  float* s_delta = s_candr + kGM * kGCand;                     // [128]
  float* s_shift = s_delta + kGM;                               // [64]
  int* s_stat = reinterpret_cast<int*>(s_shift + kGemmD);       // [4]
  unsigned long long* s_bar = reinterpret_cast<unsigned long long*>(s_stat + 4);  // [2], 8-aligned
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(s_bar + 2);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int quarter = warp & 3, cslice = warp >> 2;  // TMEM lanes 32*quarter.., columns 64*cslice..
  const GemmConst gc = *a.gc;
  const uint32_t bar0 = (uint32_t)__cvta_generic_to_shared(&s_bar[0]);
  const uint32_t bar1 = (uint32_t)__cvta_generic_to_shared(&s_bar[1]);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(s_tmem)), "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar0), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar1), "r"(1));
  }
  if (tid < 4) s_stat[tid] = 0;
  for (int j = tid; j < kGemmD; j += kGThreads) s_shift[j] = a.shift[j];
  for (int c = tid; c < kpad; c += kGThreads) s_np[c] = a.nprime[c];
  // centroid tiles, resident for the whole kernel
  for (int u = tid; u < kpad * 8; u += kGThreads) {
    const int r = u >> 3, c = u & 7;
    cp16((uint32_t)__cvta_generic_to_shared(sC + swz(r, c)), reinterpret_cast<const __nv_bfloat16*>(a.cb) + (size_t)r * kGemmD + c * 8, 16);
  }
  const int ntiles = a.ntiles;
  auto load_a = [&](int tile, int buf) {
    unsigned char* dstb = sA + buf * (kGM * 128);
    for (int u = tid; u < kGM * 8; u += kGThreads) {
      const int r = u >> 3, c = u & 7;
      const int64_t row = (int64_t)tile * kGM + r;
      const bool ok = row < a.n;
      cp16((uint32_t)__cvta_generic_to_shared(dstb + swz(r, c)), reinterpret_cast<const __nv_bfloat16*>(a.xb) + (ok ? row : 0) * kGemmD + c * 8, ok ? 16 : 0);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  if ((int)blockIdx.x < ntiles) load_a(blockIdx.x, 0);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *s_tmem;
  const uint32_t sC_addr = (uint32_t)__cvta_generic_to_shared(sC);
  uint32_t ph0 = 0, ph1 = 0;  // mbarrier phases
  bool aborted = false;
  int nflag = 0, n64 = 0, nover = 0;

  int local = 0;
  for (int tile = blockIdx.x; tile < ntiles && !aborted; tile += gridDim.x, ++local) {
    const int buf = local & 1;
    const uint32_t sA_addr = (uint32_t)__cvta_generic_to_shared(sA + buf * (kGM * 128));
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    auto issue = [&](int nt) {  // one thread: group nt into accumulator nt & 1
      const uint32_t d = tmem + (uint32_t)((nt & 1) * kGN);
      const uint32_t bbase = sC_addr + (uint32_t)(nt * kGN * 128);
#pragma unroll
      for (int kk = 0; kk < kGemmD / 16; ++kk)
        mma_bf16(d, sm_desc(sA_addr + kk * 32), sm_desc(bbase + kk * 32), kk > 0 ? 1u : 0u);
      mma_commit((nt & 1) ? bar1 : bar0);
    };
    if (tid == 0) {
      issue(0);
      if (NT > 1) issue(1);
    }
    // per-point start: threshold from the previous label, on the resident tiles
    if (tid < kGM) {
      const int p = tid;
      const int64_t i = (int64_t)tile * kGM + p;
      uint32_t thr_bits = 0u;  // rows past N keep no candidates
      if (i < a.n) {
        int z = a.labels[i];
        z = (z >= 0 && z < a.k) ? z : 0;
        const unsigned char* arow = sA + buf * (kGM * 128);
        float S = 0.f;
#pragma unroll 1
        for (int c = 0; c < 8; ++c) {
          const uint4 xv = *reinterpret_cast<const uint4*>(arow + swz(p, c));
          const uint4 cv = *reinterpret_cast<const uint4*>(sC + swz(z, c));
          const __nv_bfloat162* xh = reinterpret_cast<const __nv_bfloat162*>(&xv);
          const __nv_bfloat162* ch = reinterpret_cast<const __nv_bfloat162*>(&cv);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float2 xf = __bfloat1622float2(xh[q]), cf = __bfloat1622float2(ch[q]);
            S = __fmaf_rn(xf.x, cf.x, S);
            S = __fmaf_rn(xf.y, cf.y, S);
          }
        }
        const float A = a.xa[i];
        const float nx = sqrtf(A);
        const float delta = gc.c0 + nx * gc.c1 + A * gc.cA;
        s_delta[p] = delta;
        const float r_est = __fmaf_rn(S, gc.scale, s_np[z]);
        thr_bits = __float_as_uint(r_est + delta + nx * gc.cest);
      }
      s_thr[p] = thr_bits;
      s_cnt[p] = 0;
    }
    // prefetch the next tile's points into the other buffer (its last MMAs
    // completed in the previous tile)
    if (tile + (int)gridDim.x < ntiles) load_a(tile + gridDim.x, buf ^ 1);
    __syncthreads();

    const int p = quarter * 32 + lane;  // this thread's point (TMEM lane)
    // Two accumulators are read per round: first their chunk minima tighten
    // the point's threshold (over up to 512 centroids), then the chunks whose
    // minimum passes it are read again and their candidates collected.
    for (int nt0 = 0; nt0 < NT; nt0 += 2) {
      const int ng = min(2, NT - nt0);
      bool ok = true;
      for (int g = 0; g < ng; ++g) {
        const int nt = nt0 + g;
        ok = wait_bar((nt & 1) ? bar1 : bar0, (nt & 1) ? ph1 : ph0) && ok;
        if (nt & 1) ph1 ^= 1u; else ph0 ^= 1u;
      }
      ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld below needs the whole warp
      if (!ok) a.ls->error = 3;          // an MMA group did not complete in time
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const float delta = s_delta[p];
      float mins[2][2];
      if (ok) {
#pragma unroll
        for (int g = 0; g < 2; ++g) {
          if (g < ng) {
            const int nt = nt0 + g;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int col = cslice * 64 + h * 32;
              float v[32];
              tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)((nt & 1) * kGN + col), v);
              const int k0 = nt * kGN + col;
#pragma unroll
              for (int q = 0; q < 32; q += 4) {
                const float4 np = *reinterpret_cast<const float4*>(s_np + k0 + q);
                v[q] = __fmaf_rn(v[q], gc.scale, np.x);
                v[q + 1] = __fmaf_rn(v[q + 1], gc.scale, np.y);
                v[q + 2] = __fmaf_rn(v[q + 2], gc.scale, np.z);
                v[q + 3] = __fmaf_rn(v[q + 3], gc.scale, np.w);
              }
              float mn = fmin3g(v[0], v[1], v[2]);
#pragma unroll
              for (int q = 3; q < 31; q += 2) mn = fmin3g(mn, v[q], v[q + 1]);
              mn = fminf(mn, v[31]);
              mins[g][h] = mn;
              atomicMin(&s_thr[p], __float_as_uint(mn + delta));
            }
          }
        }
      }
      __syncthreads();
      if (ok) {
        const float thr = __uint_as_float(s_thr[p]);
#pragma unroll
        for (int g = 0; g < 2; ++g) {
          if (g < ng) {
            const int nt = nt0 + g;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              // the warp reads the chunk when any of its points needs it
              // (tcgen05.ld is warp-collective); each lane collects its own
              const bool mine = mins[g][h] <= thr;
              if (__any_sync(0xffffffffu, mine)) {
                const int col = cslice * 64 + h * 32;
                float v[32];
                tmem_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)((nt & 1) * kGN + col), v);
                const int k0 = nt * kGN + col;
#pragma unroll
                for (int q = 0; q < 32; ++q) {
                  const float r = __fmaf_rn(v[q], gc.scale, s_np[k0 + q]);
                  if (mine && r <= thr) {
                    const int slot = atomicAdd(&s_cnt[p], 1);
                    if (slot < kGCand) {
                      s_cand[p * kGCand + slot] = (uint32_t)(k0 + q);
                      s_candr[p * kGCand + slot] = r;
                    }
                  }
                }
              }
            }
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      aborted = __syncthreads_or(ok ? 0 : 1) != 0;  // block-uniform
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (aborted) break;
      if (tid == 0)
        for (int g = 0; g < 2; ++g)
          if (nt0 + 2 + g < NT) issue(nt0 + 2 + g);
    }
    if (aborted) break;
    // Resolve: 4 threads per point (16 coordinates each).  One candidate
    // decides the label; otherwise the candidates (all K after an overflow)
    // are ranked by the FP32 direct form summed over the 4 threads (its
    // bound does not depend on the summation order), then, if that is not
    // conclusive, in FP64 in the oracle's order by the point's first thread.
    {
      const int pp = tid >> 2, sub = tid & 3;
      const unsigned gmask = 0xFu << (lane & ~3);
      const int64_t i = (int64_t)tile * kGM + pp;
      if (i < a.n) {
        const float thr = __uint_as_float(s_thr[pp]);
        const int nc = s_cnt[pp];
        int nl = 0, only = -1;
        if (nc <= kGCand)
          for (int q = 0; q < nc; ++q)
            if (s_candr[pp * kGCand + q] <= thr) { ++nl; only = (int)s_cand[pp * kGCand + q]; }
        const bool over = nc > kGCand || nl == 0;  // scan all K (an empty list cannot happen; kept safe)
        int lab = only;
        if (over || nl != 1) {
          const float* xrow = a.xaos + (size_t)i * kGemmD + sub * 16;
          float xt[16];
#pragma unroll
          for (int q = 0; q < 16; q += 4) {
            const float4 v = *reinterpret_cast<const float4*>(xrow + q);
            xt[q] = __fsub_rn(v.x, s_shift[sub * 16 + q]);
            xt[q + 1] = __fsub_rn(v.y, s_shift[sub * 16 + q + 1]);
            xt[q + 2] = __fsub_rn(v.z, s_shift[sub * 16 + q + 2]);
            xt[q + 3] = __fsub_rn(v.w, s_shift[sub * 16 + q + 3]);
          }
          const int m = over ? a.k : nc;
          float best = 3.0e38f, second = 3.0e38f;
          int kb = 0;
#pragma unroll 4
          for (int q = 0; q < m; ++q) {
            int c;
            bool use = true;
            if (over) c = q;
            else {
              use = s_candr[pp * kGCand + q] <= thr;  // same decision on all 4 threads
              c = (int)s_cand[pp * kGCand + q];
            }
            const float* crow = a.ctil + (size_t)c * kGemmD + sub * 16;
            float part = 0.f;
#pragma unroll
            for (int j = 0; j < 16; j += 4) {
              const float4 cv = *reinterpret_cast<const float4*>(crow + j);
              float t = __fsub_rn(xt[j], cv.x); part = __fmaf_rn(t, t, part);
              t = __fsub_rn(xt[j + 1], cv.y); part = __fmaf_rn(t, t, part);
              t = __fsub_rn(xt[j + 2], cv.z); part = __fmaf_rn(t, t, part);
              t = __fsub_rn(xt[j + 3], cv.w); part = __fmaf_rn(t, t, part);
            }
            part = __fadd_rn(part, __shfl_xor_sync(gmask, part, 1));
            part = __fadd_rn(part, __shfl_xor_sync(gmask, part, 2));  // identical on the 4 threads
            if (use) {
              if (part < best || (part == best && c < kb)) { second = best; best = part; kb = c; }
              else if (part < second) second = part;
            }
          }
          if (sub == 0 && over) ++nover;
          lab = kb;
          const float A = a.xa[i];
          const float sA = sqrtf(A), sB = sqrtf(gc.B_max), AB = A + gc.B_max;
          const float e1 = bound64(best, sA, sB, AB), e2 = bound64(second, sA, sB, AB);
          const float lo2 = second - e2, hi1 = best + e1;
          const bool need64 = second < 3.0e38f && !((lo2 > hi1) && (lo2 - hi1 > gc.tau * (second + e2)));
          if (need64 && sub == 0) {
            const float* xr = a.xaos + (size_t)i * kGemmD;
            double bd = 0.0;
            int k64 = -1;
            for (int q = 0; q < m; ++q) {
              int c;
              if (over) c = q;
              else {
                if (!(s_candr[pp * kGCand + q] <= thr)) continue;
                c = (int)s_cand[pp * kGCand + q];
              }
              const double dd = d64row(xr, a.mu + (size_t)c * kGemmD);
              if (k64 < 0 || dd < bd || (dd == bd && c < k64)) { bd = dd; k64 = c; }
            }
            lab = k64;
            ++n64;
          }
          if (sub == 0) ++nflag;
        }
        if (sub == 0) a.labels[i] = lab;
      }
    }
    // the next tile rewrites the per-point arrays after its first barrier
  }
  // drain: every issued MMA group has been waited on unless aborted; if
  // aborted, wait (bounded) for both accumulators before releasing TMEM
  if (aborted) {
    wait_bar(bar0, ph0);
    wait_bar(bar1, ph1);
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  if (nflag) atomicAdd(&s_stat[0], nflag);
  if (n64) atomicAdd(&s_stat[1], n64);
  if (nover) atomicAdd(&s_stat[2], nover);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  if (tid == 0) {
    if (s_stat[0]) atomicAdd(&a.ls->flagged, (unsigned long long)s_stat[0]);
    if (s_stat[1]) atomicAdd(&a.ls->fp64_decided, (unsigned long long)s_stat[1]);
    if (s_stat[2]) atomicAdd(&a.ls->overflowed, (unsigned long long)s_stat[2]);
  }
}

// Points -> BF16 shifted rows, ||x~||^2 (rounded up) and an N x d FP32 copy.
__global__ void gemm_prep_points_kernel(const float* __restrict__ x, int64_t ld, int64_t n, const float* shift,
                                        __nv_bfloat16* xb, float* xa, float* xaos) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float A = 0.f;
    for (int j = 0; j < kGemmD; ++j) {
      const float v = x[(int64_t)j * ld + i];
      const float t = __fsub_rn(v, shift[j]);
      xaos[i * kGemmD + j] = v;
      xb[i * kGemmD + j] = __float2bfloat16_rn(t);
      A = __fmaf_ru(t, t, A);
    }
    xa[i] = A;
  }
}

// Tables of the next step from mu (one block): BF16 centroid rows, n'_k,
// FP32 c~ rows, the scale and the candidate-window constants.
__global__ void __launch_bounds__(256) gemm_prepare_kernel(GemmPrepArgs a) {
  __shared__ double s_b[1024];
  __shared__ double s_bmax;
  __shared__ int s_sigma;
  const int k = a.k, kpad = a.kpad;
  for (int c = threadIdx.x; c < kpad; c += blockDim.x) {
    double B = 0.0;
    for (int j = 0; j < kGemmD; ++j) {
      float cv = 0.f;
      if (c < k) {
        const double t = __dsub_rn(a.mu[(size_t)c * kGemmD + j], (double)a.shift[j]);
        cv = __double2float_rn(t);
        a.ctil[(size_t)c * kGemmD + j] = cv;
        B = __dadd_rn(B, __dmul_rn(t, t));
      }
      reinterpret_cast<__nv_bfloat16*>(a.cb)[(size_t)c * kGemmD + j] = __float2bfloat16_rn(cv);
    }
    if (c < 1024) s_b[c] = c < k ? B : 0.0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double bmax = 0.0;
    for (int c = 0; c < k; ++c) bmax = fmax(bmax, s_b[c]);
    s_bmax = bmax;
    const double P = 1.02 * ((double)a.A_max + 2.0 * bmax) + 1e-300;
    const double top = 0.5;  // binade [1, 2): M = 1.5, |2^sigma (h - 2S)| < 0.5
    int sigma = ilogb(top / P);
    if (ldexp(P, sigma) >= top) sigma -= 1;
    sigma = max(-120, min(120, sigma));
    s_sigma = sigma;
    const double u = 0x1p-24, tw = ldexp(1.0, sigma);
    const double epsS = 0x1p-7 * 1.0003 + 0x1p-16;  // BF16 products + FP32 accumulation
    const double sB = sqrt(bmax);
    const double gam = 2.0 * 4.1 * (kGemmD + 1) * 0x1p-53;
    GemmConst g;
    g.scale = -(float)ldexp(1.0, sigma + 1);
    g.M = 1.5f;
    // Delta(x) = c0 + ||x~|| c1 + ||x~||^2 cA (units of r): two screen errors
    // 2 epsS ||x~|| ||c~|| + u h each, the oracle's FP64 error, tie_rel * D2
    // with D2 <= (||x~|| + ||c~||)^2, four ulps of the binade
    g.c0 = (float)((tw * (2.0 * u * bmax + gam * bmax + a.tie_rel * bmax) + 8.0 * 0x1p-23) * (1.0 + 1e-3));
    g.c1 = (float)(tw * (4.0 * epsS * sB + 2.0 * a.tie_rel * sB) * (1.0 + 1e-3));
    g.cA = (float)(tw * (gam + a.tie_rel) * (1.0 + 1e-3));
    // start estimate (FP32 dot product in another order): 2^(sigma+1) 2^-17 ||x~|| ||c~|| + 2 ulps
    g.cest = (float)(2.0 * tw * 0x1p-17 * sB * 1.02 + 0.0);
    g.B_max = (float)(bmax * (1.0 + 1e-6));
    g.tau = (float)(a.tie_rel * (1.0 + 1e-4));
    g.pad0 = g.pad1 = 0.f;
    *a.gc = g;
  }
  __syncthreads();
  const double tw = ldexp(1.0, s_sigma);
  for (int c = threadIdx.x; c < kpad; c += blockDim.x)
    a.nprime[c] = c < k ? __double2float_rn(1.5 + tw * s_b[c]) : 1.99999988f;  // padding: top of the binade
}

}  // namespace

size_t gemm_smem_bytes(int kpad) {
  return 1024 + (size_t)kpad * 128 + 2 * kGM * 128 + (size_t)kpad * 4 + kGM * 4 * 2 + (size_t)kGM * kGCand * 8 +
         kGM * 4 + kGemmD * 4 + 16 + 32;
}

cudaError_t launch_gemm_assign(int grid, cudaStream_t st, const GemmArgs& a) {
  const size_t smem = gemm_smem_bytes(a.kpad);
  cudaError_t e = cudaFuncSetAttribute(gemm_assign_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  gemm_assign_kernel<<<grid, kGThreads, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_gemm_prep_points(const float* x, int64_t ld, int64_t n, const float* shift, void* xb, float* xa,
                                    float* xaos, cudaStream_t st) {
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 4096));
  gemm_prep_points_kernel<<<(unsigned)blocks, 256, 0, st>>>(x, ld, n, shift, reinterpret_cast<__nv_bfloat16*>(xb),
                                                            xa, xaos);
  return cudaGetLastError();
}

cudaError_t launch_gemm_prepare(cudaStream_t st, const GemmPrepArgs& a) {
  gemm_prepare_kernel<<<1, 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace km
