// tcgen05 / mbarrier / bulk-copy helpers shared by the tensor-core kernels
// (inline PTX for sm_103a).  Every wait is bounded: wait_bar gives up after
// about one second and the caller records an error instead of hanging.
#pragma once
#include <cstdint>

namespace km {
namespace {

constexpr long kWaitLimit = 1L << 22;

__device__ __forceinline__ uint64_t sm_desc(uint32_t saddr) {
  // K-major, 128-byte swizzle: start address, LBO 16 B (unused), SBO 1024 B
  // (8 rows of 128 B), fixed 0b001 at bits 46-48, layout 2 at bits 61-63
  return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void bar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void bar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void bar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// bulk global -> shared copy completing on an mbarrier (16-byte aligned
// addresses, size a multiple of 16)
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Bounded wait on an mbarrier phase: each try may suspend the thread for up
// to 20 us until the phase completes; gives up (returns false) after ~1 s.
__device__ __forceinline__ bool try_bar(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}"
               : "=r"(ok) : "r"(bar), "r"(parity), "r"(20000) : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity) {
  if (try_bar(bar, parity)) return true;
  const uint64_t t0 = gtimer();
  for (long it = 0; it < kWaitLimit; ++it) {
    if (try_bar(bar, parity)) return true;
    if (gtimer() - t0 > 1000000000ull) break;
  }
  return false;
}
// 32 consecutive TMEM columns of the warp's 32 lanes, waited for, as 16
// pairs of FP32 values (column 2q in the low half of v[q])
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, unsigned long long* v) {
  asm volatile("{\n.reg .b32 t0,t1,t2,t3,t4,t5,t6,t7,t8,t9,t10,t11,t12,t13,t14,t15,t16,t17,t18,t19,t20,t21,t22,t23,t24,t25,t26,t27,t28,t29,t30,t31;\n"
               "tcgen05.ld.sync.aligned.32x32b.x32.b32 {t0,t1,t2,t3,t4,t5,t6,t7,t8,t9,t10,t11,t12,t13,t14,t15,t16,t17,t18,t19,t20,t21,t22,t23,t24,t25,t26,t27,t28,t29,t30,t31}, [%16];\n"
               "tcgen05.wait::ld.sync.aligned;\n"
               "mov.b64 %0, {t0, t1};\nmov.b64 %1, {t2, t3};\nmov.b64 %2, {t4, t5};\nmov.b64 %3, {t6, t7};\nmov.b64 %4, {t8, t9};\nmov.b64 %5, {t10, t11};\nmov.b64 %6, {t12, t13};\nmov.b64 %7, {t14, t15};\nmov.b64 %8, {t16, t17};\nmov.b64 %9, {t18, t19};\nmov.b64 %10, {t20, t21};\nmov.b64 %11, {t22, t23};\nmov.b64 %12, {t24, t25};\nmov.b64 %13, {t26, t27};\nmov.b64 %14, {t28, t29};\nmov.b64 %15, {t30, t31};\n}"
               : "=l"(v[0]), "=l"(v[1]), "=l"(v[2]), "=l"(v[3]), "=l"(v[4]), "=l"(v[5]), "=l"(v[6]), "=l"(v[7]), "=l"(v[8]), "=l"(v[9]), "=l"(v[10]), "=l"(v[11]), "=l"(v[12]), "=l"(v[13]), "=l"(v[14]), "=l"(v[15])
               : "r"(taddr) : "memory");
}
}  // namespace
}  // namespace km
