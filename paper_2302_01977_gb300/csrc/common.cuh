// common.cuh -- device helpers shared by the libjlsketch kernels (sm_103a).
//
// * Philox4x64-10 (Salmon et al., SC'11) and Lemire's bounded integers
//   (Lemire, ACM TOMACS 2019): the counter-based streams every operator is
//   drawn from, so that R is a pure function of (seed, tag, counter).
// * device-side error flags: kernels never trap; a violated bound or a wait
//   that runs out sets a bit in the handle's flag and the kernel returns.
// * bounded mbarrier waits, TMA (cp.async.bulk.tensor) and cp.async wrappers.
#pragma once

#include <cstdint>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace jls {

// ---- error flag bits ------------------------------------------------------
enum : int { ERRF_BOUNDS = 1, ERRF_TIMEOUT = 2, ERRF_RNG = 4, ERRF_NUMERIC = 8 };

__device__ __forceinline__ void set_err(int* err, int bit) {
  if (err) atomicOr(err, bit);
}

// ---- Philox4x64-10 ---------------------------------------------------------
struct u64x4 { uint64_t x0, x1, x2, x3; };

constexpr uint64_t PHILOX_M0 = 0xD2E7470EE14C6C93ull;
constexpr uint64_t PHILOX_M1 = 0xCA5A826395121157ull;
constexpr uint64_t PHILOX_W0 = 0x9E3779B97F4A7C15ull;
constexpr uint64_t PHILOX_W1 = 0xBB67AE8584CAA73Bull;

// stream tags: ASCII name in the high 32 bits (block index in the low bits)
constexpr uint64_t TAG_SJLT = 0x534A4C54ull << 32;
constexpr uint64_t TAG_SRHT_D = 0x53524844ull << 32;
constexpr uint64_t TAG_SRHT_MU = 0x5352484Dull << 32;
constexpr uint64_t TAG_GAUSS = 0x47415553ull << 32;

__device__ __forceinline__ u64x4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3,
                                               uint64_t k0, uint64_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t lo0 = PHILOX_M0 * c0, hi0 = __umul64hi(PHILOX_M0, c0);
    const uint64_t lo1 = PHILOX_M1 * c2, hi1 = __umul64hi(PHILOX_M1, c2);
    const uint64_t n0 = hi1 ^ c1 ^ k0;
    const uint64_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += PHILOX_W0; k1 += PHILOX_W1;
  }
  return u64x4{c0, c1, c2, c3};
}

// value = floor(w * s / 2^64); rejected when the low half of the product is
// below (2^64 - s) mod s.  Returns true when accepted.
__device__ __forceinline__ bool lemire(uint64_t w, uint64_t s, uint64_t* value) {
  const uint64_t lo = w * s;
  *value = __umul64hi(w, s);
  if (lo < s) {
    const uint64_t t = (0ull - s) % s;
    if (lo < t) return false;
  }
  return true;
}

__device__ __forceinline__ double u53_open0(uint64_t w) {  // (0, 1]
  return (double)((w >> 11) + 1ull) * 0x1.0p-53;
}
__device__ __forceinline__ double u53(uint64_t w) {  // [0, 1)
  return (double)(w >> 11) * 0x1.0p-53;
}

// ---- time (ns) for bounded waits ---------------------------------------------
__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
constexpr uint64_t WAIT_LIMIT_NS = 2000000000ull;  // 2 s

// ---- shared-memory addresses -------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---- mbarrier ----------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("{ .reg .b64 st; mbarrier.arrive.shared::cta.b64 st, [%0]; }" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("{ .reg .b64 st; mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1; }" ::"r"(bar),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// try_wait that may suspend the thread for up to `ns` nanoseconds (it wakes
// early when the phase completes), so waiting warps do not spin on the issue
// slots that working warps need.
__device__ __forceinline__ bool mbar_try_wait_hint(uint32_t bar, uint32_t parity, uint32_t ns) {
  uint32_t ok;
  asm volatile(
      "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3; selp.u32 %0, 1, 0, p; }"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(ns)
      : "memory");
  return ok != 0;
}
// Wait for the phase with `parity` to complete; gives up after WAIT_LIMIT_NS,
// sets ERRF_TIMEOUT and returns false.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer_ns();
  while (true) {
    if (mbar_try_wait_hint(bar, parity, 100000u)) return true;
    if (globaltimer_ns() - t0 > WAIT_LIMIT_NS) {
      set_err(err, ERRF_TIMEOUT);
      return false;
    }
  }
}

// ---- TMA (tiled tensor copies) -------------------------------------------------
__device__ __forceinline__ void tma_prefetch_desc(const void* tmap) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(tmap)) : "memory");
}
// Ask for a 2-D tile of a tensor to be brought into L2 (a hint: nothing waits on it).
__device__ __forceinline__ void tma_prefetch_l2_2d(const void* tmap, int32_t x, int32_t y) {
  asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"(
                   reinterpret_cast<uint64_t>(tmap)),
               "r"(x), "r"(y)
               : "memory");
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void* tmap, uint32_t bar, int32_t x,
                                            int32_t y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tmap)), "r"(bar), "r"(x), "r"(y)
      : "memory");
}

// ---- cp.async (per-thread asynchronous copies) --------------------------------------
// 4-byte copy; src_bytes == 0 writes zeros without reading.
__device__ __forceinline__ void cp_async_4(uint32_t dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_8(uint32_t dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// ---- shared-memory loads by 32-bit address -----------------------------------------
__device__ __forceinline__ uint4 lds_u4(uint32_t a) {
  uint4 v;
  asm volatile("ld.shared.v4.u32 {%0,%1,%2,%3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
  return v;
}
__device__ __forceinline__ uint2 lds_u2(uint32_t a) {
  uint2 v;
  asm volatile("ld.shared.v2.u32 {%0,%1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(a));
  return v;
}
__device__ __forceinline__ float4 lds_f4(uint32_t a) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0,%1,%2,%3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
  return v;
}
__device__ __forceinline__ double2 lds_d2(uint32_t a) {
  double2 v;
  asm volatile("ld.shared.v2.f64 {%0,%1}, [%2];" : "=d"(v.x), "=d"(v.y) : "r"(a));
  return v;
}
__device__ __forceinline__ float lds_f1(uint32_t a) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ double lds_d1(uint32_t a) {
  double v;
  asm volatile("ld.shared.f64 %0, [%1];" : "=d"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ uint32_t lds_u32(uint32_t a) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
  return v;
}

__host__ __device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }

// ---- e4m3 (FP8) conversions ---------------------------------------------------------
// e4m3x2 of (lo, hi): `lo` in the lower byte (the lower address), round to
// nearest, saturating at +-448.
__device__ __forceinline__ uint32_t e4m3x2(float lo, float hi) {
  unsigned short d;
  asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(d) : "f"(hi), "f"(lo));
  return d;
}
// The two values of an e4m3x2 pair, exactly, as FP32.
__device__ __forceinline__ float2 e4m3x2_to_f2(uint32_t q) {
  uint32_t h2;
  asm("cvt.rn.f16x2.e4m3x2 %0, %1;" : "=r"(h2) : "h"((unsigned short)q));
  const __half2 h = *reinterpret_cast<const __half2*>(&h2);
  return __half22float2(h);
}
__device__ __forceinline__ bool elect_lane0() { return (threadIdx.x & 31) == 0; }

}  // namespace jls
