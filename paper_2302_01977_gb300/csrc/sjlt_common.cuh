// sjlt_common.cuh -- device pieces shared by the SJLT apply kernels
// (sjlt_apply.cu: one operator; sjlt_batch.cu: many operators in one launch):
// bulk and per-thread asynchronous copies, the reduction of per-block partial
// sums into a zeroed output, the stream-K range of a CTA and the S' (A^T R)
// accumulators of a lane's four columns.
#pragma once

#include <cstdint>

#include "common.cuh"

namespace jls {

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void cp_async_16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_mbar_arrive(uint32_t bar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}

// accumulate a contribution into the zeroed output (<= 2 contributors per cell)
__device__ __forceinline__ void red_add4(float* p, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1,%2,%3,%4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d) : "memory");
}
__device__ __forceinline__ void red_add1(float* p, float a) { atomicAdd(p, a); }
__device__ __forceinline__ void red_add1(double* p, double a) { atomicAdd(p, a); }

// Add scale * v[b] (b < nb) to output row `out_row` (columns cw0 + b).
template <int NB>
__device__ __forceinline__ void flush_row(float* out_row, const float (&v)[NB], int nb, float scale, bool vec_ok) {
#pragma unroll
  for (int b = 0; b < NB; b += 4) {
    if (b + 3 < nb && vec_ok) {
      red_add4(out_row + b, v[b] * scale, v[b + 1] * scale, v[b + 2] * scale, v[b + 3] * scale);
    } else {
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (b + u < nb) red_add1(out_row + b + u, v[b + u] * scale);
    }
  }
}
template <int NB>
__device__ __forceinline__ void flush_row(double* out_row, const double (&v)[NB], int nb, double scale, bool) {
#pragma unroll
  for (int b = 0; b < NB; ++b)
    if (b < nb) red_add1(out_row + b, v[b] * scale);
}

// Add scale * (re[b], -im[b]) (b < nb) to the complex output row `out` (FP32 pairs).
__device__ __forceinline__ void red_add2(float* p, float a, float b) {
  asm volatile("red.global.add.v2.f32 [%0], {%1,%2};" ::"l"(p), "f"(a), "f"(b) : "memory");
}
template <int NB>
__device__ __forceinline__ void flush_row_conj(float* out, const float (&re)[NB], const float (&im)[NB], int nb,
                                               float scale) {
#pragma unroll
  for (int b = 0; b < NB; ++b)
    if (b < nb) red_add2(out + 2 * b, re[b] * scale, -im[b] * scale);
}
template <int NB>
__device__ __forceinline__ void flush_row_conj(double*, const double (&)[NB], const double (&)[NB], int, double) {}

struct SplitK {  // stream-K range of this CTA
  int64_t u0, u1;
};
__device__ __forceinline__ SplitK cta_range(int64_t units) {
  const int64_t g = gridDim.x, b = blockIdx.x;
  return {units * b / g, units * (b + 1) / g};
}

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double sign_d(const uint4& r) { return __hiloint2double((int)r.z, (int)r.y); }

// What the kernels load of an entry record at shared address ea (see TiledCcs):
// FP32 tiles one word (S': x, S: w), FP64 tiles the whole record.
template <typename T>
struct CcsRec;
template <>
struct CcsRec<float> {
  __device__ __forceinline__ static uint32_t cols(uint32_t ea) { return lds_u32(ea); }
  __device__ __forceinline__ static uint32_t rows(uint32_t ea) { return lds_u32(ea + 12); }
};
template <>
struct CcsRec<double> {
  __device__ __forceinline__ static uint4 cols(uint32_t ea) { return lds_u4(ea); }
  __device__ __forceinline__ static uint4 rows(uint32_t ea) { return lds_u4(ea); }
};

// ---------------------------------------------------------------------------
// S' = A^T R : lanes over columns of A, TMA-fed.
// Accumulators per bucket: FP32 -> 2 float2 (the lane's 4 columns),
//                          FP64 -> 2 doubles (the lane's 2 columns).
template <typename T>
struct ColsAcc;
template <>
struct ColsAcc<float> {
  float2 a, b;
  __device__ __forceinline__ void zero() { a = b = make_float2(0.f, 0.f); }
  // x: the record's S' word, row offset | sign bit
  __device__ __forceinline__ void add(uint32_t xaddr, uint32_t x) {
    const float4 v = lds_f4(xaddr + (x & 0x7fffffffu));
    const float sg = __uint_as_float((x & 0x80000000u) | 0x3f800000u);
    const float2 s = f2(sg, sg);
    a = __ffma2_rn(f2(v.x, v.y), s, a);
    b = __ffma2_rn(f2(v.z, v.w), s, b);
  }
  __device__ __forceinline__ float get(int q) const { return q == 0 ? a.x : q == 1 ? a.y : q == 2 ? b.x : b.y; }
};
template <>
struct ColsAcc<double> {
  double a, b;
  __device__ __forceinline__ void zero() { a = b = 0.0; }
  __device__ __forceinline__ void add(uint32_t xaddr, const uint4& r) {
    const double2 v = lds_d2(xaddr + r.x);
    const double s = sign_d(r);
    a = fma(v.x, s, a);
    b = fma(v.y, s, b);
  }
  __device__ __forceinline__ double get(int q) const { return q == 0 ? a : b; }
};

}  // namespace jls
