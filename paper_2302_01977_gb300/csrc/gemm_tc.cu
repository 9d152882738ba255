// gemm_tc.cu -- SRHT and Gaussian sketches on tcgen05 tensor cores, with the
// FP32 input split into two bf16 terms.
//
//   S  = scale * A   * B     (Sec. 6.3 "A R")
//   S' = scale * A^T * B     (Sec. 6.3 "A* R", real A)
//
// B is the unscaled operator, held as bf16 planes [c][k] (row c of a plane is
// column c of R, rows of bf_pitch(n) elements):
//   SRHT   one plane, the sign pattern d_k (-1)^popc(k & mu_c) of the element
//          formula of Sec. 7.2 -- exact in bf16;
//   Gauss  two planes z_hi = bf16(z), z_lo = bf16(z - z_hi) of the FP32 draw z
//          (Sec. 2.4.1).
// Each FP32 value a of A is split the same way while it is staged:
// a = a_hi + a_lo + r with |r| <= 2^-16 |a|.  The kernel sums the products
//   SRHT   a_hi b + a_lo b
//   Gauss  a_hi z_hi + a_hi z_lo + a_lo z_hi       (a_lo z_lo ~ 2^-16 |a z| dropped)
// on the tensor cores with FP32 accumulation in tensor memory.
//
// Tiles: 128 output rows (TMEM lanes) x NT output columns (TMEM columns,
// NT <= 256, a multiple of 16) over K stages of 64.  Operand tiles are
// K-major with the 128-byte swizzle: row r of a tile is 128 bytes (64 bf16 of
// K), rows 8 apart are 1024 bytes apart, and 16-byte chunk j of row r sits at
// chunk j ^ (r & 7).  B tiles arrive by TMA in that layout; A tiles are written
// in it by the converter warps.
//
// Work: units are (N tile, M tile, K stage) in that order; a persistent grid
// of at most one CTA per SM takes a contiguous range of units (stream-K), so
// a tile is finished by at most two CTAs whose partial sums are added with
// red.global.add into the zeroed output -- two terms added to zero give the
// same result in either order.  Inside a CTA the MMA chain for one tile part
// is cut every FOLD stages: the epilogue warps add each chain's sum into a
// running total in a second TMEM region, so no single tensor-core
// accumulation chain covers more than FOLD * 64 values of K.
//
// Warp roles (22 warps, one CTA per SM):
//   warp 0       TMA producer for the B planes (one elected lane); the same
//                lane asks L2 for the A tile of the unit pf_dist units ahead,
//                so that the converters' loads find it there
//   warp 1       TMEM allocation; one lane issues tcgen05.mma and commits
//   warps 2..17  converters: load FP32 A (coalesced, two K stages ahead in a
//                ring of three register buffers), split, write bf16 tiles
//   warps 18..21 epilogue: tcgen05.ld, fold or scale + red.global.add
// Every wait is bounded: on a timeout the waiting role sets the error flag
// and an abort flag in shared memory, the other roles stop at their next
// unit, in-flight copies and MMAs are waited for (bounded) and TMEM is freed.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdlib>

#include "common.cuh"
#include "internal.h"
#include "tcgen05.cuh"

#ifndef JLS_TC_FOLD_STAGES
#define JLS_TC_FOLD_STAGES 16
#endif

namespace jls {

namespace {

using namespace tcx;

constexpr int TC_BM = 128;                 // output rows per tile (UMMA M)
constexpr int TC_BK = 64;                  // K per stage (one 128-byte swizzle row of bf16)
constexpr int TC_NMAX = 256;               // output columns per tile (UMMA N limit)
constexpr int TC_CONV_WARPS = 16;
constexpr int TC_CONV_THREADS = 32 * TC_CONV_WARPS;
constexpr int TC_CV = TC_BM * TC_BK / TC_CONV_THREADS;  // FP32 values a converter thread stages per K stage
constexpr int TC_EPI_WARPS = 4;
constexpr int TC_THREADS = 32 * (2 + TC_CONV_WARPS + TC_EPI_WARPS);
constexpr int TC_FOLD = JLS_TC_FOLD_STAGES;  // K stages per accumulation chain (0: no cut)
constexpr uint32_t TC_A_PLANE = TC_BM * TC_BK * 2;  // 16 KB: one bf16 term of an A tile
constexpr int TC_MAX_STAGES = 4;
constexpr long TC_SMEM_MAX = 227 * 1024;
constexpr uint32_t TC_BAR_BYTES = 256;

__device__ __forceinline__ bool fold_point(int ks) { return TC_FOLD > 0 && (ks & (TC_FOLD - 1)) == 0; }
static_assert(TC_FOLD == 0 || (TC_FOLD & (TC_FOLD - 1)) == 0, "the fold interval is a power of two");

// bf16x2 of (lo, hi): `lo` lands in the lower 16 bits (the lower address).
__device__ __forceinline__ uint32_t bf16x2(float lo, float hi) {
  uint32_t d;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}
// Split four consecutive values: hi = bf16(x), lo = bf16(x - hi) (the
// subtraction is exact), as two bf16x2 words each.
__device__ __forceinline__ void split4(float4 x, uint32_t& h01, uint32_t& h23, uint32_t& l01, uint32_t& l23) {
  h01 = bf16x2(x.x, x.y);
  h23 = bf16x2(x.z, x.w);
  const float2 m1 = make_float2(-1.f, -1.f);
  const float2 r01 = __ffma2_rn(make_float2(__uint_as_float(h01 << 16), __uint_as_float(h01 & 0xffff0000u)), m1,
                                make_float2(x.x, x.y));
  const float2 r23 = __ffma2_rn(make_float2(__uint_as_float(h23 << 16), __uint_as_float(h23 & 0xffff0000u)), m1,
                                make_float2(x.z, x.w));
  l01 = bf16x2(r01.x, r01.y);
  l23 = bf16x2(r23.x, r23.y);
}

// ---- converters: FP32 A -> bf16 (hi, lo) tiles -------------------------------------
// 512 converter threads, TC_CV = 16 values each per 128 x 64 stage.
// S  (TRANS = false): A is M x K row-major.  Thread t takes float4 j*512 + t
//    (j < 4) of the stage: row j*32 + t/16, K quad t % 16, so 16 lanes read one
//    row's 256 contiguous bytes and write its 128-byte swizzled bf16 row
//    without bank conflicts.
// S' (TRANS = true): A is K x M row-major (the tile's rows are A's columns).
//    Thread t takes tile row r = t % 128 and K quarter t / 128: 16 loads of
//    A[k][m0 + r], each a 128-byte coalesced warp access; it then owns two
//    whole 16-byte chunks of row r per plane, stored conflict-free.
// Shared-memory offsets within a tile are fixed per thread; tiles wholly
// inside A take an unchecked path.
template <bool TRANS>
struct Converter {
  const float* A;
  int64_t lda;
  int64_t m_rows, k_len;
  int ct;
  uint32_t off0;  // S: offset of row t/16 (j = 0); S': offset of row t % 128, first chunk

  __device__ __forceinline__ void setup(const float* A_, int64_t lda_, const TcWork& w, int ct_) {
    A = A_;
    lda = lda_;
    m_rows = w.m_rows;
    k_len = w.k_len;
    ct = ct_;
    if (!TRANS) {
      const uint32_t r = (uint32_t)(ct >> 4), kq = (uint32_t)(ct & 15);
      off0 = r * 128 + ((((kq >> 1) ^ (r & 7)) << 4) | ((kq & 1) << 3));
    } else {
      const uint32_t r = (uint32_t)(ct & 127);
      off0 = r * 128;
    }
  }

  __device__ __forceinline__ void load(int64_t mt, int ks, float (&v)[TC_CV]) const {
    const int64_t m0 = mt * TC_BM, k0 = (int64_t)ks * TC_BK;
    const bool full = m0 + TC_BM <= m_rows && k0 + TC_BK <= k_len;
    if (!TRANS) {
      const int64_t m = m0 + (ct >> 4);
      const int64_t k = k0 + (ct & 15) * 4;
      const float* p = A + m * lda + k;
      const int64_t step = 32 * lda;
#pragma unroll
      for (int j = 0; j < TC_CV / 4; ++j) {
        float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
        if (full) {
          x = __ldg(reinterpret_cast<const float4*>(p + j * step));
        } else if (m + 32 * j < m_rows) {
          const float* q = p + j * step;
          if (k + 3 < k_len) {
            x = __ldg(reinterpret_cast<const float4*>(q));
          } else {
            if (k < k_len) x.x = __ldg(q);
            if (k + 1 < k_len) x.y = __ldg(q + 1);
            if (k + 2 < k_len) x.z = __ldg(q + 2);
          }
        }
        v[4 * j] = x.x;
        v[4 * j + 1] = x.y;
        v[4 * j + 2] = x.z;
        v[4 * j + 3] = x.w;
      }
    } else {
      const int64_t m = m0 + (ct & 127);
      const int64_t kb = k0 + (ct >> 7) * TC_CV;
      const float* p = A + kb * lda + m;
      if (full) {
#pragma unroll
        for (int e = 0; e < TC_CV; ++e) v[e] = __ldg(p + e * lda);
      } else {
        const bool mok = m < m_rows;
#pragma unroll
        for (int e = 0; e < TC_CV; ++e) v[e] = (mok && kb + e < k_len) ? __ldg(p + e * lda) : 0.f;
      }
    }
  }

  __device__ __forceinline__ void store(uint32_t a_hi, const float (&v)[TC_CV]) const {
    const uint32_t a_lo = a_hi + TC_A_PLANE;
    if (!TRANS) {
#pragma unroll
      for (int j = 0; j < TC_CV / 4; ++j) {
        uint32_t h01, h23, l01, l23;
        split4(make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]), h01, h23, l01, l23);
        const uint32_t off = off0 + (uint32_t)j * (32 * 128);  // 32 rows on: same swizzle phase
        sts_v2(a_hi + off, h01, h23);
        sts_v2(a_lo + off, l01, l23);
      }
    } else {
      const uint32_t r7 = (uint32_t)(ct & 7), quarter = (uint32_t)(ct >> 7);
#pragma unroll
      for (int c = 0; c < TC_CV / 8; ++c) {
        const uint32_t off = off0 + (((quarter * (TC_CV / 8) + c) ^ r7) << 4);
        uint32_t h[4], l[4];
        split4(make_float4(v[8 * c], v[8 * c + 1], v[8 * c + 2], v[8 * c + 3]), h[0], h[1], l[0], l[1]);
        split4(make_float4(v[8 * c + 4], v[8 * c + 5], v[8 * c + 6], v[8 * c + 7]), h[2], h[3], l[2], l[3]);
        sts_v4(a_hi + off, h[0], h[1], h[2], h[3]);
        sts_v4(a_lo + off, l[0], l[1], l[2], l[3]);
      }
    }
  }
};

}  // namespace

template <bool TRANS, int PLANES>
__global__ void __launch_bounds__(TC_THREADS, 1)
    tc_sketch_kernel(const float* __restrict__ A, int64_t lda, const __grid_constant__ CUtensorMap tmB0,
                     const __grid_constant__ CUtensorMap tmB1, const __grid_constant__ CUtensorMap tmA,
                     const TcWork w, float scale, float* __restrict__ out, int64_t ldo, int vec_ok, int pf_dist,
                     int* err) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  const uint32_t bars = base + (uint32_t)w.stages * w.stage_bytes;
  // barrier block: full_b[S], full_a[S], empty[S], tmem_full, tmem_empty, done; tmem slot; abort flag
  auto full_b = [&](int s) { return bars + 8u * s; };
  auto full_a = [&](int s) { return bars + 8u * (TC_MAX_STAGES + s); };
  auto empty = [&](int s) { return bars + 8u * (2 * TC_MAX_STAGES + s); };
  const uint32_t tmem_full = bars + 8u * (3 * TC_MAX_STAGES);
  const uint32_t tmem_empty = tmem_full + 8u;
  const uint32_t done_bar = tmem_full + 16u;
  const uint32_t tmem_slot = tmem_full + 24u;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(smem_raw + (bars - raw) + 8u * (3 * TC_MAX_STAGES) + 28u);
  volatile uint32_t* tmem_slot_p = reinterpret_cast<volatile uint32_t*>(smem_raw + (tmem_slot - raw));

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t units = (int64_t)((w.c_hi - w.c_lo + w.nt - 1) / w.nt) * w.mtiles * w.kst;
  const int64_t u0 = units * blockIdx.x / gridDim.x;
  const int cnt = (int)(units * (blockIdx.x + 1) / gridDim.x - u0);  // units of this CTA

  if (threadIdx.x == 0) {
    for (int s = 0; s < w.stages; ++s) {
      mbar_init(full_b(s), 1);
      mbar_init(full_a(s), TC_CONV_WARPS);
      mbar_init(empty(s), 1);
    }
    mbar_init(tmem_full, 1);
    mbar_init(tmem_empty, TC_EPI_WARPS);
    mbar_init(done_bar, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 1) tmem_alloc(tmem_slot, w.tmem_cols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot_p;

  if (warp == 0) {
    // ---------------- TMA producer: B planes ----------------
    if (lane == 0) {
      tma_prefetch_desc(&tmB0);
      if (PLANES == 2) tma_prefetch_desc(&tmB1);
      if (pf_dist > 0) tma_prefetch_desc(&tmA);
      const uint32_t b_bytes = (uint32_t)PLANES * (uint32_t)w.nt * 128u;
      // A tiles into L2 ahead of the converters: units [0, pf_dist) now, unit i + pf_dist at unit i
      Cursor pc;
      pc.init(w, u0);
      int pf = 0;
      auto prefetch_a = [&]() {
        if (TRANS) tma_prefetch_l2_2d(&tmA, (int32_t)(pc.mt * TC_BM), pc.ks * TC_BK);
        else tma_prefetch_l2_2d(&tmA, pc.ks * TC_BK, (int32_t)(pc.mt * TC_BM));
        pc.next(w);
        ++pf;
      };
      while (pf < min(pf_dist, cnt)) prefetch_a();
      Cursor c;
      c.init(w, u0);
      Ring rg;
      int issued = 0;
      for (int i = 0; i < cnt; ++i, c.next(w), rg.next(w.stages)) {
        if (*abort_flag) break;
        if (pf_dist > 0 && pf < cnt) prefetch_a();
        if (!mbar_wait(empty(rg.s), rg.ph ^ 1u, err)) {
          *abort_flag = 1;
          break;
        }
        const uint32_t dst = base + (uint32_t)rg.s * w.stage_bytes + 2 * TC_A_PLANE;
        const int row = w.c_lo + c.nt * w.nt;
        mbar_arrive_expect_tx(full_b(rg.s), b_bytes);
        tma_load_2d(dst, &tmB0, full_b(rg.s), c.ks * TC_BK, row);
        if (PLANES == 2) tma_load_2d(dst + (uint32_t)w.nt * 128u, &tmB1, full_b(rg.s), c.ks * TC_BK, row);
        issued = i + 1;
      }
      // wait for every copy still in flight (the last one issued into each slot)
      for (int i = max(0, issued - w.stages); i < issued; ++i)
        mbar_wait(full_b(i % w.stages), (uint32_t)((i / w.stages) & 1), err);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(TC_BM, w.nt);
      uint32_t chain = 0;
      bool first = true;
      Cursor c;
      c.init(w, u0);
      Ring rg;
      for (int i = 0; i < cnt; ++i, c.next(w), rg.next(w.stages)) {
        if (*abort_flag) break;
        if (i == 0 || c.ks == 0 || fold_point(c.ks)) {  // a chain begins: the accumulator must be free
          if (!mbar_wait(tmem_empty, (chain & 1) ^ 1, err)) {
            *abort_flag = 1;
            break;
          }
          tc_fence_after();
          first = true;
        }
        if (!mbar_wait(full_b(rg.s), rg.ph, err) || !mbar_wait(full_a(rg.s), rg.ph, err)) {
          *abort_flag = 1;
          break;
        }
        tc_fence_after();
        const uint32_t st = base + (uint32_t)rg.s * w.stage_bytes;
        const uint32_t b0 = st + 2 * TC_A_PLANE, b1 = b0 + (uint32_t)w.nt * 128u;
#pragma unroll
        for (int kk = 0; kk < TC_BK / 16; ++kk) {
          const uint32_t ko = (uint32_t)kk * 32u;  // 16 bf16 along K inside the swizzled row
          const uint64_t dah = sw128_desc(st + ko), dal = sw128_desc(st + TC_A_PLANE + ko);
          const uint64_t db0 = sw128_desc(b0 + ko);
          umma_bf16(tmem, dah, db0, idesc, first ? 0u : 1u);
          umma_bf16(tmem, dal, db0, idesc, 1u);
          if (PLANES == 2) umma_bf16(tmem, dah, sw128_desc(b1 + ko), idesc, 1u);
          first = false;
        }
        umma_commit(empty(rg.s));
        if (i + 1 == cnt || c.ks + 1 == w.kst || fold_point(c.ks + 1)) {  // the chain ends
          umma_commit(tmem_full);
          ++chain;
        }
      }
      // all MMAs issued by this thread have completed once done_bar flips
      umma_commit(done_bar);
      mbar_wait(done_bar, 0, err);
    }
  } else if (warp < 2 + TC_CONV_WARPS) {
    // ---------------- converters ----------------
    // three register buffers: the loads of the next two stages are in flight
    // while one stage is split and stored
    Converter<TRANS> cv;
    cv.setup(A, lda, w, threadIdx.x - 64);
    float va[TC_CV], vb[TC_CV], vc[TC_CV];
    Cursor lc;  // next unit to load
    lc.init(w, u0);
    int loaded = 0;
    auto load = [&](float (&v)[TC_CV]) {
      if (loaded < cnt) {
        cv.load(lc.mt, lc.ks, v);
        lc.next(w);
        ++loaded;
      }
    };
    Ring rg;
    auto put = [&](const float (&v)[TC_CV]) -> bool {
      if (*abort_flag) return false;
      if (!warp_wait(empty(rg.s), rg.ph ^ 1u, err)) {
        *abort_flag = 1;
        return false;
      }
      cv.store(base + (uint32_t)rg.s * w.stage_bytes, v);
      fence_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive(full_a(rg.s));
      rg.next(w.stages);
      return true;
    };
    load(va);
    load(vb);
    for (int i = 0; i < cnt; i += 3) {
      load(vc);
      if (!put(va) || i + 1 >= cnt) break;
      load(va);
      if (!put(vb) || i + 2 >= cnt) break;
      load(vb);
      if (!put(vc)) break;
    }
  } else {
    // ---------------- epilogue ----------------
    const int q = warp & 3;  // TMEM lane quarter this warp may access
    const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16);
    uint32_t chain = 0;
    bool has_total = false;
    Cursor c;
    c.init(w, u0);
    for (int i = 0; i < cnt; ++i, c.next(w)) {
      if (i == 0 || c.ks == 0 || fold_point(c.ks)) has_total = !(i == 0 || c.ks == 0);
      const bool emit = (i + 1 == cnt) || (c.ks + 1 == w.kst);
      if (!emit && !fold_point(c.ks + 1)) continue;  // the chain goes on
      if (*abort_flag) break;
      if (!warp_wait(tmem_full, chain & 1, err)) {
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      const int64_t row = c.mt * TC_BM + q * 32 + lane;
      for (int cc = 0; cc < w.nt; cc += 16) {
        uint32_t v[16], t[16];
        tmem_ld16(trow + (uint32_t)cc, v);
        if (has_total) tmem_ld16(trow + (uint32_t)(w.nt + cc), t);
        tmem_wait_ld();
        if (has_total) {
#pragma unroll
          for (int j = 0; j < 16; ++j) v[j] = __float_as_uint(__uint_as_float(v[j]) + __uint_as_float(t[j]));
        }
        if (!emit) {
          tmem_st16(trow + (uint32_t)(w.nt + cc), v);
          continue;
        }
        const int c0 = w.c_lo + c.nt * w.nt + cc;
        if (row < w.m_rows && c0 < w.c_hi) {
          float* p = out + row * ldo + c0;
          if (vec_ok && c0 + 16 <= w.c_hi) {
#pragma unroll
            for (int j = 0; j < 16; j += 4)
              red_v4(p + j, scale * __uint_as_float(v[j]), scale * __uint_as_float(v[j + 1]),
                     scale * __uint_as_float(v[j + 2]), scale * __uint_as_float(v[j + 3]));
          } else {
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (c0 + j < w.c_hi) atomicAdd(p + j, scale * __uint_as_float(v[j]));
          }
        }
      }
      if (!emit) tmem_wait_st();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tmem_empty);
      ++chain;
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, w.tmem_cols);
}

namespace {

// A as FP32 tiles of one unit (128 rows x 64 of K for S, 64 of K x 128 columns
// for S'), used only for L2 prefetches.  Returns false when A's address or
// row pitch does not meet the tensor map's 16-byte rules.
bool encode_a(CUtensorMap* tm, const sk_matrix* A, bool trans) {
  PFN_encodeTiled enc = get_encode_tiled();
  if (!enc || (reinterpret_cast<uintptr_t>(A->A) & 15) != 0 || (A->ld * 4) % 16 != 0) return false;
  const cuuint64_t gdim[2] = {(cuuint64_t)A->cols, (cuuint64_t)A->rows};
  const cuuint64_t gstride[1] = {(cuuint64_t)(A->ld * 4)};
  const cuuint32_t box[2] = {(cuuint32_t)(trans ? TC_BM : TC_BK), (cuuint32_t)(trans ? TC_BK : TC_BM)};
  const cuuint32_t estr[2] = {1, 1};
  return enc(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(A->A), gdim, gstride, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Units of A prefetched into L2 ahead of the converters (JLS_TC_PREFETCH
// overrides; 0 turns the prefetch off).
int tc_prefetch_units() {
  static int v = [] {
    const char* e = std::getenv("JLS_TC_PREFETCH");
    return e ? std::max(0, std::min(64, std::atoi(e))) : 3;
  }();
  return v;
}

int encode_plane(CUtensorMap* tm, const uint16_t* plane, int64_t n, int rows, int nt) {
  PFN_encodeTiled enc = get_encode_tiled();
  if (!enc) return SK_ERR_DEVICE;
  const cuuint64_t gdim[2] = {(cuuint64_t)n, (cuuint64_t)rows};
  const cuuint64_t gstride[1] = {(cuuint64_t)(bf_pitch(n) * 2)};
  const cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)nt};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<uint16_t*>(plane), gdim, gstride, box,
                         estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? SK_OK : SK_ERR_ALIGN;
}

}  // namespace

// The tensor-core sketch of FP32 A with operator planes p0 (and p1 with
// planes == 2): rows [c_lo, c_hi) of the planes, each k_len bf16 values with
// rows of bf_pitch(k_len), are the operator's columns.
int launch_tc_planes(int* d_err, const sk_matrix* A, bool trans, int planes, const uint16_t* p0, const uint16_t* p1,
                     int64_t k_len, int c_lo, int c_hi, float scale, float* out, int64_t ldo, cudaStream_t s) {
  TcWork w{};
  w.m_rows = trans ? A->cols : A->rows;
  w.k_len = k_len;
  w.mtiles = (w.m_rows + TC_BM - 1) / TC_BM;
  w.kst = (int)((k_len + TC_BK - 1) / TC_BK);
  const int ncols = c_hi - c_lo;
  const int ntiles = (ncols + TC_NMAX - 1) / TC_NMAX;
  w.nt = ((ncols + ntiles - 1) / ntiles + 15) / 16 * 16;
  w.c_lo = c_lo;
  w.c_hi = c_hi;
  w.stage_bytes = 2 * TC_A_PLANE + (uint32_t)planes * (uint32_t)w.nt * 128u;
  const long avail = TC_SMEM_MAX - 1024 - (long)TC_BAR_BYTES;
  w.stages = (int)std::min<long>(TC_MAX_STAGES, avail / (long)w.stage_bytes);
  if (w.stages < 2) return SK_ERR_UNSUPPORTED;
  w.tmem_cols = tmem_cols_for(TC_FOLD > 0 ? 2 * w.nt : w.nt);
  if (w.tmem_cols > 512) return SK_ERR_UNSUPPORTED;

  CUtensorMap t0, t1, ta;
  JLS_CHECK(encode_plane(&t0, p0, k_len, c_hi, w.nt));
  JLS_CHECK(encode_plane(&t1, p1, k_len, c_hi, w.nt));
  const int pf_dist = encode_a(&ta, A, trans) ? tc_prefetch_units() : 0;
  if (pf_dist == 0) ta = t0;  // never read
  JLS_CHECK_CUDA(cudaMemset2DAsync(out + c_lo, ldo * sizeof(float), 0, (size_t)ncols * sizeof(float),
                                   (size_t)w.m_rows, s));
  const int64_t tiles = (int64_t)ntiles * w.mtiles;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(num_sms(), tiles));
  const size_t smem = 1024 + (size_t)w.stages * w.stage_bytes + TC_BAR_BYTES;
  const int vec_ok = ((reinterpret_cast<uintptr_t>(out) & 15) == 0 && ldo % 4 == 0 && c_lo % 4 == 0) ? 1 : 0;
  const float* a = static_cast<const float*>(A->A);
#define JLS_TC_LAUNCH(TR, PL)                                                                                \
  do {                                                                                                       \
    auto kern = tc_sketch_kernel<TR, PL>;                                                                   \
    JLS_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));     \
    kern<<<grid, TC_THREADS, smem, s>>>(a, A->ld, t0, t1, ta, w, scale, out, ldo, vec_ok, pf_dist, d_err);   \
  } while (0)
  if (trans && planes == 2) JLS_TC_LAUNCH(true, 2);
  else if (trans) JLS_TC_LAUNCH(true, 1);
  else if (planes == 2) JLS_TC_LAUNCH(false, 2);
  else JLS_TC_LAUNCH(false, 1);
#undef JLS_TC_LAUNCH
  note_launch();
  JLS_CHECK_CUDA(cudaGetLastError());
  return SK_OK;
}

namespace {

int launch_tc(sk_op* h, const sk_matrix* A, bool trans, int c_lo, int c_hi, float scale, float* out, int64_t ldo,
              cudaStream_t s) {
  const int planes = h->kind == SK_GAUSS ? 2 : 1;
  const uint16_t* p0 = h->kind == SK_GAUSS ? h->zhi : h->srht_pm1;
  const uint16_t* p1 = h->kind == SK_GAUSS ? h->zlo : h->srht_pm1;
  return launch_tc_planes(h->d_err, A, trans, planes, p0, p1, h->n, c_lo, c_hi, scale, out, ldo, s);
}

}  // namespace

int dense_apply_tc(sk_op* h, const sk_matrix* A, int which, int c_lo, int c_hi, double scale, void* S, int64_t ldS,
                   void* St, int64_t ldSt, cudaStream_t s) {
  if (A->dtype != SK_F32) return SK_ERR_DTYPE;
  if (c_hi <= c_lo) return SK_OK;
  if (h->kind == SK_GAUSS) JLS_CHECK(gen_gauss(h, 2, h->d_total, s));
  else if (h->kind == SK_SRHT) JLS_CHECK(gen_srht_pm1(h, h->d_total, s));
  else JLS_CHECK(gen_sjlt_pm1(h, h->d_total, s));  // SJLT: R's {0, +-1} pattern is exact in bf16
  if (which & SK_S) JLS_CHECK(launch_tc(h, A, false, c_lo, c_hi, (float)scale, (float*)S, ldS, s));
  if (which & SK_ST) JLS_CHECK(launch_tc(h, A, true, c_lo, c_hi, (float)scale, (float*)St, ldSt, s));
  return SK_OK;
}

}  // namespace jls
