// gemm_fp8.cu -- SRHT and Gaussian sketches on tcgen05 tensor cores in scaled
// FP8 (e4m3), with FP32 accumulation.
//
//   S  = scale * A   * B     (Sec. 6.3 "A R")
//   S' = scale * A^T * B     (Sec. 6.3 "A* R", real A)
//
// Scaling and split.  A is quantized per tile of 64 output rows x 128 values
// of K: s_A = amax(tile) / 448 (448 is e4m3's largest finite value), and each
// value y = a / s_A becomes y_hi = e4m3(y) and y_lo = e4m3(y - y_hi), both in
// the tile's units (the subtraction is exact in FP32).  B is the unscaled
// operator: the SRHT signs are exact in e4m3 (scale 1); the Gaussian z is
// quantized per (128 values of K, column) the same way, with scale s_z.  The
// MMAs of one K tile sum
//   SRHT   y_hi b + y_lo b
//   Gauss  y_hi w_hi + y_hi w_lo + y_lo w_hi          (y_lo w_lo dropped)
// into a fresh TMEM accumulator; the epilogue warps then add s_A s_z times
// that sum into a running FP32 total in a second TMEM region (scales applied
// per K tile), and write scale * total at the end of a tile part.  The K
// tile's sums for the two column halves of the tile go to separate TMEM chunks
// (MMAs of N/2), so the epilogue folds one half while the tensor core computes
// the other.  Even so the fold of every K tile (two TMEM loads and a store per
// output, about 16 dependent round trips per 256 columns) and the e4m3
// conversions of the converters cost more per K than the tensor work saves:
// on GB300 this path is slower than the bf16 split (gemm_tc.cu), which folds
// once per 16 K stages.  With three
// e4m3 mantissa bits the kept terms differ from a z by at most about
// 3 * 2^-8 |a z| plus a floor of 2^-10 s_A |z| from e4m3's subnormal spacing.
//
// Layout.  A 128-byte swizzle row holds 128 e4m3 values, so an FP8 K stage of
// 128 has the byte layout of a bf16 stage of 64: operand tiles are K-major,
// rows of 128 bytes, rows 8 apart 1024 bytes apart, 16-byte chunk j of row r
// at chunk j ^ (r & 7); an MMA covers K = 32 (32 bytes of the row).
//
// Warp roles (22 warps, one CTA per SM), as in the bf16 kernel:
//   warp 0       TMA producer for the B planes
//   warp 1       TMEM allocation; one lane issues tcgen05.mma.kind::f8f6f4
//   warps 2..17  converters: load FP32 A one K tile ahead, reduce the tile's
//                amax across the 16 warps (named barrier), quantize, store
//   warps 18..21 epilogue: per K tile, scale and fold the accumulator
// Named barriers are always reached by every warp of their group; a warp that
// saw a timeout or an abort publishes that before the barrier, so the whole
// group leaves together.  All mbarrier waits are bounded as in gemm_tc.cu.
#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "tcgen05.cuh"

namespace jls {

namespace {

using namespace tcx;

constexpr int F8_BM = 128;                 // output rows per tile
constexpr int F8_BK = 128;                 // K per stage = per scale tile
constexpr int F8_NMAX = 256;
constexpr int F8_CONV_WARPS = 16;
constexpr int F8_CONV_THREADS = 32 * F8_CONV_WARPS;
constexpr int F8_CV = F8_BM * F8_BK / 2 / F8_CONV_THREADS;  // 16 FP32 values per converter thread per half stage
constexpr int F8_EPI_WARPS = 4;  // one per TMEM lane quarter (8, two per quarter, cost the converters registers)
constexpr int F8_EPW = F8_EPI_WARPS / 4;
constexpr int F8_THREADS = 32 * (2 + F8_CONV_WARPS + F8_EPI_WARPS);
constexpr uint32_t F8_A_PLANE = F8_BM * F8_BK;  // 16 KB: one e4m3 term of an A tile
constexpr int F8_MAX_STAGES = 4;
constexpr int F8_SCALE_RING = 8;                // >= stages + 2 (see the epilogue)
constexpr long F8_SMEM_MAX = 227 * 1024;
constexpr uint32_t F8_AUX_BYTES = 4096;         // barriers, scale ring, reduction and scale staging
constexpr float F8_MAX = 448.f;

__device__ __forceinline__ void named_sync(int id, int threads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

// Quantize four consecutive values (already divided by the tile scale) into
// e4m3 hi and lo terms, packed as 4 bytes each (first value in the low byte).
__device__ __forceinline__ void quant4(float y0, float y1, float y2, float y3, uint32_t& hi, uint32_t& lo) {
  const uint32_t h01 = e4m3x2(y0, y1), h23 = e4m3x2(y2, y3);
  const float2 d01 = e4m3x2_to_f2(h01), d23 = e4m3x2_to_f2(h23);
  const uint32_t l01 = e4m3x2(y0 - d01.x, y1 - d01.y), l23 = e4m3x2(y2 - d23.x, y3 - d23.y);
  hi = h01 | (h23 << 16);
  lo = l01 | (l23 << 16);
}

__device__ __forceinline__ void sts_u32(uint32_t a, uint32_t x) {
  asm volatile("st.shared.u32 [%0], %1;" ::"r"(a), "r"(x) : "memory");
}

// ---- converters: FP32 A -> e4m3 (hi, lo) tiles -------------------------------------
// A stage (128 rows x 128 values of K) is converted in two halves of 64 rows,
// each with its own scale; 512 converter threads take F8_CV = 16 values of a
// half.
// S  (TRANS = false): A is M x K row-major.  Warp w, lane l take float4 l of
//    rows j*16 + w (j = 4h .. 4h+3 for half h): one warp reads one row's 512
//    contiguous bytes and writes its 128-byte swizzled e4m3 row, 4 bytes per
//    lane, without bank conflicts.
// S' (TRANS = true): A is K x M row-major.  Thread t takes tile row
//    r = 64h + t % 64 and K sixteenth t / 64: 16 loads of A[k][m0 + r] (128-byte
//    coalesced warp accesses), then one whole 16-byte chunk of row r per term.
template <bool TRANS>
struct Fp8Converter {
  const float* A;
  int64_t lda;
  int64_t m_rows, k_len;
  int ct;
  uint32_t off0;  // shared offset of this thread's first 4 (S) or 16 (S') bytes in half 0

  __device__ __forceinline__ void setup(const float* A_, int64_t lda_, const TcWork& w, int ct_) {
    A = A_;
    lda = lda_;
    m_rows = w.m_rows;
    k_len = w.k_len;
    ct = ct_;
    if (!TRANS) {
      const uint32_t r = (uint32_t)(ct >> 5), l = (uint32_t)(ct & 31);
      off0 = r * 128 + ((((l >> 2) ^ (r & 7)) << 4) | ((l & 3) << 2));
    } else {
      const uint32_t r = (uint32_t)(ct & 63), kq = (uint32_t)(ct >> 6);
      off0 = r * 128 + ((kq ^ (r & 7)) << 4);
    }
  }

  __device__ __forceinline__ void load(int64_t mt, int ks, int h, float (&v)[F8_CV]) const {
    const int64_t m0 = mt * F8_BM + 64 * h, k0 = (int64_t)ks * F8_BK;
    const bool full = m0 + 64 <= m_rows && k0 + F8_BK <= k_len;
    if (!TRANS) {
      const int64_t m = m0 + (ct >> 5);
      const int64_t k = k0 + (ct & 31) * 4;
      const float* p = A + m * lda + k;
      const int64_t step = 16 * lda;
#pragma unroll
      for (int j = 0; j < F8_CV / 4; ++j) {
        float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
        if (full) {
          x = __ldg(reinterpret_cast<const float4*>(p + j * step));
        } else if (m + 16 * j < m_rows) {
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
      const int64_t m = m0 + (ct & 63);
      const int64_t kb = k0 + (ct >> 6) * F8_CV;
      const float* p = A + kb * lda + m;
      if (full) {
#pragma unroll
        for (int e = 0; e < F8_CV; ++e) v[e] = __ldg(p + e * lda);
      } else {
        const bool mok = m < m_rows;
#pragma unroll
        for (int e = 0; e < F8_CV; ++e) v[e] = (mok && kb + e < k_len) ? __ldg(p + e * lda) : 0.f;
      }
    }
  }

  // Quantize half h with 1 / s = inv and store both terms into the stage at a_hi.
  __device__ __forceinline__ void store(uint32_t a_hi, int h, float inv, const float (&v)[F8_CV]) const {
    const uint32_t a_lo = a_hi + F8_A_PLANE;
    const uint32_t hoff = (uint32_t)h * (64 * 128);  // 64 rows on: same swizzle phase
    if (!TRANS) {
#pragma unroll
      for (int j = 0; j < F8_CV / 4; ++j) {
        uint32_t hi, lo;
        quant4(v[4 * j] * inv, v[4 * j + 1] * inv, v[4 * j + 2] * inv, v[4 * j + 3] * inv, hi, lo);
        const uint32_t off = off0 + hoff + (uint32_t)j * (16 * 128);  // 16 rows on: same swizzle phase
        sts_u32(a_hi + off, hi);
        sts_u32(a_lo + off, lo);
      }
    } else {
      uint32_t hq[4], lq[4];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        quant4(v[4 * q] * inv, v[4 * q + 1] * inv, v[4 * q + 2] * inv, v[4 * q + 3] * inv, hq[q], lq[q]);
      sts_v4(a_hi + off0 + hoff, hq[0], hq[1], hq[2], hq[3]);
      sts_v4(a_lo + off0 + hoff, lq[0], lq[1], lq[2], lq[3]);
    }
  }
};

}  // namespace

template <bool TRANS, int PLANES>
__global__ void __launch_bounds__(F8_THREADS, 1)
    tc_fp8_kernel(const float* __restrict__ A, int64_t lda, const __grid_constant__ CUtensorMap tmB0,
                  const __grid_constant__ CUtensorMap tmB1, const TcWork w, const float* __restrict__ zscale,
                  int64_t zs_ld, float scale, float* __restrict__ out, int64_t ldo, int vec_ok, int* err) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  const uint32_t aux = base + (uint32_t)w.stages * w.stage_bytes;
  uint8_t* aux_g = smem_raw + (aux - raw);
  // aux block: full_b[4] full_a[4] empty[4] tmem_full[2] tmem_empty[2] done | tmem slot, abort flag |
  // scale_ready[8] | s_A ring[8][2] | amax[2][16] | ok[2][16] | epilogue ok[2][4] | B scales[2][256]
  auto full_b = [&](int s) { return aux + 8u * s; };
  auto full_a = [&](int s) { return aux + 8u * (F8_MAX_STAGES + s); };
  auto empty = [&](int s) { return aux + 8u * (2 * F8_MAX_STAGES + s); };
  auto tmem_full = [&](int h) { return aux + 96u + 8u * h; };
  auto tmem_empty = [&](int h) { return aux + 112u + 8u * h; };
  const uint32_t done_bar = aux + 128u;
  const uint32_t tmem_slot = aux + 136u;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(aux_g + 140);
  auto scale_ready = [&](int j) { return aux + 144u + 8u * j; };
  volatile float* sa_ring = reinterpret_cast<volatile float*>(aux_g + 208);   // [8][2] (two row halves)
  volatile float* red_amax = reinterpret_cast<volatile float*>(aux_g + 272);  // [2][16]
  volatile int* red_ok = reinterpret_cast<volatile int*>(aux_g + 400);        // [2][16]
  volatile int* epi_ok = reinterpret_cast<volatile int*>(aux_g + 528);        // [2][8]
  volatile float* sb_stage = reinterpret_cast<volatile float*>(aux_g + 1024); // [2][256]
  volatile uint32_t* tmem_slot_p = reinterpret_cast<volatile uint32_t*>(aux_g + 136);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t units = (int64_t)((w.c_hi - w.c_lo + w.nt - 1) / w.nt) * w.mtiles * w.kst;
  const int64_t u0 = units * blockIdx.x / gridDim.x;
  const int cnt = (int)(units * (blockIdx.x + 1) / gridDim.x - u0);

  if (threadIdx.x == 0) {
    for (int s = 0; s < w.stages; ++s) {
      mbar_init(full_b(s), 1);
      mbar_init(full_a(s), F8_CONV_WARPS);
      mbar_init(empty(s), 1);
    }
    for (int h = 0; h < 2; ++h) {
      mbar_init(tmem_full(h), 1);
      mbar_init(tmem_empty(h), F8_EPI_WARPS);
    }
    mbar_init(done_bar, 1);
    for (int j = 0; j < F8_SCALE_RING; ++j) mbar_init(scale_ready(j), 1);
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
      const uint32_t b_bytes = (uint32_t)PLANES * (uint32_t)w.nt * 128u;
      Cursor c;
      c.init(w, u0);
      Ring rg;
      int issued = 0;
      for (int i = 0; i < cnt; ++i, c.next(w), rg.next(w.stages)) {
        if (*abort_flag) break;
        if (!mbar_wait(empty(rg.s), rg.ph ^ 1u, err)) {
          *abort_flag = 1;
          break;
        }
        const uint32_t dst = base + (uint32_t)rg.s * w.stage_bytes + 2 * F8_A_PLANE;
        const int row = w.c_lo + c.nt * w.nt;
        mbar_arrive_expect_tx(full_b(rg.s), b_bytes);
        tma_load_2d(dst, &tmB0, full_b(rg.s), c.ks * F8_BK, row);
        if (PLANES == 2) tma_load_2d(dst + (uint32_t)w.nt * 128u, &tmB1, full_b(rg.s), c.ks * F8_BK, row);
        issued = i + 1;
      }
      for (int i = max(0, issued - w.stages); i < issued; ++i)
        mbar_wait(full_b(i % w.stages), (uint32_t)((i / w.stages) & 1), err);
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer: one accumulation chain per K tile ----------------
    // TMEM: running total in columns [0, NT); the stage's sums for output
    // columns [0, NT/2) and [NT/2, NT) in chunks at [NT, 3NT/2) and [3NT/2, 2NT),
    // so the epilogue folds one half while the tensor core computes the other.
    if (lane == 0) {
      const int nh = w.nt / 2;
      const uint32_t idesc = idesc_e4m3(F8_BM, nh);
      Ring rg;
      for (int i = 0; i < cnt; ++i, rg.next(w.stages)) {
        if (*abort_flag) break;
        if (!mbar_wait(full_b(rg.s), rg.ph, err) || !mbar_wait(full_a(rg.s), rg.ph, err)) {
          *abort_flag = 1;
          break;
        }
        const uint32_t st = base + (uint32_t)rg.s * w.stage_bytes;
        bool fail = false;
        for (int h = 0; h < 2; ++h) {
          if (!mbar_wait(tmem_empty(h), (uint32_t)(i & 1) ^ 1u, err)) {
            fail = true;
            break;
          }
          tc_fence_after();
          const uint32_t d = tmem + (uint32_t)(w.nt + h * nh);
          const uint32_t b0 = st + 2 * F8_A_PLANE + (uint32_t)(h * nh) * 128u;  // rows h*NT/2.. of B
          const uint32_t b1 = b0 + (uint32_t)w.nt * 128u;
#pragma unroll
          for (int kk = 0; kk < F8_BK / 32; ++kk) {
            const uint32_t ko = (uint32_t)kk * 32u;  // 32 e4m3 along K inside the swizzled row
            const uint64_t dah = sw128_desc(st + ko), dal = sw128_desc(st + F8_A_PLANE + ko);
            const uint64_t db0 = sw128_desc(b0 + ko);
            umma_e4m3(d, dah, db0, idesc, kk == 0 ? 0u : 1u);
            umma_e4m3(d, dal, db0, idesc, 1u);
            if (PLANES == 2) umma_e4m3(d, dah, sw128_desc(b1 + ko), idesc, 1u);
          }
          umma_commit(tmem_full(h));
        }
        if (fail) {
          *abort_flag = 1;
          break;
        }
        umma_commit(empty(rg.s));
      }
      umma_commit(done_bar);
      mbar_wait(done_bar, 0, err);
    }
  } else if (warp < 2 + F8_CONV_WARPS) {
    // ---------------- converters ----------------
    // half stages j = 2 i + h (64 rows each); three register buffers keep the
    // loads of the next two halves in flight while one is quantized
    const int ct = threadIdx.x - 64, cw = warp - 2;
    Fp8Converter<TRANS> cv;
    cv.setup(A, lda, w, ct);
    float va[F8_CV], vb[F8_CV], vc[F8_CV];
    Cursor lc;
    lc.init(w, u0);
    int loaded = 0;  // half stages loaded
    auto load = [&](float (&v)[F8_CV]) {
      if (loaded < 2 * cnt) {
        cv.load(lc.mt, lc.ks, loaded & 1, v);
        if (loaded & 1) lc.next(w);
        ++loaded;
      }
    };
    Ring rg;
    auto put = [&](const float (&v)[F8_CV], int j) -> bool {
      const int i = j >> 1, h = j & 1;
      bool ok = !*abort_flag;
      if (h == 0 && ok && !warp_wait(empty(rg.s), rg.ph ^ 1u, err)) {
        *abort_flag = 1;
        ok = false;
      }
      float m = 0.f;
#pragma unroll
      for (int e = 0; e < F8_CV; ++e) m = fmaxf(m, fabsf(v[e]));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
      const int b = j & 1;
      if (lane == 0) {
        red_amax[b * 16 + cw] = m;
        red_ok[b * 16 + cw] = ok ? 1 : 0;
      }
      named_sync(1, F8_CONV_THREADS);
      float amax = 0.f;
      int all_ok = 1;
#pragma unroll
      for (int q = 0; q < F8_CONV_WARPS; ++q) {
        amax = fmaxf(amax, red_amax[b * 16 + q]);
        all_ok &= red_ok[b * 16 + q];
      }
      if (!all_ok) return false;
      const float inv = amax > 0.f ? F8_MAX / amax : 0.f;
      cv.store(base + (uint32_t)rg.s * w.stage_bytes, h, inv, v);
      const int r = i & (F8_SCALE_RING - 1);
      if (ct == 0) sa_ring[2 * r + h] = amax / F8_MAX;
      if (h == 1) {
        fence_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(full_a(rg.s));
        if (ct == 0) mbar_arrive(scale_ready(r));
        rg.next(w.stages);
      }
      return true;
    };
    load(va);
    load(vb);
    for (int j = 0; j < 2 * cnt; j += 3) {
      load(vc);
      if (!put(va, j) || j + 1 >= 2 * cnt) break;
      load(va);
      if (!put(vb, j + 1) || j + 2 >= 2 * cnt) break;
      load(vb);
      if (!put(vc, j + 2)) break;
    }
  } else {
    // ---------------- epilogue: scale and fold each K tile ----------------
    const int q = warp & 3;
    const int et = threadIdx.x - 32 * (2 + F8_CONV_WARPS);  // 0..255
    const int ew = et >> 5;                                   // 0..7
    const int part = ew >> 2;                                 // which 16-column groups of a half
    const int nh = w.nt / 2;
    const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16);
    // the column scales of z for unit i, into sb_stage[i & 1] (read after the next named barrier)
    auto stage_scales = [&](int i, const Cursor& cu) {
      if (PLANES == 2) {
        const int cbase = w.c_lo + cu.nt * w.nt;
        for (int j = et; j < w.nt; j += 32 * F8_EPI_WARPS) {
          const int col = cbase + j;
          sb_stage[(i & 1) * F8_NMAX + j] = col < w.c_hi ? __ldg(zscale + (int64_t)cu.ks * zs_ld + col) : 0.f;
        }
      }
    };
    Cursor c;
    c.init(w, u0);
    if (cnt > 0) stage_scales(0, c);
    bool stop = false;
    for (int i = 0; i < cnt && !stop; ++i) {
      const bool first = (i == 0) || (c.ks == 0);  // first K tile of this tile part
      const bool emit = (i + 1 == cnt) || (c.ks + 1 == w.kst);
      const int b = i & 1;
      const int64_t row = c.mt * F8_BM + q * 32 + lane;
      const int cbase = w.c_lo + c.nt * w.nt;
      for (int h = 0; h < 2; ++h) {
        bool ok = !*abort_flag;
        if (ok && (!warp_wait(tmem_full(h), (uint32_t)(i & 1), err) ||
                   (h == 0 && !warp_wait(scale_ready(i & (F8_SCALE_RING - 1)),
                                         (uint32_t)((i / F8_SCALE_RING) & 1), err)))) {
          *abort_flag = 1;
          ok = false;
        }
        if (lane == 0) epi_ok[h * 8 + ew] = ok ? 1 : 0;
        named_sync(2, 32 * F8_EPI_WARPS);
        int all_ok = 1;
#pragma unroll
        for (int e = 0; e < F8_EPI_WARPS; ++e) all_ok &= epi_ok[h * 8 + e];
        if (!all_ok) {
          stop = true;
          break;
        }
        tc_fence_after();
        const float sa = sa_ring[2 * (i & (F8_SCALE_RING - 1)) + (q >> 1)];  // lanes 64.. are the second row half
        const float* sbs = const_cast<const float*>(sb_stage) + b * F8_NMAX;  // written before the barrier
        // the warps of a lane quarter take interleaved 16-column groups of the half
        for (int cc = h * nh + 16 * part; cc < (h + 1) * nh; cc += 16 * F8_EPW) {
          uint32_t v[16], t[16];
          tmem_ld16(trow + (uint32_t)(w.nt + cc), v);
          if (!first) tmem_ld16(trow + (uint32_t)cc, t);
          tmem_wait_ld();
#pragma unroll
          for (int j4 = 0; j4 < 16; j4 += 4) {
            float4 sc = make_float4(sa, sa, sa, sa);
            if (PLANES == 2) {
              const float4 z4 = *reinterpret_cast<const float4*>(sbs + cc + j4);
              sc = make_float4(sa * z4.x, sa * z4.y, sa * z4.z, sa * z4.w);
            }
            const float s4[4] = {sc.x, sc.y, sc.z, sc.w};
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int j = j4 + u;
              v[j] = __float_as_uint(__uint_as_float(v[j]) * s4[u] + (first ? 0.f : __uint_as_float(t[j])));
            }
          }
          if (!emit) {
            tmem_st16(trow + (uint32_t)cc, v);
            continue;
          }
          const int c0 = cbase + cc;
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
        if (lane == 0) mbar_arrive(tmem_empty(h));
      }
      c.next(w);
      if (!stop && i + 1 < cnt) stage_scales(i + 1, c);
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, w.tmem_cols);
}

namespace {

int encode_plane8(CUtensorMap* tm, const uint8_t* plane, int64_t n, int rows, int nt) {
  PFN_encodeTiled enc = get_encode_tiled();
  if (!enc) return SK_ERR_DEVICE;
  const cuuint64_t gdim[2] = {(cuuint64_t)n, (cuuint64_t)rows};
  const cuuint64_t gstride[1] = {(cuuint64_t)f8_pitch(n)};
  const cuuint32_t box[2] = {(cuuint32_t)F8_BK, (cuuint32_t)nt};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<uint8_t*>(plane), gdim, gstride, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? SK_OK : SK_ERR_ALIGN;
}

int launch_fp8(sk_op* h, const sk_matrix* A, bool trans, int c_lo, int c_hi, float scale, float* out, int64_t ldo,
               cudaStream_t s) {
  const bool gauss = h->kind == SK_GAUSS;
  const int planes = gauss ? 2 : 1;
  const uint8_t* p0 = gauss ? h->z8_hi : h->srht_q8;
  const uint8_t* p1 = gauss ? h->z8_lo : h->srht_q8;
  TcWork w{};
  w.m_rows = trans ? A->cols : A->rows;
  w.k_len = h->n;
  w.mtiles = (w.m_rows + F8_BM - 1) / F8_BM;
  w.kst = (int)((h->n + F8_BK - 1) / F8_BK);
  const int ncols = c_hi - c_lo;
  const int ntiles = (ncols + F8_NMAX - 1) / F8_NMAX;
  w.nt = ((ncols + ntiles - 1) / ntiles + 31) / 32 * 32;  // two halves of N, each a multiple of 16
  w.c_lo = c_lo;
  w.c_hi = c_hi;
  w.stage_bytes = 2 * F8_A_PLANE + (uint32_t)planes * (uint32_t)w.nt * 128u;
  const long avail = F8_SMEM_MAX - 1024 - (long)F8_AUX_BYTES;
  w.stages = (int)std::min<long>(F8_MAX_STAGES, avail / (long)w.stage_bytes);
  if (w.stages < 2) return SK_ERR_UNSUPPORTED;
  w.tmem_cols = tmem_cols_for(2 * w.nt);
  if (w.tmem_cols > 512) return SK_ERR_UNSUPPORTED;

  CUtensorMap t0, t1;
  JLS_CHECK(encode_plane8(&t0, p0, h->n, c_hi, w.nt));
  JLS_CHECK(encode_plane8(&t1, p1, h->n, c_hi, w.nt));
  JLS_CHECK_CUDA(cudaMemset2DAsync(out + c_lo, ldo * sizeof(float), 0, (size_t)ncols * sizeof(float),
                                   (size_t)w.m_rows, s));
  const int64_t tiles = (int64_t)ntiles * w.mtiles;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(num_sms(), tiles));
  const size_t smem = 1024 + (size_t)w.stages * w.stage_bytes + F8_AUX_BYTES;
  const int vec_ok = ((reinterpret_cast<uintptr_t>(out) & 15) == 0 && ldo % 4 == 0 && c_lo % 4 == 0) ? 1 : 0;
  const float* a = static_cast<const float*>(A->A);
  const float* zs = gauss ? h->z8_scale : nullptr;
#define JLS_F8_LAUNCH(TR, PL)                                                                                   \
  do {                                                                                                          \
    auto kern = tc_fp8_kernel<TR, PL>;                                                                         \
    JLS_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));        \
    kern<<<grid, F8_THREADS, smem, s>>>(a, A->ld, t0, t1, w, zs, h->d_max, scale, out, ldo, vec_ok, h->d_err); \
  } while (0)
  if (trans && gauss) JLS_F8_LAUNCH(true, 2);
  else if (trans) JLS_F8_LAUNCH(true, 1);
  else if (gauss) JLS_F8_LAUNCH(false, 2);
  else JLS_F8_LAUNCH(false, 1);
#undef JLS_F8_LAUNCH
  note_launch();
  JLS_CHECK_CUDA(cudaGetLastError());
  return SK_OK;
}

}  // namespace

int dense_apply_fp8(sk_op* h, const sk_matrix* A, int which, int c_lo, int c_hi, double scale, void* S, int64_t ldS,
                    void* St, int64_t ldSt, cudaStream_t s) {
  if (A->dtype != SK_F32 || (h->kind != SK_SRHT && h->kind != SK_GAUSS)) return SK_ERR_DTYPE;
  if (c_hi <= c_lo) return SK_OK;
  if (h->kind == SK_GAUSS) JLS_CHECK(gen_gauss_fp8(h, h->d_total, s));
  else JLS_CHECK(gen_srht_fp8(h, h->d_total, s));
  if (which & SK_S) JLS_CHECK(launch_fp8(h, A, false, c_lo, c_hi, (float)scale, (float*)S, ldS, s));
  if (which & SK_ST) JLS_CHECK(launch_fp8(h, A, true, c_lo, c_hi, (float)scale, (float*)St, ldSt, s));
  return SK_OK;
}

}  // namespace jls
