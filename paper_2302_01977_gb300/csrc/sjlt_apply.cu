// sjlt_apply.cu -- S = A R and S' = A^T R for an SJLT R (Sec. 6.3), sm_103a.
//
// R is held as a tiled compressed-column structure (Sec. 6.1's CCS of B+ and
// B-, merged with the sign and cut into tiles of TILE rows of R; see
// TiledCcs): for each tile, the entries of each column of R in row order.
// Every entry adds or subtracts elements of A (the +-1 is applied by a fused
// multiply-add with the entry's sign), and the scale 1/sqrt(alpha * blocks) is
// applied once when results are written, as in the paper's binary-matrix
// design.
//
// GB300 mapping (both kernels stream A exactly once from HBM):
//  * Persistent stream-K grid, at most one CTA per SM: the (block of A, tile
//    of R) units are cut into equal contiguous ranges, so every SM streams the
//    same number of bytes; a block split between two CTAs gets two
//    contributions, added with red.global.add into a zeroed output (two terms
//    onto zero: order-independent, so results are deterministic).
//  * A consumer warp owns <= NB output columns of R and keeps their sums in
//    registers for the whole block; because a tile's entries are grouped by
//    column, the warp walks them column by column with compile-time
//    accumulator indices.  Each entry is one broadcast 4-byte shared load
//    (byte offset | sign bit), one 32-bit add for the address, one data load
//    and two paired FP32 FMAs (FFMA2).  The chain shared load -> shared load ->
//    FMA is latency-bound, so a CTA runs SJLT_WARPS = 28 warps (7 per SM
//    sub-partition, 72 registers each) with SJLT_NB = 10 columns per warp.
//  * S' (cols kernel): lanes own VEC consecutive columns of A (one 16-byte
//    vector).  Tiles of TILE rows x 32*VEC columns arrive by TMA into a dense
//    layout; an entry makes each lane read one 16-byte vector of row r
//    (conflict-free).  One producer warp runs a STAGES-deep mbarrier ring; the
//    tile's entries and column offsets ride along as bulk copies on the same
//    barrier.
//  * S (rows kernel): lanes own RPL = 4 rows of A (lane + 32 q).  Tiles of 128
//    rows x TILE columns of A (= TILE rows of R) are copied by NPROD producer
//    warps with 4/8-byte cp.async into a row pitch of TILE + 1 elements, so
//    that 32 lanes reading tile[row][j] hit 32 banks; completion is tracked
//    with cp.async.mbarrier.arrive on the same ring.
#include <cuda.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "sjlt_common.cuh"

namespace jls {

// ---------------------------------------------------------------------------
// Matrix-free tiles: GEN_WARPS warps compute the S' tile A_ij = K(p_i, q_j) =
// 2^(-c2 |p_i - q_j|^2) (+ shift where i == j) in shared memory instead of
// loading it, so the kernel sketches a Gaussian kernel matrix that is never
// written to HBM.  Lane l owns the 4 columns of its 16-byte slot (their points
// stay in registers for the whole block of A) and computes them for rows pw,
// pw + GEN_WARPS, ... of the tile; the rows' points are loaded one tile ahead,
// two per lane, and broadcast by shuffles.  Arithmetic runs on pairs of
// columns (FADD2 / FFMA2), the exponential is the MUFU ex2 instruction.  Warp 0
// lane 0 also brings the tile's entry records and column offsets by bulk copy.
// Rows and columns outside the matrix hold 0.
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

template <int TILE, int STAGES>
__device__ __forceinline__ void gen_producer(const KGen& g, int64_t rowsA, int64_t colsA, const uint4* ents,
                                             const uint32_t* offs, int64_t e_stride, int64_t o_stride, int c_lo,
                                             int c_hi, uint32_t E_BYTES, uint32_t O_BYTES, uint32_t tiles_sa,
                                             uint32_t ents_sa, uint32_t offs_sa, uint32_t full0, uint32_t empty0,
                                             int o_lo, int pw, int lane, int64_t u0, int64_t u1, int* err) {
  constexpr int BW = 128;
  constexpr uint32_t TILE_BYTES = TILE * BW * 4;
  constexpr int ROWS = (TILE + GEN_WARPS - 1) / GEN_WARPS;  // rows per warp (<= 64: two per lane)
  static_assert(ROWS <= 64, "two row points per lane");
  const int ntiles = (int)((rowsA + TILE - 1) / TILE);
  const float2 nc2 = make_float2(-g.c2, -g.c2);
  float2 nqx0, nqx1, nqy0, nqy1, nqz0, nqz1;  // minus this lane's column points, as pairs (0,1), (2,3)
  bool cin[4];
  int64_t cur_blk = -1;
  // points of rows pw + GEN_WARPS * lane and pw + GEN_WARPS * (lane + 32) of a tile
  auto load_rows = [&](int t, float (&pa)[3], float (&pb)[3]) {
#pragma unroll
    for (int h2 = 0; h2 < 2; ++h2) {
      const int r = pw + GEN_WARPS * (lane + 32 * h2);
      const int64_t i = (int64_t)t * TILE + r;
      const bool in = r < TILE && i < rowsA;
      float* dst = h2 ? pb : pa;
      dst[0] = in ? __ldg(g.P + 3 * i) : 0.f;
      dst[1] = in ? __ldg(g.P + 3 * i + 1) : 0.f;
      dst[2] = in ? __ldg(g.P + 3 * i + 2) : 0.f;
    }
  };
  float pa[3], pb[3];
  if (u1 > u0) load_rows((int)(u0 % ntiles), pa, pb);
  int k = 0;
  for (int64_t u = u0; u < u1; ++u, ++k) {
    const int s = k % STAGES;
    const int64_t blk = u / ntiles;
    const int t = (int)(u % ntiles);
    float na[3], nb[3];  // next tile's row points, in flight while this tile is computed
    if (u + 1 < u1) load_rows((int)((u + 1) % ntiles), na, nb);
    if (k >= STAGES) {
      int ok = 1;
      if (lane == 0) ok = mbar_wait(empty0 + 8 * s, ((k / STAGES) - 1) & 1, err) ? 1 : 0;
      if (!__shfl_sync(0xffffffffu, ok, 0)) break;
    }
    const uint32_t fb = full0 + 8 * s;
    if (pw == 0 && lane == 0) {
      const uint32_t lo = __ldg(offs + (int64_t)t * o_stride + c_lo), hi = __ldg(offs + (int64_t)t * o_stride + c_hi);
      uint32_t eb = (hi - lo) * 16;
      if (eb > E_BYTES) {  // host sizing guarantees this never happens
        set_err(err, ERRF_BOUNDS);
        eb = 0;
      }
      mbar_arrive_expect_tx(fb, eb + O_BYTES);
      if (eb) bulk_g2s(ents_sa + s * E_BYTES, ents + (int64_t)t * e_stride + lo, eb, fb);
      bulk_g2s(offs_sa + s * O_BYTES, offs + (int64_t)t * o_stride + o_lo, O_BYTES, fb);
    }
    if (blk != cur_blk) {
      cur_blk = blk;
      float q[4][3];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int64_t j = blk * BW + lane * 4 + c;
        cin[c] = j < colsA;
#pragma unroll
        for (int a = 0; a < 3; ++a) q[c][a] = cin[c] ? -__ldg(g.Q + 3 * j + a) : 0.f;
      }
      nqx0 = make_float2(q[0][0], q[1][0]);
      nqx1 = make_float2(q[2][0], q[3][0]);
      nqy0 = make_float2(q[0][1], q[1][1]);
      nqy1 = make_float2(q[2][1], q[3][1]);
      nqz0 = make_float2(q[0][2], q[1][2]);
      nqz1 = make_float2(q[2][2], q[3][2]);
    }
    const int64_t j0 = blk * BW + lane * 4;
    const uint32_t dst = tiles_sa + s * TILE_BYTES + lane * 16;
    const int64_t i0 = (int64_t)t * TILE;
#pragma unroll 2
    for (int uu = 0; uu < ROWS; ++uu) {
      const int r = pw + GEN_WARPS * uu;
      if (r >= TILE) break;  // uniform
      const int src = uu & 31;
      const float px = __shfl_sync(0xffffffffu, uu < 32 ? pa[0] : pb[0], src);
      const float py = __shfl_sync(0xffffffffu, uu < 32 ? pa[1] : pb[1], src);
      const float pz = __shfl_sync(0xffffffffu, uu < 32 ? pa[2] : pb[2], src);
      const float2 px2 = make_float2(px, px), py2 = make_float2(py, py), pz2 = make_float2(pz, pz);
      const float2 dx0 = __fadd2_rn(px2, nqx0), dx1 = __fadd2_rn(px2, nqx1);
      const float2 dy0 = __fadd2_rn(py2, nqy0), dy1 = __fadd2_rn(py2, nqy1);
      const float2 dz0 = __fadd2_rn(pz2, nqz0), dz1 = __fadd2_rn(pz2, nqz1);
      float2 a0 = __ffma2_rn(dx0, dx0, __ffma2_rn(dy0, dy0, __fmul2_rn(dz0, dz0)));
      float2 a1 = __ffma2_rn(dx1, dx1, __ffma2_rn(dy1, dy1, __fmul2_rn(dz1, dz1)));
      a0 = __fmul2_rn(a0, nc2);
      a1 = __fmul2_rn(a1, nc2);
      const int64_t i = i0 + r;
      const bool rin = i < rowsA;
      float v0 = (rin && cin[0]) ? ex2_approx(a0.x) : 0.f;
      float v1 = (rin && cin[1]) ? ex2_approx(a0.y) : 0.f;
      float v2 = (rin && cin[2]) ? ex2_approx(a1.x) : 0.f;
      float v3 = (rin && cin[3]) ? ex2_approx(a1.y) : 0.f;
      if (g.shift != 0.f && i >= j0 && i < j0 + 4) {  // the diagonal crosses this slot
        if (i == j0 && cin[0]) v0 += g.shift;
        if (i == j0 + 1 && cin[1]) v1 += g.shift;
        if (i == j0 + 2 && cin[2]) v2 += g.shift;
        if (i == j0 + 3 && cin[3]) v3 += g.shift;
      }
      asm volatile("st.shared.v4.f32 [%0], {%1,%2,%3,%4};" ::"r"(dst + r * (uint32_t)(BW * 4)), "f"(v0), "f"(v1),
                   "f"(v2), "f"(v3)
                   : "memory");
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(fb);
    if (u + 1 < u1) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        pa[a] = na[a];
        pb[a] = nb[a];
      }
    }
  }
}

// CPLX: A is the real view of an interleaved complex matrix (2 m real columns
// for m complex ones); lane quads hold (re, im) of two complex columns, and the
// flush writes St as complex (row j, column c = (re, -im)): S' = A* R.
template <typename T, int TILE, int NB, int STAGES, bool GEN = false, bool CPLX = false>
__global__ void __launch_bounds__((GEN ? GEN_CTA_WARPS : SJLT_WARPS) * 32, 1)
    sjlt_cols_kernel(const __grid_constant__ CUtensorMap tmA, int64_t rowsA, int64_t colsA,
                     const uint4* __restrict__ ents, const uint32_t* __restrict__ offs, int64_t e_stride,
                     int64_t o_stride, int c_lo, int c_hi, int nbw, int njobs, uint32_t E_BYTES,
                     T* __restrict__ St, int64_t ldSt, T scale, int* err, KGen gen) {
  constexpr int VEC = 16 / sizeof(T);
  constexpr int BW = 32 * VEC;  // columns of A per block
  constexpr uint32_t TILE_BYTES = TILE * BW * sizeof(T);
  static_assert(BW * sizeof(T) == CCS_ROW_BYTES, "entry offsets assume 512-byte tile rows");
  extern __shared__ __align__(1024) uint8_t smem[];
  const int o_lo = c_lo & ~3;
  const int o_cnt = ((c_hi + 1 + 3) & ~3) - o_lo;
  const uint32_t O_BYTES = (uint32_t)o_cnt * 4;
  const uint32_t tiles_sa = smem_u32(smem);
  const uint32_t ents_sa = tiles_sa + STAGES * TILE_BYTES;
  uint8_t* sh_o = smem + STAGES * (TILE_BYTES + E_BYTES);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sh_o + STAGES * O_BYTES);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntiles = (int)((rowsA + TILE - 1) / TILE);
  const int64_t nblk = (colsA + BW - 1) / BW;
  const SplitK rg = cta_range(nblk * ntiles);

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, GEN ? 1 + GEN_WARPS : 1);
      mbar_init(empty0 + 8 * s, njobs);
    }
    fence_mbar_init();
  }
  __syncthreads();

  if (GEN && warp >= njobs) {  // ---- producers that compute the tile: A_ij = K(p_i, q_j)
    if constexpr (GEN) gen_producer<TILE, STAGES>(gen, rowsA, colsA, ents, offs, e_stride, o_stride, c_lo, c_hi,
                                                  E_BYTES, O_BYTES, tiles_sa, ents_sa, smem_u32(sh_o), full0,
                                                  empty0, o_lo, warp - njobs, lane, rg.u0, rg.u1, err);
  } else if (warp == njobs) {  // ---- producer
    if (lane == 0 && rg.u1 > rg.u0) {
      tma_prefetch_desc(&tmA);
      int k = 0;
      // entry range of the next tile, loaded one tile ahead
      int t = (int)(rg.u0 % ntiles);
      uint32_t e_lo = __ldg(offs + (int64_t)t * o_stride + c_lo), e_hi = __ldg(offs + (int64_t)t * o_stride + c_hi);
      for (int64_t u = rg.u0; u < rg.u1; ++u, ++k) {
        const int s = k % STAGES;
        const int64_t blk = u / ntiles;
        t = (int)(u % ntiles);
        const uint32_t lo = e_lo, hi = e_hi;
        if (u + 1 < rg.u1) {
          const int tn = (int)((u + 1) % ntiles);
          e_lo = __ldg(offs + (int64_t)tn * o_stride + c_lo);
          e_hi = __ldg(offs + (int64_t)tn * o_stride + c_hi);
        }
        const uint32_t eb = (hi - lo) * 16;
        if (eb > E_BYTES) {  // host sizing guarantees this never happens
          set_err(err, ERRF_BOUNDS);
          break;
        }
        if (k >= STAGES && !mbar_wait(empty0 + 8 * s, ((k / STAGES) - 1) & 1, err)) break;
        const uint32_t fb = full0 + 8 * s;
        mbar_arrive_expect_tx(fb, TILE_BYTES + eb + O_BYTES);
        tma_load_2d(tiles_sa + s * TILE_BYTES, &tmA, fb, (int32_t)(blk * BW), t * TILE);
        if (eb) bulk_g2s(ents_sa + s * E_BYTES, ents + (int64_t)t * e_stride + lo, eb, fb);
        bulk_g2s(smem_u32(sh_o) + s * O_BYTES, offs + (int64_t)t * o_stride + o_lo, O_BYTES, fb);
      }
    }
  } else {  // ---- consumers
    ColsAcc<T> acc[NB];
    const int cw0 = c_lo + warp * nbw;
    const int nb = max(0, min(nbw, c_hi - cw0));
    const bool vec_ok = ((ldSt | cw0) & 3) == 0;
    const uint32_t lane_off = lane * 16;
    int k = 0;
    auto flush = [&](int64_t blk) {
      if constexpr (CPLX) {
#pragma unroll
        for (int hq = 0; hq < VEC / 2; ++hq) {
          const int64_t jc = (blk * BW + lane * VEC) / 2 + hq;  // complex column of A = row of S'
          if (2 * jc < colsA) {
            T re[NB], im[NB];
#pragma unroll
            for (int b = 0; b < NB; ++b) {
              re[b] = acc[b].get(2 * hq);
              im[b] = acc[b].get(2 * hq + 1);
            }
            flush_row_conj<NB>(St + jc * ldSt + 2 * cw0, re, im, nb, scale);
          }
        }
      } else {
#pragma unroll
        for (int q = 0; q < VEC; ++q) {
          const int64_t j = blk * BW + lane * VEC + q;
          if (j < colsA) {
            T v[NB];
#pragma unroll
            for (int b = 0; b < NB; ++b) v[b] = acc[b].get(q);
            flush_row<NB>(St + j * ldSt + cw0, v, nb, scale, vec_ok);
          }
        }
      }
    };
    bool ok = true;
    for (int64_t u = rg.u0; u < rg.u1 && ok;) {  // one block of A per outer iteration
      const int64_t blk = u / ntiles;
      const int64_t u_end = min64(rg.u1, (blk + 1) * ntiles);
#pragma unroll
      for (int b = 0; b < NB; ++b) acc[b].zero();
      for (; u < u_end; ++u, ++k) {
        const int s = k % STAGES;
        if (!mbar_wait(full0 + 8 * s, (k / STAGES) & 1, err)) {
          ok = false;
          break;
        }
        if (nb > 0) {
          const uint32_t* O = reinterpret_cast<const uint32_t*>(sh_o + s * O_BYTES) - o_lo;
          // shared address of entry index p is ebase + 16 p
          const uint32_t ebase = ents_sa + s * E_BYTES - O[c_lo] * 16;
          const uint32_t xaddr = tiles_sa + s * TILE_BYTES + lane_off;
          uint32_t p = O[cw0];
#pragma unroll
          for (int b = 0; b < NB; ++b) {
            if (b < nb) {
              const uint32_t e = O[cw0 + b + 1];
              uint32_t ea = ebase + p * 16;
              for (; p + 1 < e; p += 2, ea += 32) {
                const auto r0 = CcsRec<T>::cols(ea), r1 = CcsRec<T>::cols(ea + 16);
                acc[b].add(xaddr, r0);
                acc[b].add(xaddr, r1);
              }
              if (p < e) {
                acc[b].add(xaddr, CcsRec<T>::cols(ea));
                ++p;
              }
            }
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(empty0 + 8 * s);
      }
      if (ok && nb > 0) flush(blk);
    }
  }
  __syncthreads();  // no CTA exits while its copies may still land in shared memory
}

// ---------------------------------------------------------------------------
// S = A R : lanes over rows of A (RPL rows each), cp.async-fed, pitch TILE + 1.
constexpr int RPL = 4;  // rows per lane
constexpr int ROWS_BLK = 32 * RPL;
#ifndef SJLT_NPROD_OVERRIDE
constexpr int NPROD = 2;  // producer warps
#else
constexpr int NPROD = SJLT_NPROD_OVERRIDE;
#endif

template <typename T>
struct RowsAcc;
template <>
struct RowsAcc<float> {
  float2 a, b;  // rows (q0, q1), (q2, q3)
  __device__ __forceinline__ void zero() { a = b = make_float2(0.f, 0.f); }
  // w: the record's S word, column offset | sign bit
  template <uint32_t STEP>
  __device__ __forceinline__ void add(uint32_t raddr, uint32_t w) {
    const uint32_t x = raddr + (w & 0x7fffffffu);
    const float v0 = lds_f1(x), v1 = lds_f1(x + STEP), v2 = lds_f1(x + 2 * STEP), v3 = lds_f1(x + 3 * STEP);
    const float sg = __uint_as_float((w & 0x80000000u) | 0x3f800000u);
    const float2 s = f2(sg, sg);
    a = __ffma2_rn(f2(v0, v1), s, a);
    b = __ffma2_rn(f2(v2, v3), s, b);
  }
  __device__ __forceinline__ float get(int q) const { return q == 0 ? a.x : q == 1 ? a.y : q == 2 ? b.x : b.y; }
};
template <>
struct RowsAcc<double> {
  double v[4];
  __device__ __forceinline__ void zero() { v[0] = v[1] = v[2] = v[3] = 0.0; }
  template <uint32_t STEP>
  __device__ __forceinline__ void add(uint32_t raddr, const uint4& r) {
    const uint32_t x = raddr + r.w;
    const double s = sign_d(r);
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = fma(lds_d1(x + q * STEP), s, v[q]);
  }
  __device__ __forceinline__ double get(int q) const { return v[q]; }
};

template <typename T, int TILE, int NB, int STAGES>
__global__ void __launch_bounds__(SJLT_WARPS * 32, 1)
    sjlt_rows_kernel(const T* __restrict__ A, int64_t lda, int64_t rowsA, int64_t colsA,
                     const uint4* __restrict__ ents, const uint32_t* __restrict__ offs, int64_t e_stride,
                     int64_t o_stride, int c_lo, int c_hi, int nbw, int njobs, uint32_t E_BYTES,
                     T* __restrict__ S, int64_t ldS, T scale, int* err) {
  constexpr int P = TILE + 1;
  constexpr uint32_t TILE_BYTES = ((ROWS_BLK * P * sizeof(T)) + 127) / 128 * 128;
  constexpr uint32_t ROW_STEP = 32 * P * sizeof(T);  // bytes between a lane's rows q and q + 1
  extern __shared__ __align__(1024) uint8_t smem[];
  const int o_lo = c_lo & ~3;
  const int o_cnt = ((c_hi + 1 + 3) & ~3) - o_lo;
  const uint32_t O_BYTES = (uint32_t)o_cnt * 4;
  const uint32_t tiles_sa = smem_u32(smem);
  const uint32_t ents_sa = tiles_sa + STAGES * TILE_BYTES;
  uint8_t* sh_o = smem + STAGES * (TILE_BYTES + E_BYTES);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sh_o + STAGES * O_BYTES);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntiles = (int)((colsA + TILE - 1) / TILE);
  const int64_t nblk = (rowsA + ROWS_BLK - 1) / ROWS_BLK;
  const SplitK rg = cta_range(nblk * ntiles);

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, NPROD * 32);
      mbar_init(empty0 + 8 * s, njobs);
    }
    fence_mbar_init();
  }
  __syncthreads();

  if (warp >= njobs) {  // ---- producers: NPROD warps of cp.async
    const int pt = threadIdx.x - njobs * 32;  // 0 .. NPROD*32-1
    const int pw = pt >> 5;
    int k = 0;
    int t = rg.u1 > rg.u0 ? (int)(rg.u0 % ntiles) : 0;
    uint32_t e_lo = 0, e_hi = 0;
    if (rg.u1 > rg.u0) {
      e_lo = __ldg(offs + (int64_t)t * o_stride + c_lo);
      e_hi = __ldg(offs + (int64_t)t * o_stride + c_hi);
    }
    for (int64_t u = rg.u0; u < rg.u1; ++u, ++k) {
      const int s = k % STAGES;
      const int64_t blk = u / ntiles;
      t = (int)(u % ntiles);
      const uint32_t lo = e_lo, hi = e_hi;
      if (u + 1 < rg.u1) {  // next tile's entry range, one tile ahead
        const int tn = (int)((u + 1) % ntiles);
        e_lo = __ldg(offs + (int64_t)tn * o_stride + c_lo);
        e_hi = __ldg(offs + (int64_t)tn * o_stride + c_hi);
      }
      if (k >= STAGES && !mbar_wait(empty0 + 8 * s, ((k / STAGES) - 1) & 1, err)) break;
      const int64_t i0 = blk * ROWS_BLK, j0 = (int64_t)t * TILE;
      const uint32_t dst = tiles_sa + s * TILE_BYTES;
      if (i0 + ROWS_BLK <= rowsA && j0 + TILE <= colsA) {
        // full tile: each warp copies every NPROD-th row, 32 consecutive
        // columns per instruction (coalesced; consecutive banks)
        const T* src = A + (i0 + pw) * lda + j0 + lane;
        uint32_t d = dst + (pw * P + lane) * (uint32_t)sizeof(T);
        for (int r = pw; r < ROWS_BLK; r += NPROD, src += NPROD * lda, d += NPROD * P * (uint32_t)sizeof(T)) {
#pragma unroll
          for (int q = 0; q < TILE / 32; ++q) {
            if (sizeof(T) == 4)
              cp_async_4(d + q * 32 * 4, src + q * 32, 4);
            else
              cp_async_8(d + q * 32 * 8, src + q * 32, 8);
          }
        }
      } else {  // ragged tile: per-element bounds, zero fill outside A
        for (int r = pw; r < ROWS_BLK; r += NPROD) {
#pragma unroll
          for (int q = 0; q < TILE / 32; ++q) {
            const int c = q * 32 + lane;
            const bool in = (i0 + r < rowsA) && (j0 + c < colsA);
            const T* src = in ? A + (i0 + r) * lda + j0 + c : A;
            if (sizeof(T) == 4)
              cp_async_4(dst + (r * P + c) * 4, src, in ? 4 : 0);
            else
              cp_async_8(dst + (r * P + c) * 8, src, in ? 8 : 0);
          }
        }
      }
      uint32_t eb = (hi - lo) * 16;
      if (eb > E_BYTES) {  // host sizing guarantees this never happens
        set_err(err, ERRF_BOUNDS);
        eb = 0;
      }
      const uint8_t* se = reinterpret_cast<const uint8_t*>(ents + (int64_t)t * e_stride + lo);
      for (uint32_t q = pt; q < eb / 16; q += NPROD * 32) cp_async_16(ents_sa + s * E_BYTES + q * 16, se + q * 16);
      const uint8_t* so = reinterpret_cast<const uint8_t*>(offs + (int64_t)t * o_stride + o_lo);
      for (uint32_t q = pt; q < O_BYTES / 16; q += NPROD * 32)
        cp_async_16(smem_u32(sh_o) + s * O_BYTES + q * 16, so + q * 16);
      cp_async_mbar_arrive(full0 + 8 * s);
    }
    cp_async_wait<0>();
  } else {  // ---- consumers
    RowsAcc<T> acc[NB];
    const int cw0 = c_lo + warp * nbw;
    const int nb = max(0, min(nbw, c_hi - cw0));
    const bool vec_ok = ((ldS | cw0) & 3) == 0;
    const uint32_t lane_off = lane * P * (uint32_t)sizeof(T);
    int k = 0;
    auto flush = [&](int64_t blk) {
#pragma unroll
      for (int q = 0; q < RPL; ++q) {
        const int64_t i = blk * ROWS_BLK + lane + 32 * q;
        if (i < rowsA) {
          T v[NB];
#pragma unroll
          for (int b = 0; b < NB; ++b) v[b] = acc[b].get(q);
          flush_row<NB>(S + i * ldS + cw0, v, nb, scale, vec_ok);
        }
      }
    };
    bool ok = true;
    for (int64_t u = rg.u0; u < rg.u1 && ok;) {  // one block of A per outer iteration
      const int64_t blk = u / ntiles;
      const int64_t u_end = min64(rg.u1, (blk + 1) * ntiles);
#pragma unroll
      for (int b = 0; b < NB; ++b) acc[b].zero();
      for (; u < u_end; ++u, ++k) {
        const int s = k % STAGES;
        if (!mbar_wait(full0 + 8 * s, (k / STAGES) & 1, err)) {
          ok = false;
          break;
        }
        if (nb > 0) {
          const uint32_t* O = reinterpret_cast<const uint32_t*>(sh_o + s * O_BYTES) - o_lo;
          const uint32_t ebase = ents_sa + s * E_BYTES - O[c_lo] * 16;
          const uint32_t raddr = tiles_sa + s * TILE_BYTES + lane_off;
          uint32_t p = O[cw0];
#pragma unroll
          for (int b = 0; b < NB; ++b) {
            if (b < nb) {
              const uint32_t e = O[cw0 + b + 1];
              uint32_t ea = ebase + p * 16;
              for (; p + 1 < e; p += 2, ea += 32) {
                const auto r0 = CcsRec<T>::rows(ea), r1 = CcsRec<T>::rows(ea + 16);
                acc[b].template add<ROW_STEP>(raddr, r0);
                acc[b].template add<ROW_STEP>(raddr, r1);
              }
              if (p < e) {
                acc[b].template add<ROW_STEP>(raddr, CcsRec<T>::rows(ea));
                ++p;
              }
            }
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(empty0 + 8 * s);
      }
      if (ok && nb > 0) flush(blk);
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// host side
PFN_encodeTiled get_encode_tiled() {
  static PFN_encodeTiled fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_encodeTiled>(p);
  }
  return fn;
}

int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) sms = 1;
  }
  return sms;
}

namespace {

// SJLT_WARPS warps per CTA: the cols kernel runs SJLT_WARPS - 1 consumer warps
// + 1 TMA producer, the rows kernel SJLT_WARPS - NPROD consumer warps + NPROD
// cp.async producers, the tile-computing cols kernel GEN_JOBS consumers +
// GEN_WARPS producers.  A consumer warp owns <= NB columns.
constexpr int COLS_JOBS = SJLT_WARPS - 1;
constexpr int ROWS_JOBS = SJLT_WARPS - NPROD;
constexpr int NB_COLS = SJLT_NB;
template <typename T>
constexpr int nb_rows() {  // d = 256 (FP32) and 128 (FP64) in one launch
  return sizeof(T) == 4 ? (256 + ROWS_JOBS - 1) / ROWS_JOBS : (128 + ROWS_JOBS - 1) / ROWS_JOBS;
}
constexpr size_t ENTRY_BYTES = sizeof(uint4);
constexpr long SMEM_MAX = 227 * 1024;

// blocks of R whose entries fit next to STAGES tiles
template <int STAGES>
long blocks_that_fit(size_t tile_b, size_t o_max, size_t e_blk) {
  return ((SMEM_MAX - 2 * STAGES * 8) / STAGES - (long)tile_b - (long)o_max) / (long)e_blk;
}

struct Jobs {
  int njobs, nbw;
};
Jobs plan_jobs(int ncols, int max_jobs) {
  // spread the columns over as many warps as allowed (more warps hide more latency)
  int nj = std::min(max_jobs, ncols);
  int nbw = (ncols + nj - 1) / nj;
  nj = (ncols + nbw - 1) / nbw;
  return {nj, nbw};
}

// Column ranges one launch can take: <= jobs * NB columns and few enough
// blocks that the staged entries fit.  Each launch streams A once; ranges are
// cut at block boundaries.
struct Range {
  int lo, hi, nblk;
};
std::vector<Range> plan_ranges(const sk_op* h, int c_lo, int c_hi, int max_blk, int max_cols) {
  std::vector<Range> out;
  int c = c_lo;
  while (c < c_hi) {
    int hi = c, nblk = 0, off = 0;
    for (size_t b = 0; b < h->blocks.size(); ++b) {
      const int b_lo = off, b_hi = off + h->blocks[b];
      off = b_hi;
      if (b_hi <= c) continue;
      if (b_lo >= c_hi) break;
      if (nblk == max_blk) break;
      const int take_hi = std::min(std::min(b_hi, c_hi), c + max_cols);
      if (take_hi <= hi) break;
      hi = take_hi;
      ++nblk;
      if (hi < std::min(b_hi, c_hi)) break;  // width limit reached inside a block
    }
    out.push_back({c, hi, nblk});
    c = hi;
  }
  return out;
}

template <typename T>
int zero_columns(T* out, int64_t ld, int64_t rows, int c_lo, int c_hi, cudaStream_t s) {
  JLS_CHECK_CUDA(cudaMemset2DAsync(out + c_lo, ld * sizeof(T), 0, (size_t)(c_hi - c_lo) * sizeof(T), rows, s));
  return SK_OK;
}

template <typename T, int TILE, int STAGES, bool CPLX = false>
int launch_cols(sk_op* h, const sk_matrix* A, const TiledCcs& C, int c_lo, int c_hi, T scale, T* St,
                int64_t ldSt, cudaStream_t s) {
  constexpr int VEC = 16 / sizeof(T), BW = 32 * VEC;
  PFN_encodeTiled enc = get_encode_tiled();
  if (!enc) return SK_ERR_DEVICE;
  CUtensorMap tm;
  const cuuint64_t gdim[2] = {(cuuint64_t)A->cols, (cuuint64_t)A->rows};
  const cuuint64_t gstride[1] = {(cuuint64_t)(A->ld * sizeof(T))};
  const cuuint32_t box[2] = {(cuuint32_t)BW, (cuuint32_t)TILE};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(&tm, sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2,
                   const_cast<void*>(A->A), gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return SK_ERR_ALIGN;
  if (CPLX)  // St: A->cols / 2 complex rows, ldSt floats; columns [c_lo, c_hi) are (re, im) pairs
    JLS_CHECK(zero_columns(St, ldSt, A->cols / 2, 2 * c_lo, 2 * c_hi, s));
  else
    JLS_CHECK(zero_columns(St, ldSt, A->cols, c_lo, c_hi, s));
  const size_t tile_b = (size_t)TILE * BW * sizeof(T);
  const size_t o_max = (COLS_JOBS * NB_COLS + 8) * 4;
  const size_t e_blk = (size_t)h->alpha * TILE * ENTRY_BYTES;
  const long fit = blocks_that_fit<STAGES>(tile_b, o_max, e_blk);
  if (fit < 1) return SK_ERR_UNSUPPORTED;
  // at most one CTA per block of A keeps every block within two contiguous
  // CTA ranges, i.e. at most two contributions per output cell
  const int64_t nblk = (A->cols + BW - 1) / BW;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(num_sms(), nblk));
  for (const Range& rg : plan_ranges(h, c_lo, c_hi, (int)fit, COLS_JOBS * NB_COLS)) {
    const Jobs J = plan_jobs(rg.hi - rg.lo, COLS_JOBS);
    const uint32_t e_bytes = (uint32_t)(e_blk * rg.nblk);
    const uint32_t o_bytes = (uint32_t)((((rg.hi + 1 + 3) & ~3) - (rg.lo & ~3)) * 4);
    const size_t smem = STAGES * (tile_b + e_bytes + o_bytes) + 2 * STAGES * 8;
    if ((long)smem > SMEM_MAX) return SK_ERR_UNSUPPORTED;
    auto kern = sjlt_cols_kernel<T, TILE, NB_COLS, STAGES, false, CPLX>;
    JLS_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<grid, (J.njobs + 1) * 32, smem, s>>>(tm, A->rows, A->cols, C.ents, C.offs, C.e_stride, C.o_stride,
                                                rg.lo, rg.hi, J.nbw, J.njobs, e_bytes, St, ldSt, scale, h->d_err,
                                                KGen{});
    note_launch();
    JLS_CHECK_CUDA(cudaGetLastError());
  }
  return SK_OK;
}

template <typename T, int TILE, int STAGES>
int launch_rows(sk_op* h, const sk_matrix* A, const TiledCcs& C, int c_lo, int c_hi, T scale, T* S, int64_t ldS,
                cudaStream_t s) {
  JLS_CHECK(zero_columns(S, ldS, A->rows, c_lo, c_hi, s));
  constexpr int NB = nb_rows<T>();
  const size_t tile_b = ((ROWS_BLK * (TILE + 1) * sizeof(T)) + 127) / 128 * 128;
  const size_t o_max = (ROWS_JOBS * NB + 8) * 4;
  const size_t e_blk = (size_t)h->alpha * TILE * ENTRY_BYTES;
  const long fit = blocks_that_fit<STAGES>(tile_b, o_max, e_blk);
  if (fit < 1) return SK_ERR_UNSUPPORTED;
  const int64_t nblk = (A->rows + ROWS_BLK - 1) / ROWS_BLK;  // see launch_cols
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(num_sms(), nblk));
  for (const Range& rg : plan_ranges(h, c_lo, c_hi, (int)fit, ROWS_JOBS * NB)) {
    const Jobs J = plan_jobs(rg.hi - rg.lo, ROWS_JOBS);
    const uint32_t e_bytes = (uint32_t)(e_blk * rg.nblk);
    const uint32_t o_bytes = (uint32_t)((((rg.hi + 1 + 3) & ~3) - (rg.lo & ~3)) * 4);
    const size_t smem = STAGES * (tile_b + e_bytes + o_bytes) + 2 * STAGES * 8;
    if ((long)smem > SMEM_MAX) return SK_ERR_UNSUPPORTED;
    auto kern = sjlt_rows_kernel<T, TILE, NB, STAGES>;
    JLS_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<grid, (J.njobs + NPROD) * 32, smem, s>>>(static_cast<const T*>(A->A), A->ld, A->rows, A->cols, C.ents,
                                                    C.offs, C.e_stride, C.o_stride, rg.lo, rg.hi, J.nbw, J.njobs,
                                                    e_bytes, S, ldS, scale, h->d_err);
    note_launch();
    JLS_CHECK_CUDA(cudaGetLastError());
  }
  return SK_OK;
}

template <int STAGES>
int launch_cols_gen(sk_op* h, const KGen& g, int64_t n, int64_t m, const TiledCcs& C, int c_lo, int c_hi,
                    float scale, float* S, int64_t ldS, cudaStream_t s) {
  constexpr int TILE = SJLT_TILE_F32, BW = 128;
  JLS_CHECK(zero_columns(S, ldS, m, c_lo, c_hi, s));
  const size_t tile_b = (size_t)TILE * BW * sizeof(float);
  const size_t o_max = (GEN_JOBS * GEN_NB + 8) * 4;
  const size_t e_blk = (size_t)h->alpha * TILE * ENTRY_BYTES;
  const long fit = blocks_that_fit<STAGES>(tile_b, o_max, e_blk);
  if (fit < 1) return SK_ERR_UNSUPPORTED;
  const int64_t nblk = (m + BW - 1) / BW;  // blocks of output rows; see launch_cols
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(num_sms(), nblk));
  CUtensorMap unused{};
  for (const Range& rg : plan_ranges(h, c_lo, c_hi, (int)fit, GEN_JOBS * GEN_NB)) {
    const Jobs J = plan_jobs(rg.hi - rg.lo, GEN_JOBS);
    const uint32_t e_bytes = (uint32_t)(e_blk * rg.nblk);
    const uint32_t o_bytes = (uint32_t)((((rg.hi + 1 + 3) & ~3) - (rg.lo & ~3)) * 4);
    const size_t smem = STAGES * (tile_b + e_bytes + o_bytes) + 2 * STAGES * 8;
    if ((long)smem > SMEM_MAX) return SK_ERR_UNSUPPORTED;
    auto kern = sjlt_cols_kernel<float, TILE, GEN_NB, STAGES, true>;
    JLS_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<grid, (J.njobs + GEN_WARPS) * 32, smem, s>>>(unused, n, m, C.ents, C.offs, C.e_stride, C.o_stride,
                                                        rg.lo, rg.hi, J.nbw, J.njobs, e_bytes, S, ldS, scale,
                                                        h->d_err, g);
    note_launch();
    JLS_CHECK_CUDA(cudaGetLastError());
  }
  return SK_OK;
}

// Three stages when one block's entries fit beside them, else two.
template <typename T, int TILE>
int launch_cols_any(sk_op* h, const sk_matrix* A, const TiledCcs& C, int c_lo, int c_hi, T scale, T* St,
                    int64_t ldSt, cudaStream_t s) {
  const size_t tile_b = (size_t)TILE * 512, o_max = (COLS_JOBS * NB_COLS + 8) * 4;
  const size_t e_blk = (size_t)h->alpha * TILE * ENTRY_BYTES;
  if (blocks_that_fit<3>(tile_b, o_max, e_blk) >= 1)
    return launch_cols<T, TILE, 3>(h, A, C, c_lo, c_hi, scale, St, ldSt, s);
  return launch_cols<T, TILE, 2>(h, A, C, c_lo, c_hi, scale, St, ldSt, s);
}
template <typename T, int TILE>
int launch_rows_any(sk_op* h, const sk_matrix* A, const TiledCcs& C, int c_lo, int c_hi, T scale, T* S,
                    int64_t ldS, cudaStream_t s) {
  const size_t tile_b = ((ROWS_BLK * (TILE + 1) * sizeof(T)) + 127) / 128 * 128;
  const size_t o_max = (ROWS_JOBS * nb_rows<T>() + 8) * 4;
  const size_t e_blk = (size_t)h->alpha * TILE * ENTRY_BYTES;
  if (blocks_that_fit<3>(tile_b, o_max, e_blk) >= 1)
    return launch_rows<T, TILE, 3>(h, A, C, c_lo, c_hi, scale, S, ldS, s);
  return launch_rows<T, TILE, 2>(h, A, C, c_lo, c_hi, scale, S, ldS, s);
}

}  // namespace

int sjlt_kernel_apply(sk_op* h, const float* P, int64_t n, const float* Q, int64_t m, double hbw, double shift,
                      double scale, float* S, int64_t ldS, cudaStream_t s) {
  JLS_CHECK(build_ccs(h, 0, s));
  const TiledCcs& C = h->ccs[0];
  KGen g;
  g.P = P;
  g.Q = Q;
  g.c2 = (float)(1.4426950408889634 / (2.0 * hbw * hbw));  // log2(e) / (2 h^2)
  g.shift = (float)shift;
  const size_t tile_b = (size_t)SJLT_TILE_F32 * 512, o_max = (GEN_JOBS * GEN_NB + 8) * 4;
  const size_t e_blk = (size_t)h->alpha * SJLT_TILE_F32 * ENTRY_BYTES;
  if (blocks_that_fit<3>(tile_b, o_max, e_blk) >= 1)
    return launch_cols_gen<3>(h, g, n, m, C, 0, h->d_total, (float)scale, S, ldS, s);
  return launch_cols_gen<2>(h, g, n, m, C, 0, h->d_total, (float)scale, S, ldS, s);
}

// Complex A (interleaved FP32 parts; rows x cols complex, ld in complex
// elements; S, S' complex with ldS, ldSt in complex elements), real R:
//  * S' = A* R: the cols kernel over the real view (2 cols real columns), whose
//    lanes hold the real and imaginary parts of two complex columns, with the
//    conjugating flush;
//  * S = A R: the rows kernel over the real view with the operator R (x) I_2
//    (row 2j + t of it has R's nonzeros of row j at columns 2c + t), whose
//    output columns are the (re, im) pairs of S.
int sjlt_apply_complex(sk_op* h, const sk_matrix* A, int which, int c_lo, int c_hi, double scale, void* S,
                       int64_t ldS, void* St, int64_t ldSt, cudaStream_t s) {
  sk_matrix V = *A;  // the real view
  V.dtype = SK_F32;
  V.cols = 2 * A->cols;
  V.ld = 2 * A->ld;
  if (which & SK_ST) {
    JLS_CHECK(build_ccs(h, 0, s));
    const TiledCcs& C = h->ccs[0];
    const size_t tile_b = (size_t)SJLT_TILE_F32 * 512, o_max = (COLS_JOBS * NB_COLS + 8) * 4;
    const size_t e_blk = (size_t)h->alpha * SJLT_TILE_F32 * ENTRY_BYTES;
    if (blocks_that_fit<3>(tile_b, o_max, e_blk) >= 1)
      JLS_CHECK((launch_cols<float, SJLT_TILE_F32, 3, true>(h, &V, C, c_lo, c_hi, (float)scale, (float*)St,
                                                             2 * ldSt, s)));
    else
      JLS_CHECK((launch_cols<float, SJLT_TILE_F32, 2, true>(h, &V, C, c_lo, c_hi, (float)scale, (float*)St,
                                                             2 * ldSt, s)));
  }
  if (which & SK_S) {
    JLS_CHECK(build_ccs_complex(h, s));
    // R (x) I_2 as an operator: twice the rows, columns and block widths of R
    sk_op R2;
    R2.kind = h->kind;
    R2.n = 2 * h->n;
    R2.alpha = h->alpha;
    R2.d_total = 2 * h->d_total;
    for (int w : h->blocks) R2.blocks.push_back(2 * w);
    R2.d_err = h->d_err;
    JLS_CHECK((launch_rows_any<float, SJLT_TILE_F32>(&R2, &V, h->ccs[2], 2 * c_lo, 2 * c_hi, (float)scale,
                                                    (float*)S, 2 * ldS, s)));
  }
  return SK_OK;
}

int sjlt_apply(sk_op* h, const sk_matrix* A, int which, int c_lo, int c_hi, double scale, void* S, int64_t ldS,
               void* St, int64_t ldSt, cudaStream_t s) {
  const int tsel = A->dtype == SK_F32 ? 0 : 1;
  JLS_CHECK(build_ccs(h, tsel, s));
  const TiledCcs& C = h->ccs[tsel];
  if (which & SK_S) {
    if (A->dtype == SK_F32)
      JLS_CHECK((launch_rows_any<float, SJLT_TILE_F32>(h, A, C, c_lo, c_hi, (float)scale, (float*)S, ldS, s)));
    else
      JLS_CHECK((launch_rows_any<double, SJLT_TILE_F64>(h, A, C, c_lo, c_hi, scale, (double*)S, ldS, s)));
  }
  if (which & SK_ST) {
    if (A->dtype == SK_F32)
      JLS_CHECK((launch_cols_any<float, SJLT_TILE_F32>(h, A, C, c_lo, c_hi, (float)scale, (float*)St, ldSt, s)));
    else
      JLS_CHECK((launch_cols_any<double, SJLT_TILE_F64>(h, A, C, c_lo, c_hi, scale, (double*)St, ldSt, s)));
  }
  return SK_OK;
}

}  // namespace jls
