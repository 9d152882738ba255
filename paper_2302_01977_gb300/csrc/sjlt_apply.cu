// sjlt_apply.cu -- S = A R and S' = A^T R for an SJLT R (Sec. 6.3), sm_103a.
//
// R is held as a tiled compressed-column structure (Sec. 6.1's CCS of B+ and
// B-, merged with a sign bit and cut into tiles of TILE rows of R): for each
// tile, the entries (row-in-tile, sign) sorted by column.  No multiplications:
// every entry adds or subtracts one element of A, and the scale 1/sqrt(alpha *
// blocks) is applied once at the end, as in the paper's binary-matrix design.
//
// GB300 mapping.  Both kernels stream A exactly once from HBM and stage each
// tile in shared memory; a warp owns a range of <= NB output columns of R and
// keeps their sums in registers for the whole stream.  Because the entries of
// a tile are grouped by column, the warp walks them column by column with
// compile-time accumulator indices (no dynamic register indexing), and the
// tile element an entry names is at the same place for every lane:
//
//  * S' (cols kernel): lanes own 32 consecutive columns of A.  Tiles of TILE
//    rows x 32 columns arrive by TMA (cp.async.bulk.tensor) into a dense
//    layout; an entry (row r) makes every lane read tile[r][lane]
//    (conflict-free).  A producer warp runs a STAGES-deep mbarrier ring.
//  * S  (rows kernel): lanes own 32 consecutive rows of A.  Tiles of 32 rows x
//    TILE columns (= TILE rows of R) are copied with 4/8-byte cp.async into a
//    row pitch of TILE+1 elements, so that lanes reading tile[lane][j] hit 32
//    different banks.
//
// Results are staged in shared memory and written with coalesced stores.
#include <cuda.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace jls {

template <typename T>
__device__ __forceinline__ T flip(T v, uint32_t neg);
template <>
__device__ __forceinline__ float flip<float>(float v, uint32_t neg) {
  return __int_as_float(__float_as_int(v) ^ (int)(neg << 16));  // neg = 0 or 0x8000
}
template <>
__device__ __forceinline__ double flip<double>(double v, uint32_t neg) {
  const long long b = __double_as_longlong(v) ^ ((long long)neg << 48);
  return __longlong_as_double(b);
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void cp_async_16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}

// Walk the entries of columns [cw0, cw0 + nb) of one tile and accumulate.
// LD is the element distance between consecutive entries' rows (cols kernel:
// 32, lanes add `lane`), or 1 for the rows kernel (lane rows at lane*pitch).
template <typename T, int NB, int ROWSTRIDE>
__device__ __forceinline__ void accumulate_tile(T (&acc)[NB], const uint16_t* __restrict__ E,
                                                const uint32_t* __restrict__ O, const T* __restrict__ X,
                                                int cw0, int nb) {
  uint32_t p = O[cw0];
#pragma unroll
  for (int b = 0; b < NB; ++b) {
    if (b < nb) {
      const uint32_t e = O[cw0 + b + 1];
      T a0 = acc[b], a1 = T(0);
      for (; p + 1 < e; p += 2) {
        const uint32_t en0 = E[p], en1 = E[p + 1];
        const T v0 = X[(en0 & 0x7fff) * ROWSTRIDE];
        const T v1 = X[(en1 & 0x7fff) * ROWSTRIDE];
        a0 += flip(v0, en0 & 0x8000);
        a1 += flip(v1, en1 & 0x8000);
      }
      if (p < e) {
        const uint32_t en0 = E[p];
        a0 += flip(X[(en0 & 0x7fff) * ROWSTRIDE], en0 & 0x8000);
        ++p;
      }
      acc[b] = a0 + a1;
    }
  }
}

// ---------------------------------------------------------------------------
// S' = A^T R : lanes over columns of A, TMA-fed.
template <typename T, int TILE, int NB, int STAGES>
__global__ void __launch_bounds__(17 * 32, 1)
    sjlt_cols_kernel(const __grid_constant__ CUtensorMap tmA, int64_t rowsA, int64_t colsA,
                     const uint16_t* __restrict__ ents, const uint32_t* __restrict__ offs, int64_t e_stride,
                     int64_t o_stride, int c_lo, int c_hi, int nbw, int njobs, uint32_t E_BYTES, T* __restrict__ St,
                     int64_t ldSt, T scale, int* err) {
  extern __shared__ __align__(1024) uint8_t smem[];
  constexpr int BOXR = TILE < 256 ? TILE : 256;
  constexpr uint32_t TILE_BYTES = TILE * 32 * sizeof(T);
  // only the offsets [o_lo, o_lo + o_cnt) and the entries of columns
  // [c_lo, c_hi) of each tile are staged (16-byte aligned supersets)
  const int o_lo = c_lo & ~3;
  const int o_cnt = ((c_hi + 1 + 3) & ~3) - o_lo;
  const uint32_t O_BYTES = (uint32_t)o_cnt * 4;
  T* tiles = reinterpret_cast<T*>(smem);
  uint16_t* sh_e = reinterpret_cast<uint16_t*>(smem + STAGES * TILE_BYTES);
  uint32_t* sh_o = reinterpret_cast<uint32_t*>(smem + STAGES * (TILE_BYTES + E_BYTES));
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + STAGES * (TILE_BYTES + E_BYTES + O_BYTES));
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t j0 = (int64_t)blockIdx.x * 32;
  const int ntiles = (int)((rowsA + TILE - 1) / TILE);

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, njobs);
    }
    fence_mbar_init();
  }
  __syncthreads();

  T acc[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) acc[b] = T(0);
  const int cw0 = c_lo + warp * nbw;
  const int nb = min(nbw, c_hi - cw0);

  if (warp == njobs) {  // ---- producer
    if (lane == 0) {
      tma_prefetch_desc(&tmA);
      bool ok = true;
      int issued = 0;
      for (int t = 0; t < ntiles && ok; ++t) {
        const int s = t % STAGES;
        if (t >= STAGES) ok = mbar_wait(empty0 + 8 * s, ((t / STAGES) - 1) & 1, err);
        if (!ok) break;
        const uint32_t fb = full0 + 8 * s;
        const uint32_t* ot = offs + (int64_t)t * o_stride;
        const uint32_t e_al = __ldg(ot + c_lo) & ~7u;
        const uint32_t eb = ((__ldg(ot + c_hi) - e_al) * 2 + 15) & ~15u;
        if (eb > E_BYTES) {  // host sizing guarantees this never happens
          set_err(err, ERRF_BOUNDS);
          ok = false;
          break;
        }
        mbar_arrive_expect_tx(fb, TILE_BYTES + eb + O_BYTES);
        const uint32_t dst = smem_u32(tiles) + s * TILE_BYTES;
#pragma unroll
        for (int q = 0; q < TILE / BOXR; ++q)
          tma_load_2d(dst + q * BOXR * 32 * sizeof(T), &tmA, fb, (int32_t)j0, (int32_t)(t * TILE + q * BOXR));
        if (eb) bulk_g2s(smem_u32(sh_e) + s * E_BYTES, ents + (int64_t)t * e_stride + e_al, eb, fb);
        bulk_g2s(smem_u32(sh_o) + s * O_BYTES, ot + o_lo, O_BYTES, fb);
        issued = t + 1;
      }
      // drain: never leave the CTA with copies in flight
      for (int t = max(0, issued - STAGES); t < issued; ++t)
        mbar_wait(full0 + 8 * (t % STAGES), (t / STAGES) & 1, err);
    }
  } else {  // ---- consumers
    for (int t = 0; t < ntiles; ++t) {
      const int s = t % STAGES;
      if (!mbar_wait(full0 + 8 * s, (t / STAGES) & 1, err)) break;
      const uint32_t* O = sh_o + s * (O_BYTES / 4) - o_lo;  // indexed by absolute column
      const uint32_t e_al = O[c_lo] & ~7u;
      if (nb > 0)
        accumulate_tile<T, NB, 32>(acc, sh_e + s * (E_BYTES / 2) - e_al, O, tiles + (size_t)s * TILE * 32 + lane,
                                   cw0, nb);
      __syncwarp();
      if (lane == 0) mbar_arrive(empty0 + 8 * s);
    }
  }
  __syncthreads();
  // stage results: out[lane][col], pitch ncols + 1, then coalesced stores
  const int ncols = c_hi - c_lo, pitch = ncols + 1;
  T* out = tiles;
  if (warp < njobs) {
#pragma unroll
    for (int b = 0; b < NB; ++b)
      if (b < nb) out[lane * pitch + warp * nbw + b] = acc[b] * scale;
  }
  __syncthreads();
  for (int q = threadIdx.x; q < 32 * ncols; q += blockDim.x) {
    const int r = q / ncols, c = q % ncols;
    if (j0 + r < colsA) St[(j0 + r) * ldSt + c_lo + c] = out[r * pitch + c];
  }
}

// ---------------------------------------------------------------------------
// S = A R : lanes over rows of A, cp.async-fed, padded pitch TILE + 1.
template <typename T, int TILE, int NB, int STAGES>
__global__ void __launch_bounds__(16 * 32, 1)
    sjlt_rows_kernel(const T* __restrict__ A, int64_t lda, int64_t rowsA, int64_t colsA,
                     const uint16_t* __restrict__ ents, const uint32_t* __restrict__ offs, int64_t e_stride,
                     int64_t o_stride, int c_lo, int c_hi, int nbw, uint32_t E_BYTES, T* __restrict__ S,
                     int64_t ldS, T scale, int* err) {
  extern __shared__ __align__(1024) uint8_t smem[];
  constexpr int P = TILE + 1;
  constexpr uint32_t TILE_BYTES = ((32 * P * sizeof(T)) + 127) / 128 * 128;
  const int o_lo = c_lo & ~3;
  const int o_cnt = ((c_hi + 1 + 3) & ~3) - o_lo;
  const uint32_t O_BYTES = (uint32_t)o_cnt * 4;
  uint8_t* base_t = smem;
  uint8_t* base_e = smem + STAGES * TILE_BYTES;
  uint8_t* base_o = base_e + STAGES * E_BYTES;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nthreads = blockDim.x;
  const int64_t i0 = (int64_t)blockIdx.x * 32;
  const int ntiles = (int)((colsA + TILE - 1) / TILE);

  auto load_tile = [&](int t, int s) {
    if (t < ntiles) {
      const uint32_t dst = smem_u32(base_t + s * TILE_BYTES);
      const int64_t jb = (int64_t)t * TILE;
      for (int q = threadIdx.x; q < 32 * TILE; q += nthreads) {
        const int r = q / TILE, c = q % TILE;
        const bool in = (i0 + r < rowsA) && (jb + c < colsA);
        const T* src = in ? A + (i0 + r) * lda + jb + c : A;
        if (sizeof(T) == 4)
          cp_async_4(dst + (r * P + c) * 4, src, in ? 4 : 0);
        else
          cp_async_8(dst + (r * P + c) * 8, src, in ? 8 : 0);
      }
      const uint32_t* ot = offs + (int64_t)t * o_stride;
      const uint32_t e_al = __ldg(ot + c_lo) & ~7u;
      uint32_t eb = ((__ldg(ot + c_hi) - e_al) * 2 + 15) & ~15u;
      if (eb > E_BYTES) {  // host sizing guarantees this never happens
        set_err(err, ERRF_BOUNDS);
        eb = 0;
      }
      const uint32_t de = smem_u32(base_e + s * E_BYTES);
      const uint8_t* se = reinterpret_cast<const uint8_t*>(ents + (int64_t)t * e_stride + e_al);
      for (uint32_t q = threadIdx.x; q < eb / 16; q += nthreads) cp_async_16(de + q * 16, se + q * 16);
      const uint32_t dof = smem_u32(base_o + s * O_BYTES);
      const uint8_t* so = reinterpret_cast<const uint8_t*>(ot + o_lo);
      for (uint32_t q = threadIdx.x; q < O_BYTES / 16; q += nthreads) cp_async_16(dof + q * 16, so + q * 16);
    }
    cp_async_commit();
  };

#pragma unroll
  for (int s = 0; s < STAGES - 1; ++s) load_tile(s, s);

  T acc[NB];
#pragma unroll
  for (int b = 0; b < NB; ++b) acc[b] = T(0);
  const int cw0 = c_lo + warp * nbw;
  const int nb = min(nbw, c_hi - cw0);

  for (int t = 0; t < ntiles; ++t) {
    cp_async_wait<STAGES - 2>();
    __syncthreads();
    load_tile(t + STAGES - 1, (t + STAGES - 1) % STAGES);
    const int s = t % STAGES;
    const uint32_t* O = reinterpret_cast<const uint32_t*>(base_o + s * O_BYTES) - o_lo;
    const uint32_t e_al = O[c_lo] & ~7u;
    if (nb > 0)
      accumulate_tile<T, NB, 1>(acc, reinterpret_cast<const uint16_t*>(base_e + s * E_BYTES) - e_al, O,
                                reinterpret_cast<const T*>(base_t + s * TILE_BYTES) + lane * P, cw0, nb);
  }
  cp_async_wait<0>();
  __syncthreads();
  const int ncols = c_hi - c_lo, pitch = ncols + 1;
  T* out = reinterpret_cast<T*>(smem);
#pragma unroll
  for (int b = 0; b < NB; ++b)
    if (b < nb) out[lane * pitch + warp * nbw + b] = acc[b] * scale;
  __syncthreads();
  for (int q = threadIdx.x; q < 32 * ncols; q += nthreads) {
    const int r = q / ncols, c = q % ncols;
    if (i0 + r < rowsA) S[(i0 + r) * ldS + c_lo + c] = out[r * pitch + c];
  }
  (void)err;
}

// ---------------------------------------------------------------------------
// host side
typedef CUresult (*PFN_encodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                    const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                    CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

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

namespace {

constexpr int NB_SJLT = 32;
constexpr int MAX_JOBS = 16;

struct Jobs {
  int njobs, nbw;
};
Jobs plan_jobs(int ncols) {
  int nj = (ncols + NB_SJLT - 1) / NB_SJLT;
  nj = std::max(nj, std::min(4, ncols));
  nj = std::min(nj, MAX_JOBS);
  int nbw = (ncols + nj - 1) / nj;
  nj = (ncols + nbw - 1) / nbw;
  return {nj, nbw};
}

// Column ranges one launch can take: <= MAX_JOBS * NB columns, and few enough
// blocks that STAGES tiles plus their entries fit in shared memory.  Each
// launch streams A once; ranges are cut at block boundaries.
struct Range {
  int lo, hi, nblk;
};
std::vector<Range> plan_ranges(const sk_op* h, int c_lo, int c_hi, int max_blk) {
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
      const int take_hi = std::min(std::min(b_hi, c_hi), c + MAX_JOBS * NB_SJLT);
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

template <typename T, int TILE>
int launch_cols(sk_op* h, const sk_matrix* A, const TiledCcs& C, int c_lo, int c_hi, T scale, T* St,
                int64_t ldSt, cudaStream_t s) {
  constexpr int STAGES = 3;
  PFN_encodeTiled enc = get_encode_tiled();
  if (!enc) return SK_ERR_DEVICE;
  CUtensorMap tm;
  const cuuint64_t gdim[2] = {(cuuint64_t)A->cols, (cuuint64_t)A->rows};
  const cuuint64_t gstride[1] = {(cuuint64_t)(A->ld * sizeof(T))};
  constexpr int BOXR = TILE < 256 ? TILE : 256;
  const cuuint32_t box[2] = {32, (cuuint32_t)BOXR};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(&tm, sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2,
                   const_cast<void*>(A->A), gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return SK_ERR_ALIGN;
  const size_t tile_b = (size_t)TILE * 32 * sizeof(T);
  const size_t o_max = (MAX_JOBS * NB_SJLT + 8) * 4;
  const size_t e_blk = (size_t)h->alpha * TILE * 2;
  const size_t budget = 227 * 1024 - 2 * STAGES * 8;
  const long fit = ((long)budget / STAGES - (long)tile_b - (long)o_max - 16) / (long)e_blk;
  if (fit < 1) return SK_ERR_UNSUPPORTED;
  for (const Range& rg : plan_ranges(h, c_lo, c_hi, (int)fit)) {
    const Jobs J = plan_jobs(rg.hi - rg.lo);
    const uint32_t e_bytes = (uint32_t)((e_blk * rg.nblk + 16 + 15) & ~(size_t)15);
    const uint32_t o_bytes = (uint32_t)((((rg.hi + 1 + 3) & ~3) - (rg.lo & ~3)) * 4);
    const size_t smem = STAGES * (tile_b + e_bytes + o_bytes) + 2 * STAGES * 8;
    const size_t out_b = (size_t)32 * (rg.hi - rg.lo + 1) * sizeof(T);
    if (smem > 227 * 1024 || out_b > STAGES * tile_b) return SK_ERR_UNSUPPORTED;
    auto kern = sjlt_cols_kernel<T, TILE, NB_SJLT, STAGES>;
    JLS_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const unsigned grid = (unsigned)((A->cols + 31) / 32);
    kern<<<grid, (J.njobs + 1) * 32, smem, s>>>(tm, A->rows, A->cols, C.ents, C.offs, C.e_stride, C.o_stride,
                                                rg.lo, rg.hi, J.nbw, J.njobs, e_bytes, St, ldSt, scale, h->d_err); note_launch();
    JLS_CHECK_CUDA(cudaGetLastError());
  }
  return SK_OK;
}

template <typename T, int TILE>
int launch_rows(sk_op* h, const sk_matrix* A, const TiledCcs& C, int c_lo, int c_hi, T scale, T* S, int64_t ldS,
                cudaStream_t s) {
  constexpr int STAGES = 3;
  const size_t tile_b = ((32 * (TILE + 1) * sizeof(T)) + 127) / 128 * 128;
  const size_t o_max = (MAX_JOBS * NB_SJLT + 8) * 4;
  const size_t e_blk = (size_t)h->alpha * TILE * 2;
  const long fit = ((long)(227 * 1024) / STAGES - (long)tile_b - (long)o_max - 16) / (long)e_blk;
  if (fit < 1) return SK_ERR_UNSUPPORTED;
  for (const Range& rg : plan_ranges(h, c_lo, c_hi, (int)fit)) {
    const Jobs J = plan_jobs(rg.hi - rg.lo);
    const uint32_t e_bytes = (uint32_t)((e_blk * rg.nblk + 16 + 15) & ~(size_t)15);
    const uint32_t o_bytes = (uint32_t)((((rg.hi + 1 + 3) & ~3) - (rg.lo & ~3)) * 4);
    const size_t smem = STAGES * (tile_b + e_bytes + o_bytes);
    const size_t out_b = (size_t)32 * (rg.hi - rg.lo + 1) * sizeof(T);
    if (smem > 227 * 1024 || out_b > smem) return SK_ERR_UNSUPPORTED;
    auto kern = sjlt_rows_kernel<T, TILE, NB_SJLT, STAGES>;
    JLS_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const unsigned grid = (unsigned)((A->rows + 31) / 32);
    kern<<<grid, J.njobs * 32, smem, s>>>(static_cast<const T*>(A->A), A->ld, A->rows, A->cols, C.ents, C.offs,
                                          C.e_stride, C.o_stride, rg.lo, rg.hi, J.nbw, e_bytes, S, ldS, scale,
                                          h->d_err); note_launch();
    JLS_CHECK_CUDA(cudaGetLastError());
  }
  return SK_OK;
}

}  // namespace

int sjlt_apply(sk_op* h, const sk_matrix* A, int which, int c_lo, int c_hi, double scale, void* S, int64_t ldS,
               void* St, int64_t ldSt, cudaStream_t s) {
  const int tsel = A->dtype == SK_F32 ? 0 : 1;
  JLS_CHECK(build_ccs(h, tsel, s));
  const TiledCcs& C = h->ccs[tsel];
  if (which & SK_S) {
    if (A->dtype == SK_F32)
      JLS_CHECK((launch_rows<float, SJLT_TILE_F32>(h, A, C, c_lo, c_hi, (float)scale, (float*)S, ldS, s)));
    else
      JLS_CHECK((launch_rows<double, SJLT_TILE_F64>(h, A, C, c_lo, c_hi, scale, (double*)S, ldS, s)));
  }
  if (which & SK_ST) {
    if (A->dtype == SK_F32)
      JLS_CHECK((launch_cols<float, SJLT_TILE_F32>(h, A, C, c_lo, c_hi, (float)scale, (float*)St, ldSt, s)));
    else
      JLS_CHECK((launch_cols<double, SJLT_TILE_F64>(h, A, C, c_lo, c_hi, scale, (double*)St, ldSt, s)));
  }
  return SK_OK;
}

}  // namespace jls
