// batch_adaptive.cu -- the stopping test of Eq. (3.1) for every instance of a
// batch, on the device, and the update of the batch's item table it decides.
//
// Algorithm 1 per instance i: after the batched launch has sketched the columns
// [c_hi - dd, c_hi) of S'_i, the test takes S~ = those dd columns,
// S^ = (I - Q Q^T)^2 S~ (two block Gram-Schmidt passes, the remark after
// Eq. (3.1)) and stops when ||S^||_F < eps_abs or ||S^||_F < eps_rel ||S~||_F.
// The two passes are those of S~'s own absorption.  At eps_rel below
// kPreciseBelow (the precise steps) S~ is projected twice, the first
// difference W - Q G in double-FP32, and ||S^||_F^2 is the trace of the Gram
// matrix its first Cholesky-QR pass factors; otherwise S~ is projected,
// factored (W = W1 L1^T), projected again, and ||S^||_F^2 = tr(L1 G2 L1^T)
// with G2 the Gram matrix of (I - Q Q^T) W1.  Either way a test costs the
// absorption's projections only.
// Q is an orthonormal basis of the earlier columns, kept per instance in HBM:
// the first d0 columns are absorbed before the first test (32 at a time), and
// after a failed test the projected S^ is absorbed, so the next test starts
// from the basis of every earlier column.  A Cholesky pivot below the drop
// level (absorb_begin) drops its column (a zero column of Q, which leaves
// Q Q^T unchanged).  The decision moves the instance's column range on
// by dd, or retires it (converged, or no room left in R_i); a one-CTA kernel
// then renumbers the units of the active instances for the next batched launch.
// Nothing returns to the host between rounds, so a whole adaptive run, all
// rounds, is one CUDA graph.
//
// One thread-block cluster of ncl CTAs per instance (1 for batches of many
// instances; 4 when there are fewer instances than SMs): CTA rank k owns the
// k-th share of S'_i's rows.  The tall-skinny products Q^T W, W^T W are reduced across
// the cluster through distributed shared memory; W - Q G, the triangular
// solves and the norms are row-local.  Every CTA factors the same reduced Gram
// matrix, so all of them take the same decisions without exchanging them.
//
// Scale: the loop sketches with the per-block scale 1/sqrt(alpha); R_i with
// B blocks carries 1/sqrt(alpha B), so the norms are reported (and compared
// with eps_abs) times 1/sqrt(B), and the finished columns are rescaled once.
// An SRHT loop sketches every column with 1/sqrt(d0 + dd) and R_i[:, :d]
// carries 1/sqrt(d): the factor is sqrt((d0 + dd) / d).
#include <cooperative_groups.h>

#include "batch.cuh"
#include "common.cuh"
#include "internal.h"

namespace cg = cooperative_groups;

namespace jls {
namespace {

constexpr int CLMAX = 4;  // CTAs per instance chosen at setup, at most (a cluster; rounds with few active
                          // instances left use clusters of 8)
constexpr int AT = 512;   // threads per CTA
constexpr int QMAX = ADAPT_QSMEM;  // Q^T W in shared memory per chunk of the basis
constexpr int BW = ADAPT_BW;
constexpr int QCH = 57344;  // bytes of Q per staged chunk of Q^T W
constexpr int RCMAX = 64;   // rows per staged chunk of Q^T W, at most
constexpr int PR = 256;     // rows per pass of W - Q G
constexpr int KC = 32;      // columns of Q per staged step of W - Q G (8 for each of 4 thread groups)
constexpr int GR = 256;     // rows per staged chunk of W^T W
constexpr int QT_FLOATS = KC * (PR + 4);  // one Q^T staging buffer of W - Q G
constexpr int LD = BW + 1;  // Gram matrix and Cholesky working arrays
constexpr int LF = BW + 4;  // the factor as the solves read it (16-byte rows)
constexpr int NW = AT / 32;

// shared memory, bytes
constexpr int SM_QS = 2 * QCH;                // Q chunks, double-buffered
constexpr int SM_WS = 2 * RCMAX * BW * 4;     // W chunks
constexpr int SM_STAGE = SM_QS + SM_WS;       // also: partial products, Q^T staging, Gram partial
constexpr int SM_G = QMAX * BW * 4;           // G = Q^T W, FP32
constexpr int SM_GRAM = BW * LD * 8;          // reduced Gram matrix, FP64
constexpr int SM_L = BW * LF * 4;             // Cholesky factor, FP32
constexpr int SM_MISC = 32 * 4 + (NW + 8) * 8 + 4 * BW * 8;  // reciprocal pivots, reduction slots, Cholesky
                                                              // scratch, the block's column sums of squares (own
                                                              // part, then the cluster's)
constexpr int SM_TOTAL = SM_STAGE + SM_G + SM_GRAM + SM_L + SM_MISC;
static_assert(2 * QMAX * BW * 4 <= SM_STAGE, "the row groups' parts of G fit the staging area");
static_assert(4 * PR * BW * 4 <= SM_STAGE && 2 * QT_FLOATS * 4 <= SM_STAGE, "W - Q G staging fits");
static_assert(5 * BW * BW * 8 + 2 * GR * BW * 4 <= SM_STAGE, "Gram partials and W chunks fit");
static_assert(GR * BW / 4 % AT == 0 && AT == 512, "thread mappings assume 512 threads");
static_assert(SM_TOTAL <= 227 * 1024, "one CTA per SM");

__device__ __forceinline__ void cl_sync() { cg::this_cluster().sync(); }

// The instance's global Q^T W (ATest::G) for bases wider than QMAX, kept in
// shared memory rather than in a register for the whole kernel.
__shared__ float* s_gg;
template <typename T>
__device__ __forceinline__ T* cl_map(T* p, int rank) {
  return cg::this_cluster().map_shared_rank(p, (unsigned)rank);
}

struct Ctx {
  int ncl, rank;  // CTAs of the instance (cluster size) and this CTA's rank
  int64_t r0, r1;  // this CTA's rows of S'_i
  const float* Q;
  float* Qw;
  int64_t ldq;
  float* W;  // ld BW
  uint8_t* stage;
  float* Gs;
  double* gram;
  float* Lf;
  float* rinv;
  double* red;  // [0, NW): warp sums; [NW]: the CTA's sum, read by the cluster
  double* cs;   // Cholesky scratch (2 BW entries), then the column sums of squares (colsq: 2 BW entries)
};

__device__ __forceinline__ void cp_async_16z(uint32_t dst, const void* src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0)
               : "memory");
}

__device__ __forceinline__ void fma8x8(float (&acc)[8][8], const float4& a0, const float4& a1, const float4& b0,
                                       const float4& b1) {
  const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
  const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
}

// sum over the CTA, the same value in every thread (fixed order)
__device__ double cta_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int w = 0; w < NW; ++w) s += red[w];
  __syncthreads();
  return s;
}

// W[r][j] <- S[r][c0 + j] for j < b (zero for b <= j < BW) on this CTA's rows;
// returns the thread's share of the sum of squares.  A warp takes a row (32
// consecutive floats of S); four rows per thread are in flight at a time.
__device__ double load_block(const Ctx& c, const float* S, int64_t ldS, int c0, int b) {
  constexpr int RS = AT / 32;  // rows per sweep of the CTA
  const int j = threadIdx.x & 31;
  const bool jin = j < b;
  float ss = 0.f;
  int64_t r = c.r0 + (threadIdx.x >> 5);
  for (; r + 3 * RS < c.r1; r += 4 * RS) {
    float v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = jin ? S[(r + u * RS) * ldS + c0 + j] : 0.f;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      c.W[(r + u * RS) * BW + j] = v[u];
      ss = fmaf(v[u], v[u], ss);
    }
  }
  for (; r < c.r1; r += RS) {
    const float v = jin ? S[r * ldS + c0 + j] : 0.f;
    c.W[r * BW + j] = v;
    ss = fmaf(v, v, ss);
  }
  return (double)ss;
}

// W <- S[:, c0 : c0 + b] as load_block, and each column's sum of squares over
// all rows of S'_i (the block before its projection) into colsq(c)[j], the
// same in every CTA of the cluster (warp partials added in warp order, the
// CTAs' in rank order); returns the block's sum of squares (their sum).
__device__ __forceinline__ double* colsq(const Ctx& c) { return c.cs + 2 * BW; }
__device__ double load_block_cols(Ctx& c, const float* S, int64_t ldS, int c0, int b) {
  const double ss = load_block(c, S, ldS, c0, b);
  double* part = reinterpret_cast<double*>(c.stage);  // [NW][32]: the stage area is free while a block loads
  part[threadIdx.x] = ss;  // warp w, lane j: column j
  __syncthreads();
  double* own = colsq(c) + BW;
  if (threadIdx.x < BW) {
    double v = 0.0;
    for (int w = 0; w < NW; ++w) v += part[w * 32 + threadIdx.x];
    own[threadIdx.x] = v;
  }
  cl_sync();
  if (threadIdx.x < BW) {
    double v = 0.0;
    for (int r = 0; r < c.ncl; ++r) v += cl_map(own, r)[threadIdx.x];
    colsq(c)[threadIdx.x] = v;
  }
  cl_sync();  // own is rewritten by the next load
  double t = 0.0;
#pragma unroll 8
  for (int j = 0; j < BW; ++j) t += colsq(c)[j];
  return t;
}

// Gs <- Q[:, :q]^T W over all rows of S'_i (q a multiple of 8, <= QMAX), in
// every CTA of the cluster.  Each CTA forms the product over its rows with
// 8 x 8 register tiles, q/2 tiles in all; the rows of each staged chunk are
// split over RG = AT / (q/2) groups of threads, whose partial products are
// added in shared memory (group order).  Then CTA k adds up the k-th quarter
// of the entries over the cluster's CTAs and writes the sums into every
// CTA's Gs.
__device__ void qt_w(Ctx& c, int q, const float* Qb) {
  const int U = (q >> 3) * 4;  // tiles: 8 rows of G x 8 of its 32 columns
  const int RG = max(1, AT / U);
  const int t = threadIdx.x;
  const bool act = t < RG * U;
  const int g = act ? t / U : 0, lt = act ? t - g * U : 0;
  const int kg = lt >> 2, cg4 = lt & 3;
  int rc = 16;  // rows per chunk: QCH bytes of Q
  while (rc < RCMAX && 2 * rc * q * 4 <= QCH) rc *= 2;
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  float* Qs = reinterpret_cast<float*>(c.stage);
  float* Ws = reinterpret_cast<float*>(c.stage + SM_QS);
  const int64_t nr = c.r1 - c.r0;
  const int nch = (int)((nr + rc - 1) / rc);
  const int q4 = q >> 2;
  auto issue = [&](int ch, int buf) {
    const int64_t rb = c.r0 + (int64_t)ch * rc;
    float* qd = Qs + buf * (QCH / 4);
    float* wd = Ws + buf * RCMAX * BW;
    const int nq = rc * q4;
    for (int e = t; e < nq + rc * (BW / 4); e += AT) {
      if (e < nq) {
        const int rr = e / q4, k4 = e - rr * q4;
        const int64_t r = rb + rr;
        const bool in = r < c.r1;
        cp_async_16z(smem_u32(qd + rr * q + k4 * 4), in ? Qb + r * c.ldq + k4 * 4 : Qb, in);
      } else {
        const int e2 = e - nq, rr = e2 >> 3, j4 = e2 & 7;
        const int64_t r = rb + rr;
        const bool in = r < c.r1;
        cp_async_16z(smem_u32(wd + rr * BW + j4 * 4), in ? c.W + r * BW + j4 * 4 : c.W, in);
      }
    }
    cp_async_commit();
  };
  if (nch > 0) issue(0, 0);
  for (int ch = 0; ch < nch; ++ch) {
    if (ch + 1 < nch) {
      issue(ch + 1, (ch + 1) & 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    if (act && g < rc) {
      const float* qb = Qs + (ch & 1) * (QCH / 4) + kg * 8;
      const float* wb = Ws + (ch & 1) * RCMAX * BW + cg4 * 8;
      // the next row's operands are loaded while this row's products issue
      float4 a0 = *reinterpret_cast<const float4*>(qb + g * q);
      float4 a1 = *reinterpret_cast<const float4*>(qb + g * q + 4);
      for (int rr = g; rr < rc; rr += RG) {
        const float4 c0 = a0, c1 = a1;
        const float4 d0 = *reinterpret_cast<const float4*>(wb + rr * BW);
        const float4 d1 = *reinterpret_cast<const float4*>(wb + rr * BW + 4);
        const int rn = rr + RG < rc ? rr + RG : rr;
        a0 = *reinterpret_cast<const float4*>(qb + rn * q);
        a1 = *reinterpret_cast<const float4*>(qb + rn * q + 4);
        fma8x8(acc, c0, c1, d0, d1);
      }
    }
    __syncthreads();
  }
  // the groups' parts of G over the staging area (every thread is past its last read of it)
  float* P = reinterpret_cast<float*>(c.stage);
  const int E4 = q * BW / 4;  // float4 entries of G
  if (act) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      float4* p = reinterpret_cast<float4*>(P + ((int64_t)g * q + kg * 8 + i) * BW + cg4 * 8);
      p[0] = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
      p[1] = make_float4(acc[i][4], acc[i][5], acc[i][6], acc[i][7]);
    }
  }
  __syncthreads();
  if (RG > 1) {  // this CTA's part: the groups' sum, into group 0's slot
    float4* P4 = reinterpret_cast<float4*>(P);
    for (int e = t; e < E4; e += AT) {
      float4 s = P4[e];
      for (int gg = 1; gg < RG; ++gg) {
        const float4 v = P4[gg * E4 + e];
        s.x += v.x;
        s.y += v.y;
        s.z += v.z;
        s.w += v.w;
      }
      P4[e] = s;
    }
  }
  cl_sync();
  const int per = E4 / c.ncl;
  const int e0 = c.rank * per;
  for (int e = t; e < per; e += AT) {
    float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int r = 0; r < c.ncl; ++r) {
      const float4 v = reinterpret_cast<const float4*>(cl_map(P, r))[e0 + e];
      s.x += v.x;
      s.y += v.y;
      s.z += v.z;
      s.w += v.w;
    }
    for (int r = 0; r < c.ncl; ++r) reinterpret_cast<float4*>(cl_map(c.Gs, r))[e0 + e] = s;
  }
  cl_sync();
}

// G = Q[:, :q]^T W for any q (a multiple of 8): in shared memory (c.Gs) for
// q <= QMAX, else chunk by chunk of QMAX columns into the instance's global G
// (written by the cluster's rank 0, read by all CTAs after the closing
// cluster barrier).
template <bool WIDE>
__device__ void qt_w_all(Ctx& c, int q) {
  if constexpr (!WIDE) {
    qt_w(c, q, c.Q);
    return;
  }
  if (q <= QMAX) {
    qt_w(c, q, c.Q);
    return;
  }
  for (int q0 = 0; q0 < q; q0 += QMAX) {
    const int qc = min(QMAX, q - q0);
    qt_w(c, qc, c.Q + q0);
    if (c.rank == 0)
      for (int e = threadIdx.x; e < qc * BW / 4; e += AT)
        reinterpret_cast<float4*>(s_gg + (int64_t)q0 * BW)[e] = reinterpret_cast<const float4*>(c.Gs)[e];
    cl_sync();  // the chunk is stored before Gs is overwritten, and G is complete after the last one
  }
}

// W <- W - Q[:, :q] Gs on this CTA's rows: passes of PR rows; Q staged
// transposed KC columns at a time (the next step's loads in flight); four
// groups of threads take 8 of each step's columns with 8 x 8 register tiles,
// and their partial products are added in shared memory at the end of a pass.
template <bool GG>
__device__ void w_minus_qg(const Ctx& c, int q) {
  const float* G = GG ? s_gg : c.Gs;
  float* Qt = reinterpret_cast<float*>(c.stage);  // [2][KC][PR + 4]
  float* Pw = reinterpret_cast<float*>(c.stage);  // [4][PR][BW], after a pass's last step
  const int kq = threadIdx.x >> 7, lt = threadIdx.x & 127;
  const int rg = lt >> 2, cg = lt & 3;  // rows rg*8 .. +7, columns cg*8 .. +7
  const int srow = threadIdx.x & (PR - 1), spart = threadIdx.x / PR;  // staging: row, which KC/2 columns
  for (int64_t p0 = c.r0; p0 < c.r1; p0 += PR) {
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
    const int64_t rt = p0 + srow;
    const bool rin = rt < c.r1;
    const bool busy = p0 + rg * 8 < c.r1;  // this thread's rows are not all past the end
    float4 pre[KC / 8];
    auto fetch = [&](int k0) {
#pragma unroll
      for (int u = 0; u < KC / 8; ++u) {
        const int k = k0 + spart * (KC / 2) + 4 * u;
        pre[u] = (rin && k < q) ? *reinterpret_cast<const float4*>(c.Q + rt * c.ldq + k)
                                : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    };
    auto stage_q = [&](int buf) {
#pragma unroll
      for (int u = 0; u < KC / 8; ++u) {
        float* d = Qt + buf * QT_FLOATS + (spart * (KC / 2) + 4 * u) * (PR + 4) + srow;
        d[0] = pre[u].x;
        d[PR + 4] = pre[u].y;
        d[2 * (PR + 4)] = pre[u].z;
        d[3 * (PR + 4)] = pre[u].w;
      }
    };
    fetch(0);
    stage_q(0);
    if (KC < q) fetch(KC);
    __syncthreads();
    for (int k0 = 0, st = 0; k0 < q; k0 += KC, ++st) {
      // the next step's columns go to the other buffer while this step's are read
      if (k0 + KC < q) {
        stage_q((st + 1) & 1);
        if (k0 + 2 * KC < q) fetch(k0 + 2 * KC);
      }
      if (busy && k0 + kq * 8 < q) {  // q - k0 is a multiple of 8
        const float* Qb = Qt + (st & 1) * QT_FLOATS;
#pragma unroll
        for (int k8 = 0; k8 < 8; ++k8) {
          const int kk = kq * 8 + k8;
          const float4 a0 = *reinterpret_cast<const float4*>(Qb + kk * (PR + 4) + rg * 8);
          const float4 a1 = *reinterpret_cast<const float4*>(Qb + kk * (PR + 4) + rg * 8 + 4);
          const float4 g0 = *reinterpret_cast<const float4*>(G + (k0 + kk) * BW + cg * 8);
          const float4 g1 = *reinterpret_cast<const float4*>(G + (k0 + kk) * BW + cg * 8 + 4);
          fma8x8(acc, a0, a1, g0, g1);
        }
      }
      __syncthreads();
    }
    // the four groups' parts, then W -= their sum
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      float4* p = reinterpret_cast<float4*>(Pw + ((kq * PR) + rg * 8 + i) * BW + cg * 8);
      p[0] = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
      p[1] = make_float4(acc[i][4], acc[i][5], acc[i][6], acc[i][7]);
    }
    __syncthreads();
    const float4* P4 = reinterpret_cast<const float4*>(Pw);
    for (int f = threadIdx.x; f < PR * BW / 4; f += AT) {
      const int64_t r = p0 + (f >> 3);
      if (r < c.r1) {
        float4 s = P4[f];
#pragma unroll
        for (int gq = 1; gq < 4; ++gq) {
          const float4 v = P4[gq * (PR * BW / 4) + f];
          s.x += v.x;
          s.y += v.y;
          s.z += v.z;
          s.w += v.w;
        }
        float4* wp = reinterpret_cast<float4*>(c.W + r * BW + (f & 7) * 4);
        float4 w0 = *wp;
        w0.x -= s.x;
        w0.y -= s.y;
        w0.z -= s.z;
        w0.w -= s.w;
        *wp = w0;
      }
    }
    __syncthreads();
  }
}

// (hi, lo) <- (hi, lo) - a g as an unevaluated double-FP32 sum: the product is
// split exactly (p + pe = a g, pe from an FMA) and the subtraction of p by
// Knuth's TwoSum (s + e = hi - p exactly); lo collects e - pe.  The explicit
// _rn intrinsics keep the compiler from contracting or reassociating the steps.
__device__ __forceinline__ void df_sub(float& hi, float& lo, float a, float g) {
  const float p = __fmul_rn(a, g);
  const float pe = __fmaf_rn(a, g, -p);
  const float s = __fsub_rn(hi, p);
  const float bb = __fsub_rn(s, hi);
  const float e = __fsub_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fadd_rn(p, bb));
  lo = __fsub_rn(__fadd_rn(lo, e), pe);
  hi = s;
}

// W <- W - Q[:, :q] Gs on this CTA's rows with the difference formed in
// double-FP32 (about 44 bits of W's scale), for the first projection of a
// block: there W - Q G is small next to W, and FP32 rounding of that size
// (about 1e-7 of W, spread over every direction) would reach the residual the
// stopping test measures.  Passes of PR rows; Q staged transposed KC columns at
// a time as in w_minus_qg; a thread owns a 4 x 4 tile (rows 4 rg .. 4 rg + 3,
// columns 4 cg .. 4 cg + 3) over all q columns of Q, so no partial sums are
// exchanged.  The result is rounded to FP32 once.
template <bool GG>
__device__ void w_minus_qg_df(const Ctx& c, int q) {
  const float* G = GG ? s_gg : c.Gs;
  float* Qt = reinterpret_cast<float*>(c.stage);  // [2][KC][PR + 4]
  const int cg = threadIdx.x & 7, rg = threadIdx.x >> 3;  // 8 column groups x 64 row groups
  const int srow = threadIdx.x & (PR - 1), spart = threadIdx.x / PR;  // staging: row, which KC/2 columns
  static_assert(AT == 512 && PR == 256 && BW == 32, "a 4 x 4 tile per thread covers a pass");
  for (int64_t p0 = c.r0; p0 < c.r1; p0 += PR) {
    float hi[4][4], lo[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int64_t r = p0 + rg * 4 + i;
      const float4 w = r < c.r1 ? *reinterpret_cast<const float4*>(c.W + r * BW + cg * 4)
                                : make_float4(0.f, 0.f, 0.f, 0.f);
      hi[i][0] = w.x;
      hi[i][1] = w.y;
      hi[i][2] = w.z;
      hi[i][3] = w.w;
#pragma unroll
      for (int j = 0; j < 4; ++j) lo[i][j] = 0.f;
    }
    const int64_t rt = p0 + srow;
    const bool rin = rt < c.r1;
    const bool busy = p0 + rg * 4 < c.r1;
    float4 pre[KC / 8];
    auto fetch = [&](int k0) {
#pragma unroll
      for (int u = 0; u < KC / 8; ++u) {
        const int k = k0 + spart * (KC / 2) + 4 * u;
        pre[u] = (rin && k < q) ? *reinterpret_cast<const float4*>(c.Q + rt * c.ldq + k)
                                : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    };
    auto stage_q = [&](int buf) {
#pragma unroll
      for (int u = 0; u < KC / 8; ++u) {
        float* d = Qt + buf * QT_FLOATS + (spart * (KC / 2) + 4 * u) * (PR + 4) + srow;
        d[0] = pre[u].x;
        d[PR + 4] = pre[u].y;
        d[2 * (PR + 4)] = pre[u].z;
        d[3 * (PR + 4)] = pre[u].w;
      }
    };
    fetch(0);
    stage_q(0);
    if (KC < q) fetch(KC);
    __syncthreads();
    for (int k0 = 0, st = 0; k0 < q; k0 += KC, ++st) {
      if (k0 + KC < q) {
        stage_q((st + 1) & 1);
        if (k0 + 2 * KC < q) fetch(k0 + 2 * KC);
      }
      if (busy) {
        const float* Qb = Qt + (st & 1) * QT_FLOATS + rg * 4;
        const float* Gb = G + k0 * BW + cg * 4;
        const int kn = min(KC, q - k0);  // a multiple of 8
        for (int k8 = 0; k8 < kn; k8 += 8) {
#pragma unroll
          for (int kk = k8; kk < k8 + 8; ++kk) {
            const float4 a = *reinterpret_cast<const float4*>(Qb + kk * (PR + 4));
            const float4 g = *reinterpret_cast<const float4*>(Gb + kk * BW);
            const float av[4] = {a.x, a.y, a.z, a.w};
            const float gv[4] = {g.x, g.y, g.z, g.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
              for (int j = 0; j < 4; ++j) df_sub(hi[i][j], lo[i][j], av[i], gv[j]);
          }
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int64_t r = p0 + rg * 4 + i;
      if (r < c.r1)
        *reinterpret_cast<float4*>(c.W + r * BW + cg * 4) =
            make_float4(__fadd_rn(hi[i][0], lo[i][0]), __fadd_rn(hi[i][1], lo[i][1]),
                        __fadd_rn(hi[i][2], lo[i][2]), __fadd_rn(hi[i][3], lo[i][3]));
    }
    __syncthreads();
  }
}

// 1/sqrt(x) for x > 0: the FP32 estimate refined by Newton steps
// y <- y (3 - x y^2) / 2 in type A (two in FP64, none in FP32)
template <typename A>
__device__ __forceinline__ A rsqrt_newton(A x) {
  if constexpr (sizeof(A) == 8) {
    if (!(x > 1e-36 && x < 1e36)) return 1.0 / sqrt(x);
    double y = (double)rsqrtf((float)x);
    y = y * fma(-0.5 * x, y * y, 1.5);
    y = y * fma(-0.5 * x, y * y, 1.5);
    return y;
  } else {
    return 1.0f / sqrtf(x);
  }
}

// 1/sqrt(p_k), or 0 (the column is dropped) for a pivot at or below 1e-26 of
// the largest diagonal dmax or at or below `floor`, or an all-zero matrix;
// kept out of line so that it does not crowd the registers of the loops
// around its call
template <typename A>
__device__ __noinline__ A chol_pivot(A pk, A dmax, A floor, A col_floor) {
  const bool drop = !(pk > A(1e-26) * dmax) || !(pk > floor) || !(pk > col_floor) || !(dmax > A(0));
  return drop ? A(0) : rsqrt_newton<A>(pk);
}

// Right-looking Cholesky G = L L^T of the BW x BW matrix in L (type A,
// leading dimension LDA, overwritten), by all AT threads.  Step k: thread 0
// takes the pivot p_k (chol_pivot), then each element (i, j), k < j <= i, of
// the trailing block gets one thread, L[i][j] -= L[i][k] L[j][k] / p_k
// (column k is scaled by 1/sqrt(p_k) only at the end).  A pivot at or
// below `floor` also drops its column.  Writes the factor as FP32 into Lf (leading dimension LF, zero above the diagonal and
// in dropped columns) and the reciprocal diagonal into rinv (0 for a dropped
// column).  iv and u are shared scratch of BW entries each.
template <typename A, int LDA>
__device__ void chol_drop(A* L, float* Lf, float* rinv, A* iv, A* u, A floor, const double* colref = nullptr,
                          double tau_col = 0.0) {
  const int t = threadIdx.x;
  if (t < 32) {
    A v = L[t * LDA + t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (t == 0) u[0] = v;
  }
  __syncthreads();
  const A dmax = u[0];
  auto pivot = [&](int k) {  // thread 0
    iv[k] = chol_pivot<A>(L[k * LDA + k], dmax, floor, colref ? (A)(tau_col * colref[k]) : A(0));
  };
  __syncthreads();
  for (int k = 0; k < BW; ++k) {
    if (t == 0) pivot(k);
    __syncthreads();
    const int m = BW - 1 - k;  // order of the trailing block
    if (t < m * (m + 1) / 2) {
      int ii = min(m - 1, (int)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f));  // t = ii (ii + 1) / 2 + jj
      if (t < ii * (ii + 1) / 2) --ii;
      const int jj = t - ii * (ii + 1) / 2;
      const int i = k + 1 + ii, j = k + 1 + jj;
      const A ip = iv[k] * iv[k];
      L[i * LDA + j] -= (L[i * LDA + k] * ip) * L[j * LDA + k];
    }
    __syncthreads();
  }
  for (int e = t; e < BW * BW; e += AT) {
    const int i = e >> 5, j = e & 31;
    Lf[i * LF + j] = j <= i ? (float)(L[i * LDA + j] * iv[j]) : 0.f;
  }
  if (t < BW) rinv[t] = (float)iv[t];
  __syncthreads();
}

// c.gram <- W^T W for the b <= BW columns of W (the rest are zero), over all
// rows: FP32 runs of 4 GR rows added in FP64, the CTAs' partials added in rank
// order in every CTA.
__device__ void gram_pass(Ctx& c) {
  double* gp = reinterpret_cast<double*>(c.stage);                 // [BW][BW], this CTA's partial
  float* Wc = reinterpret_cast<float*>(c.stage + BW * BW * 8);      // [2][GR][BW], double-buffered
  double* gg = reinterpret_cast<double*>(c.stage + BW * BW * 8 + 2 * GR * BW * 4);  // [4][BW][BW], the groups'
  const int grp = threadIdx.x >> 7, lt = threadIdx.x & 127;
  const int i = lt >> 2, j0 = (lt & 3) * 8;  // entries (i, j0 .. j0 + 7); rows rr = grp (mod 4)
  double d[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) d[u] = 0.0;
  auto issue = [&](int64_t p0, int buf) {
#pragma unroll
    for (int u = 0; u < GR * BW / 4 / AT; ++u) {
      const int e = threadIdx.x + u * AT, rr = e >> 3, j4 = e & 7;
      const int64_t r = p0 + rr;
      const bool in = r < c.r1;
      cp_async_16z(smem_u32(Wc + buf * GR * BW + e * 4), in ? c.W + r * BW + j4 * 4 : c.W, in);
    }
    cp_async_commit();
  };
  if (c.r0 < c.r1) issue(c.r0, 0);
  for (int64_t p0 = c.r0, ch = 0; p0 < c.r1; p0 += GR, ++ch) {
    if (p0 + GR < c.r1) {
      issue(p0 + GR, (int)((ch + 1) & 1));
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const float* Wb = Wc + (ch & 1) * GR * BW;
    float f[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) f[u] = 0.f;
#pragma unroll 4
    for (int rr = grp; rr < GR; rr += 4) {
      const float wi = Wb[rr * BW + i];
      const float4 w0 = *reinterpret_cast<const float4*>(Wb + rr * BW + j0);
      const float4 w1 = *reinterpret_cast<const float4*>(Wb + rr * BW + j0 + 4);
      f[0] = fmaf(wi, w0.x, f[0]);
      f[1] = fmaf(wi, w0.y, f[1]);
      f[2] = fmaf(wi, w0.z, f[2]);
      f[3] = fmaf(wi, w0.w, f[3]);
      f[4] = fmaf(wi, w1.x, f[4]);
      f[5] = fmaf(wi, w1.y, f[5]);
      f[6] = fmaf(wi, w1.z, f[6]);
      f[7] = fmaf(wi, w1.w, f[7]);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) d[u] += (double)f[u];
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 8; ++u) gg[grp * BW * BW + i * BW + j0 + u] = d[u];
  __syncthreads();
  for (int e = threadIdx.x; e < BW * BW; e += AT) gp[e] = ((gg[e] + gg[BW * BW + e]) + gg[2 * BW * BW + e]) + gg[3 * BW * BW + e];
  cl_sync();
  for (int e = threadIdx.x; e < BW * BW; e += AT) {
    double s = 0.0;
    for (int r = 0; r < c.ncl; ++r) s += cl_map(gp, r)[e];
    c.gram[(e >> 5) * LD + (e & 31)] = s;
  }
  cl_sync();  // the partials are overwritten after this
}

// The factor of c.gram (FP64 in the first Cholesky-QR pass, where the Gram
// matrix squares W's condition number; FP32 in the second, where it is the
// identity up to the first pass's rounding), then W <- W L^{-T} row by row.
__device__ void factor_solve(Ctx& c, bool fp64, double floor, double tau_col = 0.0) {
  if (fp64) {
    chol_drop<double, LD>(c.gram, c.Lf, c.rinv, c.cs, c.cs + BW, floor, tau_col > 0.0 ? colsq(c) : nullptr,
                          tau_col);
  } else {
    float* Lw = reinterpret_cast<float*>(c.stage);  // FP32 working copy (the partials are no longer read)
    for (int e = threadIdx.x; e < BW * BW; e += AT) Lw[(e >> 5) * LD + (e & 31)] = (float)c.gram[(e >> 5) * LD + (e & 31)];
    __syncthreads();
    float* fs = reinterpret_cast<float*>(c.cs);
    chol_drop<float, LD>(Lw, c.Lf, c.rinv, fs, fs + BW, (float)floor);
  }
  // x_j = (w_j - sum_{m < j} x_m L[j][m]) / L[j][j], one row per thread
  for (int64_t r = c.r0 + threadIdx.x; r < c.r1; r += AT) {
    float x[BW];
    float4* wp = reinterpret_cast<float4*>(c.W + r * BW);
#pragma unroll
    for (int u = 0; u < BW / 4; ++u) {
      const float4 v = wp[u];
      x[4 * u] = v.x;
      x[4 * u + 1] = v.y;
      x[4 * u + 2] = v.z;
      x[4 * u + 3] = v.w;
    }
#pragma unroll
    for (int j = 0; j < BW; ++j) {
      float a0 = x[j], a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
      for (int m4 = 0; m4 < BW / 4; ++m4) {
        if (4 * m4 >= j) break;
        const float4 l = *reinterpret_cast<const float4*>(c.Lf + j * LF + m4 * 4);
        if (4 * m4 + 0 < j) a0 = fmaf(-x[4 * m4 + 0], l.x, a0);
        if (4 * m4 + 1 < j) a1 = fmaf(-x[4 * m4 + 1], l.y, a1);
        if (4 * m4 + 2 < j) a2 = fmaf(-x[4 * m4 + 2], l.z, a2);
        if (4 * m4 + 3 < j) a3 = fmaf(-x[4 * m4 + 3], l.w, a3);
      }
      x[j] = ((a0 + a1) + (a2 + a3)) * c.rinv[j];
    }
#pragma unroll
    for (int u = 0; u < BW / 4; ++u) wp[u] = make_float4(x[4 * u], x[4 * u + 1], x[4 * u + 2], x[4 * u + 3]);
  }
  __syncthreads();
}

// Orthonormalize W's b columns and append them to Q.  Plain steps: [project
// against Q, Cholesky-QR] twice.  Precise steps (a batch tested at eps_rel
// below kPreciseBelow): the first projection forms W - Q G in double-FP32
// (w_minus_qg_df) and is followed by a second, FP32 projection before the
// first factorization.  The FP32 difference W - Q G errs by about 1e-7 of W in
// every direction, and the FP32 product Q^T W by about sqrt(q) 2^-24 of W
// along Q; near eps_rel = 1e-6 both are as large as the residual the test
// measures.  The double-FP32 difference removes the first and the second
// projection the second, so the factored block (and the tested norm) is
// (I - Q Q^T)^2 W formed to about 1e-13 of W.  The first pass's FP32
// triangular solve can magnify rounding along Q by the block's condition
// number, and the projection before the second Cholesky-QR removes that again.
// dref: the block's sum of squares before it was projected against Q.  A
// column whose pivot is at or below the drop level times dref, or at or below
// 1e-26 of the largest pivot, is dropped (a zero column of Q, which leaves
// Q Q^T unchanged).  Plain steps: DROP_FP32 = (3.2e-7)^2, the FP32 noise level
// of the block (normalizing such a residual, rounding along Q, would cost Q
// its orthogonality).  Precise steps: DROP_PRECISE, a residual of 1e-10 of
// the block, a column that is zero in the data (an SJLT column without
// entries) or rounding; and a column whose residual is at or below 1e-7 of
// its own norm before the projection (DROP_COL on its sum of squares): the
// FP32 basis represents the span of the earlier columns only to about that
// level, so a column that lies in that span in exact arithmetic (an SJLT
// column with the one entry of an earlier column's row: the same column of S
// up to its sign) leaves a residual there, which normalized would be a basis
// direction outside the sketch's range.
// The second pass's input columns have unit norm (or are zero) before the
// projection between the passes.  A column that this projection shrinks below
// 0.1 of its length (pivot <= DROP_PASS2) was mostly rounding along Q that the
// first pass normalized: renormalizing what is left would make a basis column
// that is not orthogonal to Q, so it is dropped as well.
constexpr double DROP_FP32 = 1e-13;
constexpr double DROP_PRECISE = 1e-20;
constexpr double DROP_COL = 1e-14;  // precise steps: a pivot at or below 1e-14 of its own column's sum of squares
constexpr double DROP_PASS2 = 1e-2;

// W arrives as it is: its projection(s), the first Gram matrix, Cholesky-QR
// (with the drop rule), then the projection between the passes and its Gram
// matrix; absorb_end finishes the pass.  Returns the trace of the first Gram
// matrix (the same value in every CTA of the cluster): with the precise steps
// ||(I - Q Q^T)^2 W||_F^2.
template <bool WIDE>
__device__ double absorb_begin(Ctx& c, int q, double dref, bool precise) {
  const bool gg = WIDE && q > QMAX;
  if (q > 0) {
    qt_w_all<WIDE>(c, q);
    if (precise) {
      if (gg) w_minus_qg_df<WIDE>(c, q);
      else w_minus_qg_df<false>(c, q);
      qt_w_all<WIDE>(c, q);
    }
    if (gg) w_minus_qg<WIDE>(c, q);
    else w_minus_qg<false>(c, q);
  }
  gram_pass(c);
  double tr = 0.0;
#pragma unroll 8
  for (int i = 0; i < BW; ++i) tr += c.gram[i * LD + i];
  factor_solve(c, true, (precise ? DROP_PRECISE : DROP_FP32) * dref, precise ? DROP_COL : 0.0);
  if (q > 0) {
    qt_w_all<WIDE>(c, q);
    if (gg) w_minus_qg<WIDE>(c, q);
    else w_minus_qg<false>(c, q);
  }
  gram_pass(c);
  return tr > 0.0 ? tr : 0.0;
}

// tr(L1 G2 L1^T), L1 the first pass's factor (c.Lf) and G2 the second Gram
// matrix (c.gram): with the projected block W = W1 L1^T, this is
// ||(I - Q Q^T) W||_F^2 = ||(I - Q Q^T)^2 S~||_F^2 up to the residuals of
// dropped columns.  Every CTA of the cluster holds the same L1 and G2 and
// sums in the same order, so all of them get the same value.
__device__ double lgl_trace(Ctx& c) {
  double acc = 0.0;
  for (int e = threadIdx.x; e < BW * BW; e += AT) {
    const int i = e / BW, k = e % BW;
    double m = 0.0;  // (L1 G2)[i][k]
    for (int j = 0; j <= i; ++j) m = fma((double)c.Lf[i * LF + j], c.gram[j * LD + k], m);
    acc = fma(m, (double)c.Lf[i * LF + k], acc);
  }
  const double v = cta_sum(acc, c.red);
  return v > 0.0 ? v : 0.0;
}

// The second Cholesky-QR pass on the output of absorb_begin, then
// Q[:, q : q + b] <- W[:, :b].
__device__ void absorb_end(Ctx& c, int& q, int b) {
  factor_solve(c, false, DROP_PASS2);
  // float4 at a time (b, q and the row pitch of Q are multiples of 8)
  const int f = threadIdx.x & 7;
  if (f < (b >> 2)) {
    const float4* W4 = reinterpret_cast<const float4*>(c.W);
#pragma unroll 4
    for (int64_t r = c.r0 + (threadIdx.x >> 3); r < c.r1; r += AT / 8)
      *reinterpret_cast<float4*>(c.Qw + r * c.ldq + q + 4 * f) = W4[r * (BW / 4) + f];
  }
  __syncthreads();
  q += b;
}

// One instance per cluster of ncl CTAs (launched with that cluster size; 1: a
// CTA alone, whose cluster barriers are CTA barriers).  WIDE: some instance's
// basis may pass QMAX columns (Q^T W then goes through the instance's global
// G); a separate instantiation, so that batches of narrower bases keep the
// kernel's registers without spills.
template <bool WIDE>
__global__ void __launch_bounds__(AT, 1)
    batch_test_kernel(BItem* __restrict__ items, ATest* __restrict__ tests, const int* __restrict__ order, int ncl,
                      double eps_rel, double eps_abs, bool precise, const int* __restrict__ active, int act_lo,
                      int act_hi) {
  extern __shared__ __align__(16) uint8_t smem[];
  Ctx c;
  c.ncl = ncl;
  c.rank = (int)cg::this_cluster().block_rank();
  if (active) {  // order: the active instances, largest first (active_list_kernel); this launch's share
    const int a = *active;
    if (a < act_lo || a >= act_hi || (int)(blockIdx.x / ncl) >= a) return;  // uniform over a cluster
  }
  const int inst = order[blockIdx.x / ncl];
  ATest* T = tests + inst;
  BItem* I = items + inst;
  if (T->state != ADAPT_ACTIVE) return;  // the same in every CTA of the cluster
  const int dd = T->dd, c_end = I->c_hi, c_split = c_end - dd;
  int q = T->q, covered = T->covered;
  const int64_t n = T->rows;
  const int64_t rpr = ((n + ncl - 1) / ncl + 15) / 16 * 16;
  c.r0 = min64(n, (int64_t)c.rank * rpr);
  c.r1 = min64(n, c.r0 + rpr);
  c.Q = T->Q;
  c.Qw = T->Q;
  c.ldq = T->qcap;
  c.W = T->W;
  if (threadIdx.x == 0) s_gg = T->G;  // read after the first barrier
  c.stage = smem;
  c.Gs = reinterpret_cast<float*>(smem + SM_STAGE);
  c.gram = reinterpret_cast<double*>(smem + SM_STAGE + SM_G);
  c.Lf = reinterpret_cast<float*>(smem + SM_STAGE + SM_G + SM_GRAM);
  c.rinv = reinterpret_cast<float*>(smem + SM_STAGE + SM_G + SM_GRAM + SM_L);
  c.red = reinterpret_cast<double*>(smem + SM_STAGE + SM_G + SM_GRAM + SM_L + 32 * 4);  // NW + 1 slots
  c.cs = c.red + NW + 8;
  const float* S = T->S;
  const int64_t ldS = T->ldS;

  // columns before the tested block that Q does not cover yet (the first d0)
  while (covered < c_split) {
    const int b = min(BW, c_split - covered);
    const double dref = load_block_cols(c, S, ldS, covered, b);
    absorb_begin<WIDE>(c, q, dref, precise);
    absorb_end(c, q, b);
    covered += b;
  }
  // the test, Eq. (3.1): its two projections are those of the absorption
  const double nt2 = load_block_cols(c, S, ldS, c_split, dd);
  const double tr1 = absorb_begin<WIDE>(c, q, nt2, precise);
  const double nh2 = precise ? tr1 : lgl_trace(c);
  const double sc = T->srht ? sqrt((double)T->first_w / (double)c_end)
                            : 1.0 / sqrt((double)(1 + (c_end - T->first_w) / dd));
  const double nh = sqrt(nh2) * sc, nt = sqrt(nt2) * sc;
  const bool stop = (nh < eps_abs) || (nh < eps_rel * nt);
  const bool room = c_end + dd <= T->d_cap;
  if (!stop && room) {  // Algorithm 1 goes on: Q <- [Q, orth(S^)]
    absorb_end(c, q, dd);
    covered = c_end;
  }
  if (c.rank == 0 && threadIdx.x == 0) {
    T->nh = nh;
    T->nt = nt;
    T->tests += 1;
    T->d_reached = c_end;
    if (stop || !room) {
      T->state = stop ? ADAPT_CONVERGED : ADAPT_CAPPED;
      I->units = 0;
    } else {
      T->q = q;
      T->covered = covered;
      I->c_lo = c_end;
      I->c_hi = c_end + dd;
    }
  }
}

// Units of the active instances for the next batched launch, numbered in
// item order (one CTA): per item its blocks x tiles and its columns per warp.
__global__ void __launch_bounds__(1024)
    batch_renumber_kernel(BItem* __restrict__ items, int count, BHeader* __restrict__ hdr, int njobs, int nb,
                          int* err) {
  __shared__ int64_t part[1024];
  const int t = threadIdx.x;
  const int per = (count + 1023) / 1024;
  const int i0 = min(count, t * per), i1 = min(count, i0 + per);
  int64_t s = 0;
  for (int i = i0; i < i1; ++i) {
    BItem& I = items[i];
    if (I.units) {
      const int nbw = (I.c_hi - I.c_lo + njobs - 1) / njobs;
      if (nbw > nb) {
        set_err(err, ERRF_BOUNDS);  // the host checks dd against the shape before the run
        I.units = 0;
      } else {
        I.nbw = nbw;
        I.units = (int64_t)((I.cols + 127) / 128) * I.ntiles;
      }
    }
    s += I.units;
  }
  part[t] = s;
  __syncthreads();
  if (t == 0) {
    int64_t run = 0;
    for (int k = 0; k < 1024; ++k) {
      const int64_t v = part[k];
      part[k] = run;
      run += v;
    }
    hdr->total_units = run;
  }
  __syncthreads();
  int64_t u = part[t];
  for (int i = i0; i < i1; ++i) {
    items[i].unit0 = u;
    u += items[i].units;
  }
}

// S'_i[:, :d_reached] *= 1/sqrt(B), B = blocks of R_i[:, :d_reached] (SJLT), or
// S_i[:, :d_reached] *= sqrt(first_w / d_reached) (SRHT)
__global__ void __launch_bounds__(256) batch_rescale_kernel(const ATest* __restrict__ tests) {
  const ATest& T = tests[blockIdx.x];
  const int d = T.d_reached;
  if (d <= T.first_w) return;
  const float f = (float)(T.srht ? sqrt((double)T.first_w / (double)d)
                                 : 1.0 / sqrt((double)(1 + (d - T.first_w) / T.dd)));
  float* S = const_cast<float*>(T.S);
  for (int64_t r = blockIdx.y; r < T.rows; r += gridDim.y)
    for (int j = threadIdx.x; j < d; j += blockDim.x) S[r * T.ldS + j] *= f;
}

}  // namespace

int adaptive_prepare() {
  JLS_CHECK_CUDA(
      cudaFuncSetAttribute(batch_test_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, SM_TOTAL));
  JLS_CHECK_CUDA(cudaFuncSetAttribute(batch_test_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, SM_TOTAL));
  return SK_OK;
}

// The instances still active, in the order of `order` (largest first), and
// how many (one CTA).
__global__ void __launch_bounds__(1024)
    active_list_kernel(const ATest* __restrict__ tests, const int* __restrict__ order, int count,
                       int* __restrict__ list, int* __restrict__ n_active) {
  __shared__ int part[1024];
  const int t = threadIdx.x;
  const int per = (count + 1023) / 1024;
  const int i0 = min(count, t * per), i1 = min(count, i0 + per);
  int k = 0;
  for (int i = i0; i < i1; ++i) k += tests[order[i]].state == ADAPT_ACTIVE;
  part[t] = k;
  __syncthreads();
  if (t == 0) {
    int run = 0;
    for (int j = 0; j < 1024; ++j) {
      const int v = part[j];
      part[j] = run;
      run += v;
    }
    *n_active = run;
  }
  __syncthreads();
  int o = part[t];
  for (int i = i0; i < i1; ++i)
    if (tests[order[i]].state == ADAPT_ACTIVE) list[o++] = order[i];
}

static int launch_test(BItem* items, ATest* tests, const int* order, int count, int ncl, double eps_rel,
                       double eps_abs, bool wide, const int* active, int act_lo, int act_hi, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(count * ncl));
  cfg.blockDim = dim3(AT);
  cfg.dynamicSmemBytes = SM_TOTAL;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)ncl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const bool precise = eps_rel < kPreciseBelow;
  if (wide)
    JLS_CHECK_CUDA(cudaLaunchKernelEx(&cfg, batch_test_kernel<true>, items, tests, order, ncl, eps_rel, eps_abs, precise,
                                      active, act_lo, act_hi));
  else
    JLS_CHECK_CUDA(cudaLaunchKernelEx(&cfg, batch_test_kernel<false>, items, tests, order, ncl, eps_rel, eps_abs,
                                      precise, active, act_lo, act_hi));
  note_launch();
  return SK_OK;
}

// One round's tests.  A batch of fewer instances than SMs runs clusters of
// ncl CTAs per instance.  Larger batches list their active instances on the
// device first and then make three launches, of which only the one that fits
// the count runs: one CTA per instance while at least as many instances as
// SMs are active, clusters of 4 from a quarter of that, clusters of 8 below
// (as instances converge, the remaining ones get more SMs each).  `list`
// (count ints) and `n_active` are device scratch.
int adaptive_test_round(BItem* items, ATest* tests, const int* order, int count, int ncl, double eps_rel,
                        double eps_abs, bool wide, int* list, int* n_active, cudaStream_t s) {
  if (ncl != 1 && ncl != 2 && ncl != CLMAX) return SK_ERR_INVALID_ARG;
  const int sms = num_sms();
  if (count < sms || !list || !n_active)
    return launch_test(items, tests, order, count, ncl, eps_rel, eps_abs, wide, nullptr, 0, 0, s);
  active_list_kernel<<<1, 1024, 0, s>>>(tests, order, count, list, n_active);
  note_launch();
  JLS_CHECK_CUDA(cudaGetLastError());
  JLS_CHECK(launch_test(items, tests, list, count, 1, eps_rel, eps_abs, wide, n_active, sms, 1 << 30, s));
  JLS_CHECK(launch_test(items, tests, list, count, 4, eps_rel, eps_abs, wide, n_active, sms / 4, sms, s));
  return launch_test(items, tests, list, count, 8, eps_rel, eps_abs, wide, n_active, 0, sms / 4, s);
}

int adaptive_renumber_launch(BItem* items, int count, BHeader* hdr, int njobs, int nb, int* err, cudaStream_t s) {
  batch_renumber_kernel<<<1, 1024, 0, s>>>(items, count, hdr, njobs, nb, err);
  note_launch();
  JLS_CHECK_CUDA(cudaGetLastError());
  return SK_OK;
}

int adaptive_rescale_launch(const ATest* tests, int count, cudaStream_t s) {
  batch_rescale_kernel<<<dim3((unsigned)count, 16), 256, 0, s>>>(tests);
  note_launch();
  JLS_CHECK_CUDA(cudaGetLastError());
  return SK_OK;
}

}  // namespace jls
