// adaptive.cu -- increment rescale and the Frobenius stopping test.
//
// Stopping test (Eq. (3.1) with the two-pass projection of the
// remark after it; Algorithm 1's S~ = last Delta-d columns):
//   S^ = (I - Q Q^T)^2 S~,  stop = ||S^||_F < eps_abs or ||S^||_F < eps_rel ||S~||_F.
// Q is an orthonormal basis of the earlier sketch columns kept per handle and
// slot.  New columns are absorbed 64 at a time by [two block Gram-Schmidt
// passes against Q, Cholesky-QR, one more pass, Cholesky-QR] (the first Gram
// matrix and factor in FP64).  For FP32 data the first pass forms W - Q G in
// double-FP32: FP32 rounding of W - Q G is about 1e-7 of W, spread over every
// direction, as large as the residual near eps_rel = 1e-6; the second pass
// removes the part along Q that the FP32 product Q^T W leaves.  A column whose
// residual is below 1e-10 (FP32 data) or 1e-13 (FP64) of the block before its
// projection is dropped (a zero column of Q, which does not change Q Q^T), so
// a block with zero columns (an SJLT column without entries) adds zero columns.
// The tested block's ||S^||_F^2 = ||(I - Q Q^T)^2 S~||_F^2 is the trace of the
// Gram matrix its first Cholesky-QR pass factors, so a test costs only the
// projections of its absorption.
//
// Tall-skinny products X^T Y (rows ~ n, widths <= 512) run on CUDA cores: each
// CTA reduces a chunk of rows into a 64 x 64 tile of partial sums, chunks are
// summed in FP64 by a second kernel.  Frobenius norms are FP64 sums of squares,
// and the test synchronizes with the host once, to read them.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace jls {

constexpr int NORM_GRID_C = 256;  // CTAs of the norm and column-norm partial sums

// ---------------------------------------------------------------------------
template <typename T>
__global__ void scale_cols_kernel(T* S, int64_t rows, int64_t ld, int c0, int c1, T f) {
  const int w = c1 - c0;
  const int64_t rpb = (rows + gridDim.x - 1) / gridDim.x;
  const int64_t r_beg = (int64_t)blockIdx.x * rpb, r_end = min64(rows, r_beg + rpb);
  for (int64_t r = r_beg; r < r_end; ++r)
    for (int c = threadIdx.x; c < w; c += blockDim.x) S[r * ld + c0 + c] *= f;
}

int scale_columns(void* S, int dtype, int64_t rows, int64_t ld, int c0, int c1, double factor, cudaStream_t s) {
  if (c1 <= c0) return SK_OK;
  const unsigned grid = (unsigned)(8 * num_sms());
  if (dtype == SK_F32)
    scale_cols_kernel<float><<<grid, 256, 0, s>>>((float*)S, rows, ld, c0, c1, (float)factor);
  else
    scale_cols_kernel<double><<<grid, 256, 0, s>>>((double*)S, rows, ld, c0, c1, factor); note_launch();
  JLS_CHECK_CUDA(cudaGetLastError());
  return SK_OK;
}

// ---------------------------------------------------------------------------
// partial[chunk][i][j] = sum_{r in chunk} X[r][i] * Y[r][j]   (i < p, j < q)
// One CTA: a 64 x 64 block of (i, j) over one chunk of rows; 256 threads with
// 4 x 4 outputs each, rows staged 32 at a time (coalesced 256-byte row reads)
// and the next 32 rows loaded into registers while the current ones are used.
template <typename T>
__global__ void __launch_bounds__(256)
    tsgemm_tn_partial(const T* __restrict__ X, int64_t ldx, int p, const T* __restrict__ Y, int64_t ldy, int q,
                      int64_t rows, int64_t rows_per_chunk, double* __restrict__ part) {
  __shared__ __align__(16) T xs[32][68];
  __shared__ __align__(16) T ys[32][68];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int i0 = blockIdx.x * 64, j0 = blockIdx.y * 64;
  const int64_t r_begin = (int64_t)blockIdx.z * rows_per_chunk;
  const int64_t r_end = min64(rows, r_begin + rows_per_chunk);
  // this thread stages elements e = threadIdx.x + 256 u of each 32 x 64 tile: row e / 64, column e % 64
  const int c = threadIdx.x & 63, rb = threadIdx.x >> 6;
  const bool xin = i0 + c < p, yin = j0 + c < q;
  T xr[8], yr[8];
  auto fetch = [&](int64_t r0) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int64_t r = r0 + rb + 4 * u;
      xr[u] = (r < r_end && xin) ? X[r * ldx + i0 + c] : T(0);
      yr[u] = (r < r_end && yin) ? Y[r * ldy + j0 + c] : T(0);
    }
  };
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) acc[a][cc] = T(0);
  if (r_begin < r_end) fetch(r_begin);
  for (int64_t r0 = r_begin; r0 < r_end; r0 += 32) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      xs[rb + 4 * u][c] = xr[u];
      ys[rb + 4 * u][c] = yr[u];
    }
    __syncthreads();
    if (r0 + 32 < r_end) fetch(r0 + 32);
#pragma unroll 8
    for (int rr = 0; rr < 32; ++rr) {
      T xv[4], yv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) xv[a] = xs[rr][ty * 4 + a];
#pragma unroll
      for (int cc = 0; cc < 4; ++cc) yv[cc] = ys[rr][tx * 4 + cc];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) acc[a][cc] = fma(xv[a], yv[cc], acc[a][cc]);
    }
    __syncthreads();
  }
  double* out = part + (int64_t)blockIdx.z * p * q;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = i0 + ty * 4 + a;
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      const int j = j0 + tx * 4 + cc;
      if (i < p && j < q) out[(int64_t)i * q + j] = (double)acc[a][cc];
    }
  }
}

// out[e] = sum of the chunks' partials, added in chunk order; the loads of
// eight chunks are issued before they are added (the sums' order is unchanged).
__global__ void reduce_partials(const double* __restrict__ part, int nchunks, int64_t count, double* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    double s = 0;
    int c = 0;
    for (; c + 8 <= nchunks; c += 8) {
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = part[(int64_t)(c + u) * count + e];
#pragma unroll
      for (int u = 0; u < 8; ++u) s += v[u];
    }
    for (; c < nchunks; ++c) s += part[(int64_t)c * count + e];
    out[e] = s;
  }
}

// Y[r][j] = sum_{i < p} X[r][i] M[i][j]     (SUB = false)
// Y[r][j] -= sum_{i < p} X[r][i] M[i][j]    (SUB = true)
// for j < q <= 64; M is FP64, row-major with leading dimension ldm.  One CTA
// owns 64 rows and reads all of them before it writes, so Y may alias X.
// The next 32-wide slice of X and M is loaded into registers while the
// current one is used.
template <typename T, bool SUB>
__global__ void __launch_bounds__(256)
    rows_small_gemm(const T* X, int64_t ldx, int p, const double* __restrict__ M, int64_t ldm, int q, T* Y,
                    int64_t ldy, int64_t rows) {
  __shared__ __align__(16) T xs[32][68];  // [i][row]
  __shared__ __align__(16) T ms[32][68];  // [i][col]
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t r0 = (int64_t)blockIdx.x * 64;
  // staging: X element (row e / 32, i e % 32), M element (i e / 64, col e % 64) for e = threadIdx.x + 256 u
  const int xi = threadIdx.x & 31, xr0 = threadIdx.x >> 5;
  const int mc = threadIdx.x & 63, mi0 = threadIdx.x >> 6;
  T xv_n[8], mv_n[8];
  auto fetch = [&](int i0) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int64_t r = r0 + xr0 + 8 * u;
      xv_n[u] = (r < rows && i0 + xi < p) ? X[r * ldx + i0 + xi] : T(0);
      const int i = i0 + mi0 + 4 * u;
      mv_n[u] = (i < p && mc < q) ? (T)M[(int64_t)i * ldm + mc] : T(0);
    }
  };
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[a][c] = T(0);
  fetch(0);
  for (int i0 = 0; i0 < p; i0 += 32) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      xs[xi][xr0 + 8 * u] = xv_n[u];
      ms[mi0 + 4 * u][mc] = mv_n[u];
    }
    __syncthreads();
    if (i0 + 32 < p) fetch(i0 + 32);
#pragma unroll 8
    for (int ii = 0; ii < 32; ++ii) {
      T xv[4], mv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) xv[a] = xs[ii][ty * 4 + a];
#pragma unroll
      for (int c = 0; c < 4; ++c) mv[c] = ms[ii][tx * 4 + c];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = fma(xv[a], mv[c], acc[a][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int64_t r = r0 + ty * 4 + a;
    if (r >= rows) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j = tx * 4 + c;
      if (j < q) Y[r * ldy + j] = SUB ? Y[r * ldy + j] - acc[a][c] : acc[a][c];
    }
  }
}

// (hi, lo) <- (hi, lo) - a m as an unevaluated double-FP32 sum: the product
// is split exactly (p + pe = a m, pe from an FMA) and the subtraction of p by
// Knuth's TwoSum (s + e = hi - p exactly); lo collects e - pe.  The _rn
// intrinsics keep the compiler from contracting or reassociating the steps.
__device__ __forceinline__ void df_sub(float& hi, float& lo, float a, float m) {
  const float p = __fmul_rn(a, m);
  const float pe = __fmaf_rn(a, m, -p);
  const float s = __fsub_rn(hi, p);
  const float bb = __fsub_rn(s, hi);
  const float e = __fsub_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fadd_rn(p, bb));
  lo = __fsub_rn(__fadd_rn(lo, e), pe);
  hi = s;
}

// Y[r][j] -= sum_{i < p} X[r][i] M[i][j] for FP32 data with the difference
// formed in double-FP32 and rounded once (about 44 bits of Y's scale): the
// first projection of a block against Q, where Y - X M is small next to Y and
// FP32 rounding of Y's size would reach the residual the stopping test
// measures.  Same tiling as rows_small_gemm (M rounded to FP32); Y must not
// alias X.
__global__ void __launch_bounds__(256)
    rows_small_gemm_df(const float* __restrict__ X, int64_t ldx, int p, const double* __restrict__ M, int64_t ldm,
                       int q, float* __restrict__ Y, int64_t ldy, int64_t rows) {
  __shared__ __align__(16) float xs[32][68];  // [i][row]
  __shared__ __align__(16) float ms[32][68];  // [i][col]
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t r0 = (int64_t)blockIdx.x * 64;
  const int xi = threadIdx.x & 31, xr0 = threadIdx.x >> 5;
  const int mc = threadIdx.x & 63, mi0 = threadIdx.x >> 6;
  float xv_n[8], mv_n[8];
  auto fetch = [&](int i0) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int64_t r = r0 + xr0 + 8 * u;
      xv_n[u] = (r < rows && i0 + xi < p) ? X[r * ldx + i0 + xi] : 0.f;
      const int i = i0 + mi0 + 4 * u;
      mv_n[u] = (i < p && mc < q) ? (float)M[(int64_t)i * ldm + mc] : 0.f;
    }
  };
  float hi[4][4], lo[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int64_t r = r0 + ty * 4 + a;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j = tx * 4 + c;
      hi[a][c] = (r < rows && j < q) ? Y[r * ldy + j] : 0.f;
      lo[a][c] = 0.f;
    }
  }
  fetch(0);
  for (int i0 = 0; i0 < p; i0 += 32) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      xs[xi][xr0 + 8 * u] = xv_n[u];
      ms[mi0 + 4 * u][mc] = mv_n[u];
    }
    __syncthreads();
    if (i0 + 32 < p) fetch(i0 + 32);
#pragma unroll 4
    for (int ii = 0; ii < 32; ++ii) {
      const float4 xv = *reinterpret_cast<const float4*>(&xs[ii][ty * 4]);
      const float4 mv = *reinterpret_cast<const float4*>(&ms[ii][tx * 4]);
      const float xa[4] = {xv.x, xv.y, xv.z, xv.w};
      const float ma[4] = {mv.x, mv.y, mv.z, mv.w};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) df_sub(hi[a][c], lo[a][c], xa[a], ma[c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int64_t r = r0 + ty * 4 + a;
    if (r >= rows) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j = tx * 4 + c;
      if (j < q) Y[r * ldy + j] = __fadd_rn(hi[a][c], lo[a][c]);
    }
  }
}

// 1 / sqrt(x) for x > 0.  In FP64: Newton-Raphson steps y <- y (3 - x y^2) / 2
// from the FP32 hardware estimate (relative error <= 2^-21; one step leaves
// <= 1.5 (2^-21)^2 < 1e-12, two steps reach FP64 rounding).  GB300's FP64
// square root and division each take several hundred cycles of latency, a
// Newton step four dependent FP64 operations.  Outside FP32's exponent range
// the plain FP64 sqrt and division are used.
template <int STEPS>
__device__ __forceinline__ double rsqrt_nr(double x) {
  if (!(x > 1e-36 && x < 1e36)) return 1.0 / sqrt(x);
  double y = (double)rsqrtf((float)x);
#pragma unroll
  for (int s = 0; s < STEPS; ++s) y = y * fma(-0.5 * x, y * y, 1.5);
  return y;
}

// Cholesky G = L L^T of the b x b (b <= 64) FP64 Gram matrix, right-looking,
// in arithmetic type A, with column dropping: a pivot <= 1e-26 of the largest
// diagonal, or <= tau times the sum of the nref partials in `ref` (the
// block's sum of squares before its projection against Q), or <= floor_abs,
// or a zero Gram matrix zeroes that column of L.  Writes L (lower,
// b x b row-major, type T, zeros above the diagonal) and rinv[j] = 1 / L[j][j]
// (0 for a dropped column).  One CTA of 256 threads; the pivot of step k + 1
// is taken by thread 0 while warps 1..7 finish step k's trailing update.
template <typename A, typename T, int NR>
__global__ void __launch_bounds__(256) chol_factor_kernel(const double* __restrict__ Gm, int b, T* __restrict__ Lo,
                                                          T* __restrict__ rinv_out, const double* __restrict__ ref,
                                                          int nref, double tau, double floor_abs,
                                                          const double* __restrict__ colpart, int col_ld,
                                                          double tau_col) {
  __shared__ A L[64][65];
  __shared__ A rinv[64];
  __shared__ A s_sq[2], s_iv[2];
  __shared__ A s_dmax, s_floor;
  __shared__ A s_colfloor[64];  // tau_col times each column's sum of squares before the projection
  const int tid = threadIdx.x;
  if constexpr (sizeof(A) == 4) {
    // The FP32 factor is the second Cholesky-QR pass's: its Gram matrix is the
    // identity up to the first pass's rounding, G = I + E.  When max |E| <=
    // 1e-4, L = chol(G) is L_ij = G_ij / sqrt(G_jj) below the diagonal and
    // sqrt(G_ii) on it up to terms of order |E|^2 (below FP32 rounding), every
    // pivot is near 1 (no drop applies), and the factor is formed at once
    // instead of in b dependent steps.
    __shared__ int s_near;
    double dev = 0.0;
    for (int e = tid; e < b * b; e += 256) dev = fmax(dev, fabs(Gm[e] - (e / b == e % b ? 1.0 : 0.0)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dev = fmax(dev, __shfl_xor_sync(0xffffffffu, dev, o));
    if (tid == 0) s_near = 1;
    __syncthreads();
    if ((tid & 31) == 0 && !(dev <= 1e-4)) s_near = 0;
    __syncthreads();
    if (s_near && !colpart && floor_abs < 0.5 && nref == 0) {
      for (int e = tid; e < b * b; e += 256) {
        const int i = e / b, j = e % b;
        Lo[e] = j < i ? (T)((A)Gm[e] / sqrtf((A)Gm[j * b + j])) : j == i ? (T)sqrtf((A)Gm[e]) : T(0);
      }
      if (tid < b) rinv_out[tid] = (T)(1.0f / sqrtf((A)Gm[tid * b + tid]));
      return;
    }
  }
  for (int e = tid; e < b * b; e += 256) L[e / b][e % b] = (A)Gm[e];
  if (tid < 64) {
    double v = 0.0;
    if (colpart && tid < b)
      for (int g = 0; g < NORM_GRID_C; ++g) v += colpart[(int64_t)g * col_ld + tid];  // fixed order
    s_colfloor[tid] = (A)(tau_col * v);
  }
  __syncthreads();
  if (tid < 32) {
    A m = 0;
    for (int i = tid; i < b; i += 32) m = fmax(m, L[i][i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (tid == 0) {
      s_dmax = m;
      double dref = 0;  // the block's sum of squares before its projection (fixed order)
      for (int k = 0; k < nref; ++k) dref += ref[k];
      s_floor = (A)fmax(tau * dref, floor_abs);
    }
  }
  __syncthreads();
  auto pivot = [&](int k) {  // thread 0 only
    const A dmax = s_dmax, pk = L[k][k];
    const bool dk = !(pk > A(1e-26) * dmax) || !(pk > s_floor) || !(pk > s_colfloor[k]) || !(dmax > A(0));
    A iv = A(0);
    if (!dk) {
      if constexpr (sizeof(A) == 8) iv = rsqrt_nr<NR>(pk);
      else iv = 1.0f / sqrtf(pk);
    }
    s_iv[k & 1] = iv;
    s_sq[k & 1] = dk ? A(0) : pk * iv;
    rinv[k] = iv;
  };
  if (tid == 0) pivot(0);
  __syncthreads();
  const int w = tid >> 5;
  const int ut = tid - 32, ti = ut / 14, tj = ut % 14;  // warps 1..7: 16 x 14 update grid
  for (int k = 0; k < b; ++k) {
    const A iv = s_iv[k & 1];
    if (tid > k && tid < b) L[tid][k] *= iv;
    if (tid == k) L[k][k] = s_sq[k & 1];
    __syncthreads();
    if (k + 1 < b && tid > k && tid < b) L[tid][k + 1] -= L[tid][k] * L[k + 1][k];  // column k + 1 first
    __syncthreads();
    if (k + 1 < b) {
      if (tid == 0) {
        pivot(k + 1);
      } else if (w > 0 && ti < 16) {
        for (int i = k + 2 + ti; i < b; i += 16) {
          const A lik = L[i][k];
          for (int j = k + 2 + tj; j <= i; j += 14) L[i][j] -= lik * L[j][k];
        }
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < b * b; e += 256) {
    const int i = e / b, j = e % b;
    Lo[e] = j <= i ? (T)L[i][j] : T(0);
  }
  if (tid < b) rinv_out[tid] = (T)rinv[tid];
}

// W[r][:] <- W[r][:] L^{-T} (b <= 64 columns) in place, by forward
// substitution x_j = (w_j - sum_{i<j} x_i L[j][i]) / L[j][j], one thread per
// row, with rinv[j] = 1 / L[j][j] (0 for a dropped column, whose x_j is then 0).
// trsm_rows<T>() rows per CTA, staged through shared memory with coalesced accesses.
template <typename T>
__host__ __device__ constexpr int trsm_rows() {
  return sizeof(T) == 4 ? 64 : 16;
}
template <typename T>
__global__ void __launch_bounds__(trsm_rows<T>()) rows_trsm_kernel(T* W, int64_t ldw, int b, const T* __restrict__ Lo,
                                                                   const T* __restrict__ rinv, int64_t rows) {
  constexpr int RT = trsm_rows<T>();
  __shared__ __align__(16) T ls[64][64];
  __shared__ T rv[64];
  __shared__ T ws[RT][65];
  const int64_t r0 = (int64_t)blockIdx.x * RT;
#pragma unroll 8
  for (int e = threadIdx.x; e < 64 * 64; e += RT) {
    const int j = e >> 6, i = e & 63;
    ls[j][i] = (j < b && i < b) ? Lo[j * b + i] : T(0);
  }
  for (int j = threadIdx.x; j < 64; j += RT) rv[j] = j < b ? rinv[j] : T(0);
#pragma unroll 8
  for (int e = threadIdx.x; e < RT * 64; e += RT) {
    const int rr = e >> 6, j = e & 63;
    const int64_t r = r0 + rr;
    ws[rr][j] = (r < rows && j < b) ? W[r * ldw + j] : T(0);
  }
  __syncthreads();
  T x[64];
  const int t = threadIdx.x;
#pragma unroll
  for (int j = 0; j < 64; ++j) {
    T a0 = ws[t][j], a1 = T(0);
#pragma unroll
    for (int i = 0; i + 1 < j; i += 2) {
      a0 = fma(-x[i], ls[j][i], a0);
      a1 = fma(-x[i + 1], ls[j][i + 1], a1);
    }
    if (j & 1) a0 = fma(-x[j - 1], ls[j][j - 1], a0);
    x[j] = (a0 + a1) * rv[j];
  }
#pragma unroll
  for (int j = 0; j < 64; ++j) ws[t][j] = x[j];
  __syncthreads();
  for (int e = threadIdx.x; e < RT * 64; e += RT) {
    const int rr = e >> 6, j = e & 63;
    const int64_t r = r0 + rr;
    if (r < rows && j < b) W[r * ldw + j] = ws[rr][j];
  }
}

// Walk the b columns of rows [r_begin, r_end) with blockDim.x = 256 threads and
// no per-element division: for b <= 256, 256/b rows at a time (thread t takes
// column t % b of row t / b); for wider blocks, each row in steps of 256.
template <typename F>
__device__ __forceinline__ void for_block(int64_t r_begin, int64_t r_end, int b, F f) {
  const int t = threadIdx.x;
  if (b <= 256) {
    const int per = 256 / b;
    if (t >= per * b) return;
    const int c = t % b, ro = t / b;
    for (int64_t r = r_begin + ro; r < r_end; r += per) f(r, c);
  } else {
    for (int64_t r = r_begin; r < r_end; ++r)
      for (int c = t; c < b; c += 256) f(r, c);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) copy_block_kernel(const T* __restrict__ src, int64_t lds, T* __restrict__ dst,
                                                         int64_t ldd, int64_t rows, int b) {
  const int64_t rpb = (rows + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = (int64_t)blockIdx.x * rpb, r1 = min64(rows, r0 + rpb);
  for_block(r0, r1, b, [&](int64_t r, int c) { dst[r * ldd + c] = src[r * lds + c]; });
}

// Sum of squares of a rows x b block, one FP64 partial per CTA.  A thread
// sums its own values in T (at most rows / gridDim of them, a few hundred
// here), the CTA adds the thread sums in FP64.
template <typename T>
__global__ void __launch_bounds__(256) sumsq_partial(const T* __restrict__ W, int64_t ldw, int64_t rows, int b,
                                                     double* __restrict__ part) {
  __shared__ double red[256];
  const int64_t rpb = (rows + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = (int64_t)blockIdx.x * rpb, r1 = min64(rows, r0 + rpb);
  T s = T(0);
  for_block(r0, r1, b, [&](int64_t r, int c) {
    const T v = W[r * ldw + c];
    s = fma(v, v, s);
  });
  red[threadIdx.x] = (double)s;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// Each column's sum of squares of a rows x b block (b <= 512), one FP64
// partial per CTA and column: part[blockIdx.x * b + j].  256 threads: column
// t % w of the rows t / w (mod 256 / w), w = min(b, 256), over the CTA's rows.
template <typename T>
__global__ void __launch_bounds__(256) colsumsq_partial(const T* __restrict__ W, int64_t ldw, int64_t rows, int b,
                                                        double* __restrict__ part) {
  __shared__ double red[256];
  const int64_t rpb = (rows + gridDim.x - 1) / gridDim.x;
  const int64_t r0 = (int64_t)blockIdx.x * rpb, r1 = min64(rows, r0 + rpb);
  for (int c0 = 0; c0 < b; c0 += 256) {
    const int w = min(256, b - c0), per = 256 / w;
    const int t = threadIdx.x, j = t % w, ro = t / w;
    double acc = 0.0;
    if (t < per * w) {
      T sq = T(0);
      for (int64_t r = r0 + ro; r < r1; r += per) {
        const T v = W[r * ldw + c0 + j];
        sq = fma(v, v, sq);
      }
      acc = (double)sq;
    }
    red[t] = acc;
    __syncthreads();
    if (t < w) {
      double v = 0.0;
      for (int g = 0; g < per; ++g) v += red[g * w + t];
      part[(int64_t)blockIdx.x * b + c0 + t] = v;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
namespace {

constexpr int NORM_GRID = NORM_GRID_C;

// out[0] = tr(G) for the b x b FP64 Gram matrix G = W^T W of the tested block
// after its two projections (the precise absorption), i.e.
// ||(I - Q Q^T)^2 S~||_F^2, summed in a fixed order; out[1 .. nout) = 0.  One warp.
__global__ void gram_trace_kernel(const double* __restrict__ G, int b, double* __restrict__ out, int nout) {
  double v = 0.0;
  for (int i = threadIdx.x; i < b; i += 32) v += G[(int64_t)i * b + i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (threadIdx.x == 0) out[0] = v > 0.0 ? v : 0.0;
  for (int e = 1 + threadIdx.x; e < nout; e += 32) out[e] = 0.0;
}

// ||W2 L^T||_F^2 = tr(L G2 L^T) for the b x b factor L (row-major, type T,
// zero above the diagonal) of the first Cholesky-QR pass and the FP64 Gram
// matrix G2 = W2^T W2 of its projected output W2 = (I - Q Q^T) W L^{-T}:
// with W the block after one projection, W2 L^T = (I - Q Q^T)^2 S~ up to the
// dropped columns' residuals, so this is the test's ||S^||^2 without
// projecting the block a second time before its factorization.  One CTA of
// 256 threads; thread t takes row i = t / 4 of L G2 in the data's type T (FP32
// for FP32 data: each term l_i^T G2 l_i = ||W2 l_i||^2 is a sum of nonnegative
// parts up to rounding) with its 16 columns k = 16 (t % 4) + 0..15 as 16
// independent accumulation chains, then dots them with row i of L in FP64;
// the sum is reduced in a fixed order into out[0], out[1 .. nout) = 0.
template <typename T>
__global__ void __launch_bounds__(256) lgl_trace_kernel(const T* __restrict__ L, const double* __restrict__ G2, int b,
                                                        double* __restrict__ out, int nout) {
  __shared__ __align__(16) T Gs[64][64];
  __shared__ double red[8];
  const int t = threadIdx.x;
  for (int e = t; e < 64 * 64; e += 256) {
    const int r = e >> 6, c = e & 63;
    Gs[r][c] = (r < b && c < b) ? (T)G2[r * b + c] : (T)0;
  }
  __syncthreads();
  const int i = t >> 2, k0 = 16 * (t & 3);
  double acc = 0.0;
  if (i < b) {
    const T* Li = L + (int64_t)i * b;
    T m[16];  // (L G2)[i][k0 + kk]
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) m[kk] = (T)0;
#pragma unroll 4
    for (int j = 0; j <= i; ++j) {
      const T lj = Li[j];
#pragma unroll
      for (int kk = 0; kk < 16; ++kk) m[kk] = fma(lj, Gs[j][k0 + kk], m[kk]);
    }
#pragma unroll
    for (int kk = 0; kk < 16; ++kk)
      if (k0 + kk <= i) acc = fma((double)m[kk], (double)Li[k0 + kk], acc);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((t & 31) == 0) red[t >> 5] = acc;
  __syncthreads();
  if (t == 0) {
    double v = 0.0;
    for (int w = 0; w < 8; ++w) v += red[w];
    out[0] = v > 0.0 ? v : 0.0;
  }
  for (int e = 1 + t; e < nout; e += 256) out[e] = 0.0;
}

// Where the tested block's ||S^||^2 goes once it is known (NORM_GRID partials
// after the ||S~||^2 ones), and the host copy of both.
constexpr double kDropPass2 = 1e-2;

struct TestOut {
  double* norms;  // 2 x NORM_GRID: ||S~||^2 partials, then ||S^||^2
  double* host;
  cudaEvent_t ready;
};

struct Scratch {
  void* W;        // rows x wmax (T)
  double* part;   // partial products
  double* G;      // up to d_max x wmax
  double* U;      // Cholesky factor (64 x 64) and reciprocal pivots (64), type T
  double* norms;  // 2 x NORM_GRID partials (||S~||^2, ||S^||^2)
  double* ref;    // NORM_GRID partials: a block's sum of squares before its projection
  double* colref;  // NORM_GRID x wmax partials: each column's sum of squares before its projection
  int col_ld;      // columns per partial row of colref (the block width they were taken over)
  size_t part_elems;
};

int ensure_scratch(sk_op* h, int slot, int64_t rows, int dtype, int wmax, Scratch* sc, int nchunks) {
  const size_t es = elem_size(dtype);
  const size_t wb = ((size_t)rows * wmax * es + 255) / 256 * 256;
  const size_t part_elems = (size_t)nchunks * h->d_max * wmax;
  const size_t gb = (size_t)h->d_max * wmax * sizeof(double);
  const size_t need = wb + part_elems * sizeof(double) + gb + 64 * 65 * sizeof(double) + 3 * NORM_GRID * sizeof(double) +
                      (size_t)NORM_GRID * wmax * sizeof(double);
  if (h->scratch_bytes[slot] < need) {
    if (h->scratch[slot]) cudaFree(h->scratch[slot]);
    h->scratch[slot] = nullptr;
    h->scratch_bytes[slot] = 0;
    JLS_CHECK_CUDA(cudaMalloc(&h->scratch[slot], need));
    h->scratch_bytes[slot] = need;
  }
  uint8_t* p = static_cast<uint8_t*>(h->scratch[slot]);
  sc->W = p;
  p += wb;
  sc->part = reinterpret_cast<double*>(p);
  p += part_elems * sizeof(double);
  sc->G = reinterpret_cast<double*>(p);
  p += gb;
  sc->U = reinterpret_cast<double*>(p);
  p += 64 * 65 * sizeof(double);
  sc->norms = reinterpret_cast<double*>(p);
  sc->ref = sc->norms + 2 * NORM_GRID;
  sc->colref = sc->ref + NORM_GRID;
  sc->col_ld = wmax;
  sc->part_elems = part_elems;
  return SK_OK;
}

template <typename T>
int tsgemm(const T* X, int64_t ldx, int p, const T* Y, int64_t ldy, int q, int64_t rows, int nchunks, double* part,
           double* out, cudaStream_t s) {
  // about two CTAs per SM; nchunks bounds the partial-sum buffer
  const int blocks = ((p + 63) / 64) * ((q + 63) / 64);
  const int want = std::max(1, std::min(nchunks, (2 * num_sms() + blocks - 1) / blocks));
  const int64_t rpc = ((rows + want - 1) / want + 31) / 32 * 32;
  const int nch = (int)((rows + rpc - 1) / rpc);
  dim3 grid((p + 63) / 64, (q + 63) / 64, nch);
  tsgemm_tn_partial<T><<<grid, 256, 0, s>>>(X, ldx, p, Y, ldy, q, rows, rpc, part); note_launch();
  const unsigned rgrid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(4 * num_sms(), ((int64_t)p * q + 255) / 256));
  reduce_partials<<<rgrid, 256, 0, s>>>(part, nch, (int64_t)p * q, out); note_launch();
  JLS_CHECK_CUDA(cudaGetLastError());
  return SK_OK;
}

// W (rows x b, ld ldw) <- W - Q G for G = Q^T W (p x b, FP64, ld b), 64 columns at a time;
// with `df` (FP32 data) the difference is formed in double-FP32
template <typename T>
int sub_qg(T* W, int64_t ldw, int b, const T* Q, int64_t ldq, int p, const double* G, int64_t rows, cudaStream_t s,
           bool df = false) {
  for (int j0 = 0; j0 < b; j0 += 64) {
    const int q = std::min(64, b - j0);
    const unsigned grid = (unsigned)((rows + 63) / 64);
    if constexpr (sizeof(T) == 4) {
      if (df) {
        rows_small_gemm_df<<<grid, 256, 0, s>>>(Q, ldq, p, G + j0, b, q, W + j0, ldw, rows); note_launch();
        continue;
      }
    }
    rows_small_gemm<T, true><<<grid, 256, 0, s>>>(Q, ldq, p, G + j0, b, q, W + j0, ldw, rows); note_launch();
  }
  JLS_CHECK_CUDA(cudaGetLastError());
  return SK_OK;
}

// W (rows x b, ld ldw) <- (I - Q Q^T)^passes W.  With df_first the first
// difference is formed in double-FP32 (FP32 data): W - Q G is then exact to
// about 1e-13 of W, and the part along Q that the FP32 product Q^T W leaves
// (about sqrt(q) 2^-24 of W) is removed by the next pass.
template <typename T>
int project_passes(const sk_op* h, const Basis& B, T* W, int64_t ldw, int b, int64_t rows, const Scratch& sc,
                   int nchunks, int passes, cudaStream_t s, bool df_first = false) {
  if (B.cols == 0) return SK_OK;
  const T* Q = static_cast<const T*>(B.Q);
  for (int pass = 0; pass < passes; ++pass) {
    JLS_CHECK(tsgemm<T>(Q, h->d_max, B.cols, W, ldw, b, rows, nchunks, sc.part, sc.G, s));
    JLS_CHECK(sub_qg<T>(W, ldw, b, Q, h->d_max, B.cols, sc.G, rows, s, df_first && pass == 0));
  }
  return SK_OK;
}

// the test's two passes, (I - Q Q^T)^2 W (the first in double-FP32 with the precise steps)
template <typename T>
int project_twice(const sk_op* h, const Basis& B, T* W, int64_t ldw, int b, int64_t rows, const Scratch& sc,
                  int nchunks, cudaStream_t s) {
  return project_passes<T>(h, B, W, ldw, b, rows, sc, nchunks, 2, s, B.precise);
}

// NORM_GRID x b partial column sums of squares of W into `part` (no synchronization)
template <typename T>
int colsumsq_launch(const T* W, int64_t ldw, int64_t rows, int b, double* part, cudaStream_t s) {
  colsumsq_partial<T><<<NORM_GRID, 256, 0, s>>>(W, ldw, rows, b, part); note_launch();
  JLS_CHECK_CUDA(cudaGetLastError());
  return SK_OK;
}

// NORM_GRID partial sums of squares of W into `part` (no synchronization)
template <typename T>
int sumsq_launch(const T* W, int64_t ldw, int64_t rows, int b, double* part, cudaStream_t s) {
  sumsq_partial<T><<<NORM_GRID, 256, 0, s>>>(W, ldw, rows, b, part); note_launch();
  JLS_CHECK_CUDA(cudaGetLastError());
  return SK_OK;
}

// Orthonormalize the b <= 64 columns of W (ld ldw) and append them to Q.
// Plain steps: [project against Q, Cholesky-QR] twice.  Precise steps (FP32
// data, B.precise): [project twice, Cholesky-QR, project, Cholesky-QR], the
// first projection's difference formed in double-FP32.  With `project`, W
// arrives as it is and its first projection(s) are made here; without, W
// arrives projected (the later chunks of a wide tested block, projected twice
// for the test).
// The first factorization is in FP64 (the Gram matrix squares W's condition
// number); the second Gram matrix is the identity up to the first pass's
// rounding, so with FP32 data it is factored in FP32.  The projection between
// the passes removes the rounding along Q that the first pass's triangular
// solve magnifies by the block's condition number.  With `test`, W is the
// tested block; its ||S^||^2 = ||(I - Q Q^T)^2 S~||^2 is the trace of the
// first Gram matrix with the precise steps (gram_trace_kernel), and
// tr(L1 G2 L1^T) from the first factor and the second Gram matrix with the
// plain ones (lgl_trace_kernel: the block projected once, factored, projected
// again); it is copied to the host with ||S~||^2 and signalled.
template <typename T>
int absorb_block(sk_op* h, Basis& B, T* W, int64_t ldw, int b, int64_t rows, const Scratch& sc, int nchunks,
                 bool project, const double* ref, cudaStream_t s, const TestOut* test = nullptr,
                 const double* colref = nullptr, int col_ld = 0) {
  const bool precise = B.precise;
  if (project) JLS_CHECK(project_passes<T>(h, B, W, ldw, b, rows, sc, nchunks, precise ? 2 : 1, s, precise));
  T* Lf = reinterpret_cast<T*>(sc.U);
  T* rinv = Lf + 64 * 64;
  constexpr int RT = trsm_rows<T>();
  const unsigned tgrid = (unsigned)((rows + RT - 1) / RT);
  // The first pass drops columns whose residual is at the noise level of the
  // block before its projection (ref: NORM_GRID partials of its sum of
  // squares).  Plain steps on FP32 data: 3.2e-7 of the block, the rounding of
  // an FP32 projection (normalizing it, rounding along Q, would cost Q its
  // orthogonality).  Precise steps: 1e-10, a column that is zero in the data
  // (an SJLT column without entries) or rounding.  FP64 data: 1e-13.  The
  // second pass's columns had unit norm before the projection between the
  // passes; one that it shrinks below 0.1 (pivot <= kDropPass2) was rounding
  // along Q that the first pass normalized, and is dropped rather than
  // renormalized.
  const double tau = sizeof(T) == 8 ? 1e-26 : (precise ? 1e-20 : 1e-13);
  // Precise steps also drop a column whose residual is at or below 1e-7 of its
  // own norm before the projection (colref: each column's sum of squares):
  // the FP32 basis represents the span of the earlier columns only to about
  // that level, so a column in that span in exact arithmetic (an SJLT column
  // with the one entry of an earlier column's row) leaves a residual there,
  // which normalized would be a direction outside the sketch's range.
  const double tau_col = (precise && colref) ? 1e-14 : 0.0;
  for (int pass = 0; pass < 2; ++pass) {
    if (pass == 1) JLS_CHECK(project_passes<T>(h, B, W, ldw, b, rows, sc, nchunks, 1, s));
    JLS_CHECK(tsgemm<T>(W, ldw, b, W, ldw, b, rows, nchunks, sc.part, sc.G, s));
    if (test && pass == (precise ? 0 : 1)) {
      if (precise) {
        gram_trace_kernel<<<1, 32, 0, s>>>(sc.G, b, test->norms + NORM_GRID, NORM_GRID);
      } else {  // Lf still holds the first pass's factor
        lgl_trace_kernel<T><<<1, 256, 0, s>>>(Lf, sc.G, b, test->norms + NORM_GRID, NORM_GRID);
      }
      note_launch();
      JLS_CHECK_CUDA(cudaMemcpyAsync(test->host, test->norms, 2 * NORM_GRID * sizeof(double),
                                     cudaMemcpyDeviceToHost, s));
      JLS_CHECK_CUDA(cudaEventRecord(test->ready, s));
    }
    const double* r = pass == 0 ? ref : nullptr;
    const int nr = r ? NORM_GRID : 0;
    const double fa = pass == 0 ? 0.0 : kDropPass2;
    const double* cr = pass == 0 && tau_col > 0.0 ? colref : nullptr;
    if (sizeof(T) == 8)
      chol_factor_kernel<double, T, 2><<<1, 256, 0, s>>>(sc.G, b, Lf, rinv, r, nr, tau, fa, cr, col_ld, tau_col);
    else if (pass == 0)
      chol_factor_kernel<double, T, 1><<<1, 256, 0, s>>>(sc.G, b, Lf, rinv, r, nr, tau, fa, cr, col_ld, tau_col);
    else
      chol_factor_kernel<float, T, 0><<<1, 256, 0, s>>>(sc.G, b, Lf, rinv, r, nr, tau, fa, nullptr, 0, 0.0);
    note_launch();
    rows_trsm_kernel<T><<<tgrid, RT, 0, s>>>(W, ldw, b, Lf, rinv, rows); note_launch();
  }
  copy_block_kernel<T><<<(unsigned)(4 * num_sms()), 256, 0, s>>>(W, ldw, static_cast<T*>(B.Q) + B.cols, h->d_max,
                                                                  rows, b);
  note_launch();
  JLS_CHECK_CUDA(cudaGetLastError());
  B.cols += b;
  return SK_OK;
}

// The test of Eq. (3.1) on S~ = S[:, c_split:c_end], then Algorithm 1's
// extension of Q by the QR of S^ (made at once, so that the next test, on the
// next Delta-d columns, starts from the basis of every earlier column).
// Columns of S before c_split that Q does not cover yet (the first d0, or
// after a restart) are absorbed first.  A tested block of up to 64 columns is
// projected twice and ||S^||^2 is the trace of the Gram matrix its first
// Cholesky-QR pass factors (gram_trace_kernel); a wider one is projected
// twice and its norm summed before it is absorbed in chunks of 64.
// The two norms are copied to the slot's pinned host buffer and an event is
// recorded, while the extension of Q runs on; norm_test_finish waits for
// that event.  Each slot (S, S') has its
// own basis, scratch, host buffer and event, so the two tests can run on two
// streams at once.
template <typename T>
int norm_test_enqueue_t(sk_op* h, int slot, const T* S, int64_t rows, int64_t ldS, int dtype, double eps_rel,
                        int c_split, int c_end, cudaStream_t s) {
  Basis& B = h->basis[slot];
  // FP32 data with a tight eps_rel takes the precise steps; a basis built by
  // the other steps is started again
  const bool precise = sizeof(T) == 4 && eps_rel < kPreciseBelow;
  const bool same_shape = B.Q && B.rows == rows && B.dtype == dtype;
  if (!same_shape || c_split < B.covered || B.precise != precise) {
    if (!same_shape) {
      if (B.Q) cudaFree(B.Q);
      B.Q = nullptr;
      JLS_CHECK_CUDA(cudaMalloc(&B.Q, (size_t)rows * h->d_max * sizeof(T)));
    }
    JLS_CHECK_CUDA(cudaMemsetAsync(B.Q, 0, (size_t)rows * h->d_max * sizeof(T), s));
    B.rows = rows;
    B.dtype = dtype;
    B.cols = 0;
    B.covered = 0;
  }
  B.precise = precise;
  if (!h->host_norms[slot]) JLS_CHECK_CUDA(cudaMallocHost(&h->host_norms[slot], 2 * NORM_GRID * sizeof(double)));
  if (!h->norms_ready[slot]) JLS_CHECK_CUDA(cudaEventCreateWithFlags(&h->norms_ready[slot], cudaEventDisableTiming));
  const int bt = c_end - c_split;
  const int wmax = std::max(64, bt);
  if (bt > 512) return SK_ERR_UNSUPPORTED;
  const int nchunks = (int)std::min<int64_t>(64, (rows + 511) / 512);
  Scratch sc;
  JLS_CHECK(ensure_scratch(h, slot, rows, dtype, wmax, &sc, nchunks));
  T* W = static_cast<T*>(sc.W);
  const unsigned cgrid = (unsigned)(4 * num_sms());
  // columns [covered, c_split) not in Q yet, 64 at a time
  while (B.covered < c_split) {
    const int b = std::min(64, c_split - B.covered);
    copy_block_kernel<T><<<cgrid, 256, 0, s>>>(S + B.covered, ldS, W, 64, rows, b); note_launch();
    JLS_CHECK(sumsq_launch<T>(W, 64, rows, b, sc.ref, s));
    if (precise) JLS_CHECK(colsumsq_launch<T>(W, 64, rows, b, sc.colref, s));
    JLS_CHECK(absorb_block<T>(h, B, W, 64, b, rows, sc, nchunks, true, sc.ref, s, nullptr,
                              precise ? sc.colref : nullptr, b));
    B.covered += b;
  }
  // the test block: both norms summed on the device
  copy_block_kernel<T><<<cgrid, 256, 0, s>>>(S + c_split, ldS, W, wmax, rows, bt); note_launch();
  JLS_CHECK_CUDA(cudaGetLastError());
  JLS_CHECK(sumsq_launch<T>(W, wmax, rows, bt, sc.norms, s));
  if (precise) JLS_CHECK(colsumsq_launch<T>(W, wmax, rows, bt, sc.colref, s));
  const double* cref = precise ? sc.colref : nullptr;
  if (bt <= 64) {  // one chunk: ||S^|| from its absorption's first Gram matrix
    const TestOut out{sc.norms, h->host_norms[slot], h->norms_ready[slot]};
    JLS_CHECK(absorb_block<T>(h, B, W, wmax, bt, rows, sc, nchunks, true, sc.norms, s, &out, cref, bt));
    B.covered = c_end;
    return SK_OK;
  }
  JLS_CHECK(project_twice<T>(h, B, W, wmax, bt, rows, sc, nchunks, s));
  JLS_CHECK(sumsq_launch<T>(W, wmax, rows, bt, sc.norms + NORM_GRID, s));
  JLS_CHECK_CUDA(cudaMemcpyAsync(h->host_norms[slot], sc.norms, 2 * NORM_GRID * sizeof(double), cudaMemcpyDeviceToHost,
                                 s));
  JLS_CHECK_CUDA(cudaEventRecord(h->norms_ready[slot], s));
  // extend Q by S^ (64 columns at a time; later chunks are first made
  // orthogonal to the chunks just added)
  for (int j0 = 0; j0 < bt; j0 += 64) {
    const int b = std::min(64, bt - j0);
    JLS_CHECK(absorb_block<T>(h, B, W + j0, wmax, b, rows, sc, nchunks, j0 > 0, sc.norms, s, nullptr,
                              cref ? cref + j0 : nullptr, bt));
  }
  B.covered = c_end;
  return SK_OK;
}

}  // namespace

int norm_test_enqueue(sk_op* h, int slot, const void* S, int64_t rows, int64_t ldS, int dtype, double eps_rel,
                      int c_split, int c_end, cudaStream_t s) {
  if (dtype == SK_F32)
    return norm_test_enqueue_t<float>(h, slot, (const float*)S, rows, ldS, dtype, eps_rel, c_split, c_end, s);
  return norm_test_enqueue_t<double>(h, slot, (const double*)S, rows, ldS, dtype, eps_rel, c_split, c_end, s);
}

int norm_test_finish(sk_op* h, int slot, double eps_rel, double eps_abs, int* stop, double* nh, double* nt) {
  JLS_CHECK_CUDA(cudaEventSynchronize(h->norms_ready[slot]));
  double t2 = 0, h2 = 0;
  const double* hn = h->host_norms[slot];
  for (int i = 0; i < NORM_GRID; ++i) {  // fixed order: deterministic
    t2 += hn[i];
    h2 += hn[NORM_GRID + i];
  }
  *nt = std::sqrt(t2);
  *nh = std::sqrt(h2);
  *stop = (*nh < eps_abs) || (*nh < eps_rel * *nt);
  return SK_OK;
}

int norm_test(sk_op* h, int slot, const void* S, int64_t rows, int64_t ldS, int dtype, int c_split, int c_end,
              double eps_rel, double eps_abs, int* stop, double* nh, double* nt, cudaStream_t s) {
  JLS_CHECK(norm_test_enqueue(h, slot, S, rows, ldS, dtype, eps_rel, c_split, c_end, s));
  return norm_test_finish(h, slot, eps_rel, eps_abs, stop, nh, nt);
}

}  // namespace jls

// ---------------------------------------------------------------------------
// Allocation-free variant of the stopping test's projection and norms.
//
// Some callers cannot allocate device memory: processes whose device memory
// is fully owned by another allocator or pool, and callers that must not block
// on the device-wide synchronization cudaMalloc/cudaFree imply.  (Code inside
// CUDA stream capture is not served: the call reads its norms back to the host
// and synchronizes its stream.)  For them,
// sketch_project_norms_noalloc takes its scratch (the tall-skinny product's
// partial sums, the reduced product Q^T S and the norm partials) from the
// file-scope array below instead of a handle.  Every GPU that loads the library
// holds this array until the process exits.
namespace jls {
namespace {

constexpr int NOALLOC_MAX_Q = 1024;  // columns of Q
constexpr int NOALLOC_MAX_B = 64;    // columns of S~
constexpr int NOALLOC_CHUNKS = 8;    // row chunks of the partial products
constexpr size_t NOALLOC_PART = (size_t)NOALLOC_CHUNKS * NOALLOC_MAX_Q * NOALLOC_MAX_B;
constexpr size_t NOALLOC_G = (size_t)NOALLOC_MAX_Q * NOALLOC_MAX_B;
constexpr size_t NOALLOC_DOUBLES = NOALLOC_PART + NOALLOC_G + NORM_GRID;  // 4.5 MiB

}  // namespace

static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_DOUBLES];

namespace {

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};

// Device address of g_noalloc_scratch for the current device.  In host code
// the array's name is only a host-side stand-in, so the address is looked up
// once per device (with that device current) and cached.
int noalloc_scratch(double** out) {
  int dev = 0;
  JLS_CHECK_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return SK_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    JLS_CHECK_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_noalloc_ptr[dev];
  return SK_OK;
}

template <typename T>
int sumsq_noalloc(const T* W, int64_t ldw, int64_t rows, int b, double* partials, double* out, cudaStream_t s) {
  sumsq_partial<T><<<NORM_GRID, 256, 0, s>>>(W, ldw, rows, b, partials); note_launch();
  JLS_CHECK_CUDA(cudaGetLastError());
  double part[NORM_GRID];
  JLS_CHECK_CUDA(cudaMemcpyAsync(part, partials, sizeof(part), cudaMemcpyDeviceToHost, s));
  JLS_CHECK_CUDA(cudaStreamSynchronize(s));
  double acc = 0;
  for (int i = 0; i < NORM_GRID; ++i) acc += part[i];  // fixed order: deterministic
  *out = acc;
  return SK_OK;
}

template <typename T>
int project_norms_noalloc_t(const T* Q, int64_t ldQ, int q_cols, const T* St, int64_t ldS, int64_t rows, int b,
                            T* Sh, int64_t ldH, double* nh, double* nt, cudaStream_t s) {
  double* scratch = nullptr;
  JLS_CHECK(noalloc_scratch(&scratch));
  double* part = scratch;
  double* G = scratch + NOALLOC_PART;
  double* norms = G + NOALLOC_G;
  copy_block_kernel<T><<<(unsigned)(4 * num_sms()), 256, 0, s>>>(St, ldS, Sh, ldH, rows, b); note_launch();
  JLS_CHECK_CUDA(cudaGetLastError());
  double t2 = 0, h2 = 0;
  JLS_CHECK(sumsq_noalloc<T>(Sh, ldH, rows, b, norms, &t2, s));
  for (int pass = 0; pass < 2 && q_cols > 0; ++pass) {  // S^ <- (I - Q Q^T) S^, twice
    JLS_CHECK(tsgemm<T>(Q, ldQ, q_cols, Sh, ldH, b, rows, NOALLOC_CHUNKS, part, G, s));
    JLS_CHECK(sub_qg<T>(Sh, ldH, b, Q, ldQ, q_cols, G, rows, s));
  }
  JLS_CHECK(sumsq_noalloc<T>(Sh, ldH, rows, b, norms, &h2, s));
  *nt = std::sqrt(t2);
  *nh = std::sqrt(h2);
  return SK_OK;
}

}  // namespace

}  // namespace jls

extern "C" int sketch_project_norms_noalloc(const void* Q, int64_t ldQ, int32_t q_cols, const void* S_tilde,
                                            int64_t ldS, int64_t rows, int32_t b, int32_t dtype, void* S_hat,
                                            int64_t ldH, double eps_rel, double eps_abs, int32_t* stop,
                                            double* norm_hat, double* norm_tilde, void* stream) {
  using namespace jls;
  if (!S_tilde || !S_hat || !stop || rows < 1 || b < 1 || q_cols < 0 || ldS < b || ldH < b) return SK_ERR_INVALID_ARG;
  if (b > NOALLOC_MAX_B || q_cols > NOALLOC_MAX_Q) return SK_ERR_INVALID_ARG;  // beyond the static scratch
  if (q_cols > 0 && (!Q || ldQ < q_cols)) return SK_ERR_INVALID_ARG;
  if (dtype != SK_F32 && dtype != SK_F64) return SK_ERR_DTYPE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double nh = 0, nt = 0;
  if (dtype == SK_F32)
    JLS_CHECK(project_norms_noalloc_t<float>(static_cast<const float*>(Q), ldQ, q_cols,
                                             static_cast<const float*>(S_tilde), ldS, rows, b,
                                             static_cast<float*>(S_hat), ldH, &nh, &nt, s));
  else
    JLS_CHECK(project_norms_noalloc_t<double>(static_cast<const double*>(Q), ldQ, q_cols,
                                              static_cast<const double*>(S_tilde), ldS, rows, b,
                                              static_cast<double*>(S_hat), ldH, &nh, &nt, s));
  *stop = (nh < eps_abs) || (nh < eps_rel * nt);
  if (norm_hat) *norm_hat = nh;
  if (norm_tilde) *norm_tilde = nt;
  return SK_OK;
}
