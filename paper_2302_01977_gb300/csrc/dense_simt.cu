// dense_simt.cu -- SRHT and Gaussian sketches on CUDA cores (FP32 or FP64).
//
//   S  = scale * A   * B     (Sec. 6.3 "A R")
//   S' = scale * A^T * B     (Sec. 6.3 "A* R", real A)
// with B the unscaled operator: Gaussian z (N(0,1), Sec. 2.4.1) read from the
// stored plane, or the SRHT sign pattern d_k (-1)^popc(k & mu_c) (the element formula of Sec. 7.2)
// generated while the B tile is staged.  This is the plain path the tensor-core
// split path is measured against, and the FP64 path.  Tiles of 128 x 64
// outputs over K steps of 16, 256 threads with 8 x 4 outputs each; FP32 sums
// are kept in two levels (a chunk of 256 K values, then the running total) to
// keep the rounding of long (n = 32768) reductions near the chunk level.
#include "common.cuh"
#include "internal.h"

namespace jls {

namespace {
constexpr int BM = 128, BN = 64, BK = 16, TM = 8, TN = 4;
constexpr int CHUNK_K = 256;
}

// CPLX (S = A R for complex A, real operator): A is the real view of the
// complex matrix (K = 2n interleaved (re, im) columns) and B the operator
// R (x) I_2: B[k][c] = R[k / 2][c / 2] when k and c have the same parity, 0
// otherwise; the output columns c are the interleaved (re, im) parts of S's.
template <typename T, bool TRANS, bool SRHT, bool CPLX = false>
__global__ void __launch_bounds__(256)
    dense_simt_kernel(const T* __restrict__ A, int64_t lda, int64_t M, int64_t K, const T* __restrict__ zt,
                      const int8_t* __restrict__ diag, const int32_t* __restrict__ mu, int64_t n, int c_lo,
                      int c_hi, T scale, T* __restrict__ C, int64_t ldc) {
  __shared__ T As[BK][BM + 4];
  __shared__ T Bs[BK][BN + 4];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t m0 = (int64_t)blockIdx.x * BM;
  const int c0 = c_lo + blockIdx.y * BN;

  T acc[TM][TN], chunk[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = chunk[i][j] = T(0);

  for (int64_t k0 = 0; k0 < K; k0 += BK) {
    // ---- A tile -> As[kk][mm]
    for (int q = tid; q < BM * BK; q += 256) {
      int mm, kk;
      if (TRANS) {  // A[k][m], contiguous in m
        mm = q % BM;
        kk = q / BM;
      } else {  // A[m][k], contiguous in k
        kk = q % BK;
        mm = q / BK;
      }
      const int64_t gm = m0 + mm, gk = k0 + kk;
      T v = T(0);
      if (gm < M && gk < K) v = TRANS ? A[gk * lda + gm] : A[gm * lda + gk];
      As[kk][mm] = v;
    }
    // ---- B tile -> Bs[kk][cc]
    for (int q = tid; q < BN * BK; q += 256) {
      const int kk = q % BK, cc = q / BK;
      const int64_t gk = k0 + kk;
      const int gc = c0 + cc;
      T v = T(0);
      if (gk < K && gc < c_hi && (!CPLX || ((gk ^ gc) & 1) == 0)) {
        const int64_t rk = CPLX ? (gk >> 1) : gk;
        const int rc = CPLX ? (gc >> 1) : gc;
        if (SRHT) {
          const int neg = (__popcll((unsigned long long)rk & (unsigned long long)(uint32_t)mu[rc]) & 1) ^
                          (diag[rk] < 0);
          v = neg ? T(-1) : T(1);
        } else {
          v = zt[(int64_t)rc * n + rk];
        }
      }
      Bs[kk][cc] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty * TM + i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx * TN + j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) chunk[i][j] = fma(a[i], b[j], chunk[i][j]);
    }
    __syncthreads();
    if (((k0 + BK) % CHUNK_K) == 0) {
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) {
          acc[i][j] += chunk[i][j];
          chunk[i][j] = T(0);
        }
    }
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int64_t gm = m0 + ty * TM + i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int gc = c0 + tx * TN + j;
      if (gc < c_hi) C[gm * ldc + gc] = (acc[i][j] + chunk[i][j]) * scale;
    }
  }
}

template <typename T>
static int launch_dense(sk_op* h, const sk_matrix* A, bool trans, int c_lo, int c_hi, T scale, T* C, int64_t ldc,
                        cudaStream_t s) {
  const int64_t M = trans ? A->cols : A->rows;
  const int64_t K = trans ? A->rows : A->cols;
  dim3 grid((unsigned)((M + BM - 1) / BM), (unsigned)((c_hi - c_lo + BN - 1) / BN));
  const T* zt = nullptr;
  if (h->kind == SK_GAUSS) zt = sizeof(T) == 4 ? (const T*)h->z32 : (const T*)h->z64;
  const T* a = static_cast<const T*>(A->A);
#define JLS_LAUNCH(TR, SR)                                                                                      \
  dense_simt_kernel<T, TR, SR><<<grid, 256, 0, s>>>(a, A->ld, M, K, zt, h->srht_diag, h->srht_mu, h->n, c_lo, \
                                                    c_hi, scale, C, ldc)
  const bool srht = h->kind == SK_SRHT;
  if (trans && srht) JLS_LAUNCH(true, true);
  else if (trans) JLS_LAUNCH(true, false);
  else if (srht) JLS_LAUNCH(false, true);
  else JLS_LAUNCH(false, false);
#undef JLS_LAUNCH
  note_launch();
  JLS_CHECK_CUDA(cudaGetLastError());
  return SK_OK;
}

// S = A R for complex A (interleaved FP32 parts, rows x n complex) on CUDA
// cores: the real view times R (x) I_2, written straight into S's interleaved
// parts (columns [2 c_lo, 2 c_hi) of the real view of S).
int dense_apply_simt_complex_s(sk_op* h, const sk_matrix* A, int c_lo, int c_hi, double scale, void* S, int64_t ldS,
                               cudaStream_t s) {
  if (h->kind == SK_GAUSS) JLS_CHECK(gen_gauss(h, 0, h->d_total, s));
  const int64_t M = A->rows, K = 2 * A->cols;
  dim3 grid((unsigned)((M + BM - 1) / BM), (unsigned)((2 * (c_hi - c_lo) + BN - 1) / BN));
  const float* a = static_cast<const float*>(A->A);
  if (h->kind == SK_SRHT)
    dense_simt_kernel<float, false, true, true><<<grid, 256, 0, s>>>(
        a, 2 * A->ld, M, K, nullptr, h->srht_diag, h->srht_mu, h->n, 2 * c_lo, 2 * c_hi, (float)scale,
        static_cast<float*>(S), 2 * ldS);
  else
    dense_simt_kernel<float, false, false, true><<<grid, 256, 0, s>>>(
        a, 2 * A->ld, M, K, h->z32, h->srht_diag, h->srht_mu, h->n, 2 * c_lo, 2 * c_hi, (float)scale,
        static_cast<float*>(S), 2 * ldS);
  note_launch();
  JLS_CHECK_CUDA(cudaGetLastError());
  return SK_OK;
}

int dense_apply_simt(sk_op* h, const sk_matrix* A, int which, int c_lo, int c_hi, double scale, void* S,
                     int64_t ldS, void* St, int64_t ldSt, cudaStream_t s) {
  if (h->kind == SK_GAUSS) JLS_CHECK(gen_gauss(h, A->dtype == SK_F32 ? 0 : 1, h->d_total, s));
  if (A->dtype == SK_F32) {
    if (which & SK_S) JLS_CHECK(launch_dense<float>(h, A, false, c_lo, c_hi, (float)scale, (float*)S, ldS, s));
    if (which & SK_ST) JLS_CHECK(launch_dense<float>(h, A, true, c_lo, c_hi, (float)scale, (float*)St, ldSt, s));
  } else {
    if (which & SK_S) JLS_CHECK(launch_dense<double>(h, A, false, c_lo, c_hi, scale, (double*)S, ldS, s));
    if (which & SK_ST) JLS_CHECK(launch_dense<double>(h, A, true, c_lo, c_hi, scale, (double*)St, ldSt, s));
  }
  return SK_OK;
}

}  // namespace jls
