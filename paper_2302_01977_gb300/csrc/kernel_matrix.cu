// kernel_matrix.cu -- explicit Gaussian kernel matrix
//   A_ij = exp(-||x_i - y_j||^2 / (2 h^2)) + shift * [i + diag_off == j]
// written row-major (diag_off places a block of rows inside a larger matrix).  Store-bound: one coalesced pass over A; the y points of
// a column block are staged in shared memory once per CTA.
#include "common.cuh"
#include "internal.h"

namespace jls {

__device__ __forceinline__ float kexp(float x) { return expf(x); }
__device__ __forceinline__ double kexp(double x) { return exp(x); }

template <typename T, int COLS_PER_CTA>
__global__ void __launch_bounds__(256)
    kernel_matrix_kernel(const T* __restrict__ X, const T* __restrict__ Y, int64_t rows, int64_t cols,
                         T neg_inv_2h2, T shift, int64_t diag_off, T* __restrict__ A, int64_t ld,
                         int rows_per_cta) {
  __shared__ T ys[3 * COLS_PER_CTA];
  const int64_t c0 = (int64_t)blockIdx.x * COLS_PER_CTA;
  const int ncols = (int)min64(COLS_PER_CTA, cols - c0);
  for (int q = threadIdx.x; q < 3 * ncols; q += blockDim.x) ys[q] = Y[c0 * 3 + q];
  __syncthreads();
  const int64_t r_begin = (int64_t)blockIdx.y * rows_per_cta;
  const int64_t r_end = min64(rows, r_begin + rows_per_cta);
  for (int64_t i = r_begin; i < r_end; ++i) {
    const T x0 = X[3 * i], x1 = X[3 * i + 1], x2 = X[3 * i + 2];
    T* arow = A + i * ld + c0;
    for (int j = threadIdx.x; j < ncols; j += blockDim.x) {
      const T d0 = x0 - ys[3 * j], d1 = x1 - ys[3 * j + 1], d2 = x2 - ys[3 * j + 2];
      T a = kexp((d0 * d0 + d1 * d1 + d2 * d2) * neg_inv_2h2);
      if (i + diag_off == c0 + j) a += shift;
      arow[j] = a;
    }
  }
}

int launch_kernel_matrix(const sk_matrix* g, void* A, int64_t ld, cudaStream_t s, int64_t diag_off) {
  constexpr int CPC = 1024;
  const int rows_per_cta = 64;
  dim3 grid((unsigned)((g->cols + CPC - 1) / CPC), (unsigned)((g->rows + rows_per_cta - 1) / rows_per_cta));
  if (grid.y > 65535) return SK_ERR_UNSUPPORTED;
  const double nih = -1.0 / (2.0 * g->h * g->h);
  if (g->dtype == SK_F32)
    kernel_matrix_kernel<float, CPC><<<grid, 256, 0, s>>>(static_cast<const float*>(g->X),
                                                         static_cast<const float*>(g->Y), g->rows, g->cols,
                                                         (float)nih, (float)g->shift, diag_off,
                                                         static_cast<float*>(A), ld, rows_per_cta);
  else
    kernel_matrix_kernel<double, CPC><<<grid, 256, 0, s>>>(static_cast<const double*>(g->X),
                                                          static_cast<const double*>(g->Y), g->rows, g->cols,
                                                          nih, g->shift, diag_off, static_cast<double*>(A), ld,
                                                          rows_per_cta); note_launch();
  JLS_CHECK_CUDA(cudaGetLastError());
  return SK_OK;
}

}  // namespace jls
