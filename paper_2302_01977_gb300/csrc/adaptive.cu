// adaptive.cu -- increment rescale and the Frobenius stopping test.
//
// Stopping test (Eq. (3.1) with the two-pass projection of the
// remark after it; Algorithm 1's S~ = last Delta-d columns):
//   S^ = (I - Q Q^T)^2 S~,  stop = ||S^||_F < eps_abs or ||S^||_F < eps_rel ||S~||_F.
// Q is an orthonormal basis of the earlier sketch columns kept per handle and
// slot.  New columns are absorbed 64 at a time: two block Gram-Schmidt passes
// against Q, then two Cholesky-QR passes (Gram matrix and factor in FP64; a
// pivot below 1e-13 of the largest drops that column, so a rank-deficient
// block adds zero columns to Q, which do not change Q Q^T).
//
// Tall-skinny products X^T Y (rows ~ n, widths <= 512) run on CUDA cores: each
// CTA reduces a chunk of rows into a 32 x 32 tile of partial sums, chunks are
// summed in FP64 by a second kernel.  Frobenius norms are FP64 sums of squares.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace jls {

// ---------------------------------------------------------------------------
template <typename T>
__global__ void scale_cols_kernel(T* S, int64_t rows, int64_t ld, int c0, int c1, T f) {
  const int w = c1 - c0;
  const int64_t total = rows * w;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = q / w;
    const int c = (int)(q % w);
    S[r * ld + c0 + c] *= f;
  }
}

int scale_columns(void* S, int dtype, int64_t rows, int64_t ld, int c0, int c1, double factor, cudaStream_t s) {
  if (c1 <= c0) return SK_OK;
  const unsigned grid = 152 * 8;
  if (dtype == SK_F32)
    scale_cols_kernel<float><<<grid, 256, 0, s>>>((float*)S, rows, ld, c0, c1, (float)factor);
  else
    scale_cols_kernel<double><<<grid, 256, 0, s>>>((double*)S, rows, ld, c0, c1, factor); note_launch();
  JLS_CHECK_CUDA(cudaGetLastError());
  return SK_OK;
}

// ---------------------------------------------------------------------------
// partial[chunk][i][j] = sum_{r in chunk} X[r][i] * Y[r][j]   (i < p, j < q)
template <typename T>
__global__ void __launch_bounds__(256)
    tsgemm_tn_partial(const T* __restrict__ X, int64_t ldx, int p, const T* __restrict__ Y, int64_t ldy, int q,
                      int64_t rows, int64_t rows_per_chunk, double* __restrict__ part) {
  __shared__ T xs[32][33];
  __shared__ T ys[32][33];
  const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
  const int64_t r_begin = (int64_t)blockIdx.z * rows_per_chunk;
  const int64_t r_end = min64(rows, r_begin + rows_per_chunk);
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // ty in 0..7
  T acc[4] = {T(0), T(0), T(0), T(0)};
  for (int64_t r0 = r_begin; r0 < r_end; r0 += 32) {
    for (int rr = ty; rr < 32; rr += 8) {
      const int64_t r = r0 + rr;
      xs[rr][tx] = (r < r_end && i0 + tx < p) ? X[r * ldx + i0 + tx] : T(0);
      ys[rr][tx] = (r < r_end && j0 + tx < q) ? Y[r * ldy + j0 + tx] : T(0);
    }
    __syncthreads();
#pragma unroll 8
    for (int rr = 0; rr < 32; ++rr) {
      const T yv = ys[rr][tx];
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] = fma(xs[rr][ty + 8 * u], yv, acc[u]);
    }
    __syncthreads();
  }
  double* out = part + (int64_t)blockIdx.z * p * q;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = i0 + ty + 8 * u, j = j0 + tx;
    if (i < p && j < q) out[(int64_t)i * q + j] = (double)acc[u];
  }
}

__global__ void reduce_partials(const double* __restrict__ part, int nchunks, int64_t count, double* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
    double s = 0;
    for (int c = 0; c < nchunks; ++c) s += part[(int64_t)c * count + e];
    out[e] = s;
  }
}

// W[r][j] -= sum_i Q[r][i] * G[i][j]   (G is p x q in FP64, q <= 64)
template <typename T>
__global__ void __launch_bounds__(256)
    sub_qg_kernel(T* __restrict__ W, int64_t ldw, int q, const T* __restrict__ Q, int64_t ldq, int p,
                  const double* __restrict__ G, int64_t rows) {
  __shared__ T gs[32][64];
  __shared__ T qs[32][33];
  const int64_t r0 = (int64_t)blockIdx.x * 32;
  const int j = threadIdx.x & 63, rg = threadIdx.x >> 6;  // rg 0..3 -> 8 rows each
  T acc[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) acc[u] = T(0);
  for (int i0 = 0; i0 < p; i0 += 32) {
    for (int e = threadIdx.x; e < 32 * 64; e += 256) {
      const int ii = e / 64, jj = e % 64;
      gs[ii][jj] = (i0 + ii < p && jj < q) ? (T)G[(int64_t)(i0 + ii) * q + jj] : T(0);
    }
    for (int e = threadIdx.x; e < 32 * 32; e += 256) {
      const int rr = e / 32, ii = e % 32;
      const int64_t r = r0 + rr;
      qs[rr][ii] = (r < rows && i0 + ii < p) ? Q[r * ldq + i0 + ii] : T(0);
    }
    __syncthreads();
#pragma unroll 4
    for (int ii = 0; ii < 32; ++ii) {
      const T g = gs[ii][j];
#pragma unroll
      for (int u = 0; u < 8; ++u) acc[u] = fma(qs[rg * 8 + u][ii], g, acc[u]);
    }
    __syncthreads();
  }
  if (j < q)
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int64_t r = r0 + rg * 8 + u;
      if (r < rows) W[r * ldw + j] -= acc[u];
    }
}

// Cholesky of the b x b (b <= 64) FP64 Gram matrix with column dropping, then
// U = L^{-T} (upper triangular, dropped columns zero).  One CTA of 64 threads.
__global__ void chol_inv_kernel(const double* __restrict__ Gm, int b, double* __restrict__ U, int* err) {
  extern __shared__ double chol_sh[];
  double (*L)[65] = reinterpret_cast<double (*)[65]>(chol_sh);
  double (*Li)[65] = reinterpret_cast<double (*)[65]>(chol_sh + 64 * 65);
  __shared__ int drop[64];
  const int t = threadIdx.x;
  for (int i = 0; i < b; ++i)
    if (t < b) L[i][t] = Gm[i * b + t];
  __syncthreads();
  double dmax = 0;
  for (int i = 0; i < b; ++i) dmax = fmax(dmax, L[i][i]);
  for (int k = 0; k < b; ++k) {
    __syncthreads();
    const double pk = L[k][k];
    const bool dk = !(pk > 1e-26 * dmax) || !(dmax > 0);
    if (t == 0) drop[k] = dk;
    __syncthreads();
    const double sq = dk ? 0.0 : sqrt(pk);
    if (t >= k && t < b) L[t][k] = dk ? 0.0 : L[t][k] / sq;  // column k of L (L[k][k] = sqrt)
    __syncthreads();
    if (t > k && t < b)
      for (int j = k + 1; j <= t; ++j) L[t][j] -= L[t][k] * L[j][k];
  }
  __syncthreads();
  // Li = L^{-1} (lower), column by column: thread t solves column t
  if (t < b) {
    for (int i = 0; i < b; ++i) Li[i][t] = 0.0;
    if (!drop[t]) {
      Li[t][t] = 1.0 / L[t][t];
      for (int i = t + 1; i < b; ++i) {
        if (drop[i]) continue;
        double sacc = 0;
        for (int k = t; k < i; ++k) sacc += L[i][k] * Li[k][t];
        Li[i][t] = -sacc / L[i][i];
      }
    }
  }
  __syncthreads();
  // U = Li^T : U[i][j] = Li[j][i]
  if (t < b)
    for (int i = 0; i < b; ++i) U[i * b + t] = Li[t][i];
  (void)err;
}

// Wout[r][j] = sum_{i <= j} W[r][i] * U[i][j]  (b <= 64), U FP64; 16 rows per CTA
template <typename T>
__global__ void __launch_bounds__(256)
    mul_upper_kernel(const T* __restrict__ W, int64_t ldw, const double* __restrict__ U, int b, T* __restrict__ Wo,
                     int64_t ldo, int64_t rows) {
  __shared__ T us[64][64];
  __shared__ T ws[16][65];
  for (int e = threadIdx.x; e < 64 * 64; e += 256) {
    const int i = e / 64, j = e % 64;
    us[i][j] = (i < b && j < b) ? (T)U[i * b + j] : T(0);
  }
  const int64_t r0 = (int64_t)blockIdx.x * 16;
  for (int e = threadIdx.x; e < 16 * 64; e += 256) {
    const int rr = e / 64, i = e % 64;
    const int64_t r = r0 + rr;
    ws[rr][i] = (r < rows && i < b) ? W[r * ldw + i] : T(0);
  }
  __syncthreads();
  const int j = threadIdx.x & 63, rg = threadIdx.x >> 6;
  for (int u = 0; u < 4; ++u) {
    const int rr = rg * 4 + u;
    const int64_t r = r0 + rr;
    T acc = T(0);
    for (int i = 0; i <= j && i < b; ++i) acc = fma(ws[rr][i], us[i][j], acc);
    if (r < rows && j < b) Wo[r * ldo + j] = acc;
  }
}

template <typename T>
__global__ void copy_block_kernel(const T* __restrict__ src, int64_t lds, T* __restrict__ dst, int64_t ldd,
                                  int64_t rows, int b) {
  const int64_t total = rows * b;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / b;
    const int c = (int)(e % b);
    dst[r * ldd + c] = src[r * lds + c];
  }
}

template <typename T>
__global__ void sumsq_partial(const T* __restrict__ W, int64_t ldw, int64_t rows, int b, double* __restrict__ part) {
  __shared__ double red[256];
  double s = 0;
  const int64_t total = rows * b;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const double v = (double)W[(e / b) * ldw + (e % b)];
    s += v * v;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// ---------------------------------------------------------------------------
namespace {

constexpr int NORM_GRID = 256;
constexpr int CHOL_SMEM = 2 * 64 * 65 * sizeof(double);

struct Scratch {
  void* W;        // rows x wmax (T)
  void* W2;       // rows x 64 (T)
  double* part;   // partial products
  double* G;      // up to d_max x wmax
  double* U;      // 64 x 64
  double* norms;  // NORM_GRID partials
  size_t part_elems;
};

int ensure_scratch(sk_op* h, int64_t rows, int dtype, int wmax, Scratch* sc, int nchunks) {
  const size_t es = elem_size(dtype);
  const size_t wb = ((size_t)rows * wmax * es + 255) / 256 * 256;
  const size_t w2b = ((size_t)rows * 64 * es + 255) / 256 * 256;
  const size_t part_elems = (size_t)nchunks * h->d_max * wmax;
  const size_t gb = (size_t)h->d_max * wmax * sizeof(double);
  const size_t need = wb + w2b + part_elems * sizeof(double) + gb + 64 * 64 * sizeof(double) + NORM_GRID * sizeof(double);
  if (h->scratch_bytes < need) {
    if (h->scratch) cudaFree(h->scratch);
    h->scratch = nullptr;
    h->scratch_bytes = 0;
    JLS_CHECK_CUDA(cudaMalloc(&h->scratch, need));
    h->scratch_bytes = need;
  }
  uint8_t* p = static_cast<uint8_t*>(h->scratch);
  sc->W = p;
  p += wb;
  sc->W2 = p;
  p += w2b;
  sc->part = reinterpret_cast<double*>(p);
  p += part_elems * sizeof(double);
  sc->G = reinterpret_cast<double*>(p);
  p += gb;
  sc->U = reinterpret_cast<double*>(p);
  p += 64 * 64 * sizeof(double);
  sc->norms = reinterpret_cast<double*>(p);
  sc->part_elems = part_elems;
  return SK_OK;
}

template <typename T>
int tsgemm(const T* X, int64_t ldx, int p, const T* Y, int64_t ldy, int q, int64_t rows, int nchunks, double* part,
           double* out, cudaStream_t s) {
  const int64_t rpc = ((rows + nchunks - 1) / nchunks + 31) / 32 * 32;
  const int nch = (int)((rows + rpc - 1) / rpc);
  dim3 grid((p + 31) / 32, (q + 31) / 32, nch);
  tsgemm_tn_partial<T><<<grid, 256, 0, s>>>(X, ldx, p, Y, ldy, q, rows, rpc, part); note_launch();
  reduce_partials<<<64, 256, 0, s>>>(part, nch, (int64_t)p * q, out); note_launch();
  JLS_CHECK_CUDA(cudaGetLastError());
  return SK_OK;
}

// W (rows x b, ld ldw) <- (I - Q Q^T)^2 W
template <typename T>
int project_twice(const sk_op* h, const Basis& B, T* W, int64_t ldw, int b, int64_t rows, const Scratch& sc,
                  int nchunks, cudaStream_t s) {
  if (B.cols == 0) return SK_OK;
  const T* Q = static_cast<const T*>(B.Q);
  for (int pass = 0; pass < 2; ++pass) {
    JLS_CHECK(tsgemm<T>(Q, h->d_max, B.cols, W, ldw, b, rows, nchunks, sc.part, sc.G, s));
    for (int j0 = 0; j0 < b; j0 += 64) {
      // G is B.cols x b row-major; sub_qg reads a 64-column slab via a shifted base
      const int q = std::min(64, b - j0);
      // copy the slab into contiguous form expected by sub_qg (ld = q)
      // (sub_qg indexes G[i * q + j]); reuse part as staging
      double* slab = sc.part;
      dim3 g1((unsigned)((B.cols * 64 + 255) / 256));
      copy_block_kernel<double><<<g1, 256, 0, s>>>(sc.G + j0, b, slab, q, B.cols, q); note_launch();
      sub_qg_kernel<T><<<(unsigned)((rows + 31) / 32), 256, 0, s>>>(W + j0, ldw, q, Q, h->d_max, B.cols, slab, rows); note_launch();
    }
    JLS_CHECK_CUDA(cudaGetLastError());
  }
  return SK_OK;
}

template <typename T>
int sumsq(const T* W, int64_t ldw, int64_t rows, int b, const Scratch& sc, double* out, cudaStream_t s) {
  sumsq_partial<T><<<NORM_GRID, 256, 0, s>>>(W, ldw, rows, b, sc.norms); note_launch();
  JLS_CHECK_CUDA(cudaGetLastError());
  double part[NORM_GRID];
  JLS_CHECK_CUDA(cudaMemcpyAsync(part, sc.norms, sizeof(part), cudaMemcpyDeviceToHost, s));
  JLS_CHECK_CUDA(cudaStreamSynchronize(s));
  double acc = 0;
  for (int i = 0; i < NORM_GRID; ++i) acc += part[i];  // fixed order: deterministic
  *out = acc;
  return SK_OK;
}

template <typename T>
int norm_test_t(sk_op* h, int slot, const T* S, int64_t rows, int64_t ldS, int dtype, int c_split, int c_end,
                double eps_rel, double eps_abs, int* stop, double* nh, double* nt, cudaStream_t s) {
  Basis& B = h->basis[slot];
  if (!B.Q || B.rows != rows || B.dtype != dtype || c_split < B.covered) {
    if (B.Q) cudaFree(B.Q);
    B.Q = nullptr;
    JLS_CHECK_CUDA(cudaMalloc(&B.Q, (size_t)rows * h->d_max * sizeof(T)));
    JLS_CHECK_CUDA(cudaMemsetAsync(B.Q, 0, (size_t)rows * h->d_max * sizeof(T), s));
    B.rows = rows;
    B.dtype = dtype;
    B.cols = 0;
    B.covered = 0;
  }
  const int bt = c_end - c_split;
  const int wmax = std::max(64, bt);
  if (bt > 512) return SK_ERR_UNSUPPORTED;
  const int nchunks = (int)std::min<int64_t>(64, (rows + 511) / 512);
  Scratch sc;
  JLS_CHECK(ensure_scratch(h, rows, dtype, wmax, &sc, nchunks));
  static bool chol_attr = false;
  if (!chol_attr) {
    JLS_CHECK_CUDA(cudaFuncSetAttribute(chol_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, CHOL_SMEM));
    chol_attr = true;
  }
  T* W = static_cast<T*>(sc.W);
  T* W2 = static_cast<T*>(sc.W2);
  T* Q = static_cast<T*>(B.Q);
  const unsigned cgrid = 152 * 4;
  // absorb columns [covered, c_split) into Q, 64 at a time
  while (B.covered < c_split) {
    const int b = std::min(64, c_split - B.covered);
    copy_block_kernel<T><<<cgrid, 256, 0, s>>>(S + B.covered, ldS, W, 64, rows, b); note_launch();
    JLS_CHECK(project_twice<T>(h, B, W, 64, b, rows, sc, nchunks, s));
    for (int pass = 0; pass < 2; ++pass) {  // Cholesky QR twice
      JLS_CHECK(tsgemm<T>(W, 64, b, W, 64, b, rows, nchunks, sc.part, sc.G, s));
      chol_inv_kernel<<<1, 64, CHOL_SMEM, s>>>(sc.G, b, sc.U, h->d_err); note_launch();
      mul_upper_kernel<T><<<(unsigned)((rows + 15) / 16), 256, 0, s>>>(W, 64, sc.U, b, W2, 64, rows); note_launch();
      copy_block_kernel<T><<<cgrid, 256, 0, s>>>(W2, 64, W, 64, rows, b); note_launch();
    }
    copy_block_kernel<T><<<cgrid, 256, 0, s>>>(W, 64, Q + B.cols, h->d_max, rows, b); note_launch();
    JLS_CHECK_CUDA(cudaGetLastError());
    B.cols += b;
    B.covered += b;
  }
  // the test block
  copy_block_kernel<T><<<cgrid, 256, 0, s>>>(S + c_split, ldS, W, wmax, rows, bt); note_launch();
  JLS_CHECK_CUDA(cudaGetLastError());
  double t2 = 0, h2 = 0;
  JLS_CHECK(sumsq<T>(W, wmax, rows, bt, sc, &t2, s));
  JLS_CHECK(project_twice<T>(h, B, W, wmax, bt, rows, sc, nchunks, s));
  JLS_CHECK(sumsq<T>(W, wmax, rows, bt, sc, &h2, s));
  *nt = std::sqrt(t2);
  *nh = std::sqrt(h2);
  *stop = (*nh < eps_abs) || (*nh < eps_rel * *nt);
  return SK_OK;
}

}  // namespace

int norm_test(sk_op* h, int slot, const void* S, int64_t rows, int64_t ldS, int dtype, int c_split, int c_end,
              double eps_rel, double eps_abs, int* stop, double* nh, double* nt, cudaStream_t s) {
  if (dtype == SK_F32)
    return norm_test_t<float>(h, slot, (const float*)S, rows, ldS, dtype, c_split, c_end, eps_rel, eps_abs, stop,
                              nh, nt, s);
  return norm_test_t<double>(h, slot, (const double*)S, rows, ldS, dtype, c_split, c_end, eps_rel, eps_abs, stop,
                             nh, nt, s);
}

}  // namespace jls

// ---------------------------------------------------------------------------
// Allocation-free variant of the stopping test's projection and norms.
//
// Some callers cannot allocate device memory: code running inside CUDA stream
// capture (where cudaMalloc would break the capture), processes whose device
// memory is fully owned by another allocator or pool, and callers that must
// not block on the synchronization cudaMalloc/cudaFree imply.  For them,
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
  copy_block_kernel<T><<<152 * 4, 256, 0, s>>>(St, ldS, Sh, ldH, rows, b); note_launch();
  JLS_CHECK_CUDA(cudaGetLastError());
  double t2 = 0, h2 = 0;
  JLS_CHECK(sumsq_noalloc<T>(Sh, ldH, rows, b, norms, &t2, s));
  for (int pass = 0; pass < 2 && q_cols > 0; ++pass) {  // S^ <- (I - Q Q^T) S^, twice
    JLS_CHECK(tsgemm<T>(Q, ldQ, q_cols, Sh, ldH, b, rows, NOALLOC_CHUNKS, part, G, s));
    sub_qg_kernel<T><<<(unsigned)((rows + 31) / 32), 256, 0, s>>>(Sh, ldH, b, Q, ldQ, q_cols, G, rows); note_launch();
    JLS_CHECK_CUDA(cudaGetLastError());
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
