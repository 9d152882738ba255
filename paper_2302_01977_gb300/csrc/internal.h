// internal.h -- host-side declarations shared by the libjlsketch translation units.
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>

#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/jlsketch.h"

namespace jls {

// Tile sizes (rows of R per tile) of the tiled compressed-column structure,
// per element size (the S and S' SJLT kernels stage TILE rows or columns of A).
constexpr int SJLT_TILE_F32 = 128;
constexpr int SJLT_TILE_F64 = 64;
constexpr int SJLT_MAX_ALPHA = 32;
constexpr int MAX_D = 8192;
constexpr int MAX_BLOCKS = 256;  // SJLT blocks (initial + increments) a handle can hold

// Row pitch (elements) of the bf16 operator planes [c][k] read by the
// tensor-core path: rows start on 128-byte boundaries, as TMA wants.
__host__ __device__ inline int64_t bf_pitch(int64_t n) { return (n + 63) / 64 * 64; }
// Row pitch (bytes) of the e4m3 operator planes of the FP8 path.
__host__ __device__ inline int64_t f8_pitch(int64_t n) { return (n + 127) / 128 * 128; }
constexpr int F8_KTILE = 128;  // values of K per FP8 scale tile

// Tiled CCS of R (Sec. 6.1's compressed column storage, cut into tiles of
// `tile` rows): for tile t, entries[t*e_stride + p] sorted by column (rows
// ascending inside a column), and offs[t*o_stride + c] = first entry of
// column c (offs[.. + d_total] = count).  An entry for row r of the tile is a
// 16-byte record:
//   x = r * CCS_ROW_BYTES   (byte offset of row r in an S' kernel tile)
//   y, z = the sign as +-1.0 (FP32 tiles: the float twice; FP64 tiles: the
//          double's low and high words)
//   w = r * element size    (byte offset of column r in an S kernel tile row)
// In FP32 tiles x and w also carry the sign in bit 31, so the FP32 kernels
// read one 32-bit word per entry (a broadcast 4-byte shared load takes one
// shared-memory wavefront, a 16-byte one two); the FP64 kernels read the
// whole record.
constexpr int CCS_ROW_BYTES = 512;  // S' tiles: 128 FP32 or 64 FP64 columns per row
struct TiledCcs {
  int tile = 0;
  int built_d = -1;           // d_total it was built for
  int ntiles = 0;
  int64_t e_stride = 0;       // entries per tile
  int64_t o_stride = 0;       // uint32 offsets per tile (multiple of 4)
  uint4* ents = nullptr;
  uint32_t* offs = nullptr;
  size_t ents_cap = 0, offs_cap = 0;  // bytes
};

// Matrix-free S' tiles (sjlt_cols_kernel<..., GEN = true>): A_ij = K(p_i, q_j) =
// exp2(-c2 |p_i - q_j|^2) + shift [i == j], c2 = log2(e) / (2 h^2); P holds the
// points of the rows of R, Q the points of the output rows (FP32, 3 per point).
struct KGen {
  const float* P = nullptr;
  const float* Q = nullptr;
  float c2 = 0.f;
  float shift = 0.f;
};
// The matrix-free forward is bound by its tile-computing warps: measured at n =
// 262144, d = 256 with 16 warps per CTA, 3 producers 137 ms, 4 producers 112 ms
// (5 of 20 warps 111 ms, with spills); more warps in all only take issue slots
// from the producers (16 / 20 / 24 / 28 warps with 3 producers: 137 / 146 /
// 154 / 169 ms).
#ifndef GEN_WARPS_OVERRIDE
constexpr int GEN_WARPS = 4;   // tile-computing warps per CTA
#else
constexpr int GEN_WARPS = GEN_WARPS_OVERRIDE;
#endif
// Warps per CTA of the SJLT apply kernels and output columns per consumer warp
// (the accumulators of SJLT_NB columns, 4 values each, live in registers).  The
// consumers wait on shared-memory loads, so more warps with fewer columns each
// hide more latency; measured on GB300 (n = 32768, d = 256, S / S' ms):
// 16 x 20: 1.66 / 1.27, 20 x 16: 1.54 / 1.13, 24 x 12: 1.42 / 1.03,
// 28 x 10: 1.36 / 0.96, 32 x 9: 1.40 / 0.94 (72 registers per thread at 28).
#ifndef SJLT_WARPS_OVERRIDE
constexpr int SJLT_WARPS = 28;
constexpr int SJLT_NB = 10;
#else
constexpr int SJLT_WARPS = SJLT_WARPS_OVERRIDE;
constexpr int SJLT_NB = SJLT_NB_OVERRIDE;
#endif
// The tile-computing kernel keeps 16 warps (see GEN_WARPS).
#ifndef GEN_CTA_WARPS_OVERRIDE
constexpr int GEN_CTA_WARPS = 16;
#else
constexpr int GEN_CTA_WARPS = GEN_CTA_WARPS_OVERRIDE;
#endif
constexpr int GEN_JOBS = GEN_CTA_WARPS - GEN_WARPS;      // consumer warps beside the tile-computing ones
constexpr int GEN_NB = (256 + GEN_JOBS - 1) / GEN_JOBS;  // d = 256 in one launch

struct Basis {                // orthonormal basis Q of earlier sketch columns
  void* Q = nullptr;          // rows x d_max, row-major (ld = d_max), dtype
  int dtype = 0;
  int64_t rows = 0;
  int cols = 0;               // columns of Q so far
  int covered = 0;            // sketch columns already absorbed into Q
  bool precise = false;       // absorbed by the precise steps (FP32 data, eps_rel below kPreciseBelow)
};

// Stopping tests of FP32 data with eps_rel below this take the precise
// absorption (first projection's difference in double-FP32, a second
// projection before the first Cholesky-QR pass): the plain FP32 steps resolve
// ||S^|| / ||S~|| to about 1e-6, which decides a test to 1 % only from about
// 1e-5 up.
constexpr double kPreciseBelow = 1e-4;

}  // namespace jls

struct sk_op {
  int kind = 0;
  int64_t n = 0;
  int alpha = 1;
  int d_total = 0;
  uint32_t flags = 0;          // SK_SCALE_BLOCK, SK_SRHT_REPLACE
  int d_max = 0;
  int64_t nu = 1;
  uint64_t seed = 0;
  int device = 0;
  std::vector<int> blocks;     // block widths (first = initial d, then increments)
  int pending_old_d = -1;      // d_total before the last increment not yet applied
  int* d_err = nullptr;        // device error flag

  // SJLT: packed entries [block][n][alpha] = column | (sign < 0) << 31
  int32_t* sjlt_ents = nullptr;
  int sjlt_blocks_cap = 0;
  jls::TiledCcs ccs[3];        // [0] tile for F32, [1] tile for F64, [2] R (x) I_2 for complex S = A R
  int32_t* sjlt_ents2 = nullptr;  // entries of R (x) I_2
  size_t ents2_bytes = 0;

  // SRHT: D signs, sampled columns, sampling state (next counter)
  int8_t* srht_diag = nullptr;
  int32_t* srht_mu = nullptr;
  unsigned long long* srht_state = nullptr;

  // Gaussian: unscaled z, transposed (column c of R contiguous over rows)
  float* z32 = nullptr;
  double* z64 = nullptr;
  uint16_t* zhi = nullptr;     // bf16 bits, rows of bf_pitch(n)
  uint16_t* zlo = nullptr;
  int z32_cols = 0, z64_cols = 0, zbf_cols = 0;

  // SRHT +-1 plane for the tensor-core path (bf16 bits, d_max rows of bf_pitch(n))
  uint16_t* srht_pm1 = nullptr;
  int pm1_cols = 0;
  // complex A with SRHT / Gaussian operators: expanded tensor-core planes of
  // R (x) I_2 (2 d_max rows of bf_pitch(2n)), columns expanded so far, and the
  // V^T R buffer of S' = A* R
  void* cplx_p0 = nullptr;
  void* cplx_p1 = nullptr;
  int cplx_cols = 0;
  void* cplx_T = nullptr;
  size_t cplx_T_bytes = 0;

  // FP8 path: e4m3 planes (d_max rows of f8_pitch(n) bytes).  Gaussian: z_hi,
  // z_lo in units of the scale of each (128-value K tile, column), scales
  // [ceil(n/128)][d_max]; SRHT: the exact +-1 plane.
  uint8_t* z8_hi = nullptr;
  uint8_t* z8_lo = nullptr;
  float* z8_scale = nullptr;
  int z8_cols = 0;
  uint8_t* srht_q8 = nullptr;
  int q8_cols = 0;

  jls::Basis basis[2];
  void* scratch[2] = {nullptr, nullptr};  // stopping-test scratch, per slot (S, S')
  size_t scratch_bytes[2] = {0, 0};
  void* gen_scratch = nullptr;        // row blocks of a generated kernel matrix
  float* ksk_u = nullptr;             // kernel-sketch adjoint: second sums, n x 4
  size_t ksk_u_bytes = 0;
  size_t gen_scratch_bytes = 0;
  double* host_norms[2] = {nullptr, nullptr};       // pinned: each slot's norm partials
  cudaEvent_t norms_ready[2] = {nullptr, nullptr};  // recorded after their copy
  cudaStream_t aux_stream = nullptr;                // the S' test of adaptive_norm_test_pair
  cudaEvent_t aux_fork = nullptr, aux_join = nullptr;
};

namespace jls {

// --- operators.cu ---
int gen_sjlt_block(sk_op* h, int block, int col_off, int width, cudaStream_t s);
int build_ccs(sk_op* h, int which_tile, cudaStream_t s);
int build_ccs_complex(sk_op* h, cudaStream_t s);  // ccs[2]: R (x) I_2
int gen_srht(sk_op* h, int d_old, int d_new, cudaStream_t s);
int gen_gauss(sk_op* h, int plane, int c_end, cudaStream_t s);  // plane: 0 f32, 1 f64, 2 bf16x2
int gen_srht_pm1(sk_op* h, int c_end, cudaStream_t s);
int gen_sjlt_pm1(sk_op* h, int c_end, cudaStream_t s);  // the SJLT's +-1 plane (tensor-core route)
int gen_gauss_fp8(sk_op* h, int c_end, cudaStream_t s);
int gen_srht_fp8(sk_op* h, int c_end, cudaStream_t s);
int export_dense_R(sk_op* h, void* R_dev, int dtype, cudaStream_t s);

// --- sjlt_apply.cu ---
// S = A R (rows kernel) and S' = A^T R (cols kernel) for output columns
// [c_lo, c_hi) of R, writing scale * (signed sums).
int sjlt_apply(sk_op* h, const sk_matrix* A, int which, int c_lo, int c_hi, double scale,
               void* S, int64_t ldS, void* St, int64_t ldSt, cudaStream_t s);
// the same for an interleaved complex A (SK_C64): S = A R, S' = A* R
int sjlt_apply_complex(sk_op* h, const sk_matrix* A, int which, int c_lo, int c_hi, double scale, void* S,
                       int64_t ldS, void* St, int64_t ldSt, cudaStream_t s);

// Matrix-free S = K(Q, P; h) R (+ shift on the diagonal) for an SJLT R with n
// rows (P: n points) and m output rows (Q: m points), FP32, never forming K.
int sjlt_kernel_apply(sk_op* h, const float* P, int64_t n, const float* Q, int64_t m, double hbw,
                      double shift, double scale, float* S, int64_t ldS, cudaStream_t s);

// --- kernel_sketch.cu ---  gradient of <dS, K(X, X; h) R> in X and h (SJLT R)
int kernel_sketch_adjoint(sk_op* h, const float* X, double hbw, double scale, const float* dS, int64_t ldS,
                          float* dX, double* dh, cudaStream_t s);

// --- dense_simt.cu ---  SRHT / Gaussian on CUDA cores (FP32 or FP64)
int dense_apply_simt(sk_op* h, const sk_matrix* A, int which, int c_lo, int c_hi, double scale,
                     void* S, int64_t ldS, void* St, int64_t ldSt, cudaStream_t s);

// --- gemm_tc.cu ---  SRHT / Gaussian on tcgen05 tensor cores, bf16 hi+lo split
int dense_apply_tc(sk_op* h, const sk_matrix* A, int which, int c_lo, int c_hi, double scale,
                   void* S, int64_t ldS, void* St, int64_t ldSt, cudaStream_t s);

// --- srht_fwht.cu ---  SRHT S = A D H P / sqrt(d) by row transforms (FP32, nu in [2^14, 2^16])
int fwht_segments(int64_t nu);  // 0 if the FWHT path does not apply
int srht_apply_fwht(sk_op* h, const sk_matrix* A, int c_lo, int c_hi, double scale, float* S, int64_t ldS,
                    cudaStream_t s);

// --- gemm_fp8.cu ---  SRHT / Gaussian on tcgen05 tensor cores, e4m3 split with tile scales
int dense_apply_fp8(sk_op* h, const sk_matrix* A, int which, int c_lo, int c_hi, double scale, void* S,
                    int64_t ldS, void* St, int64_t ldSt, cudaStream_t s);

// --- kernel_matrix.cu ---
// A_ij = K(x_i, y_j) + shift [i + diag_off == j] for the generator's X, Y
int launch_kernel_matrix(const sk_matrix* g, void* A, int64_t ld, cudaStream_t s, int64_t diag_off = 0);

// --- adaptive.cu ---
int scale_columns(void* S, int dtype, int64_t rows, int64_t ld, int c0, int c1, double factor,
                  cudaStream_t s);
int norm_test(sk_op* h, int slot, const void* S, int64_t rows, int64_t ldS, int dtype, int c_split,
              int c_end, double eps_rel, double eps_abs, int* stop, double* nh, double* nt,
              cudaStream_t s);
// the same test in two parts: everything enqueued on s (no host wait), then the wait and the decision
int norm_test_enqueue(sk_op* h, int slot, const void* S, int64_t rows, int64_t ldS, int dtype, double eps_rel, int c_split,
                      int c_end, cudaStream_t s);
int norm_test_finish(sk_op* h, int slot, double eps_rel, double eps_abs, int* stop, double* nh, double* nt);

// --- sjlt_apply.cu host helpers (also used by gemm_tc.cu) ---
typedef CUresult (*PFN_encodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                    const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                    CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
PFN_encodeTiled get_encode_tiled();  // cuTensorMapEncodeTiled from the driver, or null
int num_sms();

// --- jlsketch.cu helpers ---
void note_launch();  // counts kernel launches (sketch_launch_count)
double op_scale(const sk_op* h);  // SJLT 1/sqrt(alpha * blocks); SRHT, Gaussian 1/sqrt(d_total) (block scale: see jlsketch.cu)
bool block_scaled(const sk_op* h);
int launch_tc_planes(int* d_err, const sk_matrix* A, bool trans, int planes, const uint16_t* p0, const uint16_t* p1,
                     int64_t k_len, int c_lo, int c_hi, float scale, float* out, int64_t ldo, cudaStream_t s);
int dense_apply_simt_complex_s(sk_op* h, const sk_matrix* A, int c_lo, int c_hi, double scale, void* S, int64_t ldS,
                               cudaStream_t s);
int dense_apply_complex(sk_op* h, const sk_matrix* A, int which, int prec, int c_lo, int c_hi, double scale,
                        void* S, int64_t ldS, void* St, int64_t ldSt, cudaStream_t s);  // SK_SCALE_BLOCK on an SRHT or Gaussian operator: column scales differ by block
int cuda_status(cudaError_t e);
size_t elem_size(int dtype);

}  // namespace jls

#define JLS_CHECK_CUDA(expr)                                   \
  do {                                                         \
    cudaError_t e__ = (expr);                                  \
    if (e__ != cudaSuccess) return ::jls::cuda_status(e__);    \
  } while (0)

#define JLS_CHECK(expr)                \
  do {                                 \
    int r__ = (expr);                  \
    if (r__ != SK_OK) return r__;      \
  } while (0)
