// srht_fwht.cu -- S = A D H P / sqrt(d) for the SRHT by a fast Walsh-Hadamard
// transform of each row of A (Sec. 7.1), FP32, GB300.
//
// Row i of A (zero-padded to nu = 2^ceil(log2 n)) is sign-flipped by D,
// transformed by the unnormalized Sylvester H (y_o = sum_k x_k (-1)^popc(k & o))
// and the d sampled outputs y_{mu_c} are kept, scaled by 1 / sqrt(d) -- the
// element formula of Sec. 7.2 evaluated through the transform.
//
// GB300 mapping.  A 32768-value row is 128 KB, half the register file, so a
// row is cut into nu / L sub-transforms of L = 16384 values: the butterflies of
// the top log2(nu / L) bits are applied while loading (unit (i, p) loads every
// L-segment q of the row and sums (-1)^popc(p & q) x_q), and each unit is an
// independent transform of length L whose outputs are y_{p L + o}.  A unit is
// one CTA of 128 threads x 128 values in registers (three CTAs per SM, so
// some load while others compute; the segments' second readers hit L2): seven
// butterfly stages in registers, one transpose through shared memory, seven
// more stages.  The transformed unit is written back to the buffer and the
// sampled columns whose output index falls in segment p are gathered and
// stored (plain stores: every column belongs to one unit).
//
// n not a power of two (Sec. 7.1's split, Eqs. had1 and hadiden): with
// k = 2^floor(log2 n), n = k + r and p = 2^ceil(log2 r), the padded order-2k
// transform is A_k H_k + T in its first half and A_k H_k - T in its second,
// T repeating the order-p transform of the last r columns (zero-padded to p).
// The units above then transform only the first k columns (outputs taken at
// mu mod k) and store scale (A_k H_k)_mu; a second kernel transforms each
// row's last r columns in shared memory and adds +-scale (A^ H_p)_{mu mod p}
// (+ below k, - above).  Per row that is k log k + p log p butterflies instead
// of 2k log 2k; the split is taken for r <= 8192 (p fits one CTA's shared
// memory), the padded transform otherwise.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "batch.cuh"
#include "common.cuh"
#include "internal.h"

namespace jls {

namespace {

constexpr int FW_THREADS = 128;
constexpr int FW_E = 128;                   // values per thread
constexpr int FW_L = FW_THREADS * FW_E;     // 16384: length of a unit's transform
constexpr int FW_LOG_L = 14;
constexpr int FW_MAX_SEG = 4;               // nu <= 65536
constexpr int FW_BUF = FW_L + FW_L / 128;   // exchange buffer, one pad word every 128
constexpr int FW_DWORDS = FW_MAX_SEG * 4 * FW_THREADS;  // D sign bits, per thread and segment

__device__ __forceinline__ int pad(int k) { return k + (k >> 7); }

// butterfly stage on register index bit `s` of an array of N values, two
// butterflies per FFMA2 pair (x + y and x - y as fma(y, +-1, x), exact)
template <int N>
__device__ __forceinline__ void stage(float (&x)[N], int s) {
  const float2 p1 = make_float2(1.f, 1.f), m1 = make_float2(-1.f, -1.f);
  const int d = 1 << s;
  if (d == 1) {  // partners are neighbours: pair butterflies j = 4r, 4r + 2
#pragma unroll
    for (int j = 0; j < N; j += 4) {
      const float2 a = make_float2(x[j], x[j + 2]), b = make_float2(x[j + 1], x[j + 3]);
      const float2 sum = __ffma2_rn(b, p1, a), dif = __ffma2_rn(b, m1, a);
      x[j] = sum.x;
      x[j + 2] = sum.y;
      x[j + 1] = dif.x;
      x[j + 3] = dif.y;
    }
  } else {  // pair butterflies j, j + 1 (both with bit s clear)
#pragma unroll
    for (int j = 0; j < N; j += 2) {
      if ((j >> s) & 1) continue;
      const float2 a = make_float2(x[j], x[j + 1]), b = make_float2(x[j + d], x[j + d + 1]);
      const float2 sum = __ffma2_rn(b, p1, a), dif = __ffma2_rn(b, m1, a);
      x[j] = sum.x;
      x[j + 1] = sum.y;
      x[j + d] = dif.x;
      x[j + d + 1] = dif.y;
    }
  }
}

}  // namespace

// One CTA of 128 threads per unit at a time (three CTAs per SM).  Thread t
// holds k = t + 128 j (j < 128): round A transforms bits 7..13 in registers,
// one transpose through the padded buffer (pad(k) = k + k/128, so both the
// write k = t + 128 j and the read k = j + 128 t are conflict-free) gives
// k = j + 128 t, and round B transforms bits 0..6.
__global__ void __launch_bounds__(FW_THREADS, 3)
    srht_fwht_rows_kernel(const float* __restrict__ A, int64_t lda, int64_t rows, int64_t n, int nseg,
                          const int8_t* __restrict__ diag, const int32_t* __restrict__ mu, uint32_t omask,
                          int c_lo, int c_hi, float scale, float* __restrict__ S, int64_t ldS) {
  extern __shared__ float buf[];                                        // FW_BUF floats
  uint32_t* dbits = reinterpret_cast<uint32_t*>(buf + FW_BUF);          // [seg][word][thread]
  const int t = threadIdx.x;

  // D sign bits re-laid out per thread: bit (j % 32) of dbits[(q*4 + j/32)*128 + t] is d_{qL + t + 128 j} < 0
  for (int e = t; e < nseg * 4 * FW_THREADS; e += FW_THREADS) {
    const int tt = e % FW_THREADS, wq = e / FW_THREADS, q = wq >> 2, wj = wq & 3;
    uint32_t m = 0;
    for (int b = 0; b < 32; ++b) {
      const int64_t k = (int64_t)q * FW_L + tt + FW_THREADS * (32 * wj + b);
      if (k < n && diag[k] < 0) m |= 1u << b;
    }
    dbits[e] = m;
  }
  __syncthreads();

  const int64_t units = rows * nseg;
  for (int64_t u = blockIdx.x; u < units; u += gridDim.x) {
    const int64_t i = u / nseg;
    const int p = (int)(u - i * nseg);
    const float* a = A + i * lda;
    const bool whole = (int64_t)nseg * FW_L <= n;  // no zero padding in this row
    float x[FW_E];
    // segment 1 (if any) by cp.async into this thread's round-A slots of the
    // buffer, segment 0 into registers: all loads of both are in flight at once
    const uint32_t sb = smem_u32(buf) + 4u * (uint32_t)t;  // slot of k = t + 128 j is t + 129 j
    if (nseg > 1) {
      const float* a1 = a + FW_L + t;
#pragma unroll 8
      for (int j = 0; j < FW_E; ++j) {
        const bool in = whole || FW_L + t + FW_THREADS * j < n;
        cp_async_4(sb + 4u * 129u * (uint32_t)j, in ? a1 + FW_THREADS * j : a, in ? 4u : 0u);
      }
      cp_async_commit();
    }
#pragma unroll
    for (int j = 0; j < FW_E; ++j) x[j] = (whole || t + FW_THREADS * j < n) ? __ldg(a + t + FW_THREADS * j) : 0.f;
#pragma unroll
    for (int wj = 0; wj < 4; ++wj) {
      const uint32_t m = dbits[wj * FW_THREADS + t];
#pragma unroll
      for (int b = 0; b < 32; ++b) {
        const int j = 32 * wj + b;
        x[j] = __uint_as_float(__float_as_uint(x[j]) ^ ((m << (31 - b)) & 0x80000000u));
      }
    }
    if (nseg > 1) {  // the top-bit butterfly with segment 1: sign (-1)^popc(p & 1)
      cp_async_wait<0>();
      const uint32_t flip = (uint32_t)(p & 1) << 31;
#pragma unroll
      for (int wj = 0; wj < 4; ++wj) {
        const uint32_t m = dbits[(4 + wj) * FW_THREADS + t];
#pragma unroll
        for (int b = 0; b < 32; ++b) {
          const int j = 32 * wj + b;
          x[j] += __uint_as_float(__float_as_uint(buf[t + 129 * j]) ^ ((m << (31 - b)) & 0x80000000u) ^ flip);
        }
      }
    }
    // segments 2 and 3 (nu = 65536): register loads, 16 at a time
    for (int q = 2; q < nseg; ++q) {
      const uint32_t flip = (uint32_t)(__popc(p & q) & 1) << 31;
      const float* aq = a + q * FW_L + t;
      const int kq = q * FW_L + t;
#pragma unroll
      for (int wj = 0; wj < 4; ++wj) {
        const uint32_t m = dbits[(q * 4 + wj) * FW_THREADS + t];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          float v[16];
#pragma unroll
          for (int b = 0; b < 16; ++b) {
            const int j = 32 * wj + 16 * h + b;
            v[b] = (whole || kq + FW_THREADS * j < n) ? __ldg(aq + FW_THREADS * j) : 0.f;
          }
#pragma unroll
          for (int b = 0; b < 16; ++b) {
            const int j = 32 * wj + 16 * h + b;
            x[j] += __uint_as_float(__float_as_uint(v[b]) ^ ((m << (31 - (16 * h + b))) & 0x80000000u) ^ flip);
          }
        }
      }
    }
    // round A: bits 7..13 (register index j); k = t + 128 j at pad(k) = t + 129 j
#pragma unroll
    for (int s = 0; s < 7; ++s) stage<FW_E>(x, s);
#pragma unroll
    for (int j = 0; j < FW_E; ++j) buf[t + 129 * j] = x[j];
    __syncthreads();
    // round B: bits 0..6; k = j + 128 t at pad(k) = j + 129 t (this thread's own slots from here on)
#pragma unroll
    for (int j = 0; j < FW_E; ++j) x[j] = buf[j + 129 * t];
#pragma unroll
    for (int s = 0; s < 7; ++s) stage<FW_E>(x, s);
#pragma unroll
    for (int j = 0; j < FW_E; ++j) buf[j + 129 * t] = x[j];
    __syncthreads();
    // sampled columns whose output index (mod the transform order) is in segment p
    for (int c = c_lo + t; c < c_hi; c += FW_THREADS) {
      const int o = (int)((uint32_t)mu[c] & omask);
      if ((o >> FW_LOG_L) == p) S[i * ldS + c] = scale * buf[pad(o & (FW_L - 1))];
    }
    __syncthreads();
  }
}

// The H_p part of the split: row i's columns k .. k + r - 1, sign-flipped by D
// and zero-padded to p, are transformed, and every sampled column adds
// +-scale (A^ H_p)_{mu mod p} to the scale (A_k H_k)_{mu mod k} already stored
// (one read-modify-write per output: deterministic).
constexpr int TAIL_THREADS = 128;
constexpr int TAIL_MAX = 8192;

// p = 128 E (E = 8 .. 64) values of a row in registers, 128 threads.  Thread t
// loads k^ = t + 128 j (j < E); round A transforms bits 7 .. (the register
// index) by FFMA2 butterfly pairs; a transpose through shared memory gives
// thread t' = G h + g (G = 128 / E) the values k^ = 128 h + g + G j', so round
// B1 transforms bits log2 G .. 6 in registers and round B2 bits 0 .. log2 G - 1
// across the G lanes of a group by shuffles.  The buffer index of k^ is
// k^ + G (k^ >> 7): conflict-free for both the write and the read.
template <int E>
__global__ void __launch_bounds__(TAIL_THREADS)
    srht_fwht_tail_kernel(const float* __restrict__ A, int64_t lda, int64_t rows, int64_t k, int r,
                          const int8_t* __restrict__ diag, const int32_t* __restrict__ mu, int c_lo, int c_hi,
                          float scale, float* __restrict__ S, int64_t ldS) {
  constexpr int P = 128 * E, G = 128 / E;
  constexpr int LOG_E = E == 8 ? 3 : E == 16 ? 4 : E == 32 ? 5 : 6;
  __shared__ float tb[P + E * G];
  const int t = threadIdx.x;
  auto idx = [](int kk) { return kk + G * (kk >> 7); };
  uint64_t neg = 0;  // D's sign of k^ = t + 128 j, bit j
  for (int j = 0; j < E; ++j) {
    const int kk = t + 128 * j;
    if (kk < r && diag[k + kk] < 0) neg |= 1ull << j;
  }
  const int h = t / G, g = t % G;
  for (int64_t i = blockIdx.x; i < rows; i += gridDim.x) {
    const float* a = A + i * lda + k;
    float x[E];
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const int kk = t + 128 * j;
      const float v = kk < r ? __ldg(a + kk) : 0.f;
      x[j] = ((neg >> j) & 1) ? -v : v;
    }
#pragma unroll
    for (int st = 0; st < LOG_E; ++st) stage<E>(x, st);
#pragma unroll
    for (int j = 0; j < E; ++j) tb[idx(t + 128 * j)] = x[j];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < E; ++j) x[j] = tb[idx(128 * h + g + G * j)];
#pragma unroll
    for (int st = 0; st < LOG_E; ++st) stage<E>(x, st);
#pragma unroll
    for (int b = 1; b < G; b <<= 1) {
      const bool upper = (g & b) != 0;
#pragma unroll
      for (int j = 0; j < E; ++j) {
        const float u = __shfl_xor_sync(0xffffffffu, x[j], b);
        x[j] = upper ? u - x[j] : x[j] + u;
      }
    }
    __syncthreads();  // every thread has read its transposed values
#pragma unroll
    for (int j = 0; j < E; ++j) tb[idx(128 * h + g + G * j)] = x[j];
    __syncthreads();
    for (int c = c_lo + t; c < c_hi; c += TAIL_THREADS) {
      const int o = mu[c];
      const float v = scale * tb[idx(o & (P - 1))];
      S[i * ldS + c] += o < k ? v : -v;
    }
    __syncthreads();
  }
}

// p < 1024: the transform in shared memory, log2 p butterfly stages over the CTA
__global__ void __launch_bounds__(TAIL_THREADS)
    srht_fwht_tail_small_kernel(const float* __restrict__ A, int64_t lda, int64_t rows, int64_t k, int r, int p,
                                const int8_t* __restrict__ diag, const int32_t* __restrict__ mu, int c_lo, int c_hi,
                                float scale, float* __restrict__ S, int64_t ldS) {
  __shared__ float tb[1024];
  const int t = threadIdx.x;
  for (int64_t i = blockIdx.x; i < rows; i += gridDim.x) {
    const float* a = A + i * lda + k;
    for (int j = t; j < p; j += TAIL_THREADS) tb[j] = j < r ? (diag[k + j] < 0 ? -a[j] : a[j]) : 0.f;
    __syncthreads();
    for (int hh = 1; hh < p; hh <<= 1) {
      for (int b = t; b < p / 2; b += TAIL_THREADS) {
        const int j0 = ((b & ~(hh - 1)) << 1) | (b & (hh - 1)), j1 = j0 + hh;
        const float x = tb[j0], y = tb[j1];
        tb[j0] = x + y;
        tb[j1] = x - y;
      }
      __syncthreads();
    }
    for (int c = c_lo + t; c < c_hi; c += TAIL_THREADS) {
      const int o = mu[c];
      const float v = scale * tb[o & (p - 1)];
      S[i * ldS + c] += o < k ? v : -v;
    }
    __syncthreads();
  }
}

// butterfly stage on register index bit `s`, one FADD per output: the batched
// kernel's short rows change the pairing from stage to stage, where packing
// operands for FFMA2 pairs would cost register moves
template <int N>
__device__ __forceinline__ void stage_s(float (&x)[N], int s) {
  const int d = 1 << s;
#pragma unroll
  for (int j = 0; j < N; ++j) {
    if ((j >> s) & 1) continue;
    const float a = x[j], b = x[j + d];
    x[j] = a + b;
    x[j + d] = a - b;
  }
}

// Unit length and segment count for nu; 0 if the FWHT path does not apply.
int fwht_segments(int64_t nu) {
  if (nu < FW_L || nu > (int64_t)FW_L * FW_MAX_SEG) return 0;
  return (int)(nu / FW_L);
}

int srht_apply_fwht(sk_op* h, const sk_matrix* A, int c_lo, int c_hi, double scale, float* S, int64_t ldS,
                    cudaStream_t s) {
  const int nseg = fwht_segments(h->nu);
  if (!nseg || A->dtype != SK_F32) return SK_ERR_UNSUPPORTED;
  if (c_hi <= c_lo) return SK_OK;
  // Sec. 7.1's split for n = k + r, 0 < r <= TAIL_MAX, when the order-k transform is one of ours
  int64_t k = 1;
  while (2 * k <= h->n) k *= 2;
  const int64_t r = h->n - k;
  int p = 1;
  while (p < r) p *= 2;
  const char* env = std::getenv("JLS_SRHT_SPLIT");  // "0": transform the zero-padded rows instead
  const bool split = r > 0 && r <= TAIL_MAX && fwht_segments(k) > 0 && !(env && env[0] == '0' && !env[1]);
  const size_t smem = FW_BUF * sizeof(float) + FW_DWORDS * sizeof(uint32_t);
  static bool attr = false;
  if (!attr) {
    JLS_CHECK_CUDA(cudaFuncSetAttribute(srht_fwht_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr = true;
  }
  const int segs = split ? fwht_segments(k) : nseg;
  const int64_t units = A->rows * segs;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(3 * num_sms(), units));
  srht_fwht_rows_kernel<<<grid, FW_THREADS, smem, s>>>(static_cast<const float*>(A->A), A->ld, A->rows,
                                                        split ? k : h->n, segs, h->srht_diag, h->srht_mu,
                                                        (uint32_t)((split ? k : h->nu) - 1), c_lo, c_hi,
                                                        (float)scale, S, ldS);
  note_launch();
  JLS_CHECK_CUDA(cudaGetLastError());
  if (split) {
    const unsigned tgrid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(8 * num_sms(), A->rows));
    const float* Ap = static_cast<const float*>(A->A);
    const float sc = (float)scale;
    switch (p) {
      case 8192:
        srht_fwht_tail_kernel<64><<<tgrid, TAIL_THREADS, 0, s>>>(Ap, A->ld, A->rows, k, (int)r, h->srht_diag,
                                                                  h->srht_mu, c_lo, c_hi, sc, S, ldS);
        break;
      case 4096:
        srht_fwht_tail_kernel<32><<<tgrid, TAIL_THREADS, 0, s>>>(Ap, A->ld, A->rows, k, (int)r, h->srht_diag,
                                                                  h->srht_mu, c_lo, c_hi, sc, S, ldS);
        break;
      case 2048:
        srht_fwht_tail_kernel<16><<<tgrid, TAIL_THREADS, 0, s>>>(Ap, A->ld, A->rows, k, (int)r, h->srht_diag,
                                                                  h->srht_mu, c_lo, c_hi, sc, S, ldS);
        break;
      case 1024:
        srht_fwht_tail_kernel<8><<<tgrid, TAIL_THREADS, 0, s>>>(Ap, A->ld, A->rows, k, (int)r, h->srht_diag,
                                                                 h->srht_mu, c_lo, c_hi, sc, S, ldS);
        break;
      default:
        srht_fwht_tail_small_kernel<<<tgrid, TAIL_THREADS, 0, s>>>(Ap, A->ld, A->rows, k, (int)r, p, h->srht_diag,
                                                                    h->srht_mu, c_lo, c_hi, sc, S, ldS);
    }
    note_launch();
    JLS_CHECK_CUDA(cudaGetLastError());
  }
  return SK_OK;
}


// ---------------------------------------------------------------------------
// Batches of SRHT sketches S_i = A_i D_i H_i P_i scale_i (nu_i <= 4096): the
// rows of every instance with a non-empty column range are numbered into one
// list of units (one row each, instances in order) and a persistent grid of
// 128-thread CTAs takes contiguous ranges of it.  A row of order nu = 128 E
// (E = 4 .. 32) is transformed in registers as in srht_fwht_tail_kernel; a
// row of order below 512 in shared memory.  Outputs are plain stores (each
// sampled column belongs to one row transform), so runs are deterministic.
constexpr int SB_THREADS = 128;
constexpr int SB_MAX_NU = 4096;

struct SbItem {
  const float* A;
  float* S;
  const int8_t* diag;
  const int32_t* mu;
  int64_t lda, ldS;
  int64_t unit0;  // first unit of this instance
  int64_t rows;   // units of this instance in the next run (0: left out)
  int64_t nrows;  // rows of A_i
  int32_t n, nu, c_lo, c_hi;
  float scale;
  int32_t flags;   // bit 0: rows start on 16-byte boundaries (A and lda * 4)
  int32_t tail_p;  // Sec. 7.1's split: n = k + r with k = nu / 2 and 0 < r <= k / 2, p = 2^ceil(log2 r); 0: none
};

// row r of an instance into `stg` (nu floats, zero past n) by cp.async: 16-byte
// copies when its rows start on 16-byte boundaries, 4-byte copies otherwise
template <int P>
__device__ __forceinline__ void sb_prefetch(const SbItem& it, int64_t r, float* stg) {
  const float* a = it.A + r * it.lda;
  const uint32_t st = smem_u32(stg);
  if (it.flags & 1) {
    for (int q = threadIdx.x; q < P / 4; q += SB_THREADS) {
      const int rem = it.n - 4 * q;
      const uint32_t bytes = rem >= 4 ? 16u : rem > 0 ? 4u * rem : 0u;
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(st + 16 * q),
                   "l"(bytes ? a + 4 * q : a), "r"(bytes) : "memory");
    }
  } else {
    for (int k = threadIdx.x; k < P; k += SB_THREADS) cp_async_4(st + 4 * k, k < it.n ? a + k : a, k < it.n ? 4 : 0);
  }
  cp_async_commit();
}

// rows [r0, r1) of one instance, order P = 128 E; the next row is staged by
// cp.async while this one is transformed
template <int E>
__device__ void sb_rows_reg(const SbItem& it, int64_t r0, int64_t r1, float* tb, float* stg) {
  constexpr int P = 128 * E, G = 128 / E;
  constexpr int LOG_E = E == 4 ? 2 : E == 8 ? 3 : E == 16 ? 4 : 5;
  static_assert(P <= SB_MAX_NU && G <= 32, "register path: 512 <= nu <= 4096");
  const int t = threadIdx.x;
  auto idx = [](int kk) { return kk + G * (kk >> 7); };
  uint32_t neg = 0;  // D's sign of k = t + 128 j, bit j
  for (int j = 0; j < E; ++j) {
    const int kk = t + 128 * j;
    if (kk < it.n && it.diag[kk] < 0) neg |= 1u << j;
  }
  const int h = t / G, g = t % G;
  sb_prefetch<P>(it, r0, stg);
  for (int64_t r = r0; r < r1; ++r) {
    cp_async_wait<0>();
    __syncthreads();  // row r is staged
    float x[E];
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const float v = stg[t + 128 * j];
      x[j] = ((neg >> j) & 1) ? -v : v;
    }
#pragma unroll
    for (int st = 0; st < LOG_E; ++st) stage_s<E>(x, st);
#pragma unroll
    for (int j = 0; j < E; ++j) tb[idx(t + 128 * j)] = x[j];
    __syncthreads();  // every thread has read the staged row and written tb
    if (r + 1 < r1) sb_prefetch<P>(it, r + 1, stg);
#pragma unroll
    for (int j = 0; j < E; ++j) x[j] = tb[idx(128 * h + g + G * j)];
#pragma unroll
    for (int st = 0; st < LOG_E; ++st) stage_s<E>(x, st);
#pragma unroll
    for (int b = 1; b < G; b <<= 1) {
      const float sg = (g & b) ? -1.f : 1.f;  // lower lane x + u, upper lane u - x
#pragma unroll
      for (int j = 0; j < E; ++j) x[j] = fmaf(sg, x[j], __shfl_xor_sync(0xffffffffu, x[j], b));
    }
    __syncthreads();  // every thread has read its transposed values
#pragma unroll
    for (int j = 0; j < E; ++j) tb[idx(128 * h + g + G * j)] = x[j];
    __syncthreads();
    float* srow = it.S + r * it.ldS;
    for (int c = it.c_lo + t; c < it.c_hi; c += SB_THREADS) srow[c] = it.scale * tb[idx(it.mu[c] & (P - 1))];
    __syncthreads();
  }
}

// rows [r0, r1) of one instance, order nu < 512: butterflies in shared memory
__device__ void sb_rows_smem(const SbItem& it, int64_t r0, int64_t r1, float* tb) {
  const int t = threadIdx.x, p = it.nu;
  for (int64_t r = r0; r < r1; ++r) {
    const float* a = it.A + r * it.lda;
    for (int j = t; j < p; j += SB_THREADS) tb[j] = j < it.n ? (it.diag[j] < 0 ? -__ldg(a + j) : __ldg(a + j)) : 0.f;
    __syncthreads();
    for (int hh = 1; hh < p; hh <<= 1) {
      for (int b = t; b < p / 2; b += SB_THREADS) {
        const int j0 = ((b & ~(hh - 1)) << 1) | (b & (hh - 1)), j1 = j0 + hh;
        const float x = tb[j0], y = tb[j1];
        tb[j0] = x + y;
        tb[j1] = x - y;
      }
      __syncthreads();
    }
    float* srow = it.S + r * it.ldS;
    for (int c = it.c_lo + t; c < it.c_hi; c += SB_THREADS) srow[c] = it.scale * tb[it.mu[c] & (p - 1)];
    __syncthreads();
  }
}

__global__ void __launch_bounds__(SB_THREADS, 6)
    srht_batch_kernel(const SbItem* __restrict__ items, int count, int64_t total_host,
                      const int64_t* __restrict__ total_dev) {
  const int64_t total = total_dev ? *total_dev : total_host;
  __shared__ float tb[SB_MAX_NU + SB_MAX_NU / 128 * 4];  // order 4096: P + E G = 4096 + 32 * 4
  __shared__ __align__(16) float stg[SB_MAX_NU];            // the next row, staged by cp.async
  const int64_t per = (total + gridDim.x - 1) / gridDim.x;
  const int64_t u0 = (int64_t)blockIdx.x * per, u1 = min64(total, u0 + per);
  if (u0 >= u1) return;
  int lo = 0, hi = count - 1;  // the last instance whose first unit is <= u0
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (items[mid].unit0 <= u0) lo = mid;
    else hi = mid - 1;
  }
  int64_t u = u0;
  for (int i = lo; i < count && u < u1; ++i) {
    SbItem it = items[i];
    const int64_t end = min64(u1, it.unit0 + it.rows);
    if (u >= end) continue;  // an instance left out of this run
    const int64_t r0 = u - it.unit0, r1 = end - it.unit0;
    if (it.tail_p) {  // Sec. 7.1's split: this pass transforms the first k = nu / 2 columns at order k
      it.nu /= 2;
      it.n = it.nu;
    }
    switch (it.nu) {
      case 4096: sb_rows_reg<32>(it, r0, r1, tb, stg); break;
      case 2048: sb_rows_reg<16>(it, r0, r1, tb, stg); break;
      case 1024: sb_rows_reg<8>(it, r0, r1, tb, stg); break;
      case 512: sb_rows_reg<4>(it, r0, r1, tb, stg); break;
      default: sb_rows_smem(it, r0, r1, tb);
    }
    u = end;
  }
}

// The second pass of Sec. 7.1's split (Eqs. had1, hadiden) for the rows of
// instances with tail_p > 0 (n = k + r, k = nu / 2, 0 < r <= k / 2): the
// first pass wrote scale (A_k H_k)_{mu mod k}; this adds
// +- scale (A^ H_p)_{mu mod p} (+ below k, - above), A^ the last r columns
// with D's signs, zero-padded to p.  One warp per row: lane l holds tail
// values l + 32 j (j < PER = max(1, p / 32)); the bits of j by butterflies in
// registers, the lane bits by shuffles; the transform goes through a warp-owned
// shared buffer to the lanes that add it to the sampled columns (a read and a
// write per output, after the first pass in stream order: deterministic).
// Grid: (instance, group of rows), TAIL_WARPS warps per CTA.
constexpr int TAIL_WARPS = 4;
constexpr int TAIL_ROWS_PER_CTA_Y = 32;  // gridDim.y = ceil(max rows / this)

template <int PER>
__device__ void sb_tail_row(const SbItem& it, int64_t r, float* buf) {
  const int lane = threadIdx.x & 31, k = it.nu / 2, p = it.tail_p, rr = it.n - k;
  const float* a = it.A + r * it.lda + k;
  float x[PER];
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const int i = lane + 32 * j;
    const float v = i < rr ? __ldg(a + i) : 0.f;
    x[j] = (i < rr && it.diag[k + i] < 0) ? -v : v;
  }
#pragma unroll
  for (int st = 0; (1 << st) < PER; ++st) stage_s<PER>(x, st);
#pragma unroll
  for (int b = 1; b < 32; b <<= 1) {
    if (b >= p) break;  // uniform
    const float sg = (lane & b) ? -1.f : 1.f;
#pragma unroll
    for (int j = 0; j < PER; ++j) x[j] = fmaf(sg, x[j], __shfl_xor_sync(0xffffffffu, x[j], b));
  }
#pragma unroll
  for (int j = 0; j < PER; ++j)
    if (lane + 32 * j < p) buf[lane + 32 * j] = x[j];
  __syncwarp();
  float* srow = it.S + r * it.ldS;
  for (int c = it.c_lo + lane; c < it.c_hi; c += 32) {
    const int m = it.mu[c];
    const float w = buf[m & (p - 1)];
    srow[c] += it.scale * (m < k ? w : -w);
  }
  __syncwarp();
}

__global__ void __launch_bounds__(TAIL_WARPS * 32) srht_batch_tail_kernel(const SbItem* __restrict__ items) {
  __shared__ float buf[TAIL_WARPS][SB_MAX_NU / 4];  // p <= nu / 4
  const SbItem& it = items[blockIdx.x];
  if (!it.tail_p || !it.rows || it.c_hi <= it.c_lo) return;
  const int warp = threadIdx.x >> 5;
  const int per = it.tail_p <= 32 ? 1 : it.tail_p / 32;
  for (int64_t r = (int64_t)blockIdx.y * TAIL_WARPS + warp; r < it.nrows; r += (int64_t)gridDim.y * TAIL_WARPS) {
    switch (per) {
      case 1: sb_tail_row<1>(it, r, buf[warp]); break;
      case 2: sb_tail_row<2>(it, r, buf[warp]); break;
      case 4: sb_tail_row<4>(it, r, buf[warp]); break;
      case 8: sb_tail_row<8>(it, r, buf[warp]); break;
      case 16: sb_tail_row<16>(it, r, buf[warp]); break;
      default: sb_tail_row<32>(it, r, buf[warp]); break;
    }
  }
}

// The tail order p of Sec. 7.1's split for a batched row of n values and
// padded order nu (n = k + r, k = nu / 2, 0 < r <= k / 2), or 0 (transform the
// zero-padded row).
static int srht_batch_split_p(int64_t n, int64_t nu) {
  const int64_t k = nu / 2, r = n - k;
  if (nu < 4 || r <= 0 || r > k / 2) return 0;
  int p = 1;
  while (p < r) p *= 2;
  return p;
}

// Between the rounds of the adaptive loop: the test kernel has left each
// instance's next column range (or units = 0 when it stopped) in the shared
// loop table; copy the ranges into the SRHT items and number the rows of the
// instances still active (one CTA of 1024 threads, in item order).
__global__ void __launch_bounds__(1024)
    sb_renumber_kernel(const BItem* __restrict__ bi, SbItem* __restrict__ sb, int count, int64_t* __restrict__ total) {
  __shared__ int64_t part[1024];
  const int t = threadIdx.x;
  const int per = (count + 1023) / 1024;
  const int i0 = min(count, t * per), i1 = min(count, i0 + per);
  int64_t sum = 0;
  for (int i = i0; i < i1; ++i) {
    SbItem& I = sb[i];
    I.c_lo = bi[i].c_lo;
    I.c_hi = bi[i].c_hi;
    I.rows = (bi[i].units && I.c_hi > I.c_lo) ? I.nrows : 0;
    sum += I.rows;
  }
  part[t] = sum;
  __syncthreads();
  if (t == 0) {
    int64_t run = 0;
    for (int k = 0; k < 1024; ++k) {
      const int64_t v = part[k];
      part[k] = run;
      run += v;
    }
    *total = run;
  }
  __syncthreads();
  int64_t u = part[t];
  for (int i = i0; i < i1; ++i) {
    sb[i].unit0 = u;
    u += sb[i].rows;
  }
}

}  // namespace jls

// ---------------------------------------------------------------------------
// host side of the SRHT batch
struct sk_srht_batch {
  int device = 0;
  int count = 0;
  std::vector<sk_srht_batch_item> items;
  jls::SbItem* h_items = nullptr;  // pinned mirror of the item table
  jls::SbItem* d_items = nullptr;
  int64_t total = 0;               // units of the next run
  int ctas_per_sm = 6;
  bool has_tail = false;           // some instance takes Sec. 7.1's split (a second, tail pass)
  int64_t max_rows = 0;
  float tuned_ms[6] = {};          // per tuner candidate: CTAs per SM 3, 6, 12 with the split, then without
  bool split_used = false;         // the tuner kept Sec. 7.1's split
  // the adaptive loop (sketch_srht_batch_adaptive_setup)
  bool adaptive = false;
  int max_tests = 0, a_ncl = 1;
  bool a_wide = false;  // some instance's basis passes ADAPT_QSMEM columns
  double eps_rel = 0.0, eps_abs = 0.0;
  jls::SbItem* d_sb0 = nullptr;   // round 0's items: [0, d0 + dd) at the loop's scale 1/sqrt(d0 + dd)
  jls::BItem* d_loop = nullptr;   // the loop table the test kernel updates (c_lo, c_hi, units)
  jls::BItem* d_loop0 = nullptr;
  jls::ATest* d_tests = nullptr;  // per-instance loop state, and its initial value
  jls::ATest* d_tests0 = nullptr;
  int* d_order = nullptr;         // instances, largest first
  float* d_basis = nullptr;       // Q_i and W_i of every instance
  int64_t* d_units = nullptr;     // rows of the next round
};

namespace jls {
namespace {

constexpr int SB_CTAS[3] = {3, 6, 12};  // 6 CTAs of 80 registers x 128 threads fill an SM

void sb_number(sk_srht_batch* b) {
  int64_t u = 0;
  for (int i = 0; i < b->count; ++i) {
    SbItem& I = b->h_items[i];
    I.unit0 = u;
    I.rows = I.c_hi > I.c_lo ? b->items[i].rows : 0;
    u += I.rows;
  }
  b->total = u;
}

// the tail pass of Sec. 7.1's split, after the order-k pass in stream order
int sb_tail_launch(sk_srht_batch* b, cudaStream_t s) {
  if (!b->has_tail) return SK_OK;
  const dim3 grid((unsigned)b->count,
                  (unsigned)std::max<int64_t>(1, (b->max_rows + TAIL_ROWS_PER_CTA_Y - 1) / TAIL_ROWS_PER_CTA_Y));
  srht_batch_tail_kernel<<<grid, TAIL_WARPS * 32, 0, s>>>(b->d_items);
  note_launch();
  JLS_CHECK_CUDA(cudaGetLastError());
  return SK_OK;
}

int sb_launch(sk_srht_batch* b, cudaStream_t s) {
  JLS_CHECK_CUDA(cudaMemcpyAsync(b->d_items, b->h_items, sizeof(SbItem) * b->count, cudaMemcpyHostToDevice, s));
  if (b->total == 0) return SK_OK;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((int64_t)b->ctas_per_sm * num_sms(),
                                                                         b->total));
  srht_batch_kernel<<<grid, SB_THREADS, 0, s>>>(b->d_items, b->count, b->total, nullptr);
  note_launch();
  JLS_CHECK_CUDA(cudaGetLastError());
  return sb_tail_launch(b, s);
}

// one timed run per CTAs-per-SM choice (after one untimed run); keeps the fastest
// Sets every item's tail order (Sec. 7.1's split on) or clears them (the
// zero-padded rows).
void sb_set_split(sk_srht_batch* b, bool on) {
  b->has_tail = false;
  for (int i = 0; i < b->count; ++i) {
    SbItem& I = b->h_items[i];
    I.tail_p = on ? srht_batch_split_p(I.n, I.nu) : 0;
    b->has_tail |= I.tail_p > 0;
  }
}

// CTAs per SM (3, 6 or 12) and, where some instance qualifies, Sec. 7.1's
// split on or off: each candidate is timed once on the caller's stream (after
// one untimed run) and the fastest is kept.
int sb_tune(sk_srht_batch* b, cudaStream_t s) {
  cudaEvent_t e0, e1;
  JLS_CHECK_CUDA(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return SK_ERR_DEVICE;
  }
  // JLS_SRHT_SPLIT=1 or =0 pins the split on or off instead of timing both
  const char* env = std::getenv("JLS_SRHT_SPLIT");
  const int pin = env && !env[1] ? (env[0] == '1' ? 1 : env[0] == '0' ? 0 : -1) : -1;
  sb_set_split(b, true);
  const int k_lo = (pin == 0 || !b->has_tail) ? 3 : 0, k_hi = (pin == 1 && b->has_tail) ? 3 : 6;
  int rc = SK_OK, best = k_lo;
  for (int k = k_lo; k < k_hi && rc == SK_OK; ++k) {
    b->ctas_per_sm = SB_CTAS[k % 3];
    sb_set_split(b, k < 3);
    if ((rc = sb_launch(b, s)) != SK_OK) break;
    if (cudaEventRecord(e0, s) != cudaSuccess || (rc = sb_launch(b, s)) != SK_OK ||
        cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&b->tuned_ms[k], e0, e1) != cudaSuccess) {
      rc = rc == SK_OK ? SK_ERR_DEVICE : rc;
      break;
    }
    if (k == k_lo || b->tuned_ms[k] < b->tuned_ms[best]) best = k;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->ctas_per_sm = SB_CTAS[best % 3];
  sb_set_split(b, best < 3);
  b->split_used = b->has_tail;
  return rc;
}

}  // namespace
}  // namespace jls

using namespace jls;

extern "C" {

int sketch_srht_batch_create(sk_srht_batch_handle* out, const sk_srht_batch_item* items, int32_t count,
                             void* stream) {
  if (!out || !items || count < 1) return SK_ERR_INVALID_ARG;
  *out = nullptr;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int i = 0; i < count; ++i) {
    const sk_srht_batch_item& it = items[i];
    const sk_op* h = it.op;
    if (!h || h->kind != SK_SRHT) return SK_ERR_INVALID_ARG;
    if (!it.A || !it.S || it.rows < 1 || it.ld < h->n || it.ldS < h->d_total) return SK_ERR_INVALID_ARG;
    if (it.c_lo < 0 || it.c_hi < it.c_lo || it.c_hi > h->d_total) return SK_ERR_INVALID_ARG;
    if (h->nu > SB_MAX_NU) return SK_ERR_UNSUPPORTED;
  }
  sk_srht_batch* b = new sk_srht_batch();
  b->count = count;
  b->items.assign(items, items + count);
  cudaGetDevice(&b->device);
  auto fail = [&](int code) {
    sketch_srht_batch_destroy(b);
    return code;
  };
  if (cudaMallocHost(&b->h_items, sizeof(SbItem) * count) != cudaSuccess ||
      cudaMalloc(&b->d_items, sizeof(SbItem) * count) != cudaSuccess) {
    cudaGetLastError();
    return fail(SK_ERR_NOMEM);
  }
  std::memset(b->h_items, 0, sizeof(SbItem) * count);
  for (int i = 0; i < count; ++i) {
    const sk_srht_batch_item& it = items[i];
    const sk_op* h = it.op;
    SbItem& I = b->h_items[i];
    I.A = it.A;
    I.S = it.S;
    I.diag = h->srht_diag;
    I.mu = h->srht_mu;
    I.lda = it.ld;
    I.ldS = it.ldS;
    I.n = (int32_t)h->n;
    I.nu = (int32_t)h->nu;
    I.c_lo = it.c_lo;
    I.c_hi = it.c_hi;
    I.nrows = it.rows;
    I.scale = (float)(it.scale != 0.0 ? it.scale : 1.0 / std::sqrt((double)h->d_total));
    I.flags = ((reinterpret_cast<uintptr_t>(it.A) & 15u) == 0 && (it.ld * 4) % 16 == 0) ? 1 : 0;
    b->max_rows = std::max<int64_t>(b->max_rows, it.rows);
  }
  sb_number(b);
  // six CTAs of 33 KB of shared memory per SM: ask for the largest shared-memory carveout
  if (cudaFuncSetAttribute(srht_batch_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                           (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess) {
    cudaGetLastError();
    return fail(SK_ERR_DEVICE);
  }
  const int rc = sb_tune(b, s);
  if (rc != SK_OK) return fail(rc);
  *out = b;
  return SK_OK;
}

int sketch_srht_batch_set(sk_srht_batch_handle b, const int32_t* c_lo, const int32_t* c_hi) {
  if (!b) return SK_ERR_INVALID_ARG;
  for (int i = 0; i < b->count; ++i) {
    const int lo = c_lo ? c_lo[i] : b->h_items[i].c_lo, hi = c_hi ? c_hi[i] : b->h_items[i].c_hi;
    if (lo < 0 || hi < lo || hi > b->items[i].op->d_total) return SK_ERR_INVALID_ARG;
  }
  for (int i = 0; i < b->count; ++i) {
    if (c_lo) b->h_items[i].c_lo = c_lo[i];
    if (c_hi) b->h_items[i].c_hi = c_hi[i];
  }
  sb_number(b);
  return SK_OK;
}

int sketch_srht_batch_run(sk_srht_batch_handle b, void* stream) {
  if (!b) return SK_ERR_INVALID_ARG;
  return sb_launch(b, static_cast<cudaStream_t>(stream));
}

int sketch_srht_batch_info(sk_srht_batch_handle b, int32_t* ctas_per_sm, int64_t* units, float* tuned_ms,
                           int32_t* split) {
  if (!b) return SK_ERR_INVALID_ARG;
  if (ctas_per_sm) *ctas_per_sm = b->ctas_per_sm;
  if (units) *units = b->total;
  if (tuned_ms)
    for (int k = 0; k < 6; ++k) tuned_ms[k] = b->tuned_ms[k];
  if (split) *split = b->split_used ? 1 : 0;
  return SK_OK;
}

static void sb_adaptive_free(sk_srht_batch* b) {
  void* ps[] = {b->d_sb0, b->d_loop, b->d_loop0, b->d_tests, b->d_tests0, b->d_order, b->d_basis, b->d_units};
  for (void* p : ps)
    if (p) cudaFree(p);
  b->d_sb0 = nullptr;
  b->d_loop = b->d_loop0 = nullptr;
  b->d_tests = b->d_tests0 = nullptr;
  b->d_order = nullptr;
  b->d_basis = nullptr;
  b->d_units = nullptr;
  b->adaptive = false;
}

int sketch_srht_batch_adaptive_setup(sk_srht_batch_handle b, const int32_t* d0, int32_t dd, double eps_rel,
                                     double eps_abs, void* stream) {
  if (!b || !d0 || dd < 8 || dd > ADAPT_BW || dd % 8 || !(eps_rel >= 0.0) || !(eps_abs >= 0.0))
    return SK_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int count = b->count;
  for (int i = 0; i < count; ++i) {
    const sk_op* h = b->items[i].op;
    const int first = d0[i] + dd;
    if (d0[i] < 0 || d0[i] % 8 || h->blocks.empty() || h->blocks[0] != first) return SK_ERR_INVALID_ARG;
    for (size_t j = 1; j < h->blocks.size(); ++j)
      if (h->blocks[j] != dd) return SK_ERR_INVALID_ARG;  // R_i = SRHT(d0 + dd) grown by dd-column increments
    if (b->items[i].ldS < h->d_total) return SK_ERR_INVALID_ARG;
    if (h->d_total - dd > ADAPT_QMAX) return SK_ERR_UNSUPPORTED;
  }
  JLS_CHECK_CUDA(cudaStreamSynchronize(s));
  sb_adaptive_free(b);
  std::vector<SbItem> sb0(b->h_items, b->h_items + count);
  std::vector<BItem> loop0(count);
  std::vector<ATest> a0(count);
  std::vector<size_t> off(count);
  size_t total = 0;
  bool wide = false;  // some basis passes ADAPT_QSMEM columns
  int max_tests = 0;
  for (int i = 0; i < count; ++i) {
    const sk_op* h = b->items[i].op;
    const int first = d0[i] + dd;
    sb0[i].scale = (float)(1.0 / std::sqrt((double)first));
    std::memset(&loop0[i], 0, sizeof(BItem));
    loop0[i].c_lo = 0;
    loop0[i].c_hi = first;
    loop0[i].units = 1;
    const int qcap = std::max(8, (h->d_total - dd + 7) / 8 * 8);
    off[i] = total;
    total += (size_t)b->items[i].rows * (qcap + ADAPT_BW);
    if (qcap > ADAPT_QSMEM) total += (size_t)qcap * ADAPT_BW;  // Q^T W of a wide basis
    wide |= qcap > ADAPT_QSMEM;
    ATest& T = a0[i];
    std::memset(&T, 0, sizeof(T));
    T.S = b->items[i].S;
    T.rows = b->items[i].rows;
    T.ldS = b->items[i].ldS;
    T.qcap = qcap;
    T.dd = dd;
    T.d_cap = h->d_total;
    T.first_w = first;
    T.state = ADAPT_ACTIVE;
    T.srht = 1;
    max_tests = std::max(max_tests, 1 + (h->d_total - first) / dd);
  }
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    return b->items[x].rows * (int64_t)b->items[x].op->d_total > b->items[y].rows * (int64_t)b->items[y].op->d_total;
  });
  if (cudaMalloc(&b->d_sb0, sizeof(SbItem) * count) != cudaSuccess ||
      cudaMalloc(&b->d_loop, sizeof(BItem) * count) != cudaSuccess ||
      cudaMalloc(&b->d_loop0, sizeof(BItem) * count) != cudaSuccess ||
      cudaMalloc(&b->d_tests, sizeof(ATest) * count) != cudaSuccess ||
      cudaMalloc(&b->d_tests0, sizeof(ATest) * count) != cudaSuccess ||
      cudaMalloc(&b->d_order, sizeof(int) * (2 * count + 1)) != cudaSuccess ||  // order, active list, count
      cudaMalloc(&b->d_basis, total * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&b->d_units, sizeof(int64_t)) != cudaSuccess) {
    cudaGetLastError();
    sb_adaptive_free(b);
    return SK_ERR_NOMEM;
  }
  for (int i = 0; i < count; ++i) {
    a0[i].Q = b->d_basis + off[i];
    a0[i].W = b->d_basis + off[i] + (size_t)b->items[i].rows * a0[i].qcap;
    a0[i].G = a0[i].qcap > ADAPT_QSMEM ? a0[i].W + (size_t)b->items[i].rows * ADAPT_BW : nullptr;
  }
  int rc = adaptive_prepare();
  if (rc == SK_OK &&
      (cudaMemcpy(b->d_sb0, sb0.data(), sizeof(SbItem) * count, cudaMemcpyHostToDevice) != cudaSuccess ||
       cudaMemcpy(b->d_loop0, loop0.data(), sizeof(BItem) * count, cudaMemcpyHostToDevice) != cudaSuccess ||
       cudaMemcpy(b->d_tests0, a0.data(), sizeof(ATest) * count, cudaMemcpyHostToDevice) != cudaSuccess ||
       cudaMemcpy(b->d_order, order.data(), sizeof(int) * count, cudaMemcpyHostToDevice) != cudaSuccess))
    rc = SK_ERR_DEVICE;
  if (rc != SK_OK) {
    sb_adaptive_free(b);
    return rc;
  }
  b->max_tests = max_tests;
  b->a_wide = wide;
  // the stopping test: one CTA per instance when the instances fill the GPU, else a cluster of 4
  const char* env = std::getenv("JLS_ADAPT_CLUSTER");
  b->a_ncl = env ? std::atoi(env) : (count >= num_sms() ? 1 : 4);
  if (b->a_ncl != 1 && b->a_ncl != 2 && b->a_ncl != 4) b->a_ncl = 4;
  b->eps_rel = eps_rel;
  b->eps_abs = eps_abs;
  b->adaptive = true;
  return SK_OK;
}

int sketch_srht_batch_adaptive_run(sk_srht_batch_handle b, int32_t max_rounds, void* stream) {
  if (!b || !b->adaptive || max_rounds < 0) return SK_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int count = b->count;
  const int rounds = max_rounds ? std::min<int>(max_rounds, b->max_tests) : b->max_tests;
  JLS_CHECK_CUDA(cudaMemcpyAsync(b->d_items, b->d_sb0, sizeof(SbItem) * count, cudaMemcpyDeviceToDevice, s));
  JLS_CHECK_CUDA(cudaMemcpyAsync(b->d_loop, b->d_loop0, sizeof(BItem) * count, cudaMemcpyDeviceToDevice, s));
  JLS_CHECK_CUDA(cudaMemcpyAsync(b->d_tests, b->d_tests0, sizeof(ATest) * count, cudaMemcpyDeviceToDevice, s));
  int64_t rows_all = 0;
  for (const sk_srht_batch_item& it : b->items) rows_all += it.rows;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((int64_t)b->ctas_per_sm * num_sms(), rows_all));
  for (int r = 0; r < rounds; ++r) {
    sb_renumber_kernel<<<1, 1024, 0, s>>>(b->d_loop, b->d_items, count, b->d_units);
    note_launch();
    srht_batch_kernel<<<grid, SB_THREADS, 0, s>>>(b->d_items, count, 0, b->d_units);
    note_launch();
    JLS_CHECK_CUDA(cudaGetLastError());
    JLS_CHECK(sb_tail_launch(b, s));
    JLS_CHECK(adaptive_test_round(b->d_loop, b->d_tests, b->d_order, count, b->a_ncl, b->eps_rel, b->eps_abs,
                                  b->a_wide, b->d_order + count, b->d_order + 2 * count, s));
  }
  return adaptive_rescale_launch(b->d_tests, count, s);
}

int sketch_srht_batch_adaptive_result(sk_srht_batch_handle b, int32_t* d_reached, int32_t* state, int32_t* tests,
                                      double* nh, double* nt, void* stream) {
  if (!b || !b->adaptive) return SK_ERR_INVALID_ARG;
  JLS_CHECK_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  std::vector<ATest> a(b->count);
  JLS_CHECK_CUDA(cudaMemcpy(a.data(), b->d_tests, sizeof(ATest) * b->count, cudaMemcpyDeviceToHost));
  for (int i = 0; i < b->count; ++i) {
    if (d_reached) d_reached[i] = a[i].d_reached;
    if (state) state[i] = a[i].state;
    if (tests) tests[i] = a[i].tests;
    if (nh) nh[i] = a[i].nh;
    if (nt) nt[i] = a[i].nt;
  }
  return SK_OK;
}

void sketch_srht_batch_destroy(sk_srht_batch_handle b) {
  if (!b) return;
  sb_adaptive_free(b);
  if (b->h_items) cudaFreeHost(b->h_items);
  if (b->d_items) cudaFree(b->d_items);
  delete b;
}

}  // extern "C"
