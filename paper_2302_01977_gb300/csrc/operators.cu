// operators.cu -- drawing the JL operators on the device (Sec. 2.4, Sec. 6.1-6.2, Sec. 7.2).
//
// Stream layout (identical to the host oracle's, which is written independently):
//  * SJLT row i, block b: draws t = 0, 1, ... at Philox counter (i, t, 0, 0),
//    key (seed, TAG_SJLT | b); slot k takes the next accepted draw,
//    position = lemire(word0, span) (span = width/alpha for the block
//    construction, width for the graph construction, Sec. 2.4.3); a draw is
//    skipped on Lemire rejection or, in the graph construction, on a repeated
//    column; sign = top bit of word1 (set means -1).
//  * SRHT: d_i = top bit of word0 at counter (i, 0, 0, 0), key (seed, TAG_SRHT_D);
//    sampled columns = first distinct lemire(word0, nu) over counters
//    (t, 0, 0, 0), key (seed, TAG_SRHT_MU) (Sec. 2.4.2, without replacement).
//  * Gaussian column c: counter (i, c >> 1, 0, 0), key (seed, TAG_GAUSS),
//    Box-Muller on u1 in (0,1], u2 in [0,1): cos half for even c, sin for odd.
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace jls {

// ---------------------------------------------------------------------------
// SJLT: one thread per row, alpha slots, packed entry = col | (neg << 31).
__global__ void sjlt_draw_kernel(int64_t n, int alpha, int width, int block_construction,
                                 uint64_t seed, int block, int col_off, int32_t* __restrict__ out,
                                 int* err) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t key1 = TAG_SJLT | (uint64_t)block;
  const uint64_t span = block_construction ? (uint64_t)(width / alpha) : (uint64_t)width;
  int cols[SJLT_MAX_ALPHA];
  int neg[SJLT_MAX_ALPHA];
  uint64_t t = 0;
  for (int k = 0; k < alpha; ++k) {
    int tries = 0;
    while (true) {
      if (++tries > (1 << 20)) {  // practically unreachable; never spin forever
        set_err(err, ERRF_RNG);
        return;
      }
      const u64x4 w = philox4x64_10((uint64_t)i, t, 0, 0, seed, key1);
      ++t;
      uint64_t v;
      if (!lemire(w.x0, span, &v)) continue;
      int c = block_construction ? (int)(k * span + v) : (int)v;
      bool dup = false;
      if (!block_construction)
        for (int q = 0; q < k; ++q) dup |= (cols[q] == c);
      if (dup) continue;
      cols[k] = c;
      neg[k] = (int)(w.x1 >> 63);
      break;
    }
  }
  if (!block_construction) {  // ascending columns, signs travel with them
    for (int a = 1; a < alpha; ++a) {
      const int c = cols[a], s = neg[a];
      int b = a - 1;
      while (b >= 0 && cols[b] > c) {
        cols[b + 1] = cols[b];
        neg[b + 1] = neg[b];
        --b;
      }
      cols[b + 1] = c;
      neg[b + 1] = s;
    }
  }
  int32_t* o = out + i * alpha;
  for (int k = 0; k < alpha; ++k)
    o[k] = (int32_t)((uint32_t)(cols[k] + col_off) | ((uint32_t)neg[k] << 31));
}

int gen_sjlt_block(sk_op* h, int block, int col_off, int width, cudaStream_t s) {
  if (block >= h->sjlt_blocks_cap) {
    const int new_cap = std::max(8, 2 * h->sjlt_blocks_cap);
    int32_t* p = nullptr;
    const size_t per = (size_t)h->n * h->alpha * sizeof(int32_t);
    JLS_CHECK_CUDA(cudaMalloc(&p, per * new_cap));
    if (h->sjlt_ents) {
      JLS_CHECK_CUDA(cudaMemcpyAsync(p, h->sjlt_ents, per * h->sjlt_blocks_cap,
                                     cudaMemcpyDeviceToDevice, s));
      JLS_CHECK_CUDA(cudaStreamSynchronize(s));
      cudaFree(h->sjlt_ents);
    }
    h->sjlt_ents = p;
    h->sjlt_blocks_cap = new_cap;
  }
  const int threads = 256;
  const int64_t grid = (h->n + threads - 1) / threads;
  sjlt_draw_kernel<<<(unsigned)grid, threads, 0, s>>>(
      h->n, h->alpha, width, h->kind == SK_SJLT_BLOCK, h->seed, block, col_off,
      h->sjlt_ents + (size_t)block * h->n * h->alpha, h->d_err); note_launch();
  JLS_CHECK_CUDA(cudaGetLastError());
  return SK_OK;
}

// ---------------------------------------------------------------------------
// Tiled CCS build: one CTA per tile of `tile` rows of R.  Each thread owns
// columns c = tid, tid + blockDim, ...; blocks occupy disjoint column ranges
// (offsets boff[0..nblocks]), so column c is only looked up in its own
// block's alpha slots.  Pass 1 counts, a CTA scan turns counts into offsets,
// pass 2 writes the entries of each column in ascending row order
// (deterministic).
struct BlockOffsets {
  int n;
  int off[MAX_BLOCKS + 1];
};

// One CTA (256 threads) per tile of `tile` rows of R: a counting sort of the
// tile's entries by column.  (1) count per column with shared atomics; (2)
// exclusive scan; (3) place, one block of R at a time: the block's entries are
// staged in shared memory and warp 0 walks the rows in order, so rows stay
// ascending inside a column (a row has at most one entry per column within a
// block, and blocks own disjoint columns, so the running cursors never clash).
constexpr int CCS_THREADS = 256;
constexpr int CCS_STAGE = SJLT_TILE_F32 * SJLT_MAX_ALPHA;  // staged entries of one block

__global__ void __launch_bounds__(CCS_THREADS)
    ccs_build_kernel(const int32_t* __restrict__ ents, int64_t n, int alpha, const __grid_constant__ BlockOffsets bo,
                     int d_total, int tile, int esize, int64_t e_stride, int64_t o_stride, uint4* __restrict__ out_e,
                     uint32_t* __restrict__ out_o) {
  extern __shared__ uint32_t sh_cnt[];  // d_total + 1 counters / cursors
  __shared__ uint32_t th_sum[CCS_THREADS];
  __shared__ int32_t stage[CCS_STAGE];
  const int t = blockIdx.x, tid = threadIdx.x;
  const int64_t r0 = (int64_t)t * tile;
  const int rows = (int)min64(tile, n - r0);
  const int B = bo.n;
  for (int c = tid; c <= d_total; c += CCS_THREADS) sh_cnt[c] = 0;
  __syncthreads();
  const int per_blk = rows * alpha;
  for (int b = 0; b < B; ++b) {
    const int32_t* base = ents + ((int64_t)b * n + r0) * alpha;
    for (int q = tid; q < per_blk; q += CCS_THREADS) atomicAdd(&sh_cnt[base[q] & 0x7fffffff], 1u);
  }
  __syncthreads();
  // exclusive scan: each thread owns a contiguous chunk of counters
  const int chunk = (d_total + CCS_THREADS - 1) / CCS_THREADS;
  const int c_beg = min(d_total, tid * chunk), c_end = min(d_total, c_beg + chunk);
  uint32_t local = 0;
  for (int c = c_beg; c < c_end; ++c) local += sh_cnt[c];
  th_sum[tid] = local;
  __syncthreads();
  if (tid == 0) {
    uint32_t acc = 0;
    for (int q = 0; q < CCS_THREADS; ++q) {
      const uint32_t v = th_sum[q];
      th_sum[q] = acc;
      acc += v;
    }
    sh_cnt[d_total] = acc;
  }
  __syncthreads();
  uint32_t acc = th_sum[tid];
  for (int c = c_beg; c < c_end; ++c) {
    const uint32_t v = sh_cnt[c];
    sh_cnt[c] = acc;
    acc += v;
  }
  __syncthreads();
  uint32_t* oo = out_o + (int64_t)t * o_stride;
  uint4* oe = out_e + (int64_t)t * e_stride;
  for (int c = tid; c <= d_total; c += CCS_THREADS) oo[c] = sh_cnt[c];
  __syncthreads();
  for (int b = 0; b < B; ++b) {
    const int32_t* base = ents + ((int64_t)b * n + r0) * alpha;
    for (int q = tid; q < per_blk; q += CCS_THREADS) stage[q] = base[q];
    __syncthreads();
    if (tid < 32) {
      for (int r = 0; r < rows; ++r) {
        for (int k = tid; k < alpha; k += 32) {
          const int32_t e = stage[r * alpha + k];
          const uint32_t pos = sh_cnt[e & 0x7fffffff]++;
          // {S' offset of row r, sign, sign, S offset of row r}, see TiledCcs
          uint4 rec;
          const uint32_t neg = e < 0 ? 0x80000000u : 0u;
          rec.x = (uint32_t)r * CCS_ROW_BYTES;
          rec.w = (uint32_t)(r * esize);
          if (esize == 4) {  // FP32 kernels load one word: offset | sign bit
            rec.x |= neg;
            rec.w |= neg;
            rec.y = rec.z = neg | 0x3f800000u;
          } else {
            rec.y = 0u;
            rec.z = (e < 0) ? 0xbff00000u : 0x3ff00000u;
          }
          oe[pos] = rec;
        }
        __syncwarp();
      }
    }
    __syncthreads();
  }
}

int build_ccs(sk_op* h, int which_tile, cudaStream_t s) {
  TiledCcs& C = h->ccs[which_tile];
  const int tile = which_tile == 0 ? SJLT_TILE_F32 : SJLT_TILE_F64;
  if (C.built_d == h->d_total && C.tile == tile) return SK_OK;
  const int B = (int)h->blocks.size();
  if (B > MAX_BLOCKS) return SK_ERR_UNSUPPORTED;
  C.tile = tile;
  C.ntiles = (int)((h->n + tile - 1) / tile);
  C.e_stride = (int64_t)h->alpha * B * tile;
  C.o_stride = ((int64_t)h->d_total + 1 + 3) / 4 * 4;
  const size_t eb = (size_t)C.e_stride * C.ntiles * sizeof(uint4);
  const size_t ob = (size_t)C.o_stride * C.ntiles * sizeof(uint32_t);
  if (eb > C.ents_cap) {
    if (C.ents) cudaFree(C.ents);
    C.ents = nullptr;
    C.ents_cap = 0;
    JLS_CHECK_CUDA(cudaMalloc(&C.ents, eb));
    C.ents_cap = eb;
  }
  if (ob > C.offs_cap) {
    if (C.offs) cudaFree(C.offs);
    C.offs = nullptr;
    C.offs_cap = 0;
    JLS_CHECK_CUDA(cudaMalloc(&C.offs, ob));
    C.offs_cap = ob;
  }
  BlockOffsets bo;
  bo.n = B;
  int off = 0;
  for (int b = 0; b < B; ++b) {
    bo.off[b] = off;
    off += h->blocks[b];
  }
  bo.off[B] = off;
  const size_t shm = sizeof(uint32_t) * (h->d_total + 1);
  JLS_CHECK_CUDA(cudaFuncSetAttribute(ccs_build_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  ccs_build_kernel<<<C.ntiles, CCS_THREADS, shm, s>>>(h->sjlt_ents, h->n, h->alpha, bo, h->d_total, tile,
                                              which_tile == 0 ? 4 : 8, C.e_stride, C.o_stride, C.ents, C.offs);
  note_launch();
  JLS_CHECK_CUDA(cudaGetLastError());
  C.built_d = h->d_total;
  return SK_OK;
}

// R (x) I_2 for complex data (S = A R of an interleaved complex A): row 2j + t
// of it carries row j's nonzeros at columns 2c + t with the same signs.
__global__ void sjlt_expand2_kernel(const int32_t* __restrict__ ents, int64_t n, int alpha, int blocks,
                                    int32_t* __restrict__ out) {
  const int64_t total = (int64_t)blocks * n * alpha;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = q / (n * alpha), rem = q - b * n * alpha;
    const int64_t j = rem / alpha, k = rem - j * alpha;
    const uint32_t e = (uint32_t)ents[q], col = e & 0x7fffffffu, neg = e & 0x80000000u;
#pragma unroll
    for (uint32_t t = 0; t < 2; ++t)
      out[((b * 2 * n) + 2 * j + t) * alpha + k] = (int32_t)((2 * col + t) | neg);
  }
}

int build_ccs_complex(sk_op* h, cudaStream_t s) {
  TiledCcs& C = h->ccs[2];
  if (C.built_d == h->d_total && C.tile == SJLT_TILE_F32) return SK_OK;
  const int B = (int)h->blocks.size();
  if (B > MAX_BLOCKS) return SK_ERR_UNSUPPORTED;
  const int64_t n2 = 2 * h->n;
  const int d2 = 2 * h->d_total;
  const size_t need = (size_t)B * n2 * h->alpha * sizeof(int32_t);
  if (need > h->ents2_bytes) {
    if (h->sjlt_ents2) cudaFree(h->sjlt_ents2);
    h->sjlt_ents2 = nullptr;
    h->ents2_bytes = 0;
    JLS_CHECK_CUDA(cudaMalloc(&h->sjlt_ents2, need));
    h->ents2_bytes = need;
  }
  sjlt_expand2_kernel<<<(unsigned)(4 * num_sms()), 256, 0, s>>>(h->sjlt_ents, h->n, h->alpha, B, h->sjlt_ents2);
  note_launch();
  JLS_CHECK_CUDA(cudaGetLastError());
  const int tile = SJLT_TILE_F32;
  C.tile = tile;
  C.ntiles = (int)((n2 + tile - 1) / tile);
  C.e_stride = (int64_t)h->alpha * B * tile;
  C.o_stride = ((int64_t)d2 + 1 + 3) / 4 * 4;
  const size_t eb = (size_t)C.e_stride * C.ntiles * sizeof(uint4);
  const size_t ob = (size_t)C.o_stride * C.ntiles * sizeof(uint32_t);
  if (eb > C.ents_cap) {
    if (C.ents) cudaFree(C.ents);
    C.ents = nullptr;
    C.ents_cap = 0;
    JLS_CHECK_CUDA(cudaMalloc(&C.ents, eb));
    C.ents_cap = eb;
  }
  if (ob > C.offs_cap) {
    if (C.offs) cudaFree(C.offs);
    C.offs = nullptr;
    C.offs_cap = 0;
    JLS_CHECK_CUDA(cudaMalloc(&C.offs, ob));
    C.offs_cap = ob;
  }
  BlockOffsets bo;
  bo.n = B;
  int off = 0;
  for (int b = 0; b < B; ++b) {
    bo.off[b] = off;
    off += 2 * h->blocks[b];
  }
  bo.off[B] = off;
  const size_t shm = sizeof(uint32_t) * (d2 + 1);
  JLS_CHECK_CUDA(cudaFuncSetAttribute(ccs_build_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  ccs_build_kernel<<<C.ntiles, CCS_THREADS, shm, s>>>(h->sjlt_ents2, n2, h->alpha, bo, d2, tile, 4, C.e_stride,
                                                      C.o_stride, C.ents, C.offs);
  note_launch();
  JLS_CHECK_CUDA(cudaGetLastError());
  C.built_d = h->d_total;
  return SK_OK;
}

// ---------------------------------------------------------------------------
// SRHT
__global__ void srht_diag_kernel(int64_t n, uint64_t seed, int8_t* __restrict__ diag) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const u64x4 w = philox4x64_10((uint64_t)i, 0, 0, 0, seed, TAG_SRHT_D);
  diag[i] = (w.x0 >> 63) ? (int8_t)-1 : (int8_t)1;
}

// One thread: continue the sequence of candidate columns from the saved
// counter until d_new distinct columns exist.  Membership uses an
// open-addressing table in shared memory (capacity `cap`, a power of two).
__global__ void srht_mu_kernel(int64_t nu, uint64_t seed, int d_old, int d_new, int cap, bool replace,
                               int32_t* __restrict__ mu, unsigned long long* __restrict__ state,
                               int* err) {
  extern __shared__ int32_t table[];
  if (threadIdx.x != 0) return;
  if (replace) {  // every accepted draw, repeats kept (sampling with replacement)
    unsigned long long t = state[0];
    for (int have = d_old; have < d_new;) {
      const u64x4 w = philox4x64_10((uint64_t)t, 0, 0, 0, seed, TAG_SRHT_MU);
      ++t;
      uint64_t v;
      if (lemire(w.x0, (uint64_t)nu, &v)) mu[have++] = (int32_t)v;
    }
    state[0] = t;
    return;
  }
  for (int q = 0; q < cap; ++q) table[q] = -1;
  auto insert = [&](int32_t v) -> bool {  // true if newly inserted
    uint32_t hsh = ((uint32_t)v * 2654435761u) & (cap - 1);
    while (true) {
      if (table[hsh] == v) return false;
      if (table[hsh] < 0) {
        table[hsh] = v;
        return true;
      }
      hsh = (hsh + 1) & (cap - 1);
    }
  };
  for (int q = 0; q < d_old; ++q) insert(mu[q]);
  unsigned long long t = state[0];
  int have = d_old;
  uint64_t guard = 0;
  while (have < d_new) {
    if (++guard > (1ull << 32)) {
      set_err(err, ERRF_RNG);
      return;
    }
    const u64x4 w = philox4x64_10((uint64_t)t, 0, 0, 0, seed, TAG_SRHT_MU);
    ++t;
    uint64_t v;
    if (!lemire(w.x0, (uint64_t)nu, &v)) continue;
    if (insert((int32_t)v)) mu[have++] = (int32_t)v;
  }
  state[0] = t;
}

int gen_srht(sk_op* h, int d_old, int d_new, cudaStream_t s) {
  if (!h->srht_diag) {
    JLS_CHECK_CUDA(cudaMalloc(&h->srht_diag, h->n));
    JLS_CHECK_CUDA(cudaMalloc(&h->srht_mu, sizeof(int32_t) * h->d_max));
    JLS_CHECK_CUDA(cudaMalloc(&h->srht_state, sizeof(unsigned long long)));
    JLS_CHECK_CUDA(cudaMemsetAsync(h->srht_state, 0, sizeof(unsigned long long), s));
    const int threads = 256;
    srht_diag_kernel<<<(unsigned)((h->n + threads - 1) / threads), threads, 0, s>>>(h->n, h->seed,
                                                                                    h->srht_diag); note_launch();
    JLS_CHECK_CUDA(cudaGetLastError());
  }
  const bool replace = (h->flags & SK_SRHT_REPLACE) != 0;
  int cap = 1;
  while (!replace && cap < 2 * d_new) cap <<= 1;
  const size_t shm = sizeof(int32_t) * cap;
  if (shm > 48 * 1024)
    JLS_CHECK_CUDA(
        cudaFuncSetAttribute(srht_mu_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  srht_mu_kernel<<<1, 32, shm, s>>>(h->nu, h->seed, d_old, d_new, cap, replace, h->srht_mu, h->srht_state,
                                    h->d_err); note_launch();
  JLS_CHECK_CUDA(cudaGetLastError());
  return SK_OK;
}

// ---------------------------------------------------------------------------
// Gaussian z (unscaled N(0,1)), stored transposed: plane[c * n + i].
__device__ __forceinline__ double gauss_z(int64_t i, int c, uint64_t seed) {
  const u64x4 w = philox4x64_10((uint64_t)i, (uint64_t)(c >> 1), 0, 0, seed, TAG_GAUSS);
  const double u1 = u53_open0(w.x0);
  const double u2 = u53(w.x1);
  const double rad = sqrt(-2.0 * log(u1));
  double sn, cs;
  sincospi(2.0 * u2, &sn, &cs);
  return (c & 1) ? rad * sn : rad * cs;
}

// The same draw with the transcendental steps in FP32, for the FP32 and bf16
// planes (GB300 runs FP64 at a small fraction of its FP32 rate): the uniforms
// are the same 53-bit values; -2 ln u1 takes logf(u1) below 1/2 and
// log1pf(-(1 - u1)) above it (1 - u1 is exact in FP64), so both tails keep
// FP32 relative accuracy; the angle is sincospif(2 u2).  The result differs
// from the FP64 draw by a few FP32 ulps.
__device__ __forceinline__ float gauss_z32(int64_t i, int c, uint64_t seed) {
  const u64x4 w = philox4x64_10((uint64_t)i, (uint64_t)(c >> 1), 0, 0, seed, TAG_GAUSS);
  const double u1 = u53_open0(w.x0);
  const double u2 = u53(w.x1);
  const float l = u1 < 0.5 ? logf((float)u1) : log1pf(-(float)(1.0 - u1));
  const float rad = sqrtf(-2.0f * l);
  float sn, cs;
  sincospif(2.0f * (float)u2, &sn, &cs);
  return (c & 1) ? rad * sn : rad * cs;
}

__global__ void gauss_gen_kernel(int64_t n, int c0, int c1, uint64_t seed, float* __restrict__ z32,
                                 double* __restrict__ z64, __nv_bfloat16* __restrict__ zhi,
                                 __nv_bfloat16* __restrict__ zlo) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int c = c0 + blockIdx.y;
  if (i >= n || c >= c1) return;
  const int64_t o = (int64_t)c * n + i;
  if (z64) z64[o] = gauss_z(i, c, seed);
  if (!z32 && !zhi) return;
  const float zf = gauss_z32(i, c, seed);
  if (z32) z32[o] = zf;
  if (zhi) {  // z = z_hi + z_lo + O(2^-16 |z|): the two bf16 terms of the FP32 draw
    const int64_t ob = (int64_t)c * bf_pitch(n) + i;
    const __nv_bfloat16 hi = __float2bfloat16_rn(zf);
    zhi[ob] = hi;
    zlo[ob] = __float2bfloat16_rn(zf - __bfloat162float(hi));
  }
}

int gen_gauss(sk_op* h, int plane, int c_end, cudaStream_t s) {
  const size_t cells = (size_t)h->d_max * h->n;
  const size_t bf_cells = (size_t)h->d_max * bf_pitch(h->n);
  int* have = plane == 0 ? &h->z32_cols : plane == 1 ? &h->z64_cols : &h->zbf_cols;
  if (plane == 0 && !h->z32) JLS_CHECK_CUDA(cudaMalloc(&h->z32, cells * sizeof(float)));
  if (plane == 1 && !h->z64) JLS_CHECK_CUDA(cudaMalloc(&h->z64, cells * sizeof(double)));
  if (plane == 2 && !h->zhi) {
    JLS_CHECK_CUDA(cudaMalloc(&h->zhi, bf_cells * sizeof(uint16_t)));
    JLS_CHECK_CUDA(cudaMalloc(&h->zlo, bf_cells * sizeof(uint16_t)));
  }
  if (*have >= c_end) return SK_OK;
  const int c0 = *have;
  dim3 grid((unsigned)((h->n + 255) / 256), (unsigned)(c_end - c0));
  gauss_gen_kernel<<<grid, 256, 0, s>>>(h->n, c0, c_end, h->seed, plane == 0 ? h->z32 : nullptr,
                                        plane == 1 ? h->z64 : nullptr,
                                        plane == 2 ? reinterpret_cast<__nv_bfloat16*>(h->zhi) : nullptr,
                                        plane == 2 ? reinterpret_cast<__nv_bfloat16*>(h->zlo) : nullptr); note_launch();
  JLS_CHECK_CUDA(cudaGetLastError());
  *have = c_end;
  return SK_OK;
}

// SRHT +-1 plane (bf16 bits, exact), transposed: pm1[c * bf_pitch(n) + i] = d_i (-1)^popc(i & mu_c).
__global__ void srht_pm1_kernel(int64_t n, int c0, int c1, const int8_t* __restrict__ diag,
                                const int32_t* __restrict__ mu, uint16_t* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int c = c0 + blockIdx.y;
  if (i >= n || c >= c1) return;
  const int neg = (__popcll((unsigned long long)i & (unsigned long long)(uint32_t)mu[c]) & 1) ^ (diag[i] < 0);
  out[(int64_t)c * bf_pitch(n) + i] = neg ? (uint16_t)0xBF80 : (uint16_t)0x3F80;  // bf16 -1 / +1
}

int gen_srht_pm1(sk_op* h, int c_end, cudaStream_t s) {
  if (!h->srht_pm1)
    JLS_CHECK_CUDA(cudaMalloc(&h->srht_pm1, (size_t)h->d_max * bf_pitch(h->n) * sizeof(uint16_t)));
  if (h->pm1_cols >= c_end) return SK_OK;
  dim3 grid((unsigned)((h->n + 255) / 256), (unsigned)(c_end - h->pm1_cols));
  srht_pm1_kernel<<<grid, 256, 0, s>>>(h->n, h->pm1_cols, c_end, h->srht_diag, h->srht_mu, h->srht_pm1); note_launch();
  JLS_CHECK_CUDA(cudaGetLastError());
  h->pm1_cols = c_end;
  return SK_OK;
}

// SJLT sign plane for the tensor-core route: out[c][i] = +-1 (bf16) where row i
// of R has an entry in column c, 0 elsewhere (exact in bf16; the scale is the
// product's).  One thread per row of R for one block's entries.
__global__ void sjlt_pm1_kernel(int64_t n, int alpha, const int32_t* __restrict__ ents, uint16_t* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int k = 0; k < alpha; ++k) {
    const int32_t e = ents[i * alpha + k];
    out[(int64_t)(e & 0x7fffffff) * bf_pitch(n) + i] = e < 0 ? (uint16_t)0xBF80 : (uint16_t)0x3F80;
  }
}

// The SJLT's +-1 plane up to column c_end (whole blocks; kept in the handle's
// +-1 plane buffer, which SJLT operators do not otherwise use).
int gen_sjlt_pm1(sk_op* h, int c_end, cudaStream_t s) {
  const size_t pitch_b = (size_t)bf_pitch(h->n) * sizeof(uint16_t);
  if (!h->srht_pm1) JLS_CHECK_CUDA(cudaMalloc(&h->srht_pm1, (size_t)h->d_max * pitch_b));
  if (h->pm1_cols >= c_end) return SK_OK;
  int b0 = 0;
  for (size_t b = 0; b < h->blocks.size(); ++b) {
    const int w = h->blocks[b];
    if (b0 >= h->pm1_cols && b0 < c_end) {
      JLS_CHECK_CUDA(cudaMemsetAsync(reinterpret_cast<uint8_t*>(h->srht_pm1) + (size_t)b0 * pitch_b, 0,
                                     (size_t)w * pitch_b, s));
      sjlt_pm1_kernel<<<(unsigned)((h->n + 255) / 256), 256, 0, s>>>(h->n, h->alpha,
                                                                     h->sjlt_ents + (size_t)b * h->n * h->alpha,
                                                                     h->srht_pm1);
      note_launch();
      JLS_CHECK_CUDA(cudaGetLastError());
    }
    b0 += w;
  }
  h->pm1_cols = std::max(h->pm1_cols, std::min(c_end, b0));
  return SK_OK;
}

// ---------------------------------------------------------------------------
// FP8 planes.  Gaussian: one CTA of 128 threads per (K tile of 128, column c)
// draws the tile's FP32 z (as for the FP32 plane), takes its amax, and writes
// w_hi = e4m3(z / s), w_lo = e4m3(z / s - w_hi) with s = amax / 448, and s.
// Columns are quantized independently, so an increment never changes the
// planes of earlier columns.
__global__ void gauss_fp8_kernel(int64_t n, int c0, uint64_t seed, int64_t pitch, int64_t sld, uint8_t* __restrict__ zh,
                                 uint8_t* __restrict__ zl, float* __restrict__ zs) {
  __shared__ float wmax[4];
  const int kt = blockIdx.x, c = c0 + blockIdx.y;
  const int64_t k = (int64_t)kt * F8_KTILE + threadIdx.x;
  const float z = k < n ? gauss_z32(k, c, seed) : 0.f;
  float m = fabsf(z);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
  __syncthreads();
  const float amax = fmaxf(fmaxf(wmax[0], wmax[1]), fmaxf(wmax[2], wmax[3]));
  const float inv = amax > 0.f ? 448.f / amax : 0.f;
  const float y = z * inv;
  const uint32_t h = e4m3x2(y, 0.f) & 0xffu;
  const float r = y - e4m3x2_to_f2(h).x;
  const uint32_t l = e4m3x2(r, 0.f) & 0xffu;
  if (k < n) {
    zh[(int64_t)c * pitch + k] = (uint8_t)h;
    zl[(int64_t)c * pitch + k] = (uint8_t)l;
  }
  if (threadIdx.x == 0) zs[(int64_t)kt * sld + c] = amax / 448.f;
}

int gen_gauss_fp8(sk_op* h, int c_end, cudaStream_t s) {
  const int64_t kts = (h->n + F8_KTILE - 1) / F8_KTILE;
  if (!h->z8_hi) {
    const size_t bytes = (size_t)h->d_max * f8_pitch(h->n);
    JLS_CHECK_CUDA(cudaMalloc(&h->z8_hi, bytes));
    JLS_CHECK_CUDA(cudaMalloc(&h->z8_lo, bytes));
    JLS_CHECK_CUDA(cudaMalloc(&h->z8_scale, (size_t)kts * h->d_max * sizeof(float)));
  }
  if (h->z8_cols >= c_end) return SK_OK;
  dim3 grid((unsigned)kts, (unsigned)(c_end - h->z8_cols));
  gauss_fp8_kernel<<<grid, F8_KTILE, 0, s>>>(h->n, h->z8_cols, h->seed, f8_pitch(h->n), h->d_max, h->z8_hi, h->z8_lo,
                                             h->z8_scale); note_launch();
  JLS_CHECK_CUDA(cudaGetLastError());
  h->z8_cols = c_end;
  return SK_OK;
}

// SRHT sign plane in e4m3 (exact): 0x38 = +1.0, 0xB8 = -1.0.
__global__ void srht_q8_kernel(int64_t n, int c0, int c1, const int8_t* __restrict__ diag,
                               const int32_t* __restrict__ mu, int64_t pitch, uint8_t* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int c = c0 + blockIdx.y;
  if (i >= n || c >= c1) return;
  const int neg = (__popcll((unsigned long long)i & (unsigned long long)(uint32_t)mu[c]) & 1) ^ (diag[i] < 0);
  out[(int64_t)c * pitch + i] = neg ? (uint8_t)0xB8 : (uint8_t)0x38;
}

int gen_srht_fp8(sk_op* h, int c_end, cudaStream_t s) {
  if (!h->srht_q8) JLS_CHECK_CUDA(cudaMalloc(&h->srht_q8, (size_t)h->d_max * f8_pitch(h->n)));
  if (h->q8_cols >= c_end) return SK_OK;
  dim3 grid((unsigned)((h->n + 255) / 256), (unsigned)(c_end - h->q8_cols));
  srht_q8_kernel<<<grid, 256, 0, s>>>(h->n, h->q8_cols, c_end, h->srht_diag, h->srht_mu, f8_pitch(h->n), h->srht_q8);
  note_launch();
  JLS_CHECK_CUDA(cudaGetLastError());
  h->q8_cols = c_end;
  return SK_OK;
}

// ---------------------------------------------------------------------------
// Dense R for export (scale included), row-major n x d_total.
template <typename T>
__global__ void dense_R_kernel(int kind, int64_t n, int d_total, int alpha, int nblocks, double scale,
                               const int32_t* __restrict__ ents, const int8_t* __restrict__ diag,
                               const int32_t* __restrict__ mu, uint64_t seed, T* __restrict__ R) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  T* row = R + i * d_total;
  if (kind == SK_SJLT_BLOCK || kind == SK_SJLT_GRAPH) {
    for (int c = 0; c < d_total; ++c) row[c] = T(0);
    for (int b = 0; b < nblocks; ++b)
      for (int k = 0; k < alpha; ++k) {
        const int32_t e = ents[((int64_t)b * n + i) * alpha + k];
        row[e & 0x7fffffff] = (T)((e < 0) ? -scale : scale);
      }
  } else if (kind == SK_SRHT) {
    for (int c = 0; c < d_total; ++c) {
      const int neg = (__popcll((unsigned long long)i & (unsigned long long)(uint32_t)mu[c]) & 1) ^ (diag[i] < 0);
      row[c] = (T)(neg ? -scale : scale);
    }
  } else {
    for (int c = 0; c < d_total; ++c) row[c] = (T)(gauss_z(i, c, seed) * scale);
  }
}

int export_dense_R(sk_op* h, void* R_dev, int dtype, cudaStream_t s) {
  const int threads = 128;
  const unsigned grid = (unsigned)((h->n + threads - 1) / threads);
  const bool per_block = block_scaled(h);  // written unscaled, then each block's columns at its scale
  const double sc = per_block ? 1.0 : op_scale(h);
  if (dtype == SK_F64)
    dense_R_kernel<double><<<grid, threads, 0, s>>>(h->kind, h->n, h->d_total, h->alpha,
                                                    (int)h->blocks.size(), sc, h->sjlt_ents, h->srht_diag,
                                                    h->srht_mu, h->seed, (double*)R_dev);
  else
    dense_R_kernel<float><<<grid, threads, 0, s>>>(h->kind, h->n, h->d_total, h->alpha,
                                                   (int)h->blocks.size(), sc, h->sjlt_ents, h->srht_diag,
                                                   h->srht_mu, h->seed, (float*)R_dev); note_launch();
  JLS_CHECK_CUDA(cudaGetLastError());
  if (per_block) {
    int b0 = 0;
    for (const int w : h->blocks) {
      JLS_CHECK(scale_columns(R_dev, dtype, h->n, h->d_total, b0, b0 + w, 1.0 / std::sqrt((double)w), s));
      b0 += w;
    }
  }
  return SK_OK;
}

}  // namespace jls
