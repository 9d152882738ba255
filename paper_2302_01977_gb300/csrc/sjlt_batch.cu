// sjlt_batch.cu -- many SJLT sketches S'_i = A_i^T R_i in one persistent launch, sm_103a.
//
// The batched form of the S' product of Sec. 6.3 for many independent (and
// uneven) matrices, e.g. the kernel matrices of the leaves and nodes of an HSS
// tree or a set of independent problems, each with its own SJLT operator R_i
// and its own range of columns [c_lo_i, c_hi_i) of R_i (Algorithm 1 sketches
// the first d0 + Delta-d columns, then Delta-d new columns per increment).
//
// Work units are (instance, block of 128 columns of A_i, tile of 128 rows of
// A_i); the units of all active instances are numbered in one sequence and a
// persistent grid of one CTA per SM streams equal contiguous ranges of it
// (stream-K over the whole batch, so small and large instances load-balance).
// Within a unit the kernel does what sjlt_cols_kernel does: a TMA producer
// warp fills a ring of tiles with the instance's tile of A_i (its tensor map
// lives in the device-resident item table), the tile's entry records and
// column offsets ride along as bulk copies, and consumer warps accumulate
// their columns of R_i in registers and add them into the zeroed output when
// the CTA leaves a block (atomically: a block spans several CTAs' ranges when
// the batch has fewer units than a few per CTA, so the order of those adds,
// and the last bit of the sums, can differ between runs).
//
// The item table and a header (total units, staging sizes) are device memory
// written from a pinned host mirror by the run call itself, so a captured CUDA
// graph of sketch_batch_run replays with whatever sketch_batch_set last wrote.
// The kernel shape (warps per CTA x columns per warp) is picked by measuring
// the batch at creation (the autotuner below).
#include <cuda.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "batch.cuh"
#include "common.cuh"
#include "internal.h"
#include "sjlt_common.cuh"

namespace jls {

namespace {

constexpr int BTILE = 128, BBW = 128;
constexpr uint32_t BTILE_BYTES = BTILE * BBW * 4;

// index of the item holding unit u: the first i with unit0_i + units_i > u
__device__ __forceinline__ int item_of(const BItem* items, int nitems, int64_t u) {
  int lo = 0, hi = nitems - 1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (items[mid].unit0 + items[mid].units > u)
      hi = mid;
    else
      lo = mid + 1;
  }
  return lo;
}

template <int WARPS, int NB, int STAGES>
__global__ void __launch_bounds__(WARPS * 32, 1)
    sjlt_batch_kernel(const BItem* __restrict__ items, int nitems, const BHeader* __restrict__ hdr, int* err) {
  const int njobs = WARPS - 1;
  const int64_t T = hdr->total_units;
  const uint32_t E_BYTES = hdr->e_bytes, O_BYTES = hdr->o_bytes;
  extern __shared__ __align__(1024) uint8_t smem[];
  const uint32_t tiles_sa = smem_u32(smem);
  const uint32_t ents_sa = tiles_sa + STAGES * BTILE_BYTES;
  uint8_t* sh_o = smem + STAGES * (BTILE_BYTES + E_BYTES);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sh_o + STAGES * O_BYTES);
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + STAGES);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const SplitK rg = cta_range(T);

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full0 + 8 * s, 1);
      mbar_init(empty0 + 8 * s, njobs);
    }
    fence_mbar_init();
  }
  __syncthreads();

  if (warp == njobs) {  // ---- producer
    if (lane == 0 && rg.u1 > rg.u0) {
      int it = item_of(items, nitems, rg.u0);
      int k = 0;
      for (int64_t u = rg.u0; u < rg.u1; ++u, ++k) {
        while (items[it].unit0 + items[it].units <= u) ++it;
        const BItem* I = items + it;
        const int ntiles = I->ntiles, c_lo = I->c_lo, c_hi = I->c_hi;
        const int64_t v = u - I->unit0, blk = v / ntiles;
        const int t = (int)(v - blk * ntiles);
        const uint32_t* offs_t = I->offs + (int64_t)t * I->o_stride;
        const uint32_t lo = __ldg(offs_t + c_lo), hi = __ldg(offs_t + c_hi);
        const int o_lo = c_lo & ~3;
        const uint32_t ob = (uint32_t)((((c_hi + 1 + 3) & ~3) - o_lo) * 4);
        const uint32_t eb = (hi - lo) * 16;
        if (eb > E_BYTES || ob > O_BYTES) {  // host sizing guarantees this never happens
          set_err(err, ERRF_BOUNDS);
          break;
        }
        const int s = k % STAGES;
        if (k >= STAGES && !mbar_wait(empty0 + 8 * s, ((k / STAGES) - 1) & 1, err)) break;
        const uint32_t fb = full0 + 8 * s;
        mbar_arrive_expect_tx(fb, BTILE_BYTES + eb + ob);
        tma_load_2d(tiles_sa + s * BTILE_BYTES, &I->tm, fb, (int32_t)(blk * BBW), t * BTILE);
        if (eb) bulk_g2s(ents_sa + s * E_BYTES, I->ents + (int64_t)t * I->e_stride + lo, eb, fb);
        bulk_g2s(smem_u32(sh_o) + s * O_BYTES, offs_t + o_lo, ob, fb);
      }
    }
  } else {  // ---- consumers
    ColsAcc<float> acc[NB];
    const uint32_t lane_off = lane * 16;
    // the block whose sums are in acc: its output and this warp's columns there
    float* o_St = nullptr;
    int64_t o_ld = 0, o_cols = 0, o_blk = -1;
    int o_it = -1, o_cw0 = 0, o_nb = 0;
    float o_scale = 0.f;
    auto flush = [&]() {
      if (o_it < 0 || o_nb <= 0) return;
      const bool vec_ok = ((o_ld | o_cw0) & 3) == 0;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int64_t j = o_blk * BBW + lane * 4 + q;
        if (j < o_cols) {
          float v[NB];
#pragma unroll
          for (int b = 0; b < NB; ++b) v[b] = acc[b].get(q);
          flush_row<NB>(o_St + j * o_ld + o_cw0, v, o_nb, o_scale, vec_ok);
        }
      }
    };
    int it = rg.u1 > rg.u0 ? item_of(items, nitems, rg.u0) : 0;
    int k = 0;
    bool ok = true;
    for (int64_t u = rg.u0; u < rg.u1 && ok; ++u, ++k) {
      while (items[it].unit0 + items[it].units <= u) ++it;
      const BItem* I = items + it;
      const int ntiles = I->ntiles;
      const int64_t v = u - I->unit0, blk = v / ntiles;
      if (it != o_it || blk != o_blk) {  // a new block of outputs
        flush();
#pragma unroll
        for (int b = 0; b < NB; ++b) acc[b].zero();
        o_it = it;
        o_blk = blk;
        o_St = I->St;
        o_ld = I->ldSt;
        o_cols = I->cols;
        o_scale = I->scale;
        const int nbw = I->nbw;
        o_cw0 = I->c_lo + warp * nbw;
        o_nb = max(0, min(nbw, I->c_hi - o_cw0));
      }
      const int s = k % STAGES;
      if (!mbar_wait(full0 + 8 * s, (k / STAGES) & 1, err)) {
        ok = false;
        break;
      }
      if (o_nb > 0) {
        const int c_lo = I->c_lo, o_lo = c_lo & ~3;
        const uint32_t* O = reinterpret_cast<const uint32_t*>(sh_o + s * O_BYTES) - o_lo;
        const uint32_t ebase = ents_sa + s * E_BYTES - O[c_lo] * 16;
        const uint32_t xaddr = tiles_sa + s * BTILE_BYTES + lane_off;
        uint32_t p = O[o_cw0];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          if (b < o_nb) {
            const uint32_t e = O[o_cw0 + b + 1];
            uint32_t ea = ebase + p * 16;
            for (; p + 1 < e; p += 2, ea += 32) {
              const uint32_t r0 = CcsRec<float>::cols(ea), r1 = CcsRec<float>::cols(ea + 16);
              acc[b].add(xaddr, r0);
              acc[b].add(xaddr, r1);
            }
            if (p < e) {
              acc[b].add(xaddr, CcsRec<float>::cols(ea));
              ++p;
            }
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(empty0 + 8 * s);
    }
    if (ok) flush();
  }
  __syncthreads();  // no CTA exits while its copies may still land in shared memory
}

// zero columns [c_lo, c_hi) of every active instance's output (one CTA per instance)
__global__ void batch_zero_kernel(const BItem* __restrict__ items, int nitems) {
  const int i = blockIdx.x;
  if (i >= nitems || items[i].units == 0) return;
  const BItem* I = items + i;
  const int w = I->c_hi - I->c_lo;
  const int64_t total = I->cols * w;
  for (int64_t e = threadIdx.x; e < total; e += blockDim.x) {
    const int64_t j = e / w;
    I->St[j * I->ldSt + I->c_lo + (e - j * w)] = 0.f;
  }
}

// ---- the kernel shapes the autotuner chooses among ------------------------------------
struct BConfig {
  int warps, nb;
  void (*k3)(const BItem*, int, const BHeader*, int*);
  void (*k2)(const BItem*, int, const BHeader*, int*);
};
// wide shapes take Algorithm 1's first d0 + Delta-d columns in one pass; the
// narrow one keeps 16 or more warps busy on a Delta-d = 32 increment
const BConfig kConfigs[] = {
    {24, 13, sjlt_batch_kernel<24, 13, 3>, sjlt_batch_kernel<24, 13, 2>},
    {20, 16, sjlt_batch_kernel<20, 16, 3>, sjlt_batch_kernel<20, 16, 2>},
    {16, 20, sjlt_batch_kernel<16, 20, 3>, sjlt_batch_kernel<16, 20, 2>},
    {32, 2, sjlt_batch_kernel<32, 2, 3>, sjlt_batch_kernel<32, 2, 2>},
};
constexpr int kNumConfigs = sizeof(kConfigs) / sizeof(kConfigs[0]);
constexpr long BSMEM_MAX = 227 * 1024;

}  // namespace
}  // namespace jls

struct sk_batch {
  int device = 0;
  int count = 0;
  std::vector<sk_batch_item> items;
  jls::BItem* h_items = nullptr;  // pinned mirror of the item table
  jls::BHeader* h_hdr = nullptr;
  jls::BItem* d_items = nullptr;
  jls::BHeader* d_hdr = nullptr;
  int* d_err = nullptr;
  int config = -1;  // index into kConfigs, chosen by measurement
  float tuned_ms[jls::kNumConfigs] = {};
  // the adaptive loop (sketch_batch_adaptive_setup)
  bool adaptive = false;
  int cfg_first = -1, cfg_inc = -1;  // shapes for the first sketch and for the increments
  int a_stages = 0, max_tests = 0;
  int a_ncl = 1;  // CTAs per instance in the test kernel
  bool a_wide = false;  // some instance's basis passes ADAPT_QSMEM columns
  size_t a_smem = 0;
  double eps_rel = 0.0, eps_abs = 0.0;
  jls::BItem* d_items0 = nullptr;  // the item table and header of round 0
  jls::BHeader* d_hdr0 = nullptr;
  jls::ATest* d_tests = nullptr;   // per-instance loop state, and its initial value
  jls::ATest* d_tests0 = nullptr;
  int* d_order = nullptr;          // instances, largest first (the test kernel's cluster order)
  float* d_basis = nullptr;        // Q_i and W_i of every instance
};

namespace jls {
namespace {

// staging bytes a tile of the range [lo, hi) of R's columns needs: alpha entry
// records per row for each block the range touches, and the column offsets
void range_staging(const sk_op* h, int lo, int hi, uint32_t* e_max, uint32_t* o_max) {
  int off = 0, touched = 0;
  for (int w : h->blocks) {
    if (off < hi && off + w > lo) ++touched;
    off += w;
  }
  *e_max = std::max<uint32_t>(*e_max, (uint32_t)(BTILE * h->alpha * touched * 16));
  *o_max = std::max<uint32_t>(*o_max, (uint32_t)((((hi + 1 + 3) & ~3) - (lo & ~3)) * 4));
}

int staging_fit(uint32_t e_max, uint32_t o_max, BHeader* hdr, int* stages, size_t* smem) {
  o_max = (o_max + 15) / 16 * 16;
  hdr->e_bytes = e_max;
  hdr->o_bytes = o_max;
  for (int st = 3; st >= 2; --st) {
    const size_t need = (size_t)st * (BTILE_BYTES + e_max + o_max) + 2 * st * 8;
    if ((long)need <= BSMEM_MAX) {
      *stages = st;
      *smem = need;
      return SK_OK;
    }
  }
  return SK_ERR_UNSUPPORTED;
}

int batch_layout(sk_batch* b, int* stages, size_t* smem) {
  // staging sizes for the widest column range of any active instance
  uint32_t e_max = 16, o_max = 16;
  for (int i = 0; i < b->count; ++i) {
    const BItem& I = b->h_items[i];
    if (I.units) range_staging(b->items[i].op, I.c_lo, I.c_hi, &e_max, &o_max);
  }
  return staging_fit(e_max, o_max, b->h_hdr, stages, smem);
}

int batch_launch(sk_batch* b, int cfg, cudaStream_t s) {
  int stages = 0;
  size_t smem = 0;
  JLS_CHECK(batch_layout(b, &stages, &smem));
  JLS_CHECK_CUDA(cudaMemcpyAsync(b->d_items, b->h_items, sizeof(BItem) * b->count, cudaMemcpyHostToDevice, s));
  JLS_CHECK_CUDA(cudaMemcpyAsync(b->d_hdr, b->h_hdr, sizeof(BHeader), cudaMemcpyHostToDevice, s));
  if (b->h_hdr->total_units == 0) return SK_OK;
  batch_zero_kernel<<<b->count, 256, 0, s>>>(b->d_items, b->count);
  note_launch();
  JLS_CHECK_CUDA(cudaGetLastError());
  const BConfig& C = kConfigs[cfg];
  auto kern = stages == 3 ? C.k3 : C.k2;  // shared-memory limit raised at creation
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(num_sms(), b->h_hdr->total_units));
  kern<<<grid, C.warps * 32, smem, s>>>(b->d_items, b->count, b->d_hdr, b->d_err);
  note_launch();
  JLS_CHECK_CUDA(cudaGetLastError());
  return SK_OK;
}

// zero and sketch on the device table as it stands (its units are counted on
// the device, so the grid is one CTA per SM; CTAs without units exit)
int batch_launch_device(sk_batch* b, int cfg, cudaStream_t s) {
  batch_zero_kernel<<<b->count, 256, 0, s>>>(b->d_items, b->count);
  note_launch();
  const BConfig& C = kConfigs[cfg];
  auto kern = b->a_stages == 3 ? C.k3 : C.k2;
  kern<<<num_sms(), C.warps * 32, b->a_smem, s>>>(b->d_items, b->count, b->d_hdr, b->d_err);
  note_launch();
  JLS_CHECK_CUDA(cudaGetLastError());
  return SK_OK;
}

// number the units of the active instances; per-instance columns per consumer warp
int batch_number(sk_batch* b, int cfg) {
  int64_t u = 0;
  const int njobs = kConfigs[cfg].warps - 1, nb = kConfigs[cfg].nb;
  for (int i = 0; i < b->count; ++i) {
    BItem& I = b->h_items[i];
    I.unit0 = u;
    if (I.units) {
      const int width = I.c_hi - I.c_lo;
      I.nbw = (width + njobs - 1) / njobs;
      if (I.nbw > nb) return SK_ERR_UNSUPPORTED;  // wider than this shape takes in one pass
      I.units = (int64_t)((I.cols + BBW - 1) / BBW) * I.ntiles;
      u += I.units;
    }
  }
  b->h_hdr->total_units = u;
  return SK_OK;
}

}  // namespace
}  // namespace jls

using namespace jls;

extern "C" {

// The autotuner: time every shape that takes the current ranges in one pass
// (one warm-up run, then three timed runs on `s`), keep the fastest.
static int batch_tune(sk_batch* b, cudaStream_t s) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return SK_ERR_DEVICE;
  const int prev = b->config;
  int rc = SK_OK;
  float best = 1e30f;
  b->config = -1;
  for (int c = 0; c < kNumConfigs; ++c) {
    b->tuned_ms[c] = -1.f;
    if (batch_number(b, c) != SK_OK) continue;
    if ((rc = batch_launch(b, c, s)) != SK_OK) break;  // warm-up
    cudaEventRecord(e0, s);
    for (int r = 0; r < 3 && rc == SK_OK; ++r) rc = batch_launch(b, c, s);
    cudaEventRecord(e1, s);
    if (rc != SK_OK || cudaEventSynchronize(e1) != cudaSuccess) {
      if (rc == SK_OK) rc = SK_ERR_DEVICE;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    b->tuned_ms[c] = ms / 3;
    if (ms < best) {
      best = ms;
      b->config = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc == SK_OK && b->config < 0) rc = SK_ERR_UNSUPPORTED;
  if (rc != SK_OK) {
    b->config = prev;
    if (prev >= 0) batch_number(b, prev);
    return rc;
  }
  batch_number(b, b->config);
  int flag = 0;
  if (cudaMemcpy(&flag, b->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess || flag) return SK_ERR_DEVICE;
  return SK_OK;
}

static int batch_fill(sk_batch* b, const int32_t* active, const int32_t* c_lo, const int32_t* c_hi) {
  for (int i = 0; i < b->count; ++i) {
    BItem& I = b->h_items[i];
    const sk_op* h = b->items[i].op;
    const int lo = c_lo ? c_lo[i] : I.c_lo, hi = c_hi ? c_hi[i] : I.c_hi;
    const bool on = active ? active[i] != 0 : I.units != 0;
    if (on && (lo < 0 || hi <= lo || hi > h->d_total || hi > h->ccs[0].built_d)) return SK_ERR_INVALID_ARG;
    I.c_lo = lo;
    I.c_hi = hi;
    I.units = on ? 1 : 0;  // numbered by batch_number
    const double sc = b->items[i].scale;
    I.scale = (float)(sc != 0.0 ? sc : op_scale(h));
  }
  return SK_OK;
}

static void adaptive_free(sk_batch* b) {
  if (b->d_items0) cudaFree(b->d_items0);
  if (b->d_hdr0) cudaFree(b->d_hdr0);
  if (b->d_tests) cudaFree(b->d_tests);
  if (b->d_tests0) cudaFree(b->d_tests0);
  if (b->d_order) cudaFree(b->d_order);
  if (b->d_basis) cudaFree(b->d_basis);
  b->d_items0 = nullptr;
  b->d_hdr0 = nullptr;
  b->d_tests = b->d_tests0 = nullptr;
  b->d_order = nullptr;
  b->d_basis = nullptr;
  b->adaptive = false;
}

int sketch_batch_create(sk_batch_handle* out, const sk_batch_item* items, int32_t count, void* stream) {
  if (!out || !items || count < 1) return SK_ERR_INVALID_ARG;
  *out = nullptr;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  PFN_encodeTiled enc = get_encode_tiled();
  if (!enc) return SK_ERR_DEVICE;
  for (int i = 0; i < count; ++i) {
    const sk_batch_item& it = items[i];
    const sk_op* h = it.op;
    if (!h || (h->kind != SK_SJLT_BLOCK && h->kind != SK_SJLT_GRAPH)) return SK_ERR_INVALID_ARG;
    if (!it.A || !it.St || it.rows != h->n || it.cols < 1 || it.ld < it.cols || it.ldSt < h->d_total)
      return SK_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(it.A) & 15u) || (it.ld * 4) % 16) return SK_ERR_ALIGN;
    if (it.c_lo < 0 || it.c_hi <= it.c_lo || it.c_hi > h->d_total) return SK_ERR_INVALID_ARG;
  }
  sk_batch* b = new sk_batch();
  b->count = count;
  b->items.assign(items, items + count);
  cudaGetDevice(&b->device);
  int rc = SK_OK;
  auto fail = [&](int code) {
    sketch_batch_destroy(b);
    return code;
  };
  if (cudaMallocHost(&b->h_items, sizeof(BItem) * count) != cudaSuccess ||
      cudaMallocHost(&b->h_hdr, sizeof(BHeader)) != cudaSuccess || cudaMalloc(&b->d_items, sizeof(BItem) * count) != cudaSuccess ||
      cudaMalloc(&b->d_hdr, sizeof(BHeader)) != cudaSuccess || cudaMalloc(&b->d_err, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return fail(SK_ERR_NOMEM);
  }
  std::memset(b->h_items, 0, sizeof(BItem) * count);
  std::memset(b->h_hdr, 0, sizeof(BHeader));
  if (cudaMemsetAsync(b->d_err, 0, sizeof(int), s) != cudaSuccess) return fail(SK_ERR_DEVICE);
  for (int i = 0; i < count; ++i) {
    const sk_batch_item& it = items[i];
    sk_op* h = it.op;
    if ((rc = build_ccs(h, 0, s)) != SK_OK) return fail(rc);
    const TiledCcs& C = h->ccs[0];
    BItem& I = b->h_items[i];
    const cuuint64_t gdim[2] = {(cuuint64_t)it.cols, (cuuint64_t)it.rows};
    const cuuint64_t gstride[1] = {(cuuint64_t)(it.ld * 4)};
    const cuuint32_t box[2] = {(cuuint32_t)BBW, (cuuint32_t)BTILE};
    const cuuint32_t estr[2] = {1, 1};
    if (enc(&I.tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(it.A), gdim, gstride, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return fail(SK_ERR_ALIGN);
    I.ents = C.ents;
    I.offs = C.offs;
    I.e_stride = C.e_stride;
    I.o_stride = C.o_stride;
    I.St = it.St;
    I.rows = it.rows;
    I.cols = it.cols;
    I.ldSt = it.ldSt;
    I.ntiles = C.ntiles;
    I.c_lo = it.c_lo;
    I.c_hi = it.c_hi;
    I.units = 1;
  }
  if ((rc = batch_fill(b, nullptr, nullptr, nullptr)) != SK_OK) return fail(rc);
  // the run path issues copies and kernels only (capturable): set the kernels' shared-memory limit now
  for (const BConfig& C : kConfigs)
    if (cudaFuncSetAttribute(C.k3, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BSMEM_MAX) != cudaSuccess ||
        cudaFuncSetAttribute(C.k2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BSMEM_MAX) != cudaSuccess) {
      cudaGetLastError();
      return fail(SK_ERR_DEVICE);
    }
  if ((rc = batch_tune(b, s)) != SK_OK) return fail(rc);
  *out = b;
  return SK_OK;
}

int sketch_batch_tune(sk_batch_handle b, void* stream) {
  if (!b) return SK_ERR_INVALID_ARG;
  return batch_tune(b, static_cast<cudaStream_t>(stream));
}

int sketch_batch_set(sk_batch_handle b, const int32_t* active, const int32_t* c_lo, const int32_t* c_hi) {
  if (!b) return SK_ERR_INVALID_ARG;
  JLS_CHECK(batch_fill(b, active, c_lo, c_hi));
  return batch_number(b, b->config);
}

int sketch_batch_run(sk_batch_handle b, void* stream) {
  if (!b) return SK_ERR_INVALID_ARG;
  return batch_launch(b, b->config, static_cast<cudaStream_t>(stream));
}

int sketch_batch_info(sk_batch_handle b, int32_t* warps, int32_t* cols_per_warp, int64_t* units, float* tuned_ms) {
  if (!b) return SK_ERR_INVALID_ARG;
  if (warps) *warps = kConfigs[b->config].warps;
  if (cols_per_warp) *cols_per_warp = kConfigs[b->config].nb;
  if (units) *units = b->h_hdr->total_units;
  if (tuned_ms)
    for (int c = 0; c < kNumConfigs; ++c) tuned_ms[c] = b->tuned_ms[c];  // kNumConfigs = 4
  return SK_OK;
}

int sketch_batch_status(sk_batch_handle b, void* stream) {
  if (!b) return SK_ERR_INVALID_ARG;
  JLS_CHECK_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  int flag = 0;
  JLS_CHECK_CUDA(cudaMemcpy(&flag, b->d_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (flag) JLS_CHECK_CUDA(cudaMemset(b->d_err, 0, sizeof(int)));
  if (flag & ERRF_TIMEOUT) return SK_ERR_TIMEOUT;
  return flag ? SK_ERR_DEVICE : SK_OK;
}

void sketch_batch_destroy(sk_batch_handle b) {
  if (!b) return;
  cudaDeviceSynchronize();
  if (b->h_items) cudaFreeHost(b->h_items);
  if (b->h_hdr) cudaFreeHost(b->h_hdr);
  if (b->d_items) cudaFree(b->d_items);
  if (b->d_hdr) cudaFree(b->d_hdr);
  if (b->d_err) cudaFree(b->d_err);
  adaptive_free(b);
  delete b;
}

// ---- the adaptive loop ----------------------------------------------------------------

int sketch_batch_adaptive_setup(sk_batch_handle b, const int32_t* d0, int32_t dd, double eps_rel, double eps_abs,
                                void* stream) {
  if (!b || !d0 || dd < 8 || dd > ADAPT_BW || dd % 8 || !(eps_rel >= 0.0) || !(eps_abs >= 0.0))
    return SK_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int count = b->count;
  for (int i = 0; i < count; ++i) {
    const sk_op* h = b->items[i].op;
    const int first = d0[i] + dd;
    if (d0[i] < 0 || d0[i] % 8 || h->blocks.empty() || h->blocks[0] != first) return SK_ERR_INVALID_ARG;
    for (size_t j = 1; j < h->blocks.size(); ++j)
      if (h->blocks[j] != dd) return SK_ERR_INVALID_ARG;  // R_i = JL(d0 + dd) grown by dd-column increments
    if (b->items[i].ldSt < h->d_total) return SK_ERR_INVALID_ARG;
    if (h->d_total - dd > ADAPT_QMAX) return SK_ERR_UNSUPPORTED;
  }
  JLS_CHECK_CUDA(cudaStreamSynchronize(s));
  adaptive_free(b);
  // operators grown since the batch was made: rebuild their tiles, refresh the table
  for (int i = 0; i < count; ++i) {
    sk_op* h = b->items[i].op;
    JLS_CHECK(build_ccs(h, 0, s));
    const TiledCcs& C = h->ccs[0];
    BItem& I = b->h_items[i];
    I.ents = C.ents;
    I.offs = C.offs;
    I.e_stride = C.e_stride;
    I.o_stride = C.o_stride;
    I.ntiles = C.ntiles;
  }
  // the kernel shapes: one for the increments [d0 + dd, d0 + 2 dd), one for the first sketch [0, d0 + dd)
  std::vector<int32_t> act(count), lo(count), hi(count);
  bool any = false;
  for (int i = 0; i < count; ++i) {
    const bool on = d0[i] + 2 * dd <= b->items[i].op->d_total;
    act[i] = on;
    lo[i] = on ? d0[i] + dd : 0;
    hi[i] = on ? d0[i] + 2 * dd : dd;
    any |= on;
  }
  if (any) {
    JLS_CHECK(batch_fill(b, act.data(), lo.data(), hi.data()));
    JLS_CHECK(batch_tune(b, s));
  }
  const int cfg_inc = b->config;
  for (int i = 0; i < count; ++i) {
    act[i] = 1;
    lo[i] = 0;
    hi[i] = d0[i] + dd;
  }
  JLS_CHECK(batch_fill(b, act.data(), lo.data(), hi.data()));
  JLS_CHECK(batch_tune(b, s));
  const int cfg_first = b->config;
  if ((kConfigs[cfg_inc].warps - 1) * kConfigs[cfg_inc].nb < dd) return SK_ERR_UNSUPPORTED;
  // staging for every range the loop can sketch
  uint32_t e_max = 16, o_max = 16;
  int max_tests = 0;
  for (int i = 0; i < count; ++i) {
    const sk_op* h = b->items[i].op;
    range_staging(h, 0, d0[i] + dd, &e_max, &o_max);
    for (int c = d0[i] + dd; c + dd <= h->d_total; c += dd) range_staging(h, c, c + dd, &e_max, &o_max);
    max_tests = std::max(max_tests, 1 + (h->d_total - d0[i] - dd) / dd);
  }
  BHeader hdr0 = *b->h_hdr;  // units of round 0, numbered for cfg_first by the tuner
  int stages = 0;
  size_t smem = 0;
  JLS_CHECK(staging_fit(e_max, o_max, &hdr0, &stages, &smem));
  // round 0's table: every instance sketches [0, d0 + dd) at the per-block scale 1/sqrt(alpha)
  std::vector<BItem> t0(b->h_items, b->h_items + count);
  for (int i = 0; i < count; ++i) t0[i].scale = (float)(1.0 / std::sqrt((double)b->items[i].op->alpha));
  // per-instance state; Q_i (cols_i x qcap_i) and W_i (cols_i x 32) in one allocation
  std::vector<ATest> a0(count);
  std::vector<size_t> off(count);
  size_t total = 0;
  bool wide = false;  // some basis passes ADAPT_QSMEM columns
  for (int i = 0; i < count; ++i) {
    const sk_op* h = b->items[i].op;
    const int qcap = std::max(8, (h->d_total - dd + 7) / 8 * 8);
    off[i] = total;
    total += (size_t)b->items[i].cols * (qcap + ADAPT_BW);
    if (qcap > ADAPT_QSMEM) total += (size_t)qcap * ADAPT_BW;  // Q^T W of a wide basis
    wide |= qcap > ADAPT_QSMEM;
    ATest& T = a0[i];
    std::memset(&T, 0, sizeof(T));
    T.S = b->items[i].St;
    T.rows = b->items[i].cols;
    T.ldS = b->items[i].ldSt;
    T.qcap = qcap;
    T.dd = dd;
    T.d_cap = h->d_total;
    T.first_w = d0[i] + dd;
    T.state = ADAPT_ACTIVE;
  }
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    return b->items[x].cols * (int64_t)b->items[x].op->d_total > b->items[y].cols * (int64_t)b->items[y].op->d_total;
  });
  if (cudaMalloc(&b->d_items0, sizeof(BItem) * count) != cudaSuccess ||
      cudaMalloc(&b->d_hdr0, sizeof(BHeader)) != cudaSuccess ||
      cudaMalloc(&b->d_tests, sizeof(ATest) * count) != cudaSuccess ||
      cudaMalloc(&b->d_tests0, sizeof(ATest) * count) != cudaSuccess ||
      cudaMalloc(&b->d_order, sizeof(int) * (2 * count + 1)) != cudaSuccess ||  // order, active list, count
      cudaMalloc(&b->d_basis, total * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    adaptive_free(b);
    return SK_ERR_NOMEM;
  }
  for (int i = 0; i < count; ++i) {
    const int qcap = a0[i].qcap;
    a0[i].Q = b->d_basis + off[i];
    a0[i].W = b->d_basis + off[i] + (size_t)b->items[i].cols * qcap;
    a0[i].G = qcap > ADAPT_QSMEM ? a0[i].W + (size_t)b->items[i].cols * ADAPT_BW : nullptr;
  }
  int rc = adaptive_prepare();
  if (rc == SK_OK &&
      (cudaMemcpy(b->d_items0, t0.data(), sizeof(BItem) * count, cudaMemcpyHostToDevice) != cudaSuccess ||
       cudaMemcpy(b->d_hdr0, &hdr0, sizeof(BHeader), cudaMemcpyHostToDevice) != cudaSuccess ||
       cudaMemcpy(b->d_tests0, a0.data(), sizeof(ATest) * count, cudaMemcpyHostToDevice) != cudaSuccess ||
       cudaMemcpy(b->d_order, order.data(), sizeof(int) * count, cudaMemcpyHostToDevice) != cudaSuccess))
    rc = SK_ERR_DEVICE;
  if (rc != SK_OK) {
    adaptive_free(b);
    return rc;
  }
  b->cfg_first = cfg_first;
  b->cfg_inc = cfg_inc;
  b->a_stages = stages;
  b->a_smem = smem;
  b->max_tests = max_tests;
  b->a_wide = wide;
  // the stopping test: one CTA per instance amortizes its fixed costs best; a
  // cluster of 4 per instance when the instances would not fill the GPU
  const char* env = std::getenv("JLS_ADAPT_CLUSTER");
  b->a_ncl = env ? std::atoi(env) : (count >= num_sms() ? 1 : 4);
  if (b->a_ncl != 1 && b->a_ncl != 2 && b->a_ncl != 4) b->a_ncl = 4;
  b->eps_rel = eps_rel;
  b->eps_abs = eps_abs;
  b->adaptive = true;
  return SK_OK;
}

int sketch_batch_adaptive_run(sk_batch_handle b, int32_t max_rounds, void* stream) {
  if (!b || !b->adaptive || max_rounds < 0) return SK_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int count = b->count;
  const int rounds = max_rounds ? std::min<int>(max_rounds, b->max_tests) : b->max_tests;
  JLS_CHECK_CUDA(cudaMemcpyAsync(b->d_items, b->d_items0, sizeof(BItem) * count, cudaMemcpyDeviceToDevice, s));
  JLS_CHECK_CUDA(cudaMemcpyAsync(b->d_hdr, b->d_hdr0, sizeof(BHeader), cudaMemcpyDeviceToDevice, s));
  JLS_CHECK_CUDA(cudaMemcpyAsync(b->d_tests, b->d_tests0, sizeof(ATest) * count, cudaMemcpyDeviceToDevice, s));
  const BConfig& Ci = kConfigs[b->cfg_inc];
  for (int r = 0; r < rounds; ++r) {
    JLS_CHECK(batch_launch_device(b, r == 0 ? b->cfg_first : b->cfg_inc, s));
    JLS_CHECK(adaptive_test_round(b->d_items, b->d_tests, b->d_order, count, b->a_ncl, b->eps_rel, b->eps_abs,
                                  b->a_wide, b->d_order + count, b->d_order + 2 * count, s));
    if (r + 1 < rounds) JLS_CHECK(adaptive_renumber_launch(b->d_items, count, b->d_hdr, Ci.warps - 1, Ci.nb, b->d_err, s));
  }
  return adaptive_rescale_launch(b->d_tests, count, s);
}

int sketch_batch_adaptive_result(sk_batch_handle b, int32_t* d_reached, int32_t* state, int32_t* tests, double* nh,
                                 double* nt, void* stream) {
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
  return sketch_batch_status(b, stream);
}

}  // extern "C"
