// kernel_sketch.cu -- gradient of the matrix-free kernel sketch, sm_103a.
//
// For S = K(X, X; h) R with K_ij = exp(-|x_i - x_j|^2 / (2 h^2)) and an SJLT R
// (the forward pass is sjlt_cols_kernel with computed tiles, sjlt_apply.cu),
// the upstream gradient dS gives L = <dS, S> = sum_mp G_mp K_mp, G = dS R^T, and
//
//   dX_m = (1/h^2) sum_p (G_mp + G_pm) K_mp (x_p - x_m)
//   dh   = (1/h^3) sum_mp G_mp K_mp |x_m - x_p|^2.
//
// One sweep over the ordered pairs (m, p) evaluates every w_mp = G_mp K_mp
// once.  A CTA owns 128 points m (4 per lane) and keeps their rows of dS in
// shared memory, one column c per 528-byte row, so that
// G_mp = scale * sum_k s_pk dS[m, c_pk] is alpha conflict-free 16-byte loads
// (the nonzeros (c_pk, s_pk) of row p of R are the same for the whole warp).
// K_mp is recomputed, never stored.  Each w_mp feeds
//   * the first sum of dX_m:  sum_p w_mp (x_p - x_m)  -- lane-local registers;
//   * the second sum of dX_p: sum_m w_mp (x_m - x_p)  -- a sum over the lanes:
//     each warp reduces 8 points p at a time with a 31-step butterfly and adds
//     the result to an n x 4 buffer U = (sum w, -sum w x_m) (red.global.add);
//     a last kernel adds -(U_a + x_pa U_0) / h^2 to dX_p;
//   * dh:  sum w_mp |x_m - x_p|^2, FP32 per batch, FP64 across batches and CTAs.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace jls {
namespace {

__device__ __forceinline__ float ex2_approx(float x) {  // the MUFU ex2 instruction (2^x)
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

constexpr int ADJ_MB = 128;     // points m per CTA (32 lanes x 4)
constexpr int ADJ_WARPS = 16;   // warps; warp w takes p = w, w + 16, ...
constexpr int ADJ_PITCH = 132;  // floats per column of the dS tile (16-byte aligned rows)
constexpr int ADJ_BATCH = 8;    // points p per butterfly reduction (8 x 4 values = one per lane)
constexpr int ADJ_MAX_D = 384;  // columns of dS the tile holds (203 KB)
constexpr int ADJ_MAX_ENT = 32; // nonzeros per row of R (alpha * blocks)

template <bool ALPHA4_ONE_BLOCK>
__global__ void __launch_bounds__(ADJ_WARPS * 32, 1)
    ksk_adjoint_kernel(const float* __restrict__ X, int64_t n, const float* __restrict__ dS, int64_t ldS, int d,
                       const int32_t* __restrict__ ents, int alpha, int blocks, float scale, float c2,
                       float inv_h2, double inv_h3, float* __restrict__ dX, float* __restrict__ U,
                       double* __restrict__ dh_acc, int* err) {
  extern __shared__ __align__(16) float sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t m0 = (int64_t)blockIdx.x * ADJ_MB;

  // rows m0 .. m0 + 127 of dS, transposed: sm[c * ADJ_PITCH + (m - m0)]
  for (int idx = threadIdx.x; idx < ADJ_MB * d; idx += blockDim.x) {
    const int mm = idx / d, c = idx - mm * d;
    const int64_t m = m0 + mm;
    sm[c * ADJ_PITCH + mm] = m < n ? __ldg(dS + m * ldS + c) : 0.f;
  }
  __syncthreads();

  // this lane's points m0 + 4 lane + q, negated, as pairs (q = 0,1) and (2,3)
  float2 nx[2], ny[2], nz[2];
#pragma unroll
  for (int h2 = 0; h2 < 2; ++h2) {
    float c[2][3];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const int64_t m = m0 + 4 * lane + 2 * h2 + e;
#pragma unroll
      for (int a = 0; a < 3; ++a) c[e][a] = m < n ? -__ldg(X + 3 * m + a) : 0.f;
    }
    nx[h2] = make_float2(c[0][0], c[1][0]);
    ny[h2] = make_float2(c[0][1], c[1][1]);
    nz[h2] = make_float2(c[0][2], c[1][2]);
  }
  const float2 nc2 = make_float2(-c2, -c2), z2 = make_float2(0.f, 0.f);
  float2 T0[2] = {z2, z2}, T1[2] = {z2, z2}, T2[2] = {z2, z2}, T3[2] = {z2, z2};
  double H = 0.0;
  const uint32_t tile = smem_u32(sm) + lane * 16;
  const uint32_t col_bytes = ADJ_PITCH * 4;

  for (int64_t p = warp; p < n; p += (int64_t)ADJ_BATCH * ADJ_WARPS) {
    float v[ADJ_BATCH * 4];
    float2 Hb = z2;
#pragma unroll
    for (int b = 0; b < ADJ_BATCH; ++b) {
      const int64_t pb = p + (int64_t)b * ADJ_WARPS;
      float u0 = 0.f, u1 = 0.f, u2 = 0.f, u3 = 0.f;
      if (pb < n) {  // uniform over the warp
        // G_mp = scale * sum_k s_pk dS[m, c_pk] for this lane's 4 points m
        float2 G0 = z2, G1 = z2;
        auto add = [&](int32_t e) {
          const uint32_t col = (uint32_t)e & 0x7fffffffu;
          const float sg = e < 0 ? -scale : scale;
          const float4 t = lds_f4(tile + col * col_bytes);
          const float2 s2 = make_float2(sg, sg);
          G0 = __ffma2_rn(make_float2(t.x, t.y), s2, G0);
          G1 = __ffma2_rn(make_float2(t.z, t.w), s2, G1);
        };
        if (ALPHA4_ONE_BLOCK) {
          const int4 e4 = __ldg(reinterpret_cast<const int4*>(ents) + pb);
          add(e4.x);
          add(e4.y);
          add(e4.z);
          add(e4.w);
        } else {
          for (int bl = 0; bl < blocks; ++bl) {
            const int32_t* er = ents + ((int64_t)bl * n + pb) * alpha;
            for (int k = 0; k < alpha; ++k) add(__ldg(er + k));
          }
        }
        const float px = __ldg(X + 3 * pb), py = __ldg(X + 3 * pb + 1), pz = __ldg(X + 3 * pb + 2);
        const float2 px2 = make_float2(px, px), py2 = make_float2(py, py), pz2 = make_float2(pz, pz);
        const float2 G[2] = {G0, G1};
        float2 su0 = z2, su1 = z2, su2 = z2, su3 = z2;
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2) {
          const float2 dx = __fadd2_rn(px2, nx[h2]), dy = __fadd2_rn(py2, ny[h2]), dz = __fadd2_rn(pz2, nz[h2]);
          const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
          const float2 a = __fmul2_rn(r2, nc2);
          const float2 w = __fmul2_rn(G[h2], make_float2(ex2_approx(a.x), ex2_approx(a.y)));
          T0[h2] = __fadd2_rn(T0[h2], w);
          T1[h2] = __ffma2_rn(w, px2, T1[h2]);
          T2[h2] = __ffma2_rn(w, py2, T2[h2]);
          T3[h2] = __ffma2_rn(w, pz2, T3[h2]);
          Hb = __ffma2_rn(w, r2, Hb);
          su0 = __fadd2_rn(su0, w);
          su1 = __ffma2_rn(w, nx[h2], su1);  // minus sum w x_m (coordinates are held negated)
          su2 = __ffma2_rn(w, ny[h2], su2);
          su3 = __ffma2_rn(w, nz[h2], su3);
        }
        u0 = su0.x + su0.y;
        u1 = su1.x + su1.y;
        u2 = su2.x + su2.y;
        u3 = su3.x + su3.y;
      }
      v[4 * b] = u0;
      v[4 * b + 1] = u1;
      v[4 * b + 2] = u2;
      v[4 * b + 3] = u3;
    }
    // reduce-scatter over the lanes: afterwards lane l holds the warp's sum of v[l]
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
      const bool up = (lane & w) != 0;
#pragma unroll
      for (int k = 0; k < w; ++k) {
        const float send = up ? v[k] : v[k + w];
        const float keep = up ? v[k + w] : v[k];
        v[k] = keep + __shfl_xor_sync(0xffffffffu, send, w);
      }
    }
    const int64_t pb = p + (int64_t)(lane >> 2) * ADJ_WARPS;
    if (pb < n) atomicAdd(U + 4 * pb + (lane & 3), v[0]);
    H += (double)Hb.x + (double)Hb.y;
  }

  // first sums: combine the warps, finish rows m of dX
  __syncthreads();
  float* red = sm;  // [ADJ_WARPS][ADJ_MB][4]
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float* r = red + ((size_t)warp * ADJ_MB + 4 * lane + q) * 4;
    const int h2 = q >> 1;
    const bool hi = q & 1;
    r[0] = hi ? T0[h2].y : T0[h2].x;
    r[1] = hi ? T1[h2].y : T1[h2].x;
    r[2] = hi ? T2[h2].y : T2[h2].x;
    r[3] = hi ? T3[h2].y : T3[h2].x;
  }
  __syncthreads();
  for (int mm = threadIdx.x; mm < ADJ_MB; mm += blockDim.x) {
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
    for (int w = 0; w < ADJ_WARPS; ++w) {
      const float* r = red + ((size_t)w * ADJ_MB + mm) * 4;
      s0 += r[0];
      s1 += r[1];
      s2 += r[2];
      s3 += r[3];
    }
    const int64_t m = m0 + mm;
    if (m < n) {
      dX[3 * m] = inv_h2 * (s1 - X[3 * m] * s0);
      dX[3 * m + 1] = inv_h2 * (s2 - X[3 * m + 1] * s0);
      dX[3 * m + 2] = inv_h2 * (s3 - X[3 * m + 2] * s0);
    }
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) H += __shfl_xor_sync(0xffffffffu, H, o);
  if (lane == 0) atomicAdd(dh_acc, H * inv_h3);
  (void)err;
}

// dX_p += the second sum / h^2, complete once every CTA has added to U
__global__ void ksk_finish_kernel(const float* __restrict__ X, int64_t n, const float* __restrict__ U, float inv_h2,
                                  float* __restrict__ dX) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const float4 u = reinterpret_cast<const float4*>(U)[p];
  // U_p = (sum_m w_mp, -sum_m w_mp x_m): the second sum is -U_p,a - x_pa U_p,0
  dX[3 * p] -= inv_h2 * (u.y + X[3 * p] * u.x);
  dX[3 * p + 1] -= inv_h2 * (u.z + X[3 * p + 1] * u.x);
  dX[3 * p + 2] -= inv_h2 * (u.w + X[3 * p + 2] * u.x);
}

}  // namespace

int kernel_sketch_adjoint(sk_op* h, const float* X, double hbw, double scale, const float* dS, int64_t ldS,
                          float* dX, double* dh, cudaStream_t s) {
  if (h->kind != SK_SJLT_BLOCK && h->kind != SK_SJLT_GRAPH) return SK_ERR_UNSUPPORTED;
  const int d = h->d_total, blocks = (int)h->blocks.size();
  if (d > ADJ_MAX_D || h->alpha * blocks > ADJ_MAX_ENT) return SK_ERR_UNSUPPORTED;
  const int64_t n = h->n;
  const size_t ubytes = (size_t)n * 4 * sizeof(float);
  if (h->ksk_u_bytes < ubytes) {
    if (h->ksk_u) cudaFree(h->ksk_u);
    h->ksk_u = nullptr;
    h->ksk_u_bytes = 0;
    JLS_CHECK_CUDA(cudaMalloc(&h->ksk_u, ubytes));
    h->ksk_u_bytes = ubytes;
  }
  JLS_CHECK_CUDA(cudaMemsetAsync(h->ksk_u, 0, ubytes, s));
  JLS_CHECK_CUDA(cudaMemsetAsync(dh, 0, sizeof(double), s));
  const size_t smem = std::max((size_t)d * ADJ_PITCH * 4, (size_t)ADJ_WARPS * ADJ_MB * 4 * 4);
  const float c2 = (float)(1.4426950408889634 / (2.0 * hbw * hbw));  // log2(e) / (2 h^2)
  const float inv_h2 = (float)(1.0 / (hbw * hbw));
  const double inv_h3 = 1.0 / (hbw * hbw * hbw);
  const unsigned grid = (unsigned)((n + ADJ_MB - 1) / ADJ_MB);
  const bool fast = h->alpha == 4 && blocks == 1;
  auto kern = fast ? ksk_adjoint_kernel<true> : ksk_adjoint_kernel<false>;
  JLS_CHECK_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<grid, ADJ_WARPS * 32, smem, s>>>(X, n, dS, ldS, d, h->sjlt_ents, h->alpha, blocks, (float)scale, c2,
                                          inv_h2, inv_h3, dX, h->ksk_u, dh, h->d_err);
  note_launch();
  JLS_CHECK_CUDA(cudaGetLastError());
  ksk_finish_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(X, n, h->ksk_u, inv_h2, dX);
  note_launch();
  JLS_CHECK_CUDA(cudaGetLastError());
  return SK_OK;
}

}  // namespace jls
