// dense_complex.cu -- SRHT and Gaussian sketches of complex A (Sec. 2,
// A in C^{m x n}; the products A R and A* R of Sec. 6.3 with a real operator R).
//
// A is complex64 with interleaved FP32 parts; its real view V is rows x 2n.
//  * S = A R: V (R (x) I_2) is S's real view, so the real product of V with
//    the expanded operator writes S's interleaved parts directly: on CUDA
//    cores the operator tile is expanded while it is staged
//    (dense_apply_simt_complex_s); on tensor cores the bf16 planes are
//    expanded once into planes of 2 d rows and 2 n values (expand_plane_kernel).
//  * S' = A* R: V^T R (2n x w, by the real transpose product) holds Re(A)^T R
//    in its even rows and Im(A)^T R in its odd ones; S'[j][c] =
//    (V^T R)[2j][c] - i (V^T R)[2j + 1][c] (conj_interleave_kernel).
#include "common.cuh"
#include "internal.h"

namespace jls {

namespace {

// E[2c][2k] = E[2c + 1][2k + 1] = P[c][k], E[2c][2k + 1] = E[2c + 1][2k] = 0,
// for columns [c0, c1) of the operator; rows of P have bf_pitch(n) values,
// rows of E bf_pitch(2n).
__global__ void expand_plane_kernel(const uint16_t* __restrict__ P, int64_t n, int c0, int c1,
                                    uint16_t* __restrict__ E) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int c = c0 + (int)blockIdx.y;
  if (k >= n || c >= c1) return;
  const uint32_t v = P[(int64_t)c * bf_pitch(n) + k];
  const int64_t pe = bf_pitch(2 * n);
  *reinterpret_cast<uint32_t*>(E + (int64_t)(2 * c) * pe + 2 * k) = v;              // (v, 0)
  *reinterpret_cast<uint32_t*>(E + (int64_t)(2 * c + 1) * pe + 2 * k) = v << 16;    // (0, v)
}

// St[j][c] = (T[2j][c - c_lo], -T[2j + 1][c - c_lo]) for c in [c_lo, c_hi);
// T is 2n x w (ld w), St complex (interleaved, ld ldSt in complex elements)
__global__ void conj_interleave_kernel(const float* __restrict__ T, int64_t n, int c_lo, int c_hi,
                                       float* __restrict__ St, int64_t ldSt) {
  const int w = c_hi - c_lo;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n * w) return;
  const int64_t j = e / w;
  const int c = (int)(e - j * w);
  const float re = T[(2 * j) * w + c], im = T[(2 * j + 1) * w + c];
  *reinterpret_cast<float2*>(St + 2 * (j * ldSt + c_lo + c)) = make_float2(re, -im);
}

int ensure_bytes(void** p, size_t* have, size_t need) {
  if (*have >= need) return SK_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *have = 0;
  JLS_CHECK_CUDA(cudaMalloc(p, need));
  *have = need;
  return SK_OK;
}

}  // namespace

int dense_apply_complex(sk_op* h, const sk_matrix* A, int which, int prec, int c_lo, int c_hi, double scale,
                        void* S, int64_t ldS, void* St, int64_t ldSt, cudaStream_t s) {
  if (h->kind != SK_SRHT && h->kind != SK_GAUSS) return SK_ERR_DTYPE;
  if (prec != SK_PREC_NATIVE && prec != SK_PREC_BF16X2) return SK_ERR_DTYPE;
  if (c_hi <= c_lo) return SK_OK;
  sk_matrix V = *A;  // the real view
  V.dtype = SK_F32;
  V.cols = 2 * A->cols;
  V.ld = 2 * A->ld;
  const bool tc = prec == SK_PREC_BF16X2;
  if (which & SK_ST) {
    const int w = c_hi - c_lo;
    const size_t need = (size_t)2 * A->cols * w * sizeof(float);
    JLS_CHECK(ensure_bytes(&h->cplx_T, &h->cplx_T_bytes, need));
    // V^T R into T: rows 2 n, columns [c_lo, c_hi) stored from T's column 0
    float* Tc = static_cast<float*>(h->cplx_T) - c_lo;
    if (tc)
      JLS_CHECK(dense_apply_tc(h, &V, SK_ST, c_lo, c_hi, scale, nullptr, 0, Tc, w, s));
    else
      JLS_CHECK(dense_apply_simt(h, &V, SK_ST, c_lo, c_hi, scale, nullptr, 0, Tc, w, s));
    const int64_t cnt = A->cols * (int64_t)w;
    conj_interleave_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, s>>>(static_cast<const float*>(h->cplx_T),
                                                                         A->cols, c_lo, c_hi,
                                                                         static_cast<float*>(St), ldSt);
    note_launch();
    JLS_CHECK_CUDA(cudaGetLastError());
  }
  if (which & SK_S) {
    if (!tc) return dense_apply_simt_complex_s(h, A, c_lo, c_hi, scale, S, ldS, s);
    const int planes = h->kind == SK_GAUSS ? 2 : 1;
    if (h->kind == SK_GAUSS) JLS_CHECK(gen_gauss(h, 2, h->d_total, s));
    else JLS_CHECK(gen_srht_pm1(h, h->d_total, s));
    const size_t plane_b = (size_t)2 * h->d_max * bf_pitch(2 * h->n) * sizeof(uint16_t);
    if (!h->cplx_p0) {
      JLS_CHECK_CUDA(cudaMalloc(&h->cplx_p0, plane_b));
      JLS_CHECK_CUDA(cudaMemsetAsync(h->cplx_p0, 0, plane_b, s));
      if (planes == 2) {
        JLS_CHECK_CUDA(cudaMalloc(&h->cplx_p1, plane_b));
        JLS_CHECK_CUDA(cudaMemsetAsync(h->cplx_p1, 0, plane_b, s));
      }
    }
    if (h->cplx_cols < h->d_total) {
      const dim3 grid((unsigned)((h->n + 255) / 256), (unsigned)(h->d_total - h->cplx_cols));
      const uint16_t* src0 = h->kind == SK_GAUSS ? h->zhi : h->srht_pm1;
      expand_plane_kernel<<<grid, 256, 0, s>>>(src0, h->n, h->cplx_cols, h->d_total,
                                               static_cast<uint16_t*>(h->cplx_p0));
      note_launch();
      if (planes == 2) {
        expand_plane_kernel<<<grid, 256, 0, s>>>(h->zlo, h->n, h->cplx_cols, h->d_total,
                                                 static_cast<uint16_t*>(h->cplx_p1));
        note_launch();
      }
      JLS_CHECK_CUDA(cudaGetLastError());
      h->cplx_cols = h->d_total;
    }
    const uint16_t* e0 = static_cast<const uint16_t*>(h->cplx_p0);
    const uint16_t* e1 = planes == 2 ? static_cast<const uint16_t*>(h->cplx_p1) : e0;
    JLS_CHECK(launch_tc_planes(h->d_err, &V, false, planes, e0, e1, 2 * h->n, 2 * c_lo, 2 * c_hi, (float)scale,
                               static_cast<float*>(S), 2 * ldS, s));
  }
  return SK_OK;
}

}  // namespace jls
