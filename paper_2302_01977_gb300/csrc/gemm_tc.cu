// gemm_tc.cu -- SRHT / Gaussian sketches on tcgen05 tensor cores (bf16 split).
#include "common.cuh"
#include "internal.h"

namespace jls {

int dense_apply_tc(sk_op* h, const sk_matrix* A, int which, int c_lo, int c_hi, double scale, void* S, int64_t ldS,
                   void* St, int64_t ldSt, cudaStream_t s) {
  (void)h; (void)A; (void)which; (void)c_lo; (void)c_hi; (void)scale; (void)S; (void)ldS; (void)St; (void)ldSt;
  (void)s;
  return SK_ERR_UNSUPPORTED;
}

}  // namespace jls
