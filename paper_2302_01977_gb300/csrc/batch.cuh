// batch.cuh -- the device tables of a batch of SJLT sketches S'_i = A_i^T R_i
// and of the adaptive loop (Algorithm 1 run per instance on the device) that
// batches of SJLT sketches and of SRHT sketches S_i = A_i R_i share.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace jls {

// One instance of the batched sketch: its tensor map, CCS tiles, output and
// the column range [c_lo, c_hi) of R_i the next launch sketches.
struct alignas(128) BItem {
  CUtensorMap tm;  // A_i: cols (inner) x rows, box 128 x 128, FP32
  const uint4* ents;
  const uint32_t* offs;
  float* St;
  int64_t e_stride, o_stride;
  int64_t rows, cols, ldSt;
  int64_t unit0, units;  // this instance's units in the batch order (0 when inactive)
  int32_t ntiles, c_lo, c_hi, nbw;
  float scale;
  int32_t pad[3];
};
struct BHeader {
  int64_t total_units;
  uint32_t e_bytes, o_bytes;  // staging per stage: entry records, column offsets
};

// Per-instance state of the adaptive loop.  The test of round r acts on the
// columns [c_hi - dd, c_hi) of S'_i that the round's batched launch sketched;
// columns [covered, c_hi - dd) are first absorbed into the basis Q.
struct alignas(16) ATest {
  const float* S;   // S'_i: rows x ldS (the batch item's output)
  float* Q;         // rows x qcap: orthonormal basis of S'_i[:, :covered] (zero columns where a pivot dropped)
  float* W;         // rows x 32: the block under test or being absorbed
  float* G;         // qcap x 32: Q^T W when the basis is wider than ADAPT_QSMEM (else unused, may be null)
  int64_t rows, ldS;
  int32_t qcap, q, covered, dd;
  int32_t d_cap;    // columns of R_i (the loop stops, unconverged, when the next increment would pass it)
  int32_t first_w;  // width of R_i's first block, d0 + dd; later blocks are dd wide
  int32_t state;    // ADAPT_ACTIVE, ADAPT_CONVERGED or ADAPT_CAPPED
  int32_t tests;    // stopping tests taken
  int32_t d_reached;
  int32_t srht;     // the scale the loop sketches with: 0 (SJLT) 1/sqrt(alpha) per block, R_i[:, :d] carries
                    // 1/sqrt(alpha B); 1 (SRHT) 1/sqrt(first_w), R_i[:, :d] carries 1/sqrt(d)
  double nh, nt;    // ||S^||_F and ||S~||_F of the last test, at the scale of R_i[:, :d_reached]
};
enum : int32_t { ADAPT_ACTIVE = 0, ADAPT_CONVERGED = 1, ADAPT_CAPPED = 2 };

constexpr int ADAPT_QMAX = 8192;  // basis columns per instance
constexpr int ADAPT_QSMEM = 512;  // basis columns whose Q^T W stays in shared memory; wider bases keep it in G
constexpr int ADAPT_BW = 32;     // widest increment dd

// Kernels of batch_adaptive.cu (all asynchronous on `s`, capturable).
int adaptive_prepare();  // shared-memory limit of the test kernel (call outside capture)
// a round's tests with the cluster size picked on the device by the active count (list, n_active: scratch)
int adaptive_test_round(BItem* items, ATest* tests, const int* order, int count, int ncl, double eps_rel,
                        double eps_abs, bool wide, int* list, int* n_active, cudaStream_t s);
int adaptive_renumber_launch(BItem* items, int count, BHeader* hdr, int njobs, int nb, int* err, cudaStream_t s);
int adaptive_rescale_launch(const ATest* tests, int count, cudaStream_t s);

}  // namespace jls
