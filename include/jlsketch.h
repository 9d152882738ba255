/*
 * jlsketch.h -- C ABI of libjlsketch, Johnson-Lindenstrauss sketching of dense
 * matrices on one NVIDIA GB300 (sm_103a).
 *
 * The library computes the random samples of adaptive randomized HSS
 * construction (Yaniv, Ghysels, Malik, Boateng, Li, "Construction of HSS matrix
 * representation using adaptive Johnson-Lindenstrauss sketching"):
 *
 *     S  = A R        (sketch of the rows of A,    Sec. 6.3 "A R")
 *     S' = A^T R      (sketch of the columns of A, Sec. 6.3 "A* R"; real A)
 *
 * for three JL operators R (n x d): the SJLT (Sec. 2.4.3, data structure
 * Sec. 6.1), the SRHT R = D H P (Sec. 2.4.2; element formula of Sec. 7.2) and the
 * Gaussian operator N(0, 1/d) (Sec. 2.4.1); R grows by Delta-d columns
 * (Sec. 6.2, Algorithm 1: R <- [R R_bar], S <- [S A R_bar]) until the Frobenius
 * stopping test of Eq. (3.1) passes.
 *
 * Conventions for every entry point:
 *  - Matrices are row-major.  A is rows x cols with leading dimension ld
 *    (elements); S and S' are n x d_total with leading dimensions ldS, ldSt.
 *  - Pointers named "device" must be CUDA device (or managed) memory of the
 *    current device; "host" pointers are ordinary host memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Calls that only launch work are asynchronous on that stream; calls that
 *    return data to the host synchronize it and say so.
 *  - Every call returns SK_OK (0) or a negative SK_ERR_* code and never throws.
 *    A handle whose device work reported an error (an internal bound or wait
 *    limit, see sketch_device_status) refuses further work with SK_ERR_DEVICE.
 *  - The caller owns A, X, Y, S, S' and the stream.  A handle owns its
 *    operator arrays, its orthonormal bases for the stopping test and its
 *    scratch, all in device memory, and frees them in sketch_destroy.
 *  - There is no CPU fallback: without a usable GPU, calls fail with
 *    SK_ERR_DEVICE.
 */
#ifndef JLSKETCH_H
#define JLSKETCH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define SK_OK                 0
#define SK_ERR_INVALID_ARG   -1  /* bad size, kind, alpha, which, null pointer */
#define SK_ERR_ALIGN         -2  /* pointer or leading dimension not aligned as required */
#define SK_ERR_DTYPE         -3  /* unsupported element type / precision combination */
#define SK_ERR_NOMEM         -4  /* device allocation failed */
#define SK_ERR_D_MAX         -5  /* an increment would exceed the d_max given at creation */
#define SK_ERR_STATE         -6  /* call out of order (e.g. increment apply before increment) */
#define SK_ERR_TIMEOUT       -7  /* a bounded device-side wait gave up */
#define SK_ERR_DEVICE        -8  /* CUDA error or device-side error flag */
#define SK_ERR_UNSUPPORTED   -9  /* valid request this library does not implement */

/* ---- operator kinds (Sec. 2.4) ------------------------------------------ */
#define SK_SJLT_GRAPH 1  /* alpha distinct positions uniform in each row's block  */
#define SK_SJLT_BLOCK 2  /* one position in each of alpha chunks of width/alpha    */
#define SK_SRHT       3  /* R = D H P, nu = 2^ceil(log2 n), columns w/o replacement
                            unless SK_SRHT_REPLACE */
#define SK_GAUSS      4  /* i.i.d. N(0, 1/d)                                      */

/* ---- element types ------------------------------------------------------ */
#define SK_F64 1
#define SK_F32 2
#define SK_C64 3  /* complex with FP32 real and imaginary parts, interleaved (re, im);
                     leading dimensions count complex elements.  Explicit A with an
                     SJLT operator and SK_PREC_NATIVE: S = A R and S' = A* R, the
                     conjugate transpose of Sec. 6.3 (R is real).               */

/* ---- arithmetic of an apply -------------------------------------------- */
#define SK_PREC_NATIVE 0  /* F64 data: FP64; F32 data: FP32 on CUDA cores          */
#define SK_PREC_BF16X2 3  /* F32 data: A = A_hi + A_lo (bf16), R likewise (Gaussian)
                             or exact (+-1, SRHT; {0, +-1}, SJLT); tcgen05 tensor
                             cores, FP32 accumulation.  SRHT and Gaussian always
                             take it; an SJLT product takes it where the route
                             pick measures it faster (sketch_sjlt_route), else
                             the SJLT kernels in FP32.  The kernel asks L2 for
                             A's tiles a few units ahead of use (3; the
                             environment variable JLS_TC_PREFETCH=0..64 sets
                             the distance, 0 turns it off)                        */
#define SK_PREC_FP8    4  /* F32 data: e4m3 hi + lo terms of A per 128 x 128 tile
                             scale and of z per (128 x 1) scale, SRHT signs exact;
                             tcgen05 tensor cores, FP32 accumulation, scales
                             applied per 128-value K tile; SRHT and Gaussian only;
                             relative error of order 1e-3 (tolerance 2e-2)         */

/* ---- which sketch ------------------------------------------------------- */
/* Creation flags (sketch_create_flags), combined by bitwise or. */
#define SK_SCALE_BLOCK  1u  /* every block of R keeps the scale of a JL operator of its own width
                               (Algorithm 1 appends an independent JL(Delta-d)): SJLT 1/sqrt(alpha),
                               SRHT 1/sqrt(w_b), Gaussian variance 1/w_b for a block of width w_b;
                               increments leave earlier columns unscaled.  Default: the grown R is
                               renormalized to one JL operator of width d_total (Sec. 6.2). */
#define SK_SRHT_REPLACE 2u  /* SRHT columns sampled with replacement ("independently and
                               uniformly", Sec. 2.4.2): the sampled index mu_j is the j-th accepted
                               draw, repeats kept, and d_max may exceed nu.  Default: without
                               replacement, the first d distinct draws.  SRHT operators only. */

#define SK_S    1  /* S  = A R   */
#define SK_ST   2  /* S' = A^T R */
#define SK_BOTH 3

typedef struct sk_op* sk_handle;

/* An input matrix: explicit, or generated from points (a Gaussian kernel). */
typedef struct sk_matrix {
  int32_t dtype;       /* SK_F32, SK_F64 (also the type of X, Y), or SK_C64 (explicit) */
  int32_t generator;   /* 0: explicit A; 1: A_ij = exp(-|x_i-y_j|^2/(2h^2)) + shift*[i==j] */
  int64_t rows, cols;  /* A is rows x cols                                          */
  const void* A;       /* explicit: device, row-major, 16-byte aligned               */
  int64_t ld;          /* explicit: leading dimension >= cols; ld*elem_size % 16 == 0 */
  const void* X;       /* generator: device, rows x 3, row-major                     */
  const void* Y;       /* generator: device, cols x 3, row-major                     */
  double h;            /* generator: kernel width h > 0                              */
  double shift;        /* generator: diagonal shift                                  */
} sk_matrix;

/*
 * sketch_create -- draw a JL operator R of size n x d on the device.
 *   kind   SK_SJLT_GRAPH | SK_SJLT_BLOCK | SK_SRHT | SK_GAUSS (Sec. 2.4).
 *   n      rows of R (= cols of A for S, rows of A for S'), 1 <= n < 2^31.
 *   d      initial columns (Algorithm 1 starts with d0 + Delta-d), 1 <= d <= d_max.
 *   alpha  SJLT nonzeros per row and block, 1 <= alpha <= min(d, 32); block
 *          construction needs alpha | d (Sec. 2.4.3).  Ignored otherwise.
 *   seed   64-bit seed; R is a pure function of (kind, n, d, alpha, seed) and
 *          the increments applied (Philox4x64-10 streams).
 *   d_max  capacity in columns, d <= d_max <= 8192; SRHT needs d_max <= nu.
 *   stream where the generation kernels run (asynchronous).
 * Out: *out receives the handle.  Errors: INVALID_ARG, NOMEM, DEVICE.
 */
int sketch_create(sk_handle* out, int32_t kind, int64_t n, int32_t d, int32_t alpha,
                  uint64_t seed, int32_t d_max, void* stream);

/*
 * sketch_create_flags -- sketch_create with creation flags (the scale mode and
 * the SRHT sampling; the paper's readings in the flag definitions above).
 *   flags  0, or SK_SCALE_BLOCK and/or SK_SRHT_REPLACE; sketch_create is
 *          flags == 0.  With SK_SRHT_REPLACE, d_max <= 8192 only.
 * Errors: INVALID_ARG (unknown flag bits; SK_SRHT_REPLACE on a non-SRHT
 * kind; as sketch_create otherwise), NOMEM, DEVICE.
 */
int sketch_create_flags(sk_handle* out, int32_t kind, int64_t n, int32_t d, int32_t alpha,
                        uint64_t seed, int32_t d_max, uint32_t flags, void* stream);

/*
 * sketch_increment -- append Delta-d columns to R (Algorithm 1, R <- [R R_bar]).
 *   SJLT: a new block of alpha nonzeros per row in the new columns; the scale
 *   becomes 1/sqrt(alpha * blocks) ("adjusting the scaling factor", Sec. 6.2).
 *   SRHT: the next delta_d distinct sampled columns of the same D H (with
 *   SK_SRHT_REPLACE: the next delta_d draws).
 *   Gaussian: delta_d new N(0,1) columns; all columns scale as 1/sqrt(d_total).
 *   With SK_SCALE_BLOCK no column is rescaled: the new block takes its own
 *   scale (see the flag).
 *   Block SJLT needs alpha | delta_d; SRHT without replacement needs d_total <= nu.
 * Errors: INVALID_ARG, D_MAX, NOMEM, DEVICE.
 */
int sketch_increment(sk_handle h, int32_t delta_d, void* stream);

/*
 * sketch_apply -- S = A R and/or S' = A^T R for the current R (Sec. 6.3).
 *   A      explicit (generator == 0) or kernel generator; rows x cols with
 *          cols == n for S and rows == n for S'.  A generated K(X, Y) is
 *          written in blocks of rows (at least 20480, or 2 GiB) to scratch the
 *          handle owns and each block is sketched; S' is computed as the S
 *          product of K(Y, X), which equals K^T.
 *   which  SK_S, SK_ST or SK_BOTH.
 *   prec   SK_PREC_NATIVE, or SK_PREC_BF16X2 (F32; SJLT by measured route) /
 *          SK_PREC_FP8 (F32, SRHT/Gaussian).
 *   S      device, rows x d_total (ldS >= d_total) of A's dtype; used if which & SK_S.
 *   St     device, cols x d_total (ldSt >= d_total);             used if which & SK_ST.
 *          For SK_C64 data S = A R and S' = A* R are complex (interleaved FP32
 *          pairs, leading dimensions in complex elements).  S' runs the S'
 *          kernel over the real view of A and conjugates while writing; S runs
 *          the S kernel over the real view with R (x) I_2.
 * Asynchronous.  Errors: INVALID_ARG, ALIGN, DTYPE, UNSUPPORTED, NOMEM, DEVICE.
 */
int sketch_apply(sk_handle h, const sk_matrix* A, int32_t which, int32_t prec,
                 void* S, int64_t ldS, void* St, int64_t ldSt, void* stream);

/*
 * sketch_apply_increment -- after sketch_increment, bring S (S') from the
 * operator before the last increment to the grown one without recomputing
 * the old columns: the d_old existing columns are rescaled to the new scale
 * and only the delta_d new columns A R_bar are computed (Algorithm 1,
 * S <- [S A R_bar]).  S must hold the sketch of the previous operator (same
 * A); call it once per sketch buffer and increment.
 * Errors: as sketch_apply, plus STATE when no increment has been made.
 */
int sketch_apply_increment(sk_handle h, const sk_matrix* A, int32_t which, int32_t prec,
                           void* S, int64_t ldS, void* St, int64_t ldSt, void* stream);

/*
 * adaptive_norm_test -- the Frobenius stopping test (Eq. (3.1))
 * on the global sketch held in S (rows x d_total, device, dtype, row-major):
 *   S~ = the last delta_d columns of S (Algorithm 1's "last Delta-d columns"),
 *   S^ = (I - Q Q^T)^2 S~ with Q an orthonormal basis of the first
 *        d_total - delta_d columns (two block Gram-Schmidt passes, the remark
 *        after the equation), and
 *   stop = ||S^||_F < eps_abs  or  ||S^||_F < eps_rel ||S~||_F.
 *   slot   0 or 1: which basis Q the handle keeps (use 0 for S, 1 for S').
 * Q is kept in the handle and only the columns not yet in it are
 * orthonormalised (block Gram-Schmidt twice + Cholesky QR twice, 64 columns at
 * a time), so successive calls cost one projection each; Q is rebuilt from
 * scratch when the split point moves backwards or `rows` changes.  Norms and
 * Gram matrices accumulate in FP64.  Synchronizes `stream`; writes *stop and,
 * if not NULL, *norm_hat = ||S^||_F and *norm_tilde = ||S~||_F (host).
 * Errors: INVALID_ARG, STATE (delta_d < 1 or >= d_total), DEVICE.
 */
int adaptive_norm_test(sk_handle h, int32_t slot, const void* S, int64_t rows, int64_t ldS,
                       int32_t dtype, int32_t delta_d, double eps_rel, double eps_abs,
                       int32_t* stop, double* norm_hat, double* norm_tilde, void* stream);

/*
 * adaptive_norm_test_pair -- the test of adaptive_norm_test on S (slot 0) and
 * on S' (slot 1) at once, for callers that sketch both (Algorithm 1 stops when
 * both tests pass).  The S' test runs on a stream the handle owns, started
 * after the work already queued on `stream`, the S test on `stream`; the two
 * chains of small kernels overlap on the GPU.  Before returning, `stream` is
 * made to wait for all of the S' test, so later work on `stream` (the next
 * increment) is ordered after both.  rows_S / rows_St: rows of S and S';
 * ldS, ldSt: their leading dimensions (>= d_total).  Host outputs: stop[2],
 * norm_hat[2], norm_tilde[2] (index 0 for S, 1 for S'; the norm arrays may be
 * NULL).  Synchronizes on the two norm copies only.  The results equal two
 * adaptive_norm_test calls'.  Errors: as adaptive_norm_test.
 */
int adaptive_norm_test_pair(sk_handle h, const void* S, int64_t rows_S, int64_t ldS, const void* St, int64_t rows_St,
                            int64_t ldSt, int32_t dtype, int32_t delta_d, double eps_rel, double eps_abs, int32_t* stop,
                            double* norm_hat, double* norm_tilde, void* stream);

/*
 * sketch_project_norms_noalloc -- the projection and norms of the stopping
 * test, for callers that cannot allocate device memory.  (The paper has no
 * counterpart: this is an interface variant of adaptive_norm_test's arithmetic.)
 *
 * Who needs it: processes whose device memory is owned by another allocator or
 * a fixed pool (a framework's caching allocator, an embedding application that
 * hands the library no memory of its own), and callers that must not take the
 * device-wide synchronization that cudaMalloc/cudaFree can imply.  This call
 * allocates nothing: no cudaMalloc, no cudaFree, no allocating library routine.
 * Its scratch is a file-scope device array of 4.5 MiB inside the library, which
 * every GPU that loads the library holds until the process exits.
 * It is not a call for code inside CUDA stream capture: it reads its norm
 * partials back into pageable host memory and synchronizes `stream`, twice per
 * call, and neither is allowed on a capturing stream.
 *
 *   Q        device, rows x q_cols, row-major (ldQ >= q_cols): an orthonormal
 *            basis supplied by the caller (may be NULL when q_cols == 0).
 *   S_tilde  device, rows x b (ldS >= b): the block to test.
 *   S_hat    device, rows x b (ldH >= b): receives (I - Q Q^T)^2 S_tilde.
 *   Writes *stop = ||S_hat||_F < eps_abs or ||S_hat||_F < eps_rel ||S_tilde||_F
 *   and, if not NULL, *norm_hat and *norm_tilde (host; FP64 sums).
 * Limits: q_cols <= 1024 and b <= 64 (larger requests return
 * SK_ERR_INVALID_ARG without touching the device); device ordinals 0 .. 63
 * (the per-device address cache has 64 entries; a call with a higher ordinal
 * current returns SK_ERR_UNSUPPORTED).  The first call on each device looks up
 * the array's device address (cudaGetSymbolAddress) with that device current
 * and caches it.  Q, S_tilde and S_hat must have the same dtype and row count
 * and S_hat at least b columns: the call sees only their pointers.  All calls
 * share the one array and nothing in it needs to start at zero (each call
 * writes every element it reads), but calls whose work overlaps on the GPU
 * (other streams, other host threads) race on it: serialize them.
 * Synchronizes `stream` (twice).  Errors: INVALID_ARG, DTYPE, UNSUPPORTED, DEVICE.
 */
int sketch_project_norms_noalloc(const void* Q, int64_t ldQ, int32_t q_cols,
                                 const void* S_tilde, int64_t ldS, int64_t rows, int32_t b,
                                 int32_t dtype, void* S_hat, int64_t ldH,
                                 double eps_rel, double eps_abs, int32_t* stop,
                                 double* norm_hat, double* norm_tilde, void* stream);

/*
 * kernel_matrix -- write the explicit matrix of a generator descriptor:
 * A_ij = exp(-||x_i - y_j||^2 / (2 h^2)) + shift * [i == j]  (device, row-major,
 * ld >= cols, dtype of the descriptor).  Asynchronous.
 */
int kernel_matrix(const sk_matrix* gen, void* A, int64_t ld, void* stream);

/*
 * sketch_kernel_apply -- matrix-free sketch of a Gaussian kernel matrix that is
 * never formed (the matrix-free setting of Sec. 1.1, kernel matrices of points
 * as in Sec. 8.1):
 *     S = K(X, Y; h) R,  K_ij = exp(-||x_i - y_j||^2 / (2 h^2)) + shift [i == j],
 * for an SJLT operator R (Sec. 2.4.3, n = the handle's n).  Tiles of K are
 * computed in shared memory next to the SJLT product of Sec. 6.3 and
 * discarded; K is never written to device memory.
 *   X      device FP32, m x 3, row-major: points of the rows of S, m >= 1.
 *   Y      device FP32, n x 3: points of the rows of R (X == Y is allowed).
 *   h_bw   kernel width h > 0;  shift  added where i == j (0 for a pure kernel).
 *   S      device FP32, m x d_total (ldS >= d_total), overwritten.
 * Asynchronous on `stream`.  FP32 arithmetic (exp2 of FP32 squared distances),
 * relative error of order 1e-6 against the FP64 definition.
 * Errors: INVALID_ARG, UNSUPPORTED (not an SJLT handle), NOMEM, DEVICE.
 */
int sketch_kernel_apply(sk_handle h, const float* X, int64_t m, const float* Y, double h_bw,
                        double shift, float* S, int64_t ldS, void* stream);

/*
 * sketch_kernel_adjoint -- gradient of L = <dS, K(X, X; h) R> (shift 0) with
 * respect to the points X and the width h, for an SJLT R (the adjoint of
 * sketch_kernel_apply with X == Y; the paper does not differentiate the
 * sketch, this is the chain rule of its definition):
 *     G = dS R^T,
 *     dX_i = (1/h^2) sum_j (G_ij + G_ji) K_ij (x_j - x_i),
 *     dh   = (1/h^3) sum_ij G_ij K_ij ||x_i - x_j||^2.
 * K is recomputed tile by tile, never stored.
 *   X    device FP32, n x 3 (n = the handle's n).
 *   dS   device FP32, n x d_total (ldS >= d_total): the upstream gradient.
 *   dX   device FP32, n x 3, overwritten (must not alias X).
 *   dh   device FP64, one value, overwritten.
 * Needs d_total <= 384 and alpha * blocks <= 32 (else UNSUPPORTED).  The handle
 * keeps an n x 4 FP32 scratch buffer for the sums over the second index.
 * Asynchronous on `stream`.  Errors: INVALID_ARG, UNSUPPORTED, NOMEM, DEVICE.
 */
int sketch_kernel_adjoint(sk_handle h, const float* X, double h_bw, const float* dS, int64_t ldS,
                          float* dX, double* dh, void* stream);

/* ---- batches: many independent SJLT sketches in one launch ------------------ */

typedef struct sk_batch* sk_batch_handle;

/* One instance of a batch: S'_i = A_i^T R_i for columns [c_lo, c_hi) of R_i. */
typedef struct sk_batch_item {
  sk_handle op;        /* SJLT operator R_i (SK_SJLT_BLOCK or SK_SJLT_GRAPH), n_i rows      */
  const float* A;      /* device FP32, rows x cols, row-major, 16-byte aligned, ld*4 % 16 == 0 */
  int64_t rows, cols;  /* rows == n_i                                                       */
  int64_t ld;          /* leading dimension of A (elements), >= cols                          */
  float* St;           /* device FP32, cols x d_total(R_i), leading dimension ldSt          */
  int64_t ldSt;
  int32_t c_lo, c_hi;  /* columns of R_i to sketch, 0 <= c_lo < c_hi <= d_total(R_i)          */
  double scale;        /* multiplies the signed sums; 0 = the operator's 1/sqrt(alpha*blocks) */
} sk_batch_item;

/*
 * sketch_batch_create -- prepare a batch of independent, uneven S' = A^T R
 * products (Sec. 6.3) to run as ONE persistent kernel launch (for example the
 * sketches of Algorithm 1's first d0 + Delta-d columns, then of each Delta-d
 * increment, for many kernel matrices; a symmetric A_i gives S_i = S'_i).
 * Builds each operator's tiled CCS for its current d_total, encodes a TMA
 * tensor map per A_i, copies the item table to the device, and picks the
 * kernel shape (warps per CTA x columns per warp) by timing the batch once per
 * shape (the autotuner; it writes the outputs).  Synchronizes `stream`.  The
 * operators must not be incremented or applied to other data of a different
 * d_total while the batch exists (their CCS arrays are referenced).  Every
 * range c_hi - c_lo must be at most 300 columns (the widest shape's 15 x 20).
 * Errors: INVALID_ARG, ALIGN, NOMEM, UNSUPPORTED, DEVICE.
 */
int sketch_batch_create(sk_batch_handle* out, const sk_batch_item* items, int32_t count, void* stream);

/*
 * sketch_batch_set -- host-only update of the next run: per instance an active
 * flag and a column range (host arrays of `count` values; NULL keeps the
 * current values).  Inactive instances are skipped.  Writes the pinned host
 * mirror of the item table that sketch_batch_run copies to the device, so call
 * it only when no earlier run is still pending on the GPU.
 * Errors: INVALID_ARG (range outside d_total), UNSUPPORTED (range too wide).
 */
int sketch_batch_set(sk_batch_handle b, const int32_t* active, const int32_t* c_lo, const int32_t* c_hi);

/*
 * sketch_batch_run -- copy the item table to the device, zero the columns
 * [c_lo, c_hi) of every active output, and run the batched sketch: one
 * persistent launch whose CTAs (one per SM) stream equal shares of all active
 * instances' (block, tile) units.  Asynchronous, allocates nothing and takes
 * no host synchronization, so it can be captured in a CUDA graph; a replay
 * uses the table sketch_batch_set last wrote, with the shared-memory staging
 * sized at capture: ranges set later must touch no more blocks of their
 * operators than the captured ones did (otherwise the kernel sets the device
 * flag that sketch_batch_status reports).  Errors: INVALID_ARG, DEVICE.
 */
int sketch_batch_run(sk_batch_handle b, void* stream);

/*
 * sketch_batch_tune -- rerun the autotuner on the ranges sketch_batch_set last
 * wrote (each shape: one warm-up and three timed runs on `stream`, which write
 * the outputs) and keep the fastest shape for later runs; e.g. once for the
 * first sketch and once for the Delta-d increments, before capturing a graph
 * of the latter.  Synchronizes `stream`; not capturable.  The paper has no
 * counterpart.  Errors: UNSUPPORTED (no shape takes the ranges), DEVICE.
 */
int sketch_batch_tune(sk_batch_handle b, void* stream);

/* sketch_batch_info -- the chosen shape, the active units of the next run and
 * the autotuner's measured ms per run for each shape, in the order 24 x 13,
 * 20 x 16, 16 x 20, 32 x 2 warps x columns (-1 = not eligible; `tuned_ms`
 * holds 4 floats).  Any pointer may be NULL.  The paper has no counterpart. */
int sketch_batch_info(sk_batch_handle b, int32_t* warps, int32_t* cols_per_warp, int64_t* units,
                      float* tuned_ms);

/* sketch_batch_status -- synchronize `stream`, report and clear the batch's
 * device error flag: SK_OK, SK_ERR_TIMEOUT or SK_ERR_DEVICE. */
int sketch_batch_status(sk_batch_handle b, void* stream);

/*
 * sketch_batch_adaptive_setup -- prepare Algorithm 1's adaptive loop for every
 * instance of the batch, run on the device by sketch_batch_adaptive_run.
 * Instance i's operator must be R_i = JL(d0[i] + dd) grown by dd-column
 * increments (sketch_increment) up to the most columns the loop may use,
 * d_total(R_i) (the increments are drawn up front; the loop sketches them one
 * at a time).  The test of Eq. (3.1) runs on S'_i = A_i^T R_i (S_i for a
 * symmetric A_i) with eps_rel and eps_abs (0 disables the absolute test).
 * d0[i] (host array of `count`) and dd are multiples of 8, 8 <= dd <= 32, and
 * d_total(R_i) - dd <= 8192.  Rebuilds the tiles of operators grown since the
 * batch was made, tunes the kernel shape for the first sketch and for the
 * increments (the tuning runs write the outputs), allocates each instance's
 * orthonormal basis (cols_i x (d_total_i - dd) FP32), a cols_i x 32 block and,
 * for bases wider than 512 columns, a (d_total_i - dd) x 32 product Q^T W,
 * and leaves the batch's ranges at [0, d0[i] + dd).  The stopping test runs one
 * CTA per instance when the batch has at least as many instances as the GPU
 * has SMs, a thread-block cluster of 4 CTAs per instance otherwise (the
 * environment variable JLS_ADAPT_CLUSTER=1, 2 or 4 overrides the choice).
 * Synchronizes `stream`.  Errors: INVALID_ARG, UNSUPPORTED, NOMEM, DEVICE.
 */
int sketch_batch_adaptive_setup(sk_batch_handle b, const int32_t* d0, int32_t dd, double eps_rel, double eps_abs,
                                void* stream);

/*
 * sketch_batch_adaptive_run -- enqueue the whole loop on `stream`: reset the
 * device tables, then per round one batched sketch launch (round 0: columns
 * [0, d0 + dd); later rounds: the next dd columns of the instances still
 * active), one launch of the stopping test (a cluster of CTAs per instance:
 * the columns before the tested block are absorbed into the instance's basis,
 * S^ = (I - Q Q^T)^2 S~, the decision, and on failure Q <- [Q, orth(S^)]) and
 * one launch that renumbers the active instances' work for the next round; a
 * final launch rescales S'_i[:, :d_i] to R_i[:, :d_i]'s scale 1/sqrt(alpha B_i).
 * At most max_rounds rounds (0 = until every instance could have finished);
 * finished instances cost nothing in later rounds.  No host synchronization,
 * no allocation: capturable in one CUDA graph.  Columns of S'_i past d_i are
 * left as they were.  Errors: INVALID_ARG (no setup), DEVICE.
 */
int sketch_batch_adaptive_run(sk_batch_handle b, int32_t max_rounds, void* stream);

/*
 * sketch_batch_adaptive_result -- synchronize `stream` and read each
 * instance's outcome (host arrays of `count`; any may be NULL): d_reached =
 * the columns of S'_i sketched (d + dd at the last test), state = 1 converged,
 * 2 stopped because R_i has no further increment, 0 still running when
 * max_rounds ran out; tests = stopping tests taken; nh, nt = ||S^||_F and
 * ||S~||_F of the last test.  Then reports the device error flag as
 * sketch_batch_status does.  Errors: INVALID_ARG, TIMEOUT, DEVICE.
 */
int sketch_batch_adaptive_result(sk_batch_handle b, int32_t* d_reached, int32_t* state, int32_t* tests, double* nh,
                                 double* nt, void* stream);

/* sketch_batch_destroy -- free the batch (NULL is a no-op); the operators are
 * not freed. */
void sketch_batch_destroy(sk_batch_handle b);

/* ---- batches of SRHT sketches: S_i = A_i R_i in one launch ------------------
 *
 * The SRHT of Sec. 2.4.2 applied through the row transform of Sec. 7.1: row r
 * of A_i, sign-flipped by D_i and zero-padded to nu_i = 2^ceil(log2 n_i), is
 * transformed by the unnormalized Sylvester-Hadamard matrix and the outputs at
 * the sampled columns mu_c are kept, S_i[r, c] = scale * sum_k A_i[r, k] d_k
 * (-1)^popcount(k & mu_c) (the element formula of Sec. 7.2).  This is the
 * product S = A R; for a symmetric A_i (a kernel matrix K(X, X)) it equals
 * S' = A_i^T R_i, the product the SJLT batch computes.  Orders nu_i <= 4096.
 */
typedef struct sk_srht_batch* sk_srht_batch_handle;

typedef struct sk_srht_batch_item {
  sk_handle op;        /* SRHT operator R_i (SK_SRHT), n_i rows, nu_i <= 4096             */
  const float* A;      /* device FP32, rows x n_i, row-major                             */
  int64_t rows;        /* rows of A_i (>= 1)                                             */
  int64_t ld;          /* leading dimension of A (elements), >= n_i                     */
  float* S;            /* device FP32, rows x d_total(R_i), leading dimension ldS        */
  int64_t ldS;
  int32_t c_lo, c_hi;  /* columns of R_i to sketch, 0 <= c_lo <= c_hi <= d_total(R_i)     */
  double scale;        /* multiplies the transform; 0 = the operator's 1/sqrt(d_total)   */
} sk_srht_batch_item;

/*
 * sketch_srht_batch_create -- prepare a batch of independent, uneven SRHT
 * sketches (synchronous set-up on `stream`).  The rows of all instances with
 * a non-empty column range are numbered into one list of units that one
 * persistent launch of 128-thread CTAs splits into contiguous ranges; the
 * number of CTAs per SM (3, 6 or 12) is picked by timing one run of each.
 * The items are copied; A_i, S_i and the operators must outlive the batch,
 * and the operators must not grow past the columns named here while it
 * exists.  Errors: INVALID_ARG (a kind other than SK_SRHT, bad sizes or
 * ranges), UNSUPPORTED (nu_i > 4096), NOMEM, DEVICE.
 */
int sketch_srht_batch_create(sk_srht_batch_handle* out, const sk_srht_batch_item* items, int32_t count,
                             void* stream);

/*
 * sketch_srht_batch_set -- host-only update of the next run's column ranges
 * (NULL keeps an array; c_lo == c_hi leaves that instance out of the run).
 * Writes the pinned host mirror that sketch_srht_batch_run copies to the
 * device, so call it only when no earlier run is still pending on the GPU.
 * Errors: INVALID_ARG (a range outside [0, d_total]).
 */
int sketch_srht_batch_set(sk_srht_batch_handle b, const int32_t* c_lo, const int32_t* c_hi);

/*
 * sketch_srht_batch_run -- copy the item table from its pinned host mirror
 * to the device and launch the batched transform on `stream` (asynchronous;
 * copies and one kernel only, so a CUDA graph can capture it and replay the
 * ranges sketch_srht_batch_set last wrote).  Columns [c_lo, c_hi) of every
 * S_i are overwritten; other columns are untouched.  Errors: INVALID_ARG,
 * DEVICE.
 */
int sketch_srht_batch_run(sk_srht_batch_handle b, void* stream);

/* sketch_srht_batch_info -- the chosen CTAs per SM, the units (rows) of the
 * next run, the tuner's times (ms; 6 floats: 3, 6 and 12 CTAs per SM with
 * Sec. 7.1's split of rows with n = k + r, 0 < r <= k / 2, k = nu / 2, then
 * the same without it, on zero-padded rows; 0 where not timed) and whether
 * the split was kept (*split = 1); any pointer may be NULL.  The split
 * transforms such a row at orders k and p = 2^ceil(log2 r) in two passes (the
 * second adds +-(A^ H_p)_{mu mod p} to the sampled outputs) instead of at
 * order nu. */
int sketch_srht_batch_info(sk_srht_batch_handle b, int32_t* ctas_per_sm, int64_t* units, float* tuned_ms,
                           int32_t* split);

/*
 * sketch_srht_batch_adaptive_setup -- prepare Algorithm 1's adaptive loop for
 * every instance of an SRHT batch (Sec. 6.2, Algorithm 1; Eq. (3.1)), run on
 * the device by sketch_srht_batch_adaptive_run.  Each operator must have been
 * created with d0[i] + dd columns and grown by dd-column increments up to the
 * columns the loop may use (the increments of Algorithm 1 are
 * data-independent draws).  Round 0 sketches S_i[:, 0 : d0 + dd); each round
 * tests the last dd columns sketched against an orthonormal basis of the
 * earlier ones (kept per instance on the device), stops the instance when
 * ||S^|| < eps_abs or ||S^|| < eps_rel ||S~||, and otherwise extends the
 * basis and sketches the next dd columns.  The loop sketches every column with
 * 1/sqrt(d0 + dd); norms are reported at the scale of R_i[:, :d] (1/sqrt(d))
 * and the finished columns are rescaled once, so S_i[:, :d] = A_i R_i[:, :d].
 * The loop is the SJLT batch's (same test kernel, FP32 sketch and basis, FP64
 * norms).  Limits: 8 <= dd <= 32, dd and d0 multiples of 8, d_total - dd <=
 * 8192.  Synchronous, not capturable.  Errors: INVALID_ARG, UNSUPPORTED,
 * NOMEM, DEVICE.
 */
int sketch_srht_batch_adaptive_setup(sk_srht_batch_handle b, const int32_t* d0, int32_t dd, double eps_rel,
                                     double eps_abs, void* stream);

/*
 * sketch_srht_batch_adaptive_run -- enqueue the whole loop on `stream`
 * (asynchronous; copies and kernels only, so one CUDA graph can capture every
 * round): reset the device tables, then per round the numbering of the active
 * instances' rows, one batched transform and the stopping test of every
 * active instance; max_rounds = 0 runs until every instance has stopped.
 * Errors: INVALID_ARG, DEVICE.
 */
int sketch_srht_batch_adaptive_run(sk_srht_batch_handle b, int32_t max_rounds, void* stream);

/*
 * sketch_srht_batch_adaptive_result -- synchronize `stream` and read each
 * instance's columns sketched (d_reached), state (1 converged, 2 out of
 * columns, 0 still running), stopping tests taken and the last test's
 * ||S^||_F and ||S~||_F (host arrays of `count` values; any may be NULL).
 * Errors: INVALID_ARG, DEVICE.
 */
int sketch_srht_batch_adaptive_result(sk_srht_batch_handle b, int32_t* d_reached, int32_t* state, int32_t* tests,
                                      double* nh, double* nt, void* stream);

/* sketch_srht_batch_destroy -- free the batch (NULL is a no-op); the operators
 * are not freed. */
void sketch_srht_batch_destroy(sk_srht_batch_handle b);

/* sketch_dims -- shape of the current operator (host outputs; any may be NULL). */
int sketch_dims(sk_handle h, int32_t* kind, int64_t* n, int32_t* d_total, int32_t* alpha,
                int32_t* blocks);

/*
 * sketch_export -- host copies of the operator for checking (synchronizes):
 *   cols, signs  SJLT: n x (alpha*blocks) int32 global column / int8 +-1, block
 *                by block, each block's entries in chunk order (block) or
 *                ascending column order (graph); the Sec. 6.1 structure.
 *   diag, mu     SRHT: n int8 signs d_i and d_total int32 sampled columns.
 *   R, R_dtype   dense R (n x d_total, row-major, host) of SK_F32/SK_F64, the
 *                values the apply kernels use (scale included).
 * Pointers that do not apply to the kind, or are NULL, are skipped.
 */
int sketch_export(sk_handle h, int32_t* cols, int8_t* signs, int8_t* diag, int32_t* mu,
                  void* R, int32_t R_dtype);

/* sketch_device_status -- synchronize `stream` and report (and clear) the
 * handle's device-side error flag: SK_OK, SK_ERR_TIMEOUT or SK_ERR_DEVICE. */
int sketch_device_status(sk_handle h, void* stream);

/* sketch_selftest_wait -- exercise the failure path of the device-side waits:
 * one thread waits, with the same bounded wait the kernels use, on a barrier
 * that nothing completes; after the limit (2 s) it sets the error flag and the
 * kernel returns.  Expected result: SK_ERR_TIMEOUT, with the context still
 * usable.  Synchronizes `stream`.  A diagnostic; the paper has no counterpart. */
int sketch_selftest_wait(void* stream);

/* sketch_launch_count -- number of kernels this library has launched in the
 * process so far (all handles); a diagnostic for counting device work. */
int64_t sketch_launch_count(void);

/* sketch_srht_route -- which route the SRHT S = A R product takes for a shape
 * (nu = 2^ceil(log2 n), A's rows and cols, the number of columns applied, and
 * prec): 1 the row FWHT of Sec. 7.1, 0 the +-1 product of the element formula
 * of Sec. 7.2, -1 not measured yet.  The first apply of a shape times both
 * routes on its stream (one synchronization) and keeps the faster; only FP32
 * data with nu in [2^14, 2^16] and SK_PREC_NATIVE or SK_PREC_BF16X2 has both
 * routes.  For n not a power of two the FWHT takes Sec. 7.1's split into
 * transforms of orders k = 2^floor(log2 n) and p = 2^ceil(log2(n - k)) when
 * n - k <= 8192 and k >= 2^14 (otherwise, or with JLS_SRHT_SPLIT=0 in the
 * environment, it transforms the zero-padded rows; both give the same S).
 * The environment variable JLS_SRHT_ROUTE=fwht or =product pins the route for
 * the process (shapes served that way are not recorded, and report -1).  A
 * diagnostic query; the paper has no counterpart. */
int sketch_srht_route(int64_t nu, int64_t rows, int64_t cols, int32_t width, int32_t prec);

/* sketch_sjlt_route -- which route an SJLT product of FP32 data with
 * SK_PREC_BF16X2 takes for a shape (kind, n = rows of R, A's rows and cols,
 * the number of columns applied, which = SK_S or SK_ST): 1 the tensor-core
 * +-1 product (R's {0, +-1} pattern is exact in bf16, A is split into bf16
 * hi + lo), 0 the SJLT kernels (FP32 sums over R's entries), -1 not measured
 * yet.  The first product of a shape times both routes on its stream (one
 * synchronization) and keeps the faster; SK_PREC_NATIVE always takes the SJLT
 * kernels.  JLS_SJLT_ROUTE=tc or =sjlt pins the route for the process (shapes
 * served that way are not recorded, and report -1).  A diagnostic query; the
 * paper has no counterpart. */
int sketch_sjlt_route(int32_t kind, int64_t n, int64_t rows, int64_t cols, int32_t width, int32_t which);

/* ---- per-node adaptive HSS compression (Algorithm 1) -------------------- */
/*
 * hss_compress_adaptive -- Algorithm 1 (HSSCompressAdaptive, Supplementary D)
 * for a symmetric A: compress every node of a binary cluster tree from one
 * growing global sketch S = A R.
 *   Tree: node [lo, hi) with more than `leaf` indices splits into
 *   [lo, lo + (hi-lo)/2) and the rest; level(root) = 0.
 *   Per node tau, visited level by level from the leaves (the nodes of a
 *   level together):
 *     leaf      S_tau(:, iota) = S(I_tau, iota) - D_tau R(I_tau, iota), D_tau = A(I_tau, I_tau)
 *     internal  S_tau(:, iota) = [S_nu1(J_nu1, iota) - B_tau R_nu2(:, iota);
 *                                 S_nu2(J_nu2, iota) - B_tau^T R_nu1(:, iota)],
 *               B_tau = A(I~_nu1, I~_nu2)
 *     (iota = all d + Delta-d columns on the first visit, the new Delta-d later);
 *     a node not yet compressed takes the test of Eq. (3.1) with
 *     eps^tau = eps / level(tau): S~ = its last Delta-d columns,
 *     S^ = (I - Q Q^T)^2 S~ against a basis Q of the earlier columns' range;
 *     passed, or min |diag Om^| of {Q^, Om^} = QR(S^) below eps_abs^tau or
 *     eps_rel^tau |(Om_tau)_11| (the rank-deficiency test): compress by the row
 *     interpolative decomposition S_tau ~ U_tau S_tau(J_tau, :) (column-pivoted
 *     QR of S_tau^T, rank = pivots above eps_abs^tau and eps_rel^tau |R_11|),
 *     R_tau = U_tau^T R(I_tau) or U_tau^T [R_nu1; R_nu2],
 *     I~_tau = I_tau(J_tau) or [I~_nu1, I~_nu2](J_tau).
 *     Otherwise the sweep ends after this level, R grows by Delta-d columns
 *     (each block keeps its own scale, SK_SCALE_BLOCK), S <- [S  A R_bar],
 *     d <- d + Delta-d, and the next sweep starts from the leaves; the loop
 *     also ends, unconverged, when R would exceed d_max columns.
 *   A      device, n x n FP64, row-major, symmetric (not checked), 16-byte
 *          aligned, lda >= n with lda * 8 % 16 == 0.  Read during the call
 *          only (D and B are copied).
 *   leaf   1 .. 4096; kind, alpha, seed as sketch_create; d0, dd >= 1 with
 *          d0 + dd <= d_max <= 2048, d_max even.
 *   eps_rel, eps_abs >= 0: the tolerances before the level division.
 * Every step runs on the device in FP64; the host reads each level's
 * outcomes and ranks (it synchronizes `stream` a few times per level).
 * Out: *out owns the generators until hss_destroy.  Errors: INVALID_ARG,
 * ALIGN, UNSUPPORTED (a local sketch of more than 4096 rows), NOMEM, DEVICE.
 */
typedef struct sk_hss* sk_hss_handle;
int hss_compress_adaptive(sk_hss_handle* out, const double* A, int64_t n, int64_t lda, int32_t leaf,
                          int32_t kind, int32_t d0, int32_t dd, int32_t alpha, uint64_t seed, int32_t d_max,
                          double eps_rel, double eps_abs, void* stream);

/* hss_info -- host outputs (each may be NULL): node count, final d, columns
 * of R, sweeps run, converged (1: the root was reached), stopping tests run. */
int hss_info(sk_hss_handle h, int32_t* nodes, int32_t* d, int32_t* d_total, int32_t* sweeps,
             int32_t* converged, int32_t* tests);

/* hss_node -- node `node` (0 = root, preorder): lohi[2] = {lo, hi} and
 * info[7] = {level, parent, child 1, child 2 (-1: none), state (0 untouched,
 * 1 partially compressed, 2 compressed), m = rows of S_tau, k = rank}. */
int hss_node(sk_hss_handle h, int32_t node, int64_t* lohi, int32_t* info);

/* hss_node_get -- copy one generator of a node to host memory `dst`:
 *   SK_HSS_U   U_tau, m x k FP64 row-major        SK_HSS_J   J_tau, k int32 (0-based rows of S_tau)
 *   SK_HSS_IT  I~_tau, k int32 (rows of A)        SK_HSS_D   D_tau (leaf), m x m FP64 column-major
 *   SK_HSS_B   B_tau (internal, root), k_nu1 x k_nu2 FP64 column-major
 *   SK_HSS_S   S_tau, m x (d + Delta-d) FP64 column-major
 *   SK_HSS_R   R_tau, k x (d + Delta-d) FP64 column-major
 * Synchronous.  Errors: INVALID_ARG, STATE (not computed for this node). */
#define SK_HSS_U  1
#define SK_HSS_J  2
#define SK_HSS_IT 3
#define SK_HSS_D  4
#define SK_HSS_B  5
#define SK_HSS_S  6
#define SK_HSS_R  7
int hss_node_get(sk_hss_handle h, int32_t node, int32_t what, void* dst);

/* hss_history -- the stopping tests in the order run: ints[4 t] = {sweep,
 * level, node, outcome (0 passed Eq. (3.1), 1 compressed by the rank test,
 * 2 needs more columns)}, reals[3 t] = {||S^||_F, ||S~||_F, min |diag Om^|
 * (0 when not computed)}; host arrays of hss_info's `tests` records. */
int hss_history(sk_hss_handle h, int32_t* ints, double* reals);

/* hss_launch_count -- kernels the handle launched (the sketch kernels of S
 * excluded). */
int64_t hss_launch_count(sk_hss_handle h);

/* hss_profile -- device time (ms, from CUDA events on the stream around each
 * launch), algorithmic FP64 FLOPs, launches and SM-milliseconds (the SMs a
 * launch's grid occupies, at most one CTA per SM counted, times its ms) per
 * kind of work, host arrays of 6 entries each (any may be NULL):
 *   0 copies of D_tau and B_tau from A     1 local sketches (GEMM)
 *   2 stopping and rank tests              3 interpolative decompositions
 *   4 R_tau (GEMM)                         5 global sketch S = A R, its
 *                                            increments and R's dense copy
 * FLOPs: 2 M N K per GEMM; 8 m q per vector projected twice against q basis
 * columns; 2 m C for a decomposition's row norms plus 4 C per remaining row and
 * pivot step, plus the triangular solves; 2 n^2 per column of S (dense count,
 * also for SJLT).  sm_ms / ms is the average number of SMs a kind of work held. */
int hss_profile(sk_hss_handle h, double* ms, double* flops, int64_t* launches, double* sm_ms);

/* hss_destroy -- free the generators and scratch (NULL is a no-op). */
void hss_destroy(sk_hss_handle h);

/* sketch_destroy -- free the handle and its device memory (NULL is a no-op). */
void sketch_destroy(sk_handle h);

/* sketch_strerror -- static text for a status code. */
const char* sketch_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* JLSKETCH_H */
