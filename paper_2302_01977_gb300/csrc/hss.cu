// hss.cu -- the per-node adaptive loop of Algorithm 1 (HSSCompressAdaptive,
// Supplementary D) on the device, in FP64, for a symmetric explicit A.
//
// The nodes of one level of the cluster tree are processed together (the
// leaves of the walk-through are compressed in parallel): one launch computes
// every local sketch of the level, one launch runs every node's stopping and
// rank-deficiency tests, one launch the interpolative decompositions of the
// nodes that compress, one launch their R_tau columns.  The host reads each
// level's outcomes (a few bytes) to decide the next launch; a node that needs
// more columns ends the sweep after its level, R grows by Delta-d columns
// (S <- [S  A R_bar] by the sketch kernels) and the next sweep starts again
// from the leaves.
//
// Per node tau (m rows of the local sketch, k = rank after compression):
//   S_tau  m x d_max, column-major          local sketch (leaf: S(I, iota) - D R(I, iota);
//                                            internal: [S_nu1(J_nu1) - B R_nu2; S_nu2(J_nu2) - B^T R_nu1])
//   Q_tau  m x (min(m, d_max) + Delta-d),   orthonormal basis of the tested columns' range
//          column-major
//   U_tau  m x k, row-major                 row interpolative decomposition S_tau ~ U_tau S_tau(J_tau, :)
//   J_tau  k positions in 0..m-1;  I~_tau  k global indices
//   R_tau  k x d_max, column-major          U_tau^T R(I_tau) (leaf) or U_tau^T [R_nu1; R_nu2]
//   D_tau  (leaf) m x m, B_tau (internal, root) k_nu1 x k_nu2, column-major, copied from A
//
// All FP64: the local sketch is a difference of two large terms (S(I, :)
// holds the diagonal block's product), and the tests and the decomposition
// resolve eps / level(tau) relative to it.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include <cooperative_groups.h>

#include "common.cuh"
#include "internal.h"

namespace cg = cooperative_groups;

namespace jls {
namespace {

constexpr int HSS_MAX_ROWS = 4096;  // rows of a node's local sketch (a column lives in shared memory)
constexpr int HSS_MAX_D = 2048;     // columns of R
constexpr int HT = 256;             // threads of the per-node kernels
constexpr int GT = 64;              // GEMM tile (rows and columns of the output)
constexpr int GK = 16;              // GEMM tile depth

// ---- operands of the batched GEMM jobs -------------------------------------
// Element (r, c) of an operand: rows [0, split) come from p (row r -> idx[r]
// when idx is set), rows [split, ...) from p2 the same way, at
// base[row * rs + c * cs].
struct Opnd {
  const double* p = nullptr;
  int64_t rs = 0, cs = 0;
  const int32_t* idx = nullptr;
  int32_t split = 1 << 30;
  const double* p2 = nullptr;
  int64_t rs2 = 0, cs2 = 0;
  const int32_t* idx2 = nullptr;
};

__device__ __forceinline__ double opnd_at(const Opnd& o, int r, int c) {
  if (r < o.split) {
    const int64_t rr = o.idx ? o.idx[r] : r;
    return o.p[rr * o.rs + (int64_t)c * o.cs];
  }
  r -= o.split;
  const int64_t rr = o.idx2 ? o.idx2[r] : r;
  return o.p2[rr * o.rs2 + (int64_t)c * o.cs2];
}

// out(r, c) = [c_in(r, c)] + alpha * sum_k a(r, k) b(k, c), r < M, c < N.
struct GemmJob {
  Opnd a, b, c;
  double* out = nullptr;
  int64_t ors = 1, ocs = 0;
  int32_t M = 0, N = 0, K = 0;
  int32_t has_c = 0;
  double alpha = 1.0;
  int32_t tile0 = 0, tiles_n = 0;
};

// One 64 x 64 output tile per CTA; 256 threads, 4 x 4 outputs each.
__global__ void __launch_bounds__(256) hss_gemm_kernel(const GemmJob* __restrict__ jobs, int njobs) {
  __shared__ double As[GK][GT + 1];
  __shared__ double Bs[GK][GT + 1];
  const int tile = blockIdx.x;
  int lo = 0, hi = njobs - 1;  // last job with tile0 <= tile
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (jobs[mid].tile0 <= tile) lo = mid; else hi = mid - 1;
  }
  const GemmJob& J = jobs[lo];
  const int t = tile - J.tile0;
  const int m0 = (t / J.tiles_n) * GT, n0 = (t % J.tiles_n) * GT;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[4][4] = {};
  for (int k0 = 0; k0 < J.K; k0 += GK) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int e = threadIdx.x + 256 * u;
      const int kk = e / GT, mm = e % GT;
      const int r = m0 + mm, k = k0 + kk;
      As[kk][mm] = (r < J.M && k < J.K) ? opnd_at(J.a, r, k) : 0.0;
      const int cc = n0 + mm;
      Bs[kk][mm] = (cc < J.N && k < J.K) ? opnd_at(J.b, k, cc) : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      double av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) av[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = m0 + ty * 4 + i;
    if (r >= J.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = n0 + tx * 4 + j;
      if (c >= J.N) continue;
      double v = J.alpha * acc[i][j];
      if (J.has_c) v += opnd_at(J.c, r, c);
      J.out[(int64_t)r * J.ors + (int64_t)c * J.ocs] = v;
    }
  }
}

// ---- gathers of A's entries: out(r, c) = A(row(r), col(c)), column-major ---
struct GatherJob {
  double* out = nullptr;
  int32_t rows = 0, cols = 0;
  const int32_t* ri = nullptr;  // global row indices, or rows r0 + r
  const int32_t* ci = nullptr;
  int64_t r0 = 0, c0 = 0;
};

__global__ void hss_gather_kernel(const GatherJob* __restrict__ jobs, const double* __restrict__ A, int64_t lda) {
  const GatherJob& J = jobs[blockIdx.x];
  const int64_t total = (int64_t)J.rows * J.cols;
  for (int64_t e = threadIdx.x; e < total; e += blockDim.x) {
    const int r = (int)(e % J.rows), c = (int)(e / J.rows);
    const int64_t gr = J.ri ? J.ri[r] : J.r0 + r;
    const int64_t gc = J.ci ? J.ci[c] : J.c0 + c;
    J.out[e] = A[gr * lda + gc];
  }
}

// ---- block and cluster reductions ----------------------------------------
// The per-node kernels run one thread-block cluster of ncl CTAs per node
// (ncl = 1 .. 16, chosen by the host from the level's node count); CTA r of
// the cluster owns the rows [r0, r1) of the node's local sketch.  A sum over
// the node's rows is a CTA partial per CTA, published in a double-buffered
// shared-memory slot, a cluster barrier, and the partials added in rank order
// by every CTA, so every CTA holds the same sums and takes the same decisions.
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// Sum over each half of the warp (lanes 0..15 and 16..31 separately).
__device__ __forceinline__ double half_sum(double v) {
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the CTA; every thread gets the result.  red: >= 33 doubles.
__device__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int w = threadIdx.x / 32, l = threadIdx.x % 32;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    double x = l < (int)(blockDim.x / 32) ? red[l] : 0.0;
    x = warp_sum(x);
    if (l == 0) red[32] = x;
  }
  __syncthreads();
  return red[32];
}

constexpr int HPS = HSS_MAX_D + 128;  // doubles per partial slot

struct Cl {
  int ncl, rank;
  int r0, r1;        // this CTA's rows
  int par;           // partial slot in use
  double* hp;        // 2 slots of HPS doubles, read by the cluster
  double* red;
};

__device__ __forceinline__ void cl_sync() { cg::this_cluster().sync(); }

// out[j] = sum over the cluster's CTAs of slot[j], j < count (after every CTA
// wrote its partials into c.hp + c.par * HPS).
__device__ void cl_finish(Cl& c, int count, double* out) {
  cl_sync();
  const double* base = c.hp + c.par * HPS;
  for (int j = threadIdx.x; j < count; j += blockDim.x) {
    double s = 0.0;
    for (int r0 = 0; r0 < c.ncl; r0 += 8) {  // 8 remote loads in flight, added in rank order
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        v[u] = r0 + u < c.ncl ? *cg::this_cluster().map_shared_rank(base + j, (unsigned)(r0 + u)) : 0.0;
#pragma unroll
      for (int u = 0; u < 8; ++u) s += v[u];
    }
    out[j] = s;
  }
  c.par ^= 1;
  __syncthreads();
}

// Sum of v over the node's rows (v: this thread's partial over its rows).
__device__ double cl_sum(Cl& c, double v, double* scal) {
  const double b = block_sum(v, c.red);
  if (threadIdx.x == 0) c.hp[c.par * HPS] = b;
  cl_finish(c, 1, scal);
  return scal[0];
}

// w <- (I - Q Q^T)^2 w against the columns [c_lo, c_hi) of Q; Qb points at
// this CTA's rows of column 0 (column j at Qb + j ld: the CTA's cache in
// shared memory or Q itself), w and the coefficients h (>= c_hi - c_lo
// doubles) in shared memory, w holding this CTA's rows only.
__device__ void project2(Cl& c, const double* __restrict__ Qb, int64_t ld, int c_lo, int c_hi, double* w,
                         double* h, double* gp) {
  const int nw = blockDim.x / 32, wid = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int mr = c.r1 - c.r0;
  for (int pass = 0; pass < 2; ++pass) {
    double* part = c.hp + c.par * HPS;
    // Q^T w: a warp takes 4 columns at a time, so that each lane has 4
    // (times the unrolled rows) independent loads in flight
    // each half-warp takes a quad of columns, its 16 lanes over the rows
    // (rows come in 16s, so few lanes idle when a CTA holds a few dozen rows)
    const int hw = lane >> 4, hl = lane & 15;
    for (int jb = c_lo + 8 * wid; jb < c_hi; jb += 8 * nw) {
      const int j0 = jb + 4 * hw;
      const int nj = max(0, min(4, c_hi - j0));
      const double* q = Qb + (int64_t)j0 * ld;
      double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
      if (nj > 0) {
#pragma unroll 2
        for (int i = hl; i < mr; i += 16) {
          const double wi = w[i];
          s0 = fma(q[i], wi, s0);
          if (nj > 1) s1 = fma(q[ld + i], wi, s1);
          if (nj > 2) s2 = fma(q[2 * ld + i], wi, s2);
          if (nj > 3) s3 = fma(q[3 * ld + i], wi, s3);
        }
      }
      s0 = half_sum(s0);
      s1 = half_sum(s1);
      s2 = half_sum(s2);
      s3 = half_sum(s3);
      if (hl == 0 && nj > 0) {
        part[j0 - c_lo] = s0;
        if (nj > 1) part[j0 + 1 - c_lo] = s1;
        if (nj > 2) part[j0 + 2 - c_lo] = s2;
        if (nj > 3) part[j0 + 3 - c_lo] = s3;
      }
    }
    cl_finish(c, c_hi - c_lo, h);
    // w -= Q h: G groups of threads split the columns, each thread of a
    // group a row; the groups' sums (gp: G x mr) are added in group order
    const int G = mr > 0 ? max(1, min((int)blockDim.x / mr, 8)) : 1;
    const int g = threadIdx.x / max(mr, 1);
    if (mr > 0 && g < G) {
      for (int i = threadIdx.x % mr; i < mr; i += blockDim.x) {
        // 8 independent loads in flight per thread
        const double* q = Qb + i;
        double a[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
        int j = c_lo + g;
        for (; j + 7 * G < c_hi; j += 8 * G) {
#pragma unroll
          for (int u = 0; u < 8; ++u) a[u] = fma(q[(int64_t)(j + u * G) * ld], h[j + u * G - c_lo], a[u]);
        }
        for (; j < c_hi; j += G) a[0] = fma(q[(int64_t)j * ld], h[j - c_lo], a[0]);
        gp[g * mr + i] = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < mr; i += blockDim.x) {
      double s = 0.0;
      for (int u = 0; u < G; ++u) s += gp[u * mr + i];
      w[i] -= s;
    }
    __syncthreads();
  }
}

// The same two passes for g <= 8 columns at once (independent columns, all
// against the same q columns of Q): wg holds them at stride wld; one cluster
// sum per pass serves all g columns (h: g x q coefficients).
constexpr int GMAX = 8;
__device__ void project2_group(Cl& c, const double* __restrict__ Qb, int64_t ld, int q, double* wg, int wld, int g,
                               double* h) {
  const int nw = blockDim.x / 32, wid = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int mr = c.r1 - c.r0;
  for (int pass = 0; pass < 2; ++pass) {
    double* part = c.hp + c.par * HPS;
    const int hw = lane >> 4, hl = lane & 15;
    for (int jb = 8 * wid; jb < q; jb += 8 * nw) {  // a half-warp per quad of columns
      const int j0 = jb + 4 * hw;
      const int nj = max(0, min(4, q - j0));
      const double* qc = Qb + (int64_t)j0 * ld;
      double sacc[4][GMAX];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int u = 0; u < GMAX; ++u) sacc[a][u] = 0.0;
      for (int i = hl; i < mr && nj > 0; i += 16) {
        double qv[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) qv[a] = a < nj ? qc[a * ld + i] : 0.0;
#pragma unroll
        for (int u = 0; u < GMAX; ++u) {
          if (u < g) {
            const double wv = wg[u * wld + i];
#pragma unroll
            for (int a = 0; a < 4; ++a) sacc[a][u] = fma(qv[a], wv, sacc[a][u]);
          }
        }
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int u = 0; u < GMAX; ++u)
          if (u < g) {  // uniform over the warp
            const double v = half_sum(sacc[a][u]);
            if (hl == 0 && a < nj) part[u * q + j0 + a] = v;
          }
    }
    cl_finish(c, g * q, h);
    // w_u -= Q h_u over (row, column) pairs, 8 loads in flight per thread
    for (int pr = threadIdx.x; pr < mr * g; pr += blockDim.x) {
      const int i = pr % mr, u = pr / mr;
      const double* hu = h + u * q;
      const double* qi = Qb + i;
      double a[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
      int j = 0;
      for (; j + 8 <= q; j += 8) {
#pragma unroll
        for (int v = 0; v < 8; ++v) a[v] = fma(qi[(int64_t)(j + v) * ld], hu[j + v], a[v]);
      }
      for (; j < q; ++j) a[0] = fma(qi[(int64_t)j * ld], hu[j], a[0]);
      wg[u * wld + i] -= ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
    }
    __syncthreads();
  }
}

__device__ __forceinline__ void cl_rows(Cl& c, int m) {
  const cg::cluster_group cl = cg::this_cluster();
  c.ncl = (int)cl.num_blocks();
  c.rank = (int)cl.block_rank();
  c.r0 = (int)((int64_t)m * c.rank / c.ncl);
  c.r1 = (int)((int64_t)m * (c.rank + 1) / c.ncl);
  c.par = 0;
}

// ---- per-node stopping and rank-deficiency tests ----------------------------
struct TestJob {
  const double* S = nullptr;  // local sketch, m x ..., column-major, ld = m
  double* Q = nullptr;        // basis, ld = m
  int32_t m = 0, d = 0, dd = 0;
  int32_t q = -1;             // basis columns so far; -1: build it from S(:, 0:d)
  int32_t qcap = 0;           // columns Q can hold
  double er = 0, ea = 0;
  double om11 = 0;            // |(Omega_tau)_11| once the basis exists
};
struct TestOut {
  double nh, nt, mind, om11;
  int32_t q, outcome;         // outcome: 0 passed (Eq. (3.1)), 1 rank-deficient, 2 needs more columns
};

// Shared memory of the test kernel, laid out per launch from the largest rows
// per CTA (mrx) and basis columns (qx, the basis after this test included):
// w (this CTA's rows), h, 2 partial slots, red, the projection's group sums
// (G x mr <= max(mrx, blockDim)), and this CTA's rows of Q (mrx x qx) when they
// fit (qsm).
struct TestLayout {
  int mrx, qx, qsm;
  int gw;  // columns of the tested block projected together (the w buffer holds gw x mrx)
};
__host__ __device__ inline size_t test_smem_bytes(const TestLayout& L) {
  return sizeof(double) * ((size_t)L.gw * L.mrx + 3 * HPS + 40 + (size_t)(L.mrx > HT ? L.mrx : HT) +
                           (L.qsm ? (size_t)L.mrx * L.qx : 0));
}
constexpr size_t TEST_SMEM_MAX = 220 * 1024;

__global__ void __launch_bounds__(HT) hss_test_kernel(const TestJob* __restrict__ jobs, TestOut* __restrict__ outs,
                                                      TestLayout L) {
  extern __shared__ double sm[];
  const int node = (int)(blockIdx.x / cg::this_cluster().num_blocks());
  const TestJob J = jobs[node];
  const int m = J.m;
  Cl c;
  cl_rows(c, m);
  double* w = sm;                   // this CTA's rows (gw columns of them for the tested block)
  double* h = w + (size_t)L.gw * L.mrx;  // coefficients
  c.hp = h + HPS;                   // 2 partial slots
  c.red = c.hp + 2 * HPS;           // 33 + scalar out
  double* scal = c.red + 36;
  double* gp = c.red + 40;          // group sums
  double* Qs = gp + (L.mrx > HT ? L.mrx : HT);
  const int mr = c.r1 - c.r0;
  // this CTA's rows of the basis: cached in shared memory (qsm) or read from Q
  const double* Qb = L.qsm ? Qs : J.Q + c.r0;
  const int64_t ldb = L.qsm ? L.mrx : m;
  auto put_col = [&](int j, double scale) {  // Q(:, j) = w / scale over this CTA's rows
    for (int i = threadIdx.x; i < mr; i += blockDim.x) {
      const double v = scale == 1.0 ? w[i] : w[i] / scale;
      J.Q[(int64_t)j * m + c.r0 + i] = v;
      if (L.qsm) Qs[(int64_t)j * L.mrx + i] = v;
    }
  };
  int q = J.q;
  double om11 = J.om11;
  if (L.qsm && q > 0) {
    for (int64_t e = threadIdx.x; e < (int64_t)mr * q; e += blockDim.x) {
      const int i = (int)(e % mr), j = (int)(e / mr);
      Qs[(int64_t)j * L.mrx + i] = J.Q[(int64_t)j * m + c.r0 + i];
    }
    __syncthreads();
  }
  if (q < 0) {
    // Q_tau: orthonormal basis of the range of S_tau(:, 0:d), columns kept
    // above max(m, d) eps ||S_tau(:, 0:d)||_F (two Gram-Schmidt passes each)
    double f2 = 0.0;
    for (int j = 0; j < J.d; ++j)
      for (int i = threadIdx.x; i < mr; i += blockDim.x) {
        const double v = J.S[(int64_t)j * m + c.r0 + i];
        f2 = fma(v, v, f2);
      }
    f2 = cl_sum(c, f2, scal);
    const double thr = (double)max(m, J.d) * 2.220446049250313e-16 * sqrt(f2);
    q = 0;
    for (int j = 0; j < J.d; ++j) {
      double c2 = 0.0;
      for (int i = threadIdx.x; i < mr; i += blockDim.x) {
        const double v = J.S[(int64_t)j * m + c.r0 + i];
        w[i] = v;
        c2 = fma(v, v, c2);
      }
      if (j == 0) om11 = sqrt(cl_sum(c, c2, scal));
      __syncthreads();
      if (q > 0) project2(c, Qb, ldb, 0, q, w, h, gp);
      double r2 = 0.0;
      for (int i = threadIdx.x; i < mr; i += blockDim.x) r2 = fma(w[i], w[i], r2);
      const double r = sqrt(cl_sum(c, r2, scal));
      if (r > thr && r > 0.0) {
        put_col(q, r);
        ++q;
      }
      __syncthreads();
    }
  }
  if (q + J.dd > J.qcap || (L.qsm && q + J.dd > L.qx)) {
    // more basis columns than Q holds: only when q = m (the basis spans all
    // of R^m and S^ = 0); counted as passed with ||S^|| = 0
    if (threadIdx.x == 0 && c.rank == 0) {
      TestOut o;
      o.nh = 0.0; o.nt = 0.0; o.mind = 0.0; o.om11 = om11; o.q = q; o.outcome = 0;
      outs[node] = o;
    }
    cl_sync();  // no CTA leaves while its partial slots may still be read
    return;
  }
  // S~ = S_tau(:, d : d + dd), S^ = (I - Q Q^T)^2 S~ into Q(:, q : q + dd): the columns are
  // projected against the same Q, gw at a time; ||S~||^2 and ||S^||^2 are summed over this CTA's
  // rows on the way and over the cluster once at the end
  double nt2p = 0.0, nh2p = 0.0;
  const int gq = q > 0 ? max(1, min(L.gw, HPS / q)) : L.gw;
  for (int jj0 = 0; jj0 < J.dd; jj0 += gq) {
    const int g = min(gq, J.dd - jj0);
    for (int pr = threadIdx.x; pr < mr * g; pr += blockDim.x) {
      const int i = pr % mr, u = pr / mr;
      const double v = J.S[(int64_t)(J.d + jj0 + u) * m + c.r0 + i];
      w[u * L.mrx + i] = v;
      nt2p = fma(v, v, nt2p);
    }
    __syncthreads();
    if (q > 0) project2_group(c, Qb, ldb, q, w, L.mrx, g, h);
    for (int pr = threadIdx.x; pr < mr * g; pr += blockDim.x) {
      const int i = pr % mr, u = pr / mr;
      const double v = w[u * L.mrx + i];
      nh2p = fma(v, v, nh2p);
      J.Q[(int64_t)(q + jj0 + u) * m + c.r0 + i] = v;
      if (L.qsm) Qs[(int64_t)(q + jj0 + u) * L.mrx + i] = v;
    }
    __syncthreads();
  }
  {
    const double t2 = block_sum(nt2p, c.red);
    const double h2 = block_sum(nh2p, c.red);
    if (threadIdx.x == 0) {
      c.hp[c.par * HPS] = t2;
      c.hp[c.par * HPS + 1] = h2;
    }
    cl_finish(c, 2, scal);
  }
  const double nt2 = scal[0], nh2 = scal[1];
  const double nh = sqrt(nh2), nt = sqrt(nt2);
  int outcome = 0;
  double mind = 0.0;
  if (!(nt == 0.0 || nh < J.ea || nh < J.er * nt)) {
    // {Q^, Om^} = QR(S^) column by column; |diag Om^| = the residual norms
    mind = INFINITY;
    for (int jj = 0; jj < J.dd; ++jj) {
      for (int i = threadIdx.x; i < mr; i += blockDim.x) w[i] = Qb[(int64_t)(q + jj) * ldb + i];
      __syncthreads();
      if (jj > 0) project2(c, Qb, ldb, q, q + jj, w, h, gp);
      double r2 = 0.0;
      for (int i = threadIdx.x; i < mr; i += blockDim.x) r2 = fma(w[i], w[i], r2);
      const double r = sqrt(cl_sum(c, r2, scal));
      mind = fmin(mind, r);
      if (r > 0.0) {
        put_col(q + jj, r);
      } else {
        for (int i = threadIdx.x; i < mr; i += blockDim.x) w[i] = 0.0;
        put_col(q + jj, 1.0);
      }
      __syncthreads();
    }
    if (mind < J.ea || mind < J.er * om11) {
      outcome = 1;
    } else {
      outcome = 2;
      q += J.dd;
    }
  }
  if (threadIdx.x == 0 && c.rank == 0) {
    TestOut o;
    o.nh = nh; o.nt = nt; o.mind = mind; o.om11 = om11; o.q = q; o.outcome = outcome;
    outs[node] = o;
  }
  cl_sync();  // no CTA leaves while its partial slots may still be read
}

// ---- row interpolative decomposition S ~ U S(J, :) --------------------------
// Column-pivoted QR of S^T by modified Gram-Schmidt on the rows of S: the
// pivot is the remaining row of largest partial norm (the lowest index on a
// tie); the partial norms are downdated, |a_i|^2 <- |a_i|^2 - r_ti^2, and
// summed afresh when the downdate has cancelled below 1e-8 of the last exact
// value (the safeguard of LAPACK's column-pivoted QR); rank k = the pivots
// whose exact norm exceeds eps_a and eps_r |R_11|; U^T = [I, R11^{-1} R12] P^T.  The rows are spread over the
// cluster; every CTA finds the same pivot from the CTAs' candidates and reads
// the pivot row itself (the same arithmetic in every CTA), so one cluster
// barrier per pivot step orders the row updates.
struct IdJob {
  const double* S = nullptr;  // m x C, column-major, ld = m
  int32_t m = 0, C = 0;
  double er = 0, ea = 0;
  double* W = nullptr;        // m x C scratch, row-major (ld = C)
  double* Rf = nullptr;       // min(m, C) x m scratch: Rf[t m + i] = r_ti
  double* R11 = nullptr;      // min(m, C)^2 scratch: R11 in pivot order, row-major
  double* U = nullptr;        // m x min(m, C) output, row-major (ld = k)
  int32_t* Jl = nullptr;      // local pivots
  int32_t* It = nullptr;      // global skeleton indices
  int64_t lo = 0;             // leaf: I_tau = lo + [0, m)
  const int32_t* It1 = nullptr;  // internal: [I~_nu1, I~_nu2]
  const int32_t* It2 = nullptr;
  int32_t k1 = 0;
};

// Shared memory of the decomposition kernel, laid out per launch from the
// largest C, rows per CTA (mr) and pivots (kx) of its nodes: qv (the pivot
// row), red, 2 candidate slots, nrm and ref (this CTA's rows), this CTA's
// rows of W when they fit (wsm), perm (every pivot), used (this CTA's rows).
struct IdLayout {
  int Cx, mrx, kx, wsm;
};
__host__ __device__ inline size_t id_smem_bytes(const IdLayout& L) {
  return sizeof(double) * ((size_t)L.Cx + 44 + 2 * (size_t)L.mrx + (L.wsm ? (size_t)L.mrx * L.Cx : 0)) +
         sizeof(int) * ((size_t)L.kx + L.mrx);
}
constexpr size_t ID_SMEM_MAX = 200 * 1024;

__global__ void __launch_bounds__(HT) hss_id_kernel(const IdJob* __restrict__ jobs, int32_t* __restrict__ ranks,
                                                    IdLayout L) {
  extern __shared__ double sm[];
  const int node = (int)(blockIdx.x / cg::this_cluster().num_blocks());
  const IdJob J = jobs[node];
  const int m = J.m, C = J.C, kmax = min(m, C);
  Cl c;
  cl_rows(c, m);
  const int mr = c.r1 - c.r0;
  double* qv = sm;                     // C
  double* red = qv + L.Cx;             // 40
  double* cand = red + 40;             // 2 slots x (value, index)
  double* nrm = cand + 4;              // this CTA's rows: partial norms
  double* ref = nrm + L.mrx;           // their last exact values
  double* Wsm = ref + L.mrx;           // this CTA's rows of W (wsm)
  int* perm = reinterpret_cast<int*>(Wsm + (L.wsm ? (size_t)L.mrx * L.Cx : 0));
  int* used = perm + L.kx;             // this CTA's rows
  // this CTA's rows of W: in shared memory when they fit, else in J.W
  double* Wmine = L.wsm ? Wsm : J.W + (int64_t)c.r0 * C;
  __shared__ int s_arg;
  const int nw = blockDim.x / 32, wid = threadIdx.x / 32, lane = threadIdx.x % 32;
  // W = S (row-major) for this CTA's rows, their norms
  for (int64_t e = threadIdx.x; e < (int64_t)mr * C; e += blockDim.x) {
    const int i = (int)(e % mr), cc = (int)(e / mr);
    Wmine[(int64_t)i * C + cc] = J.S[(int64_t)cc * m + c.r0 + i];
  }
  __syncthreads();
  for (int i = wid; i < mr; i += nw) {
    const double* row = Wmine + (int64_t)i * C;
    double s = 0.0;
    for (int cc = lane; cc < C; cc += 32) s = fma(row[cc], row[cc], s);
    s = warp_sum(s);
    if (lane == 0) { nrm[i] = s; ref[i] = s; used[i] = 0; }
  }
  __syncthreads();
  int k = 0;
  double r11 = 0.0;
  for (int t = 0; t < kmax; ++t) {
    // this CTA's candidate: the largest partial norm among its unused rows
    double bv = -1.0;
    int bi = m;
    for (int i = threadIdx.x; i < mr; i += blockDim.x)
      if (!used[i] && nrm[i] > bv) { bv = nrm[i]; bi = c.r0 + i; }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
    if (lane == 0) { red[wid] = bv; red[16 + wid] = (double)bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double b = -1.0;
      int a = m;
      for (int u = 0; u < nw; ++u) {
        const double v = red[u];
        const int ai = (int)red[16 + u];
        if (v > b || (v == b && ai < a)) { b = v; a = ai; }
      }
      cand[2 * (t & 1)] = b;
      cand[2 * (t & 1) + 1] = (double)a;
    }
    cl_sync();  // candidates and the previous step's row updates are visible
    if (threadIdx.x == 0) {
      double b = -1.0;
      int a = m;
      for (int r = 0; r < c.ncl; ++r) {
        const double* rc = cg::this_cluster().map_shared_rank(cand + 2 * (t & 1), (unsigned)r);
        const double v = rc[0];
        const int ai = (int)rc[1];
        if (v > b || (v == b && ai < a)) { b = v; a = ai; }
      }
      s_arg = a;
    }
    __syncthreads();
    const int p = s_arg;
    if (p >= m) break;
    // the pivot row and its exact norm (the same in every CTA)
    const double* prow;
    if (L.wsm) {
      int owner = 0;
      while ((int64_t)m * (owner + 1) / c.ncl <= p) ++owner;
      const int o0 = (int)((int64_t)m * owner / c.ncl);
      prow = cg::this_cluster().map_shared_rank(Wsm, (unsigned)owner) + (int64_t)(p - o0) * C;
    } else {
      prow = J.W + (int64_t)p * C;
    }
    double s = 0.0;
    for (int cc = threadIdx.x; cc < C; cc += blockDim.x) {
      const double v = prow[cc];
      qv[cc] = v;
      s = fma(v, v, s);
    }
    const double rpp = sqrt(block_sum(s, red));
    if (t == 0) r11 = rpp;
    if (!(rpp > J.ea) || !(rpp > J.er * r11)) break;
    for (int cc = threadIdx.x; cc < C; cc += blockDim.x) qv[cc] /= rpp;
    if (threadIdx.x == 0) {
      perm[t] = p;
      if (p >= c.r0 && p < c.r1) {
        used[p - c.r0] = 1;
        J.Rf[(int64_t)t * m + p] = rpp;
      }
    }
    __syncthreads();
    for (int i = wid; i < mr; i += nw) {
      if (used[i]) continue;
      double* row = Wmine + (int64_t)i * C;
      double r = 0.0;
      if (C <= 512) {
        // the lane's 16 entries of the row in registers: one load each
        double v[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const int cc = lane + 32 * u;
          v[u] = cc < C ? row[cc] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const int cc = lane + 32 * u;
          if (cc < C) r = fma(v[u], qv[cc], r);
        }
        r = warp_sum(r);
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const int cc = lane + 32 * u;
          if (cc < C) row[cc] = fma(-r, qv[cc], v[u]);
        }
      } else {
#pragma unroll 4
        for (int cc = lane; cc < C; cc += 32) r = fma(row[cc], qv[cc], r);
        r = warp_sum(r);
#pragma unroll 4
        for (int cc = lane; cc < C; cc += 32) row[cc] = fma(-r, qv[cc], row[cc]);
      }
      // downdate; the whole warp takes the same branch (r and nrm[i] are uniform)
      double n2 = nrm[i] - r * r;
      if (!(n2 > 1e-8 * ref[i])) {
        __syncwarp();
        n2 = 0.0;
        for (int cc = lane; cc < C; cc += 32) n2 = fma(row[cc], row[cc], n2);
        n2 = warp_sum(n2);
        if (lane == 0) ref[i] = n2;
      }
      __syncwarp();
      if (lane == 0) {
        J.Rf[(int64_t)t * m + c.r0 + i] = r;
        nrm[i] = n2;
      }
    }
    k = t + 1;
    __syncthreads();
  }
  // R11 in pivot order (row-major, k x k upper triangle), rows split over the cluster
  cl_sync();
  for (int s2 = c.rank; s2 < k; s2 += c.ncl)
    for (int t = s2 + threadIdx.x; t < k; t += blockDim.x)
      J.R11[(int64_t)s2 * k + t] = J.Rf[(int64_t)s2 * m + perm[t]];
  cl_sync();
  // U (row-major, ld = k): identity rows at the pivots, X = R11^{-1} R12 elsewhere
  for (int i = wid; i < mr; i += nw) {
    double* x = J.U + (int64_t)(c.r0 + i) * k;
    if (used[i]) {
      for (int s2 = lane; s2 < k; s2 += 32) x[s2] = 0.0;
      continue;
    }
    for (int s2 = k - 1; s2 >= 0; --s2) {
      const double* rr = J.R11 + (int64_t)s2 * k;
      double acc = 0.0;
      for (int t = s2 + 1 + lane; t < k; t += 32) acc = fma(rr[t], x[t], acc);
      acc = warp_sum(acc);
      if (lane == 0) x[s2] = (J.Rf[(int64_t)s2 * m + c.r0 + i] - acc) / rr[s2];
      __syncwarp();
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < k; t += blockDim.x) {
    const int p = perm[t];
    if (p >= c.r0 && p < c.r1) J.U[(int64_t)p * k + t] = 1.0;
    if (c.rank == 0) {
      J.Jl[t] = p;
      J.It[t] = J.It1 ? (p < J.k1 ? J.It1[p] : J.It2[p - J.k1]) : (int32_t)(J.lo + p);
    }
  }
  if (threadIdx.x == 0 && c.rank == 0) ranks[node] = k;
  cl_sync();  // no CTA leaves while its candidates may still be read
}


}  // namespace
}  // namespace jls

using namespace jls;

namespace {

enum { UNTOUCHED = 0, PARTIAL = 1, COMPRESSED = 2 };
// kinds of work timed separately (hss_profile)
enum { CAT_GATHER = 0, CAT_LOCAL = 1, CAT_TEST = 2, CAT_ID = 3, CAT_RTAU = 4, CAT_SKETCH = 5, HSS_CATS = 6 };

struct HssNode {
  int64_t lo = 0, hi = 0;
  int level = 0, parent = -1, c1 = -1, c2 = -1;
  int state = UNTOUCHED;
  int m = 0, q = -1, k = 0, qcap = 0;
  double om11 = 0.0;
  double *S = nullptr, *Q = nullptr, *U = nullptr, *R = nullptr, *B = nullptr, *D = nullptr;
  int32_t *J = nullptr, *It = nullptr;
};

struct HssRecord {
  int32_t sweep, level, node, outcome;
  double nh, nt, mind;
};

// Device memory in chunks with a bump pointer (256-byte aligned pieces).
struct Arena {
  std::vector<void*> chunks;
  char* cur = nullptr;
  size_t left = 0;
  int take(size_t bytes, void** out) {
    bytes = (bytes + 255) / 256 * 256;
    if (bytes == 0) bytes = 256;
    if (bytes > left) {
      const size_t sz = std::max(bytes, (size_t)256 << 20);
      void* p = nullptr;
      if (cudaMalloc(&p, sz) != cudaSuccess) {
        cudaGetLastError();
        return SK_ERR_NOMEM;
      }
      chunks.push_back(p);
      cur = static_cast<char*>(p);
      left = sz;
    }
    *out = cur;
    cur += bytes;
    left -= bytes;
    return SK_OK;
  }
  void release() {
    for (void* p : chunks) cudaFree(p);
    chunks.clear();
    cur = nullptr;
    left = 0;
  }
};

template <class T>
int take(Arena& a, size_t count, T** out) {
  void* p = nullptr;
  JLS_CHECK(a.take(count * sizeof(T), &p));
  *out = static_cast<T*>(p);
  return SK_OK;
}

}  // namespace

struct sk_hss {
  int64_t n = 0, lda = 0;
  const double* A = nullptr;
  int leaf = 0, kind = 0, alpha = 1, d0 = 0, dd = 0, d_max = 0;
  double eps_rel = 0, eps_abs = 0;
  sk_handle op = nullptr;
  std::vector<HssNode> nodes;                 // preorder; node 0 is the root
  std::vector<std::vector<int>> levels;
  std::vector<HssRecord> history;
  int d = 0, sweeps = 0, converged = 0;
  Arena arena;       // per-node generators
  Arena scratch;     // per-level decomposition scratch, released after each level
  double* S = nullptr;   // n x d_max, row-major
  double* Rd = nullptr;  // n x d_total, row-major (exported after each increment)
  void* jobs_dev = nullptr;
  size_t jobs_cap = 0;
  void* host_pin = nullptr;
  size_t host_cap = 0;
  int64_t launches = 0;
  int max_ncl_test = 8, max_ncl_id = 8;
  size_t test_smem16 = 0, id_smem16 = 0;  // shared memory a 16-CTA cluster of each kernel may take
  // device time per kind of work, from events around every launch
  struct Span { cudaEvent_t a, b; int cat; int sms; };
  std::vector<Span> spans;
  std::vector<cudaEvent_t> events;  // free events
  double ms[HSS_CATS] = {}, flops[HSS_CATS] = {};
  double sm_ms[HSS_CATS] = {};  // SMs a launch's grid occupies (at most one CTA each) times its ms
  int64_t cat_launches[HSS_CATS] = {};
};

namespace {

int ensure_jobs(sk_hss* H, size_t bytes) {
  if (bytes <= H->jobs_cap) return SK_OK;
  if (H->jobs_dev) cudaFree(H->jobs_dev);
  H->jobs_dev = nullptr;
  H->jobs_cap = 0;
  const size_t cap = std::max(bytes, (size_t)1 << 16);
  JLS_CHECK_CUDA(cudaMalloc(&H->jobs_dev, cap));
  H->jobs_cap = cap;
  return SK_OK;
}

int ensure_pinned(sk_hss* H, size_t bytes) {
  if (bytes <= H->host_cap) return SK_OK;
  if (H->host_pin) cudaFreeHost(H->host_pin);
  H->host_pin = nullptr;
  H->host_cap = 0;
  const size_t cap = std::max(bytes, (size_t)1 << 16);
  JLS_CHECK_CUDA(cudaMallocHost(&H->host_pin, cap));
  H->host_cap = cap;
  return SK_OK;
}

cudaEvent_t take_event(sk_hss* H) {
  if (!H->events.empty()) {
    cudaEvent_t e = H->events.back();
    H->events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

// Bracket work on s with events; span_end adds the algorithmic FLOPs.
int span_begin(sk_hss* H, cudaStream_t s) {
  sk_hss::Span sp{take_event(H), take_event(H), -1, 0};
  if (sp.a) cudaEventRecord(sp.a, s);
  H->spans.push_back(sp);
  return (int)H->spans.size() - 1;
}

void span_end(sk_hss* H, cudaStream_t s, int span, int cat, double flops, int launches, int64_t ctas = 0) {
  sk_hss::Span& sp = H->spans[span];
  if (sp.b) cudaEventRecord(sp.b, s);
  sp.cat = cat;
  sp.sms = (int)std::min<int64_t>(ctas > 0 ? ctas : num_sms(), num_sms());
  H->flops[cat] += flops;
  H->cat_launches[cat] += launches;
}

// After a synchronization of the stream: add up the finished spans.
void spans_collect(sk_hss* H) {
  for (sk_hss::Span& sp : H->spans) {
    float t = 0.f;
    if (sp.a && sp.b && sp.cat >= 0 && cudaEventElapsedTime(&t, sp.a, sp.b) == cudaSuccess) {
      H->ms[sp.cat] += t;
      H->sm_ms[sp.cat] += (double)sp.sms * t;
    }
    cudaGetLastError();
    if (sp.a) H->events.push_back(sp.a);
    if (sp.b) H->events.push_back(sp.b);
  }
  H->spans.clear();
}

// Copy a job array to the device (through pinned memory; the stream is
// synchronized before the pinned buffer is reused).
template <class T>
int upload(sk_hss* H, const std::vector<T>& v, cudaStream_t s) {
  const size_t bytes = v.size() * sizeof(T);
  JLS_CHECK(ensure_jobs(H, bytes));
  JLS_CHECK_CUDA(cudaStreamSynchronize(s));
  JLS_CHECK(ensure_pinned(H, bytes));
  std::memcpy(H->host_pin, v.data(), bytes);
  JLS_CHECK_CUDA(cudaMemcpyAsync(H->jobs_dev, H->host_pin, bytes, cudaMemcpyHostToDevice, s));
  return SK_OK;
}

int run_gemms(sk_hss* H, std::vector<GemmJob>& jobs, cudaStream_t s, int cat) {
  std::vector<GemmJob> live;
  int tiles = 0;
  double flops = 0.0;
  for (GemmJob j : jobs) {
    flops += 2.0 * j.M * j.N * j.K;
    if (j.M <= 0 || j.N <= 0) continue;
    j.tiles_n = (j.N + GT - 1) / GT;
    j.tile0 = tiles;
    tiles += ((j.M + GT - 1) / GT) * j.tiles_n;
    live.push_back(j);
  }
  if (live.empty()) return SK_OK;
  JLS_CHECK(upload(H, live, s));
  const int sp = span_begin(H, s);
  hss_gemm_kernel<<<tiles, 256, 0, s>>>(static_cast<const GemmJob*>(H->jobs_dev), (int)live.size());
  span_end(H, s, sp, cat, flops, 1, tiles);
  note_launch();
  ++H->launches;
  JLS_CHECK_CUDA(cudaGetLastError());
  return SK_OK;
}

int run_gathers(sk_hss* H, std::vector<GatherJob>& jobs, cudaStream_t s) {
  std::vector<GatherJob> live;
  for (const GatherJob& j : jobs)
    if (j.rows > 0 && j.cols > 0) live.push_back(j);
  if (live.empty()) return SK_OK;
  JLS_CHECK(upload(H, live, s));
  const int sp = span_begin(H, s);
  hss_gather_kernel<<<(unsigned)live.size(), 256, 0, s>>>(static_cast<const GatherJob*>(H->jobs_dev), H->A, H->lda);
  span_end(H, s, sp, CAT_GATHER, 0.0, 1, (int64_t)live.size());
  note_launch();
  ++H->launches;
  JLS_CHECK_CUDA(cudaGetLastError());
  return SK_OK;
}

// Cluster size for a launch over `nodes` nodes of up to mmax rows: the
// largest power of two that keeps nodes x ncl within the SMs and min_rows rows
// per CTA, at most max_ncl.
int pick_ncl(int max_ncl, int nodes, int mmax, int min_rows) {
  const int sms = num_sms();
  int ncl = 1;
  while (ncl < max_ncl && nodes * ncl * 2 <= sms && mmax >= min_rows * ncl * 2) ncl *= 2;
  return ncl;
}

template <typename... KArgs, typename... Args>
int launch_cl(void (*kern)(KArgs...), unsigned nodes, int ncl, size_t smem, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nodes * (unsigned)ncl);
  cfg.blockDim = dim3(HT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)ncl;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  JLS_CHECK_CUDA(cudaLaunchKernelEx(&cfg, kern, args...));
  note_launch();
  return SK_OK;
}

// Opt in to the shared memory and cluster sizes of the per-node kernels:
// clusters of 16 where the device can place one (with the kernel's shared
// memory, or with smaller row caches), else 8.
bool cluster16_fits(const void* kern, size_t smem) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(16);
  cfg.blockDim = dim3(HT);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 16;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  const bool ok = cudaOccupancyMaxActiveClusters(&n, kern, &cfg) == cudaSuccess && n > 0;
  cudaGetLastError();
  return ok;
}

int kernel_setup(sk_hss* H) {
  JLS_CHECK_CUDA(cudaFuncSetAttribute(hss_test_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TEST_SMEM_MAX));
  JLS_CHECK_CUDA(cudaFuncSetAttribute(hss_id_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ID_SMEM_MAX));
  JLS_CHECK_CUDA(cudaFuncSetAttribute(hss_test_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  JLS_CHECK_CUDA(cudaFuncSetAttribute(hss_id_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  // the largest shared memory (of 220 / 200, 118, 64 KB) at which a 16-CTA
  // cluster of each kernel fits, else clusters of 8
  const size_t tries_test[3] = {TEST_SMEM_MAX, 118 * 1024, 64 * 1024};
  const size_t tries_id[3] = {ID_SMEM_MAX, 118 * 1024, 64 * 1024};
  H->max_ncl_test = H->max_ncl_id = 8;
  H->test_smem16 = H->id_smem16 = 0;
  for (size_t b : tries_test)
    if (H->test_smem16 == 0 && cluster16_fits((const void*)hss_test_kernel, b)) {
      H->max_ncl_test = 16;
      H->test_smem16 = b;
    }
  for (size_t b : tries_id)
    if (H->id_smem16 == 0 && cluster16_fits((const void*)hss_id_kernel, b)) {
      H->max_ncl_id = 16;
      H->id_smem16 = b;
    }
  return SK_OK;
}

void build_tree(sk_hss* H) {
  H->nodes.clear();
  std::vector<int> stack;
  HssNode root;
  root.lo = 0;
  root.hi = H->n;
  H->nodes.push_back(root);
  stack.push_back(0);
  // preorder numbering: children are appended as they are split
  std::vector<int> order;
  while (!stack.empty()) {
    const int i = stack.back();
    stack.pop_back();
    const int64_t lo = H->nodes[i].lo, hi = H->nodes[i].hi;
    if (hi - lo <= H->leaf) continue;
    const int64_t mid = lo + (hi - lo) / 2;
    HssNode a, b;
    a.lo = lo; a.hi = mid; a.level = H->nodes[i].level + 1; a.parent = i;
    b.lo = mid; b.hi = hi; b.level = a.level; b.parent = i;
    const int ia = (int)H->nodes.size();
    H->nodes.push_back(a);
    H->nodes.push_back(b);
    H->nodes[i].c1 = ia;
    H->nodes[i].c2 = ia + 1;
    stack.push_back(ia + 1);
    stack.push_back(ia);
  }
  int depth = 0;
  for (const HssNode& nd : H->nodes) depth = std::max(depth, nd.level);
  H->levels.assign(depth + 1, {});
  // left to right inside a level: sort each level's nodes by lo
  for (int i = 0; i < (int)H->nodes.size(); ++i) H->levels[H->nodes[i].level].push_back(i);
  for (auto& L : H->levels)
    std::sort(L.begin(), L.end(), [&](int x, int y) { return H->nodes[x].lo < H->nodes[y].lo; });
}

// One sweep over the levels (leaves first); returns through *grow whether a
// node needs more columns.
int sweep(sk_hss* H, cudaStream_t s, bool* grow) {
  *grow = false;
  const int d = H->d, dd = H->dd, dcap = H->d_max;
  const int64_t ldS = H->d_max, ldR = H->op->d_total;
  for (int L = (int)H->levels.size() - 1; L >= 1; --L) {
    const std::vector<int>& lv = H->levels[L];
    // first visits: sizes, storage, D_tau / B_tau
    std::vector<GatherJob> gathers;
    for (int i : lv) {
      HssNode& nd = H->nodes[i];
      if (nd.state != UNTOUCHED) continue;
      const bool leaf = nd.c1 < 0;
      nd.m = leaf ? (int)(nd.hi - nd.lo) : H->nodes[nd.c1].k + H->nodes[nd.c2].k;
      if (nd.m > HSS_MAX_ROWS) return SK_ERR_UNSUPPORTED;
      nd.qcap = std::min(nd.m, dcap) + dd;
      JLS_CHECK(take(H->arena, (size_t)nd.m * dcap, &nd.S));
      JLS_CHECK(take(H->arena, (size_t)nd.m * nd.qcap, &nd.Q));
      GatherJob g;
      if (leaf) {
        JLS_CHECK(take(H->arena, (size_t)nd.m * nd.m, &nd.D));
        g.out = nd.D; g.rows = nd.m; g.cols = nd.m; g.r0 = nd.lo; g.c0 = nd.lo;
      } else {
        const HssNode& a = H->nodes[nd.c1];
        const HssNode& b = H->nodes[nd.c2];
        JLS_CHECK(take(H->arena, (size_t)std::max(1, a.k * b.k), &nd.B));
        g.out = nd.B; g.rows = a.k; g.cols = b.k; g.ri = a.It; g.ci = b.It;
      }
      gathers.push_back(g);
    }
    JLS_CHECK(run_gathers(H, gathers, s));
    // local sketches of the level
    std::vector<GemmJob> gj;
    for (int i : lv) {
      HssNode& nd = H->nodes[i];
      const int c0 = nd.state == UNTOUCHED ? 0 : d;
      const int nc = d + dd - c0;
      if (nd.c1 < 0) {
        GemmJob j;
        j.out = nd.S + (int64_t)c0 * nd.m; j.ors = 1; j.ocs = nd.m;
        j.c.p = H->S + nd.lo * ldS + c0; j.c.rs = ldS; j.c.cs = 1; j.has_c = 1;
        j.a.p = nd.D; j.a.rs = 1; j.a.cs = nd.m;
        j.b.p = H->Rd + nd.lo * ldR + c0; j.b.rs = ldR; j.b.cs = 1;
        j.M = nd.m; j.N = nc; j.K = nd.m; j.alpha = -1.0;
        gj.push_back(j);
      } else {
        const HssNode& a = H->nodes[nd.c1];
        const HssNode& b = H->nodes[nd.c2];
        GemmJob top;  // S_nu1(J_nu1, iota) - B R_nu2(:, iota)
        top.out = nd.S + (int64_t)c0 * nd.m; top.ors = 1; top.ocs = nd.m;
        top.c.p = a.S + (int64_t)c0 * a.m; top.c.rs = 1; top.c.cs = a.m; top.c.idx = a.J; top.has_c = 1;
        top.a.p = nd.B; top.a.rs = 1; top.a.cs = std::max(1, a.k);
        top.b.p = b.R + (int64_t)c0 * b.k; top.b.rs = 1; top.b.cs = b.k;
        top.M = a.k; top.N = nc; top.K = b.k; top.alpha = -1.0;
        GemmJob bot;  // S_nu2(J_nu2, iota) - B^T R_nu1(:, iota)
        bot.out = nd.S + (int64_t)c0 * nd.m + a.k; bot.ors = 1; bot.ocs = nd.m;
        bot.c.p = b.S + (int64_t)c0 * b.m; bot.c.rs = 1; bot.c.cs = b.m; bot.c.idx = b.J; bot.has_c = 1;
        bot.a.p = nd.B; bot.a.rs = std::max(1, a.k); bot.a.cs = 1;
        bot.b.p = a.R + (int64_t)c0 * a.k; bot.b.rs = 1; bot.b.cs = a.k;
        bot.M = b.k; bot.N = nc; bot.K = a.k; bot.alpha = -1.0;
        if (b.k == 0) { top.K = 0; }
        if (a.k == 0) { bot.K = 0; }
        gj.push_back(top);
        gj.push_back(bot);
      }
    }
    JLS_CHECK(run_gemms(H, gj, s, CAT_LOCAL));
    // stopping and rank-deficiency tests of the nodes not yet compressed
    std::vector<int> tested;
    std::vector<TestJob> tj;
    for (int i : lv) {
      HssNode& nd = H->nodes[i];
      if (nd.state == COMPRESSED) continue;
      TestJob t;
      t.S = nd.S; t.Q = nd.Q; t.m = nd.m; t.d = d; t.dd = dd;
      t.q = nd.state == UNTOUCHED ? -1 : nd.q;
      t.qcap = nd.qcap;
      t.er = H->eps_rel / nd.level; t.ea = H->eps_abs / nd.level;
      t.om11 = nd.om11;
      tj.push_back(t);
      tested.push_back(i);
    }
    std::vector<int> compress;
    if (!tj.empty()) {
      JLS_CHECK(upload(H, tj, s));
      TestOut* outs = nullptr;
      JLS_CHECK(take(H->scratch, tj.size(), &outs));
      const int sp = span_begin(H, s);
      int mmax = 0, qx = 0;
      for (const TestJob& t : tj) {
        mmax = std::max(mmax, t.m);
        qx = std::max(qx, (t.q < 0 ? std::min(t.m, d) : t.q) + dd);
      }
      const int ncl = pick_ncl(H->max_ncl_test, (int)tj.size(), mmax, 32);
      const int mrx = (mmax + ncl - 1) / ncl;
      TestLayout lay{mrx, qx, 1, std::max(1, std::min(GMAX, 4096 / std::max(1, mrx)))};
      if (test_smem_bytes(lay) > (ncl == 16 ? H->test_smem16 : TEST_SMEM_MAX)) lay.qsm = 0;
      JLS_CHECK(launch_cl(hss_test_kernel, (unsigned)tj.size(), ncl, test_smem_bytes(lay), s,
                          static_cast<const TestJob*>(H->jobs_dev), outs, lay));
      const int64_t test_ctas = (int64_t)tj.size() * ncl;
      ++H->launches;
      JLS_CHECK_CUDA(cudaGetLastError());
      std::vector<TestOut> ho(tj.size());
      JLS_CHECK_CUDA(cudaMemcpyAsync(ho.data(), outs, sizeof(TestOut) * ho.size(), cudaMemcpyDeviceToHost, s));
      JLS_CHECK_CUDA(cudaStreamSynchronize(s));
      // algorithmic FLOPs: a projection pass of one m-vector against q
      // columns is 4 m q (dots and update), two passes per vector
      double tf = 0.0;
      for (size_t u = 0; u < tested.size(); ++u) {
        const TestJob& t = tj[u];
        const double m = t.m;
        const double q0 = t.q < 0 ? std::min(ho[u].q - (ho[u].outcome == 2 ? dd : 0), d) : t.q;
        if (t.q < 0)
          for (int j = 0; j < d; ++j) tf += 8.0 * m * std::min<double>(j, q0) + 2.0 * m;
        tf += dd * (8.0 * m * q0 + 4.0 * m);
        if (ho[u].mind != 0.0 || ho[u].outcome != 0) tf += 8.0 * m * dd * (dd - 1) / 2.0 + 3.0 * m * dd;
      }
      span_end(H, s, sp, CAT_TEST, tf, 1, test_ctas);
      for (size_t u = 0; u < tested.size(); ++u) {
        HssNode& nd = H->nodes[tested[u]];
        const TestOut& o = ho[u];
        nd.q = o.q;
        nd.om11 = o.om11;
        H->history.push_back(HssRecord{H->sweeps, L, tested[u], o.outcome, o.nh, o.nt, o.mind});
        if (o.outcome == 2) {
          nd.state = PARTIAL;
          *grow = true;
        } else {
          compress.push_back(tested[u]);
        }
      }
    }
    // interpolative decompositions of the nodes that compress now
    if (!compress.empty()) {
      std::vector<IdJob> ij;
      const int C = d + dd;
      for (int i : compress) {
        HssNode& nd = H->nodes[i];
        const int kmax = std::min(nd.m, C);
        IdJob j;
        j.S = nd.S; j.m = nd.m; j.C = C;
        j.er = H->eps_rel / nd.level; j.ea = H->eps_abs / nd.level;
        JLS_CHECK(take(H->scratch, (size_t)nd.m * C, &j.W));
        JLS_CHECK(take(H->scratch, (size_t)kmax * nd.m, &j.Rf));
        JLS_CHECK(take(H->scratch, (size_t)std::max(1, kmax * kmax), &j.R11));
        JLS_CHECK(take(H->arena, (size_t)nd.m * kmax, &nd.U));
        JLS_CHECK(take(H->arena, (size_t)kmax, &nd.J));
        JLS_CHECK(take(H->arena, (size_t)kmax, &nd.It));
        j.U = nd.U; j.Jl = nd.J; j.It = nd.It; j.lo = nd.lo;
        if (nd.c1 >= 0) {
          j.It1 = H->nodes[nd.c1].It; j.It2 = H->nodes[nd.c2].It; j.k1 = H->nodes[nd.c1].k;
        }
        ij.push_back(j);
      }
      JLS_CHECK(upload(H, ij, s));
      int32_t* ranks = nullptr;
      JLS_CHECK(take(H->scratch, ij.size(), &ranks));
      const int sp = span_begin(H, s);
      int mmax = 0;
      for (const IdJob& t : ij) mmax = std::max(mmax, t.m);
      // a decomposition's arithmetic does not depend on how its rows are split
      // (each row's dots and updates stay in one warp), so it takes clusters
      // down to 16 rows per CTA, one row per warp
      const int ncl = pick_ncl(H->max_ncl_id, (int)ij.size(), mmax, 16);
      IdLayout lay{C, (mmax + ncl - 1) / ncl, std::min(mmax, C), 1};
      if (id_smem_bytes(lay) > (ncl == 16 ? H->id_smem16 : ID_SMEM_MAX)) lay.wsm = 0;
      JLS_CHECK(launch_cl(hss_id_kernel, (unsigned)ij.size(), ncl, id_smem_bytes(lay), s,
                          static_cast<const IdJob*>(H->jobs_dev), ranks, lay));
      const int64_t id_ctas = (int64_t)ij.size() * ncl;
      ++H->launches;
      JLS_CHECK_CUDA(cudaGetLastError());
      std::vector<int32_t> hk(ij.size());
      JLS_CHECK_CUDA(cudaMemcpyAsync(hk.data(), ranks, sizeof(int32_t) * hk.size(), cudaMemcpyDeviceToHost, s));
      JLS_CHECK_CUDA(cudaStreamSynchronize(s));
      // algorithmic FLOPs: the row norms (2 m C), per pivot step a dot and an
      // update over the remaining rows (4 (m - t) C), then the triangular
      // solves (m - k) k^2
      double idf = 0.0;
      for (size_t u = 0; u < compress.size(); ++u) {
        const double m = ij[u].m, k = hk[u];
        idf += 2.0 * m * C + 4.0 * C * (m * k - k * (k - 1) / 2.0) + (m - k) * k * k;
      }
      span_end(H, s, sp, CAT_ID, idf, 1, id_ctas);
      for (size_t u = 0; u < compress.size(); ++u) {
        HssNode& nd = H->nodes[compress[u]];
        nd.k = hk[u];
        JLS_CHECK(take(H->arena, (size_t)std::max(1, nd.k) * dcap, &nd.R));
      }
    }
    // R_tau over the columns it lacks: all of them for the nodes that just
    // compressed, the new Delta-d for the earlier ones
    std::vector<GemmJob> rj;
    for (int i : lv) {
      HssNode& nd = H->nodes[i];
      const bool now = std::find(compress.begin(), compress.end(), i) != compress.end();
      if (!now && nd.state != COMPRESSED) continue;
      const int c0 = now ? 0 : d;
      GemmJob j;
      j.out = nd.R + (int64_t)c0 * nd.k; j.ors = 1; j.ocs = nd.k;
      j.a.p = nd.U; j.a.rs = 1; j.a.cs = nd.k;  // U^T, U row-major
      if (nd.c1 < 0) {
        j.b.p = H->Rd + nd.lo * ldR + c0; j.b.rs = ldR; j.b.cs = 1;
      } else {
        const HssNode& a = H->nodes[nd.c1];
        const HssNode& b = H->nodes[nd.c2];
        j.b.p = a.R + (int64_t)c0 * a.k; j.b.rs = 1; j.b.cs = a.k; j.b.split = a.k;
        j.b.p2 = b.R + (int64_t)c0 * b.k; j.b.rs2 = 1; j.b.cs2 = b.k;
      }
      j.M = nd.k; j.N = d + dd - c0; j.K = nd.m; j.alpha = 1.0;
      rj.push_back(j);
    }
    JLS_CHECK(run_gemms(H, rj, s, CAT_RTAU));
    for (int i : compress) H->nodes[i].state = COMPRESSED;
    JLS_CHECK_CUDA(cudaStreamSynchronize(s));
    spans_collect(H);
    H->scratch.release();
    if (*grow) return SK_OK;
  }
  return SK_OK;
}

}  // namespace

extern "C" {

int hss_compress_adaptive(sk_hss_handle* out, const double* A, int64_t n, int64_t lda, int32_t leaf, int32_t kind,
                          int32_t d0, int32_t dd, int32_t alpha, uint64_t seed, int32_t d_max, double eps_rel,
                          double eps_abs, void* stream) {
  if (!out) return SK_ERR_INVALID_ARG;
  *out = nullptr;
  if (!A || n < 1 || n >= (1ll << 31) || lda < n || leaf < 1 || leaf > HSS_MAX_ROWS) return SK_ERR_INVALID_ARG;
  if (d0 < 1 || dd < 1 || d_max < d0 + dd || d_max > HSS_MAX_D || d_max % 2) return SK_ERR_INVALID_ARG;
  if (!(eps_rel >= 0.0) || !(eps_abs >= 0.0)) return SK_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(A) & 15u) || (lda * 8) % 16) return SK_ERR_ALIGN;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  sk_hss* H = new (std::nothrow) sk_hss();
  if (!H) return SK_ERR_NOMEM;
  H->n = n; H->lda = lda; H->A = A; H->leaf = leaf; H->kind = kind; H->alpha = alpha;
  H->d0 = d0; H->dd = dd; H->d_max = d_max; H->eps_rel = eps_rel; H->eps_abs = eps_abs;
  int rc = sketch_create_flags(&H->op, kind, n, d0 + dd, alpha, seed, d_max, SK_SCALE_BLOCK, stream);
  sk_matrix Am;
  std::memset(&Am, 0, sizeof(Am));
  Am.dtype = SK_F64; Am.rows = n; Am.cols = n; Am.A = A; Am.ld = lda;
  if (rc == SK_OK) rc = kernel_setup(H);
  if (rc == SK_OK) rc = cuda_status(cudaMalloc(&H->S, sizeof(double) * n * d_max));
  if (rc == SK_OK) rc = cuda_status(cudaMalloc(&H->Rd, sizeof(double) * n * d_max));
  if (rc == SK_OK) {
    const int sp = span_begin(H, s);
    const long long l0 = sketch_launch_count();
    rc = sketch_apply(H->op, &Am, SK_S, SK_PREC_NATIVE, H->S, d_max, nullptr, 0, stream);
    if (rc == SK_OK) rc = export_dense_R(H->op, H->Rd, SK_F64, s);
    span_end(H, s, sp, CAT_SKETCH, 2.0 * n * n * (d0 + dd), (int)(sketch_launch_count() - l0));
  }
  if (rc == SK_OK) {
    build_tree(H);
    H->d = d0;
  }
  while (rc == SK_OK) {
    if (H->levels.size() <= 1) {  // the root is a leaf: D = A
      H->converged = 1;
      HssNode& r = H->nodes[0];
      rc = take(H->arena, (size_t)n * n, &r.D);
      std::vector<GatherJob> g(1);
      g[0].out = r.D; g[0].rows = (int)n; g[0].cols = (int)n;
      if (rc == SK_OK) rc = run_gathers(H, g, s);
      r.state = COMPRESSED;
      r.m = (int)n;
      break;
    }
    bool grow = false;
    rc = sweep(H, s, &grow);
    if (rc != SK_OK) break;
    if (!grow) {
      HssNode& r = H->nodes[0];
      const HssNode& a = H->nodes[r.c1];
      const HssNode& b = H->nodes[r.c2];
      rc = take(H->arena, (size_t)std::max(1, a.k * b.k), &r.B);
      std::vector<GatherJob> g(1);
      g[0].out = r.B; g[0].rows = a.k; g[0].cols = b.k; g[0].ri = a.It; g[0].ci = b.It;
      if (rc == SK_OK) rc = run_gathers(H, g, s);
      r.state = COMPRESSED;
      H->converged = 1;
      ++H->sweeps;
      break;
    }
    ++H->sweeps;
    if (H->op->d_total + dd > d_max) break;
    const int sp = span_begin(H, s);
    const long long l0 = sketch_launch_count();
    rc = sketch_increment(H->op, dd, stream);
    if (rc == SK_OK) rc = sketch_apply_increment(H->op, &Am, SK_S, SK_PREC_NATIVE, H->S, d_max, nullptr, 0, stream);
    if (rc == SK_OK) rc = export_dense_R(H->op, H->Rd, SK_F64, s);
    span_end(H, s, sp, CAT_SKETCH, 2.0 * n * n * dd, (int)(sketch_launch_count() - l0));
    H->d += dd;
  }
  if (rc == SK_OK) rc = cuda_status(cudaStreamSynchronize(s));
  if (rc == SK_OK) spans_collect(H);
  if (rc == SK_OK) rc = sketch_device_status(H->op, stream);
  if (rc != SK_OK) {
    hss_destroy(H);
    return rc;
  }
  *out = H;
  return SK_OK;
}

int hss_info(sk_hss_handle h, int32_t* nodes, int32_t* d, int32_t* d_total, int32_t* sweeps, int32_t* converged,
             int32_t* tests) {
  if (!h) return SK_ERR_INVALID_ARG;
  if (nodes) *nodes = (int32_t)h->nodes.size();
  if (d) *d = h->d;
  if (d_total) *d_total = h->op ? h->op->d_total : 0;
  if (sweeps) *sweeps = h->sweeps;
  if (converged) *converged = h->converged;
  if (tests) *tests = (int32_t)h->history.size();
  return SK_OK;
}

int hss_node(sk_hss_handle h, int32_t node, int64_t* lohi, int32_t* info) {
  if (!h || node < 0 || node >= (int32_t)h->nodes.size()) return SK_ERR_INVALID_ARG;
  const HssNode& nd = h->nodes[node];
  if (lohi) { lohi[0] = nd.lo; lohi[1] = nd.hi; }
  if (info) {
    info[0] = nd.level; info[1] = nd.parent; info[2] = nd.c1; info[3] = nd.c2;
    info[4] = nd.state; info[5] = nd.m; info[6] = nd.k;
  }
  return SK_OK;
}

int hss_node_get(sk_hss_handle h, int32_t node, int32_t what, void* dst) {
  if (!h || !dst || node < 0 || node >= (int32_t)h->nodes.size()) return SK_ERR_INVALID_ARG;
  const HssNode& nd = h->nodes[node];
  const void* src = nullptr;
  size_t bytes = 0;
  switch (what) {
    case SK_HSS_U: src = nd.U; bytes = sizeof(double) * nd.m * nd.k; break;  // row-major
    case SK_HSS_J: src = nd.J; bytes = sizeof(int32_t) * nd.k; break;
    case SK_HSS_IT: src = nd.It; bytes = sizeof(int32_t) * nd.k; break;
    case SK_HSS_D: src = nd.D; bytes = sizeof(double) * nd.m * nd.m; break;
    case SK_HSS_B: {
      if (nd.c1 < 0) return SK_ERR_INVALID_ARG;
      src = nd.B;
      bytes = sizeof(double) * h->nodes[nd.c1].k * h->nodes[nd.c2].k;
      break;
    }
    case SK_HSS_S: src = nd.S; bytes = sizeof(double) * nd.m * (h->d + h->dd); break;
    case SK_HSS_R: src = nd.R; bytes = sizeof(double) * nd.k * (h->d + h->dd); break;
    default: return SK_ERR_INVALID_ARG;
  }
  if (bytes == 0) return SK_OK;
  if (!src) return SK_ERR_STATE;
  JLS_CHECK_CUDA(cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost));
  return SK_OK;
}

int hss_history(sk_hss_handle h, int32_t* ints, double* reals) {
  if (!h) return SK_ERR_INVALID_ARG;
  for (size_t u = 0; u < h->history.size(); ++u) {
    const HssRecord& r = h->history[u];
    if (ints) { ints[4 * u] = r.sweep; ints[4 * u + 1] = r.level; ints[4 * u + 2] = r.node; ints[4 * u + 3] = r.outcome; }
    if (reals) { reals[3 * u] = r.nh; reals[3 * u + 1] = r.nt; reals[3 * u + 2] = r.mind; }
  }
  return SK_OK;
}

int64_t hss_launch_count(sk_hss_handle h) { return h ? h->launches : 0; }

int hss_profile(sk_hss_handle h, double* ms, double* flops, int64_t* launches, double* sm_ms) {
  if (!h) return SK_ERR_INVALID_ARG;
  for (int c = 0; c < HSS_CATS; ++c) {
    if (sm_ms) sm_ms[c] = h->sm_ms[c];
    if (ms) ms[c] = h->ms[c];
    if (flops) flops[c] = h->flops[c];
    if (launches) launches[c] = h->cat_launches[c];
  }
  return SK_OK;
}

void hss_destroy(sk_hss_handle h) {
  if (!h) return;
  cudaDeviceSynchronize();
  if (h->op) sketch_destroy(h->op);
  h->arena.release();
  h->scratch.release();
  if (h->S) cudaFree(h->S);
  if (h->Rd) cudaFree(h->Rd);
  if (h->jobs_dev) cudaFree(h->jobs_dev);
  if (h->host_pin) cudaFreeHost(h->host_pin);
  spans_collect(h);
  for (cudaEvent_t e : h->events) cudaEventDestroy(e);
  delete h;
}

}  // extern "C"
