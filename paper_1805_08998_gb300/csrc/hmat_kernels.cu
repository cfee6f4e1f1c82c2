// hmat_kernels.cu -- device kernels of the H-matrix product (sm_103a).
//
// Kernels, in the order the product runs them (paper references are to Doelz, Harbrecht,
// Multerer, "On the best approximation of the hierarchical matrix product"):
//   k_kernel_dense  near leaves of an input matrix, evaluated entry by entry
//   k_aca           far leaves of an input matrix by adaptive cross approximation (Alg. 6)
//   k_term_jobs     the low-rank products A|tau' x rho' * B|rho' x sigma' that the restriction
//                   of Algorithm 3 creates when one factor is far (cost: Lemma 5.1)
//   k_near_eval     evaluate() of Algorithm 4 for near leaves: S(b) applied to the identity
//   k_gaussian      Gaussian test matrices Omega (counter-based, splitmix64 + Box-Muller)
//   k_apply         (hmat_apply.cu) S(b) Omega or S(b)^T Q for every far target b
//   k_orth          project the new samples against the basis twice and orthonormalise them by
//                   Gram-Schmidt twice with dropping, all in FP64 (the projection step of Alg. 8)
//   k_absorb_w      append W_new = S^T Q_new and apply the blocked stop test eq. (truncaca)
//   k_aca_*         the cross approximation compressor (Alg. 6) on the sum-expressions: start,
//                   row step (pivot column), column step (stop test, next pivot row), QR of L
//   k_lz_*          the Lanczos bidiagonalization compressor (Alg. 7): start vector, q step,
//                   w step (stop test), and the projection W = S^T Q in column blocks
//   k_final         core truncation: eigen-decomposition of W^T W (Jacobi, FP64), eps-rank,
//                   U = Q V_k, V = W V_k (the small SVD of Algorithm 5 on the sampled core)
//   k_write_far     copy the truncated factors into the output H-matrix
//
// Block size is 256 threads everywhere; every block-level helper must be reached by all
// threads of the block (they contain __syncthreads()).
#include <cstdint>
#include <cuda_runtime.h>

#include "hmat_internal.h"

namespace hm {

constexpr int NT = 256;     // threads per block
constexpr int ACA_KMAX = 128;  // largest rank of the input ACA (hmat_build rejects larger aca_kmax)
constexpr int KC = 32;      // rows staged per chunk in the SIMT contractions
constexpr int PMAX = 32;    // max right-hand-side columns per contraction call
constexpr int RMAX = 128;   // max rank / leaf size handled by one contraction call

// ---------------------------------------------------------------------------------------
// small block-level SIMT contractions
// ---------------------------------------------------------------------------------------

// Out[i + c*ldo] += sum_k M[i + k*ldm] * X[k + c*ldx] for i < mr, c < p, k < kc.
// X is staged through xs[KC * PMAX]. All threads of the block must call.
template <typename T>
__device__ void gemm_nn_acc(T *Out, int64_t ldo, const T *M, int64_t ldm, const T *X, int64_t ldx,
                            int mr, int kc, int p, T *xs) {
  constexpr int OPT = 2;
  const int tid = threadIdx.x;
  const int p4 = (p + 3) >> 2;
  const int nout = mr * p4;
  for (int ob = 0; ob < nout; ob += NT * OPT) {
    T acc[OPT][4];
#pragma unroll
    for (int j = 0; j < OPT; j++)
#pragma unroll
      for (int q = 0; q < 4; q++) acc[j][q] = T(0);
    for (int k0 = 0; k0 < kc; k0 += KC) {
      const int kk = min(KC, kc - k0);
      __syncthreads();
      for (int e = tid; e < kk * p; e += NT) {
        const int k = e % kk, c = e / kk;
        xs[k * PMAX + c] = X[(k0 + k) + (int64_t)c * ldx];
      }
      __syncthreads();
#pragma unroll
      for (int j = 0; j < OPT; j++) {
        const int o = ob + tid + j * NT;
        if (o < nout) {
          const int i = o % mr, cg = o / mr;
          const T *mp = M + i + (int64_t)k0 * ldm;
          const T *xp = xs + 4 * cg;
          for (int k = 0; k < kk; k++) {
            const T a = mp[(int64_t)k * ldm];
#pragma unroll
            for (int q = 0; q < 4; q++) acc[j][q] += a * xp[k * PMAX + q];
          }
        }
      }
    }
#pragma unroll
    for (int j = 0; j < OPT; j++) {
      const int o = ob + tid + j * NT;
      if (o < nout) {
        const int i = o % mr, cg = o / mr;
#pragma unroll
        for (int q = 0; q < 4; q++) {
          const int c = 4 * cg + q;
          if (c < p) Out[i + (int64_t)c * ldo] += acc[j][q];
        }
      }
    }
  }
  __syncthreads();
}

// Cs[q + c*r] = sum_k M[k + q*ldm] * X[k + c*ldx] for q < r (<= RMAX), c < p (<= PMAX),
// k < kc. Cs lives in shared memory (r*p entries). ms[KC*RMAX], xs[KC*PMAX] are staging.
template <typename T>
__device__ void gemm_tn(T *Cs, const T *M, int64_t ldm, const T *X, int64_t ldx, int kc, int r, int p,
                        T *ms, T *xs) {
  constexpr int OPT = (RMAX * PMAX + NT - 1) / NT;
  const int tid = threadIdx.x;
  const int nout = r * p;
  T acc[OPT];
#pragma unroll
  for (int j = 0; j < OPT; j++) acc[j] = T(0);
  for (int k0 = 0; k0 < kc; k0 += KC) {
    const int kk = min(KC, kc - k0);
    __syncthreads();
    for (int e = tid; e < kk * r; e += NT) {
      const int k = e % kk, q = e / kk;
      ms[k * RMAX + q] = M[(k0 + k) + (int64_t)q * ldm];
    }
    for (int e = tid; e < kk * p; e += NT) {
      const int k = e % kk, c = e / kk;
      xs[k * PMAX + c] = X[(k0 + k) + (int64_t)c * ldx];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < OPT; j++) {
      const int o = tid + j * NT;
      if (o < nout) {
        const int q = o % r, c = o / r;
        T s = T(0);
        for (int k = 0; k < kk; k++) s += ms[k * RMAX + q] * xs[k * PMAX + c];
        acc[j] += s;
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < OPT; j++) {
    const int o = tid + j * NT;
    if (o < nout) Cs[o] = acc[j];
  }
  __syncthreads();
}

// Out[q + c*ldo] += Cs[q + c*r]
template <typename T>
__device__ void add_small(T *Out, int64_t ldo, const T *Cs, int r, int p) {
  for (int o = threadIdx.x; o < r * p; o += NT) {
    const int q = o % r, c = o / r;
    Out[q + (int64_t)c * ldo] += Cs[o];
  }
  __syncthreads();
}

template <typename T>
__device__ void zero_mat(T *Out, int64_t ld, int rows, int cols) {
  for (int64_t o = threadIdx.x; o < (int64_t)rows * cols; o += NT) {
    const int64_t i = o % rows, c = o / rows;
    Out[i + c * ld] = T(0);
  }
  __syncthreads();
}

struct Smem {
  // carve-up of the dynamic shared memory used by the apply-type kernels
  template <typename T>
  __device__ static void get(T *base, T *&cs, T *&ms, T *&xs) {
    cs = base;
    ms = cs + RMAX * PMAX;
    xs = ms + KC * RMAX;
  }
  template <typename T>
  static constexpr size_t bytes() { return sizeof(T) * (RMAX * PMAX + KC * RMAX + KC * PMAX); }
};

// Apply the H-matrix block whose subtree holds leaves [lo, hi) (origin row0, col0) to X:
//   trans = false:  Out[rows of leaf] += leaf * X[cols of leaf]      (Algorithm 2)
//   trans = true:   Out[cols of leaf] += leaf^T * X[rows of leaf]
// X has p <= PMAX columns. Leaves are taken one at a time by the whole block.
template <typename T>
__device__ void hblock_apply(const LeafDev *leaves, const T *data, int lo, int hi, int64_t row0, int64_t col0,
                             bool trans, const T *X, int64_t ldx, int p, T *Out, int64_t ldo, T *cs, T *ms,
                             T *xs) {
  for (int l = lo; l < hi; l++) {
    const LeafDev lf = leaves[l];
    const int64_t ro = lf.row - row0, co = lf.col - col0;
    if (lf.rank < 0) {
      const T *D = data + lf.off_u;
      if (!trans) {
        gemm_nn_acc(Out + ro, ldo, D, lf.m, X + co, ldx, lf.m, lf.n, p, xs);
      } else {
        gemm_tn(cs, D, lf.m, X + ro, ldx, lf.m, lf.n, p, ms, xs);
        add_small(Out + co, ldo, cs, lf.n, p);
      }
    } else if (lf.rank > 0) {
      const T *U = data + lf.off_u, *V = data + lf.off_v;
      if (!trans) {
        gemm_tn(cs, V, lf.n, X + co, ldx, lf.n, lf.rank, p, ms, xs);
        gemm_nn_acc(Out + ro, ldo, U, lf.m, cs, lf.rank, lf.m, lf.rank, p, xs);
      } else {
        gemm_tn(cs, U, lf.m, X + ro, ldx, lf.m, lf.rank, p, ms, xs);
        gemm_nn_acc(Out + co, ldo, V, lf.n, cs, lf.rank, lf.n, lf.rank, p, xs);
      }
    }
  }
}

// ---------------------------------------------------------------------------------------
// input assembly: dense near leaves and ACA far leaves
// ---------------------------------------------------------------------------------------

__device__ __forceinline__ double kernel_eval(int kernel, const double *x, const double *y, int dim) {
  if (kernel == 2) {
    double ip = 0.0;
    for (int d = 0; d < dim; d++) ip += x[d] * y[d];
    return (1.0 + ip) * (1.0 + ip);
  }
  double r2 = 0.0;
  for (int d = 0; d < dim; d++) {
    const double e = x[d] - y[d];
    r2 += e * e;
  }
  if (kernel == 0) return exp(-sqrt(r2));
  return 1.0 / (1.0 + r2);
}

template <typename T>
__global__ void __launch_bounds__(NT) k_kernel_dense(int kernel, const double *pts, int dim,
                                                     const LeafDev *leaves, const int32_t *ids, T *data) {
  const LeafDev lf = leaves[ids[blockIdx.x]];
  T *D = data + lf.off_u;
  for (int64_t o = threadIdx.x; o < (int64_t)lf.m * lf.n; o += NT) {
    const int64_t i = o % lf.m, j = o / lf.m;
    D[o] = T(kernel_eval(kernel, pts + (lf.row + i) * dim, pts + (lf.col + j) * dim, dim));
  }
}

// warp-wide sum, the result in every lane
__device__ __forceinline__ double warp_sum(double v) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// block-wide reductions (NT threads)
__device__ double block_sum(double v, double *red) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    v = lane < NT / 32 ? red[lane] : 0.0;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) red[0] = v;
  }
  __syncthreads();
  const double r = red[0];
  __syncthreads();
  return r;
}

// argmax of |v| with the smallest index on ties; returns index (or -1 if every v < 0 marker)
__device__ int64_t block_argmax(double v, int64_t idx, double *redv, int64_t *redi) {
  for (int off = 16; off > 0; off >>= 1) {
    const double ov = __shfl_down_sync(0xffffffffu, v, off);
    const int64_t oi = __shfl_down_sync(0xffffffffu, idx, off);
    if (ov > v || (ov == v && oi >= 0 && (idx < 0 || oi < idx))) { v = ov; idx = oi; }
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) { redv[w] = v; redi[w] = idx; }
  __syncthreads();
  if (w == 0) {
    v = lane < NT / 32 ? redv[lane] : -1.0;
    idx = lane < NT / 32 ? redi[lane] : -1;
    for (int off = 16; off > 0; off >>= 1) {
      const double ov = __shfl_down_sync(0xffffffffu, v, off);
      const int64_t oi = __shfl_down_sync(0xffffffffu, idx, off);
      if (ov > v || (ov == v && oi >= 0 && (idx < 0 || oi < idx))) { v = ov; idx = oi; }
    }
    if (lane == 0) { redv[0] = v; redi[0] = idx; }
  }
  __syncthreads();
  const int64_t r = redi[0];
  __syncthreads();
  return r;
}

// Algorithm 6 with partial pivoting, one block per far leaf, FP64. Same reading as the
// oracle: first pivot row = first row; column pivot = argmax |u_hat_r| (first on ties);
// next pivot row = argmax |l_r| over unused rows; all-zero residual rows are skipped; stop
// when ||l_{k+1}|| ||u_{k+1}|| <= eps ||L_k U_k||_F (eq. (truncaca)), keeping that term.
// L (m x kmax) and R (n x kmax) live in scratch; `used` flags live after them.
__global__ void __launch_bounds__(NT) k_aca(int kernel, const double *pts, int dim, const LeafDev *leaves,
                                            const int32_t *ids, int base, double eps, int kmax, double *scratch,
                                            const int64_t *soff, int32_t *ranks) {
  __shared__ double redv[NT / 32];
  __shared__ int64_t redi[NT / 32];
  __shared__ double red[NT / 32];
  __shared__ double dots[2][ACA_KMAX][NT / 32];  // per warp: L_q . l_k and R_q . r_k, q <= k
  const int f = base + blockIdx.x;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const LeafDev lf = leaves[ids[f]];
  const int64_t m = lf.m, n = lf.n;
  double *L = scratch + soff[f];
  double *R = L + m * kmax;
  double *usedf = R + n * kmax;  // m flags stored as doubles (0 / 1)
  const int cap = (int)min((int64_t)kmax, min(m, n));
  for (int64_t i = threadIdx.x; i < m; i += NT) usedf[i] = 0.0;
  __syncthreads();
  double norm2 = 0.0;
  int k = 0;
  int64_t ipiv = 0;
  while (k < cap) {
    // pivot row with a nonzero residual row
    int64_t jpiv = -1;
    while (true) {
      if (ipiv < 0 || usedf[ipiv] != 0.0) {
        int64_t cand = m;
        for (int64_t i = threadIdx.x; i < m; i += NT)
          if (usedf[i] == 0.0) { cand = i; break; }
        // min over threads
        double cv = -(double)cand;
        int64_t best = block_argmax(cv, cand < m ? cand : -1, redv, redi);
        ipiv = best;
        if (ipiv < 0) break;
      }
      const double *x = pts + (lf.row + ipiv) * dim;
      double bv = -1.0;
      int64_t bi = -1;
      for (int64_t j = threadIdx.x; j < n; j += NT) {
        double v = kernel_eval(kernel, x, pts + (lf.col + j) * dim, dim);
        for (int q = 0; q < k; q++) v -= L[q * m + ipiv] * R[q * n + j];
        R[k * n + j] = v;
        const double a = fabs(v);
        if (a > bv) { bv = a; bi = j; }
      }
      __syncthreads();
      if (threadIdx.x == 0) usedf[ipiv] = 1.0;
      jpiv = block_argmax(bv, bi, redv, redi);
      const double best = jpiv >= 0 ? fabs(R[k * n + jpiv]) : 0.0;
      if (best > 0.0) break;
      ipiv = -1;
      jpiv = -1;
    }
    if (ipiv < 0 || jpiv < 0) break;
    const double piv = R[k * n + jpiv];
    __syncthreads();
    for (int64_t j = threadIdx.x; j < n; j += NT) R[k * n + j] = R[k * n + j] / piv;
    __syncthreads();
    const double *y = pts + (lf.col + jpiv) * dim;
    for (int64_t i = threadIdx.x; i < m; i += NT) {
      double v = kernel_eval(kernel, pts + (lf.row + i) * dim, y, dim);
      for (int q = 0; q < k; q++) v -= R[q * n + jpiv] * L[q * m + i];
      L[k * m + i] = v;
    }
    __syncthreads();
    // ||L_{k+1} U_{k+1}^T||_F^2 = ||L_k U_k^T||_F^2 + 2 sum_{q<k} (L_q . l_k)(R_q . r_k) + |l_k|^2 |r_k|^2:
    // every dot of this step (q <= k) reduced within each warp, then across the warps once
    for (int q = 0; q <= k; q++) {
      double a = 0.0, b = 0.0;
      for (int64_t i = threadIdx.x; i < m; i += NT) a += L[q * m + i] * L[k * m + i];
      for (int64_t j = threadIdx.x; j < n; j += NT) b += R[q * n + j] * R[k * n + j];
      a = warp_sum(a);
      b = warp_sum(b);
      if (lane == 0) {
        dots[0][q][w] = a;
        dots[1][q][w] = b;
      }
    }
    __syncthreads();
    double nl = 0.0, nu = 0.0;
    for (int x = 0; x < NT / 32; x++) {
      nl += dots[0][k][x];
      nu += dots[1][k][x];
    }
    double part = 0.0;
    for (int q = threadIdx.x; q < k; q += NT) {
      double a = 0.0, b = 0.0;
      for (int x = 0; x < NT / 32; x++) {
        a += dots[0][q][x];
        b += dots[1][q][x];
      }
      part += a * b;
    }
    const double cross = block_sum(part, red);  // (its barriers also end this step's reads of dots)
    const double prev = norm2;
    norm2 = prev + 2.0 * cross + nl * nu;
    k++;
    if (sqrt(nl) * sqrt(nu) <= eps * sqrt(prev)) break;
    double bv = -1.0;
    int64_t bi = -1;
    for (int64_t i = threadIdx.x; i < m; i += NT)
      if (usedf[i] == 0.0) {
        const double a = fabs(L[(k - 1) * m + i]);
        if (a > bv) { bv = a; bi = i; }
      }
    ipiv = block_argmax(bv, bi, redv, redi);
    if (ipiv < 0) break;
  }
  if (threadIdx.x == 0) ranks[f] = k;
}

// (value, index) of the largest value over the warp, the smallest index on ties; entries without
// a candidate carry (-1, -1)
__device__ __forceinline__ void warp_argmax(double &v, int &idx) {
  for (int off = 16; off > 0; off >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, v, off);
    const int oi = __shfl_xor_sync(0xffffffffu, idx, off);
    if (ov > v || (ov == v && oi >= 0 && (idx < 0 || oi < idx))) {
      v = ov;
      idx = oi;
    }
  }
}

// The same Algorithm 6 for far leaves of at most 64 x 64, one warp per leaf (eight leaves per
// block): each lane owns rows and columns lane and lane + 32, the used rows are one 64-bit mask,
// and every reduction is a warp exchange, so no step waits at a block barrier. Same pivoting,
// stop test and scratch layout as k_aca.
__global__ void __launch_bounds__(NT) k_aca_warp(int kernel, const double *pts, int dim, const LeafDev *leaves,
                                                 const int32_t *ids, int count, double eps, int kmax,
                                                 double *scratch, const int64_t *soff, int32_t *ranks) {
  const int f = blockIdx.x * (NT / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (f >= count) return;  // a whole warp: nothing below waits on the rest of the block
  const LeafDev lf = leaves[ids[f]];
  const int m = lf.m, n = lf.n;
  double *L = scratch + soff[f];
  double *R = L + (int64_t)m * kmax;
  const int cap = min(kmax, min(m, n));
  const uint64_t rows = m == 64 ? ~0ull : ((1ull << m) - 1);
  uint64_t used = 0;
  double norm2 = 0.0;
  int k = 0, ipiv = 0;
  while (k < cap) {
    int jpiv = -1;
    while (true) {
      if (ipiv < 0 || ((used >> ipiv) & 1ull)) {
        const uint64_t free_rows = rows & ~used;
        ipiv = free_rows ? __ffsll((long long)free_rows) - 1 : -1;
        if (ipiv < 0) break;
      }
      const double *x = pts + (lf.row + ipiv) * dim;
      double bv = -1.0;
      int bi = -1;
#pragma unroll
      for (int h = 0; h < 2; h++) {
        const int j = lane + 32 * h;
        if (j < n) {
          double v = kernel_eval(kernel, x, pts + (lf.col + j) * dim, dim);
          for (int q = 0; q < k; q++) v -= L[q * m + ipiv] * R[q * n + j];
          R[k * n + j] = v;
          const double a = fabs(v);
          if (a > bv) {
            bv = a;
            bi = j;
          }
        }
      }
      used |= 1ull << ipiv;
      warp_argmax(bv, bi);
      jpiv = bi;
      __syncwarp();
      const double best = jpiv >= 0 ? fabs(R[k * n + jpiv]) : 0.0;
      if (best > 0.0) break;
      ipiv = -1;
      jpiv = -1;
    }
    if (ipiv < 0 || jpiv < 0) break;
    const double piv = R[k * n + jpiv];
    __syncwarp();
#pragma unroll
    for (int h = 0; h < 2; h++) {
      const int j = lane + 32 * h;
      if (j < n) R[k * n + j] = R[k * n + j] / piv;
    }
    __syncwarp();
    const double *y = pts + (lf.col + jpiv) * dim;
#pragma unroll
    for (int h = 0; h < 2; h++) {
      const int i = lane + 32 * h;
      if (i < m) {
        double v = kernel_eval(kernel, pts + (lf.row + i) * dim, y, dim);
        for (int q = 0; q < k; q++) v -= R[q * n + jpiv] * L[q * m + i];
        L[k * m + i] = v;
      }
    }
    __syncwarp();
    // ||L_{k+1} U_{k+1}^T||_F^2 = ||L_k U_k^T||_F^2 + 2 sum_{q<k} (L_q . l_k)(R_q . r_k) + |l_k|^2 |r_k|^2
    double nl = 0.0, nu = 0.0, cross = 0.0;
    for (int q = 0; q <= k; q++) {
      double a = 0.0, b = 0.0;
#pragma unroll
      for (int h = 0; h < 2; h++) {
        const int i = lane + 32 * h;
        if (i < m) a += L[q * m + i] * L[k * m + i];
        if (i < n) b += R[q * n + i] * R[k * n + i];
      }
      a = warp_sum(a);
      b = warp_sum(b);
      if (q < k) cross += a * b;
      else {
        nl = a;
        nu = b;
      }
    }
    const double prev = norm2;
    norm2 = prev + 2.0 * cross + nl * nu;
    k++;
    if (sqrt(nl) * sqrt(nu) <= eps * sqrt(prev)) break;
    double bv = -1.0;
    int bi = -1;
#pragma unroll
    for (int h = 0; h < 2; h++) {
      const int i = lane + 32 * h;
      if (i < m && !((used >> i) & 1ull)) {
        const double a = fabs(L[(k - 1) * m + i]);
        if (a > bv) {
          bv = a;
          bi = i;
        }
      }
    }
    warp_argmax(bv, bi);
    ipiv = bi;
    if (ipiv < 0) break;
  }
  if (lane == 0) ranks[f] = k;
}

template <typename T>
__global__ void __launch_bounds__(NT) k_aca_compact(const LeafDev *leaves, const int32_t *ids,
                                                    const double *scratch, const int64_t *soff, int kmax,
                                                    T *data) {
  const LeafDev lf = leaves[ids[blockIdx.x]];
  const double *L = scratch + soff[blockIdx.x];
  const double *R = L + (int64_t)lf.m * kmax;
  for (int64_t o = threadIdx.x; o < (int64_t)lf.m * lf.rank; o += NT) data[lf.off_u + o] = T(L[o]);
  for (int64_t o = threadIdx.x; o < (int64_t)lf.n * lf.rank; o += NT) data[lf.off_v + o] = T(R[o]);
}

// ---------------------------------------------------------------------------------------
// a2: low-rank products created by the restriction (Algorithm 3)
// ---------------------------------------------------------------------------------------

template <typename T>
__global__ void __launch_bounds__(NT) k_term_jobs(const TermJob *jobs, const int32_t *ids, const LeafDev *leafA,
                                                  const LeafDev *leafB, const BlockDev *blocks, const T *dataA,
                                                  const T *dataB, T *terms) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *cs, *ms, *xs;
  Smem::get((T *)smem_raw, cs, ms, xs);
  const TermJob jb = jobs[ids[blockIdx.x]];
  T *out = terms + jb.out;
  for (int64_t o = threadIdx.x; o < jb.rows * jb.rank; o += NT) out[o] = T(0);  // outputs accumulate
  __syncthreads();
  if (jb.type == JOB_FF_R || jb.type == JOB_FF_L) {
    const LeafDev a = leafA[jb.a], b = leafB[jb.b];
    const T *Ua = dataA + a.off_u, *Va = dataA + a.off_v;
    const T *Ub = dataB + b.off_u, *Vb = dataB + b.off_v;
    const int rho = a.n;  // = b.m
    if (jb.type == JOB_FF_R) {
      // R_new (n' x ka) = V_b M^T, M = V_a^T U_b; chunk over columns q of M^T: U_b^T V_a[:, q]
      for (int c0 = 0; c0 < a.rank; c0 += PMAX) {
        const int pc = min(PMAX, a.rank - c0);
        gemm_tn(cs, Ub, rho, Va + (int64_t)c0 * rho, rho, rho, b.rank, pc, ms, xs);  // (kb x pc)
        gemm_nn_acc(out + (int64_t)c0 * b.n, b.n, Vb, b.n, cs, b.rank, b.n, b.rank, pc, xs);
      }
    } else {
      // L_new (m' x kb) = U_a M, M = V_a^T U_b (ka x kb)
      for (int c0 = 0; c0 < b.rank; c0 += PMAX) {
        const int pc = min(PMAX, b.rank - c0);
        gemm_tn(cs, Va, rho, Ub + (int64_t)c0 * rho, rho, rho, a.rank, pc, ms, xs);  // (ka x pc)
        gemm_nn_acc(out + (int64_t)c0 * a.m, a.m, Ua, a.m, cs, a.rank, a.m, a.rank, pc, xs);
      }
    }
  } else if (jb.type == JOB_FH) {
    // R_new (n' x ka) = B|rho' x sigma'^T V_a
    const LeafDev a = leafA[jb.a];
    const BlockDev bb = blocks[jb.b];
    const T *Va = dataA + a.off_v;
    for (int c0 = 0; c0 < a.rank; c0 += PMAX) {
      const int pc = min(PMAX, a.rank - c0);
      hblock_apply(leafB, dataB, bb.leaf_lo, bb.leaf_hi, bb.row, bb.col, true, Va + (int64_t)c0 * a.n, a.n, pc,
                   out + (int64_t)c0 * bb.n, bb.n, cs, ms, xs);
    }
  } else {
    // L_new (m' x kb) = A|tau' x rho' U_b
    const LeafDev b = leafB[jb.b];
    const BlockDev ba = blocks[jb.a];
    const T *Ub = dataB + b.off_u;
    for (int c0 = 0; c0 < b.rank; c0 += PMAX) {
      const int pc = min(PMAX, b.rank - c0);
      hblock_apply(leafA, dataA, ba.leaf_lo, ba.leaf_hi, ba.row, ba.col, false, Ub + (int64_t)c0 * b.m, b.m, pc,
                   out + (int64_t)c0 * ba.m, ba.m, cs, ms, xs);
    }
  }
}

// ---------------------------------------------------------------------------------------
// a8: near leaves, C|b = S(b) applied to the identity (Algorithm 4, evaluate())
// ---------------------------------------------------------------------------------------

// Accumulate C (m x n, column-major in shared memory, m, n <= 64 per tile) += L R^T where L is
// m x K and R is n x K; L(i,q) = Lp[i*sl_i + q*sl_q], R(j,q) = Rp[j*sr_j + q*sr_q].
template <typename T>
__device__ void acc_outer(T (&acc)[4][4], const T *Lp, int64_t sl_i, int64_t sl_q, const T *Rp, int64_t sr_j,
                          int64_t sr_q, int m, int n, int K, T *ls, T *rs) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // 16 x 16 threads, 4 x 4 outputs each
  for (int q0 = 0; q0 < K; q0 += KC) {
    const int kk = min(KC, K - q0);
    __syncthreads();
    for (int e = threadIdx.x; e < kk * 64; e += NT) {
      const int i = e & 63, q = e >> 6;
      ls[q * 64 + i] = i < m ? Lp[i * sl_i + (int64_t)(q0 + q) * sl_q] : T(0);
      rs[q * 64 + i] = i < n ? Rp[i * sr_j + (int64_t)(q0 + q) * sr_q] : T(0);
    }
    __syncthreads();
    for (int q = 0; q < kk; q++) {
      T a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; u++) { a[u] = ls[q * 64 + tx + 16 * u]; b[u] = rs[q * 64 + ty + 16 * u]; }
#pragma unroll
      for (int u = 0; u < 4; u++)
#pragma unroll
        for (int v = 0; v < 4; v++) acc[u][v] += a[u] * b[v];
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(NT) k_near_eval(const TargetDev *tg, const int2 *blk_terms, const TermDev *terms,
                                                  const PairDev *pairs, const BlockDev *blocks, const LeafDev *leafA,
                                                  const LeafDev *leafB, const T *dataA, const T *dataB,
                                                  const LeafDev *leafC, T *dataC) {
  __shared__ T ls[KC * 64], rs[KC * 64];
  const TargetDev t = tg[blockIdx.x];
  const LeafDev lc = leafC[t.leaf];
  T *C = dataC + lc.off_u;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  for (int i0 = 0; i0 < t.m; i0 += 64)
    for (int j0 = 0; j0 < t.n; j0 += 64) {
      const int mt = min(64, t.m - i0), nt = min(64, t.n - j0);
      // FP32: every term's (and pair's) contribution is summed on its own, then added to the block
      // with a compensated (Neumaier) sum, so the error does not grow with the number of terms;
      // FP64: one running sum
      constexpr bool COMP = sizeof(T) == 4;
      T acc[4][4], cmp[4][4];
#pragma unroll
      for (int u = 0; u < 4; u++)
#pragma unroll
        for (int v = 0; v < 4; v++) { acc[u][v] = T(0); cmp[u][v] = T(0); }
      auto fold = [&](T (&part)[4][4]) {
#pragma unroll
        for (int u = 0; u < 4; u++)
#pragma unroll
          for (int v = 0; v < 4; v++) {
            const T x = part[u][v], s0 = acc[u][v], s1 = s0 + x;
            cmp[u][v] += fabs(s0) >= fabs(x) ? (s0 - s1) + x : (x - s1) + s0;
            acc[u][v] = s1;
            part[u][v] = T(0);
          }
      };
      T part[4][4];
#pragma unroll
      for (int u = 0; u < 4; u++)
#pragma unroll
        for (int v = 0; v < 4; v++) part[u][v] = T(0);
      for (int blk = t.blk; blk >= 0; blk = blocks[blk].parent) {
        const int2 rg = blk_terms[blk];
        for (int ti = rg.x; ti < rg.y; ti++) {
          const TermDev tm = terms[ti];
          const T *L = (const T *)tm.L + (t.row - tm.row0) + i0;
          const T *R = (const T *)tm.R + (t.col - tm.col0) + j0;
          acc_outer(COMP ? part : acc, L, 1, tm.ldL, R, 1, tm.ldR, mt, nt, tm.rank, ls, rs);
          if (COMP) fold(part);
        }
      }
      for (int pi = t.pair_lo; pi < t.pair_hi; pi++) {
        const PairDev pr = pairs[pi];
        const BlockDev ba = blocks[pr.blkA], bb = blocks[pr.blkB];
        // near x near at the leaf level: both blocks are dense leaves
        const LeafDev la = leafA[ba.leaf_lo], lb = leafB[bb.leaf_lo];
        const T *DA = dataA + la.off_u + i0;                  // m x rho, ld m
        const T *DB = dataB + lb.off_u + (int64_t)j0 * lb.m;  // rho x n, ld rho; R(j, q) = DB[q + j*rho]
        acc_outer(COMP ? part : acc, DA, 1, la.m, DB, lb.m, 1, mt, nt, la.n, ls, rs);
        if (COMP) fold(part);
      }
      if (COMP)
#pragma unroll
        for (int u = 0; u < 4; u++)
#pragma unroll
          for (int v = 0; v < 4; v++) acc[u][v] += cmp[u][v];
#pragma unroll
      for (int u = 0; u < 4; u++)
#pragma unroll
        for (int v = 0; v < 4; v++) {
          const int i = tx + 16 * u, j = ty + 16 * v;
          if (i < mt && j < nt) C[(i0 + i) + (int64_t)(j0 + j) * t.m] = acc[u][v];
        }
      __syncthreads();
    }
}

// ---------------------------------------------------------------------------------------
// Gaussian test matrices
// ---------------------------------------------------------------------------------------

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Entry (i, c) of the Gaussian test matrix Omega of target leaf L in round rd (Alg. 8 draws
// standard normal samples): two splitmix64 outputs of the counter ((L * 64 + rd) * 64 + c) * 2^24
// + i, their top 24 bits as uniforms u1 in (0, 1] and u2 in [0, 1), then Box-Muller in FP32.
__device__ __forceinline__ float omega(uint64_t seed, int leaf, int rd, int c, int i) {
  const uint64_t ctr = ((((uint64_t)leaf * 64u + (uint64_t)rd) * 64u + (uint64_t)c) << 24) + (uint64_t)i;
  const uint64_t z1 = mix64(seed + (2 * ctr + 1) * 0x9E3779B97F4A7C15ull);
  const uint64_t z2 = mix64(seed + (2 * ctr + 2) * 0x9E3779B97F4A7C15ull);
  const float u1 = (float)((z1 >> 40) + 1) * 0x1.0p-24f;
  const float u2 = (float)(z2 >> 40) * 0x1.0p-24f;
  return sqrtf(-2.f * logf(u1)) * cospif(2.f * u2);
}

// Omega of every active target, n x p column-major at x_off (round 0: p0 columns)
template <typename T>
__global__ void __launch_bounds__(NT) k_gaussian(const TargetDev *tg, const TargetState *st, int p, uint64_t seed,
                                                 int round, T *x_base) {
  const int b = blockIdx.x;
  if (st[b].active == 0) return;
  const TargetDev t = tg[b];
  if (round == 0) p = t.p0;
  T *X = x_base + t.x_off;
  // all n p entries over the block's threads (a 64-row target would otherwise keep a quarter busy)
  for (int o = threadIdx.x; o < t.n * p; o += NT) {
    const int c = o / t.n, i = o - c * t.n;
    X[o] = T(omega(seed, t.leaf, round, c, i));
  }
}

// ---------------------------------------------------------------------------------------
// a4: orthogonalisation of the new samples (FP64)
// ---------------------------------------------------------------------------------------

// A sample column projected against the basis keeps components along it of the order of the
// rounding of its original norm, u ||y||, which normalisation scales by ||y|| / ||v||. A kept
// column with ||v|| < kappa ||y||, kappa = 1000 u / eps, is therefore projected once more against
// the whole basis (old and new columns) before it is normalised, so that the basis stays
// orthonormal well below eps: about 1e-7 at eps = 1e-6 (rarely met: such columns are dropped),
// about 0.1 at eps = 1e-12 (met by most late samples, whose energy is mostly in the basis).
__device__ __forceinline__ double orth_recheck_ratio(double eps) { return 1000.0 * 0x1.0p-53 / eps; }

// Q buffer of target b: qw + q_off, m x rmax FP64; the new columns are built in place at
// columns r .. r+p-1. Also writes Q_new in T precision into x_base (input of the S^T pass).
template <typename T>
__global__ void __launch_bounds__(NT) k_orth(const TargetDev *tg, const int32_t *ids, TargetState *st, int p,
                                             double eps, const T *y_base, double *qw, T *x_base, int round,
                                             int side, int fresh) {
  __shared__ double G[PMAX];
  constexpr int QCH = 64;  // basis columns projected per chunk
  __shared__ double Cm[QCH * PMAX];
  __shared__ double red[NT / 32];
  __shared__ double ny2c[PMAX];  // each sample column's squared norm before any projection
  const int b = ids[blockIdx.x];
  if (st[b].active == 0) return;
  const TargetDev t = tg[b];
  const int64_t m = side ? t.n : t.m;  // side 1: the column side (basis in the W buffer)
  const int r = fresh ? 0 : st[b].r;   // fresh: orthonormalise the block on its own
  if (round == 0) p = t.p0;
  double *Q = qw + (side ? t.w_off : t.q_off);
  double *Y = Q + (int64_t)r * m;  // m x p workspace inside Q
  const T *Ys = y_base + t.y_off;
  double ny2 = 0.0;
  for (int c = 0; c < p; c++) {
    double part = 0.0;
    for (int64_t i = threadIdx.x; i < m; i += NT) {
      const double v = (double)Ys[i + (int64_t)c * m];
      Y[i + (int64_t)c * m] = v;
      part += v * v;
    }
    const double nc = block_sum(part, red);
    if (threadIdx.x == 0) ny2c[c] = nc;
    ny2 += nc;
  }
  if (round == 0 && threadIdx.x == 0) st[b].est2 = ny2 / p;
  __syncthreads();
  const double est2 = st[b].est2;
  // project against the basis, twice: Y -= Q (Q^T Y)
  for (int pass = 0; pass < 2 && r > 0; pass++) {
    for (int c0 = 0; c0 < r; c0 += QCH) {
      const int rc = min(QCH, r - c0);
      // Cm (rc x p) = Q[:, c0:c0+rc]^T Y, one warp per output, lanes over rows
      const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
      for (int o = w; o < rc * p; o += NT / 32) {
        const int q = o % rc, c = o / rc;
        const double *qc = Q + (int64_t)(c0 + q) * m, *yc = Y + (int64_t)c * m;
        double s = 0.0;
        for (int64_t i = lane; i < m; i += 32) s += qc[i] * yc[i];
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
        if (lane == 0) Cm[o] = s;
      }
      __syncthreads();
      for (int64_t o = threadIdx.x; o < m * p; o += NT) {
        const int64_t i = o % m, c = o / m;
        double s = 0.0;
        for (int q = 0; q < rc; q++) s += Q[(int64_t)(c0 + q) * m + i] * Cm[q + c * rc];
        Y[o] -= s;
      }
      __syncthreads();
    }
  }
  // Orthonormalise the projected block column by column by classical Gram-Schmidt applied
  // twice against the columns already accepted in this round (stable while a column keeps more
  // than ~u of its norm; no Gram squaring). A column whose remaining norm is at most
  // drop = 0.1 * eps * sqrt(est2) carries negligible energy for the eps target and is dropped;
  // the block's kept columns are compacted to the front.
  const double drop2 = (0.1 * eps) * (0.1 * eps) * est2;
  const double kappa = orth_recheck_ratio(eps), kappa2 = kappa * kappa;
  int kept = 0;
  for (int j = 0; j < p; j++) {
    double *y = Y + (int64_t)j * m;
    // passes 0, 1: against the columns kept in this round; pass 2 (only for a column that kept
    // less than kappa of its norm): once more against the whole basis, old and new
    double nrm2 = 0.0;
    for (int pass = 0; pass < 3; pass++) {
      if (pass == 2) {
        if (!(nrm2 > drop2 && nrm2 < kappa2 * ny2c[j])) break;
        const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (int c0 = 0; c0 < r; c0 += QCH) {
          const int rc = min(QCH, r - c0);
          for (int q = w; q < rc; q += NT / 32) {
            const double *qc = Q + (int64_t)(c0 + q) * m;
            double s = 0.0;
            for (int64_t i = lane; i < m; i += 32) s += qc[i] * y[i];
            for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
            if (lane == 0) Cm[q] = s;
          }
          __syncthreads();
          for (int64_t i = threadIdx.x; i < m; i += NT) {
            double s = 0.0;
            for (int q = 0; q < rc; q++) s += Q[(int64_t)(c0 + q) * m + i] * Cm[q];
            y[i] -= s;
          }
          __syncthreads();
        }
      }
      if (kept > 0) {
        const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (int l = w; l < kept; l += NT / 32) {
          const double *ql = Y + (int64_t)l * m;
          double s = 0.0;
          for (int64_t i = lane; i < m; i += 32) s += ql[i] * y[i];
          for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
          if (lane == 0) G[l] = s;
        }
        __syncthreads();
        for (int64_t i = threadIdx.x; i < m; i += NT) {
          double s = 0.0;
          for (int l = 0; l < kept; l++) s += Y[i + (int64_t)l * m] * G[l];
          y[i] -= s;
        }
        __syncthreads();
      }
      if (pass >= 1) {
        double part2 = 0.0;
        for (int64_t i = threadIdx.x; i < m; i += NT) part2 += y[i] * y[i];
        nrm2 = block_sum(part2, red);
      }
    }
    if (nrm2 > drop2) {
      const double inv = 1.0 / sqrt(nrm2);
      double *dst = Y + (int64_t)kept * m;
      for (int64_t i = threadIdx.x; i < m; i += NT) dst[i] = y[i] * inv;
      kept++;
    }
    __syncthreads();
  }
  for (int64_t o = threadIdx.x; o < m * (p - kept); o += NT) Y[(int64_t)kept * m + o] = 0.0;
  __syncthreads();
  // Q_new in T precision for the transpose pass (zero padded to p columns)
  T *Xo = x_base + t.x_off;
  for (int64_t o = threadIdx.x; o < m * p; o += NT) {
    const int64_t c = o / m;
    Xo[o] = c < kept ? T(Y[o]) : T(0);
  }
  if (threadIdx.x == 0) {
    st[b].p_new = kept;
    st[b].nfwd += 1;
    if (kept == 0) st[b].active = 0;
  }
}

// The same step for targets of at most 64 rows, one warp per target: each lane holds rows lane
// and lane + 32 of the p new columns in registers. The projection against the basis runs column
// by column (modified Gram-Schmidt), twice; the new columns are orthonormalised by Gram-Schmidt
// twice with the same dropping rule; kept columns are compacted when written.
constexpr int OW = 16;  // max columns per round
template <typename T>
__global__ void __launch_bounds__(NT) k_orth_warp(const TargetDev *tg, const int32_t *ids, int nids,
                                                  TargetState *st, int p_round, double eps, const T *y_base,
                                                  double *qw, T *x_base, int round, int side, int fresh) {
  const int wi = blockIdx.x * (NT / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (wi >= nids) return;  // whole warps only
  const int b = ids[wi];
  if (st[b].active == 0) return;
  const TargetDev t = tg[b];
  const int m = side ? t.n : t.m, r = fresh ? 0 : st[b].r;
  const int p = round == 0 ? t.p0 : p_round;
  double *Q = qw + (side ? t.w_off : t.q_off);
  const T *Ys = y_base + t.y_off;
  const int i0 = lane, i1 = lane + 32;
  const bool v0 = i0 < m, v1 = i1 < m;
  double y[OW][2];
  double part = 0.0;
  double nyl = 0.0;  // lane c holds the squared norm of sample column c before any projection
#pragma unroll
  for (int c = 0; c < OW; c++) {
    y[c][0] = (c < p && v0) ? (double)Ys[i0 + (int64_t)c * m] : 0.0;
    y[c][1] = (c < p && v1) ? (double)Ys[i1 + (int64_t)c * m] : 0.0;
    const double nc = warp_sum(y[c][0] * y[c][0] + y[c][1] * y[c][1]);
    if (lane == c) nyl = nc;
    part += nc;
  }
  const double ny2 = part;
  double est2;
  if (round == 0) {
    est2 = ny2 / p;
    if (lane == 0) st[b].est2 = est2;
  } else {
    est2 = st[b].est2;
  }
  // project against the basis, twice
  for (int pass = 0; pass < 2; pass++)
    for (int q = 0; q < r; q++) {
      const double *qc = Q + (int64_t)q * m;
      const double q0 = v0 ? qc[i0] : 0.0, q1 = v1 ? qc[i1] : 0.0;
#pragma unroll
      for (int c = 0; c < OW; c++) {
        if (c >= p) break;
        const double d = warp_sum(q0 * y[c][0] + q1 * y[c][1]);
        y[c][0] -= d * q0;
        y[c][1] -= d * q1;
      }
    }
  // Gram-Schmidt twice among the new columns, with dropping
  const double drop2 = (0.1 * eps) * (0.1 * eps) * est2;
  const double kappa = orth_recheck_ratio(eps), kappa2 = kappa * kappa;
  unsigned keep = 0u;
#pragma unroll
  for (int j = 0; j < OW; j++) {
    if (j >= p) break;
    for (int pass = 0; pass < 2; pass++) {
#pragma unroll
      for (int l = 0; l < OW; l++) {
        if (l >= j) break;
        if (!((keep >> l) & 1u)) continue;
        const double d = warp_sum(y[l][0] * y[j][0] + y[l][1] * y[j][1]);
        y[j][0] -= d * y[l][0];
        y[j][1] -= d * y[l][1];
      }
    }
    double nrm2 = warp_sum(y[j][0] * y[j][0] + y[j][1] * y[j][1]);
    const double nyj = __shfl_sync(0xffffffffu, nyl, j);
    if (nrm2 > drop2 && nrm2 < kappa2 * nyj) {
      // once more against the whole basis (see orth_recheck_ratio)
      for (int q = 0; q < r; q++) {
        const double *qc = Q + (int64_t)q * m;
        const double q0 = v0 ? qc[i0] : 0.0, q1 = v1 ? qc[i1] : 0.0;
        const double d = warp_sum(q0 * y[j][0] + q1 * y[j][1]);
        y[j][0] -= d * q0;
        y[j][1] -= d * q1;
      }
#pragma unroll
      for (int l = 0; l < OW; l++) {
        if (l >= j) break;
        if (!((keep >> l) & 1u)) continue;
        const double d = warp_sum(y[l][0] * y[j][0] + y[l][1] * y[j][1]);
        y[j][0] -= d * y[l][0];
        y[j][1] -= d * y[l][1];
      }
      nrm2 = warp_sum(y[j][0] * y[j][0] + y[j][1] * y[j][1]);
    }
    if (nrm2 > drop2) {
      const double inv = 1.0 / sqrt(nrm2);
      y[j][0] *= inv;
      y[j][1] *= inv;
      keep |= 1u << j;
    }
  }
  // kept columns, compacted, into Q (FP64, columns r..) and Q_new (T, zero padded to p columns)
  const int kept = __popc(keep);
  double *Y = Q + (int64_t)r * m;
  T *Xo = x_base + t.x_off;
  int pos = 0;
#pragma unroll
  for (int j = 0; j < OW; j++) {
    if (j >= p) break;
    if ((keep >> j) & 1u) {
      if (v0) { Y[i0 + (int64_t)pos * m] = y[j][0]; Xo[i0 + (int64_t)pos * m] = T(y[j][0]); }
      if (v1) { Y[i1 + (int64_t)pos * m] = y[j][1]; Xo[i1 + (int64_t)pos * m] = T(y[j][1]); }
      pos++;
    }
  }
  for (int c = kept; c < p; c++) {
    if (v0) { Y[i0 + (int64_t)c * m] = 0.0; Xo[i0 + (int64_t)c * m] = T(0); }
    if (v1) { Y[i1 + (int64_t)c * m] = 0.0; Xo[i1 + (int64_t)c * m] = T(0); }
  }
  if (lane == 0) {
    st[b].p_new = kept;
    st[b].nfwd += 1;
    if (kept == 0) st[b].active = 0;
  }
}

// a5 + append: W_new = S^T Q_new arrives in y_base (n x p, T). Copy into W (FP64) at columns
// r .. r+p_new-1, update ||W||_F^2 and apply the blocked stop test eq. (truncaca):
// stop when ||W_new||_F <= eps_stop * ||W_old||_F.
template <typename T>
__global__ void __launch_bounds__(NT) k_absorb_w(const TargetDev *tg, TargetState *st, int p, double eps_stop,
                                                 const T *y_base, double *qw, int round, int max_rounds,
                                                 int32_t *active_count, int fixed) {
  __shared__ double red[NT / 32];
  const int b = blockIdx.x;
  const int was_active = st[b].active;
  const int pn = st[b].p_new;
  if (was_active == 0 || pn == 0) return;
  const TargetDev t = tg[b];
  const int r = st[b].r;
  double *W = qw + t.w_off + (int64_t)r * t.n;
  const T *Ws = y_base + t.y_off;
  double part = 0.0;
  for (int64_t o = threadIdx.x; o < (int64_t)t.n * pn; o += NT) {
    const double v = (double)Ws[o];
    W[o] = v;
    part += v * v;
  }
  const double nw2 = block_sum(part, red);
  // a first round wider than p holds a verification block: its last v = p/2 kept columns. Their
  // energy against the rest's (the proposed rank plus p/2 columns of oversampling) is the
  // blocked eq. (truncaca) within the round.
  const int v = (round == 0 && t.p0 > p && pn >= 2) ? min(max(p / 2, 1), pn - 1) : 0;
  double last2 = 0.0;
  if (v > 0) {
    double pl = 0.0;
    for (int64_t o = (int64_t)t.n * (pn - v) + threadIdx.x; o < (int64_t)t.n * pn; o += NT) pl += W[o] * W[o];
    last2 = block_sum(pl, red);
  }
  if (threadIdx.x == 0) {
    const double old = st[b].nrm2;
    st[b].nrm2 = old + nw2;
    const int rn = r + pn;
    st[b].r = rn;
    int act = 1;
    if (nw2 <= eps_stop * eps_stop * old) act = 0;
    if (v > 0 && last2 <= eps_stop * eps_stop * (nw2 - last2)) act = 0;
    if (rn >= min(t.m, t.n)) act = 0;                       // range exhausted: exact
    if (fixed) act = 0;                                      // fixed rank: one pass, no test
    if (rn + p > t.rmax || round + 1 >= max_rounds) {
      if (act) st[b].rank = -2;                              // marks "hit a cap"
      act = 0;
    }
    st[b].active = act;
    if (act) atomicAdd(active_count, 1);
  }
}

// ---------------------------------------------------------------------------------------
// a7: core truncation (FP64)
// ---------------------------------------------------------------------------------------

constexpr int JMAX = 96;  // max basis size handled by the Jacobi core solver (even)

// Whether the eps-rank needs a second Gram. The computed Gram of W carries rounding of order
// r sqrt(n) u trace(W^T W) in its entries, so its small eigenvalues are known only to that
// absolute level. When that level exceeds a tenth of the truncation threshold eps^2 trace
// (which would move the tail sum, and so the error reached, by up to a few per cent), Q and W
// are first rotated by the Gram's eigenvectors; the rotated W has columns
// orthogonal up to that rounding, and the Gram of such a matrix carries rounding relative to
// each pair of columns' own norms (Demmel and Veselic, "Jacobi's method is more accurate than
// QR"), which resolves eigenvalues far below eps^2 trace.
__device__ __forceinline__ bool core_needs_refinement(double eps, int r, int64_t n) {
  return eps * eps < 10.0 * r * sqrt((double)n) * 0x1.0p-53;
}

// Eigen-decomposition of G = W^T W (r x r) by cyclic Jacobi with a round-robin ordering
// (r/2 disjoint rotations per step, all applied at once), then the eps-rank: the smallest k
// with sum_{i >= k} lambda_i <= eps^2 sum_i lambda_i; finally Q <- Q V_k and W <- W V_k in place.
// With core_needs_refinement, the Gram and Jacobi run twice: the first pass's eigenvectors
// rotate all r columns of Q and W in place, and the eps-rank and V_k come from the second.
__global__ void __launch_bounds__(NT) k_final(const TargetDev *tg, TargetState *st, const int32_t *ids, double eps,
                                              double *qw) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double *G = (double *)smem_raw;          // JMAX x JMAX
  double *V = G + JMAX * JMAX;             // JMAX x JMAX
  double *cs = V + JMAX * JMAX;            // JMAX/2 cos, JMAX/2 sin
  int *pr = (int *)(cs + JMAX);            // JMAX pairing
  int *order = pr + JMAX;                  // JMAX
  __shared__ int rank_s, changed_s;
  const int b = ids[blockIdx.x];
  const TargetDev t = tg[b];
  const int r = st[b].r;
  const int64_t m = t.m, n = t.n;
  double *Q = qw + t.q_off, *W = qw + t.w_off;
  if (r == 0) {
    if (threadIdx.x == 0) { st[b].rank = 0; st[b].tail2 = 0.0; }
    return;
  }
  const int rr = r + (r & 1);  // padded to even
  const int npass = core_needs_refinement(eps, r, n) ? 2 : 1;
  int sweeps_total = 0;
  for (int pass = 0; pass < npass; pass++) {
  if (pass == 1) {
    // Q <- Q V and W <- W V with every column (V from the first pass); rows are independent
    for (int mat = 0; mat < 2; mat++) {
      double *M = mat == 0 ? Q : W;
      const int64_t rows = mat == 0 ? m : n;
      for (int64_t i = threadIdx.x; i < rows; i += NT) {
        double row[JMAX];
        for (int q = 0; q < r; q++) row[q] = M[i + (int64_t)q * rows];
        for (int j = 0; j < r; j++) {
          double sum = 0.0;
          for (int q = 0; q < r; q++) sum += row[q] * V[q + j * JMAX];
          M[i + (int64_t)j * rows] = sum;
        }
      }
    }
    __syncthreads();
  }
  // G = W^T W
  {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int o = w; o < rr * rr; o += NT / 32) {
      const int i = o % rr, j = o / rr;
      if (i > j) continue;
      double s = 0.0;
      if (i < r && j < r) {
        const double *wi = W + (int64_t)i * n, *wj = W + (int64_t)j * n;
        for (int64_t k = lane; k < n; k += 32) s += wi[k] * wj[k];
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
      }
      if (lane == 0) { G[i + j * JMAX] = s; G[j + i * JMAX] = s; }
    }
  }
  for (int o = threadIdx.x; o < rr * rr; o += NT) {
    const int i = o % rr, j = o / rr;
    V[i + j * JMAX] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  // Off-diagonal entries below skip = 1e-2 eps^2 trace(G) / r move no eigenvalue by more than a
  // hundredth of the truncation threshold eps^2 trace(G): rotations on them are skipped, so the
  // sweeps end once the entries that matter have converged.
  double trace = 0.0;
  for (int i = 0; i < r; i++) trace += G[i + i * JMAX];
  const double skip = 1e-2 * eps * eps * trace / r;
  const int npair = rr / 2;
  int pass_sweeps = 0;
  for (int sweep = 0; sweep < 40; sweep++) {
    if (threadIdx.x == 0) changed_s = 0;
    __syncthreads();
    for (int step = 0; step < rr - 1; step++) {
      // round-robin pairing: position 0 fixed, others rotate
      for (int k = threadIdx.x; k < npair; k += NT) {
        int a = (k == 0) ? 0 : 1 + ((k - 1 + step) % (rr - 1));
        int c = 1 + ((rr - 2 - k + step) % (rr - 1));
        if (a > c) { const int tmp = a; a = c; c = tmp; }
        pr[2 * k] = a;
        pr[2 * k + 1] = c;
        const double app = G[a + a * JMAX], aqq = G[c + c * JMAX], apq = G[a + c * JMAX];
        double co = 1.0, si = 0.0;
        if (apq != 0.0 && fabs(apq) > 1e-15 * sqrt(fabs(app * aqq)) && fabs(apq) > skip) {
          const double zeta = (aqq - app) / (2.0 * apq);
          const double tt = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          co = 1.0 / sqrt(1.0 + tt * tt);
          si = co * tt;
          changed_s = 1;
        }
        cs[k] = co;
        cs[JMAX / 2 + k] = si;
      }
      __syncthreads();
      // columns: G <- G J   (for each pair (a, c): col_a' = co col_a - si col_c, col_c' = si col_a + co col_c)
      for (int o = threadIdx.x; o < npair * rr; o += NT) {
        const int k = o / rr, i = o % rr;
        const int a = pr[2 * k], c = pr[2 * k + 1];
        const double co = cs[k], si = cs[JMAX / 2 + k];
        const double ga = G[i + a * JMAX], gc = G[i + c * JMAX];
        G[i + a * JMAX] = co * ga - si * gc;
        G[i + c * JMAX] = si * ga + co * gc;
        const double va = V[i + a * JMAX], vc = V[i + c * JMAX];
        V[i + a * JMAX] = co * va - si * vc;
        V[i + c * JMAX] = si * va + co * vc;
      }
      __syncthreads();
      // rows: G <- J^T G
      for (int o = threadIdx.x; o < npair * rr; o += NT) {
        const int k = o / rr, j = o % rr;
        const int a = pr[2 * k], c = pr[2 * k + 1];
        const double co = cs[k], si = cs[JMAX / 2 + k];
        const double ga = G[a + j * JMAX], gc = G[c + j * JMAX];
        G[a + j * JMAX] = co * ga - si * gc;
        G[c + j * JMAX] = si * ga + co * gc;
      }
      __syncthreads();
    }
    const int ch = changed_s;
    __syncthreads();
    pass_sweeps = sweep + 1;
    if (!ch) break;
  }
  sweeps_total += pass_sweeps;
  }  // pass
  if (threadIdx.x == 0) st[b].sweeps = sweeps_total;
  // order eigenvalues descending, eps-rank
  if (threadIdx.x == 0) {
    for (int i = 0; i < rr; i++) order[i] = i;
    for (int i = 1; i < rr; i++) {
      const int x = order[i];
      const double lx = G[x + x * JMAX];
      int j = i - 1;
      while (j >= 0 && G[order[j] + order[j] * JMAX] < lx) { order[j + 1] = order[j]; j--; }
      order[j + 1] = x;
    }
    double tot = 0.0;
    for (int i = 0; i < rr; i++) tot += fmax(G[i + i * JMAX], 0.0);
    double tail = 0.0;
    int k = rr;
    for (int i = rr - 1; i >= 0; i--) {
      const double nt = tail + fmax(G[order[i] + order[i] * JMAX], 0.0);
      if (nt <= eps * eps * tot) { tail = nt; k = i; }
      else break;
    }
    if (k > r) k = r;
    rank_s = k;
    st[b].tail2 = tail;
  }
  __syncthreads();
  const int k = rank_s;
  // in-place Q <- Q V(:, order[0:k]), W <- W V(:, order[0:k]); rows are independent
  double *Vk = G;  // reuse G storage: r x k, column-major ld JMAX
  for (int o = threadIdx.x; o < r * k; o += NT) {
    const int i = o % r, j = o / r;
    Vk[i + j * JMAX] = V[i + order[j] * JMAX];
  }
  __syncthreads();
  for (int mat = 0; mat < 2; mat++) {
    double *M = mat == 0 ? Q : W;
    const int64_t rows = mat == 0 ? m : n;
    for (int64_t i = threadIdx.x; i < rows; i += NT) {
      double row[JMAX];
      for (int q = 0; q < r; q++) row[q] = M[i + (int64_t)q * rows];
      for (int j = 0; j < k; j++) {
        double s = 0.0;
        for (int q = 0; q < r; q++) s += row[q] * Vk[q + j * JMAX];
        M[i + (int64_t)j * rows] = s;
      }
    }
  }
  if (threadIdx.x == 0) {
    if (st[b].rank != -2) st[b].rank = k;
    else st[b].rank = -(k + 3);  // cap hit: encode rank as -(k+3)
  }
}


// The same core truncation with one warp per target for bases of at most 32 columns (the
// common case): Gram, round-robin Jacobi, eps-rank and the in-place rotation of Q and W, with
// warp synchronisation only.
constexpr int WJ = 32;
constexpr int WF_WARPS = 4;
struct WarpFinalSmem {
  double G[WJ * WJ];
  double V[WJ * WJ];
  double co[WJ / 2], si[WJ / 2];
  int pa[WJ / 2], pc[WJ / 2];
  int order[WJ];
};

// Q <- Q V_k and W <- W V_k in place (rows of Q and W held by lanes), V_k = Vk[q + j*WJ] for
// q < r <= RW, j < k; RW bounds the unrolled row length so that no FP64 work is spent on padding.
template <int RW>
__device__ __forceinline__ void warp_rotate_rows(double *Q, double *W, int64_t m, int64_t n, int r, int k,
                                                 const double *Vk) {
  const int lane = threadIdx.x & 31;
  for (int mat = 0; mat < 2; mat++) {
    double *M = mat == 0 ? Q : W;
    const int64_t rows = mat == 0 ? m : n;
    for (int64_t i = lane; i < rows; i += 32) {
      double row[RW];
#pragma unroll
      for (int q = 0; q < RW; q++) row[q] = q < r ? M[i + (int64_t)q * rows] : 0.0;
      for (int j = 0; j < k; j++) {
        double sum = 0.0;
#pragma unroll
        for (int q = 0; q < RW; q++) sum += row[q] * Vk[q + j * WJ];
        M[i + (int64_t)j * rows] = sum;
      }
    }
  }
}

__global__ void __launch_bounds__(WF_WARPS * 32) k_final_warp(const TargetDev *tg, TargetState *st, const int32_t *ids,
                                                              int nids, double eps, double *qw) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int idx = blockIdx.x * WF_WARPS + w;
  if (idx >= nids) return;  // whole warps; no block barrier in this kernel
  WarpFinalSmem &S = ((WarpFinalSmem *)smem_raw)[w];
  const int b = ids[idx];
  const TargetDev t = tg[b];
  const int r = st[b].r;
  const int64_t m = t.m, n = t.n;
  double *Q = qw + t.q_off, *W = qw + t.w_off;
  if (r == 0) {
    if (lane == 0) { st[b].rank = 0; st[b].tail2 = 0.0; }
    return;
  }
  const int rr = r + (r & 1);
  const int npass = core_needs_refinement(eps, r, n) ? 2 : 1;
  int sweeps_total = 0;
  for (int pass = 0; pass < npass; pass++) {
  if (pass == 1) {
    // Q <- Q V and W <- W V with every column: V from the first pass, staged in G's storage
    // with zero rows from r to WJ (rows of S.V beyond rr were never written)
    for (int o = lane; o < WJ * r; o += 32) {
      const int i = o % WJ, j = o / WJ;
      S.G[i + j * WJ] = i < r ? S.V[i + j * WJ] : 0.0;
    }
    __syncwarp();
    if (r <= 8) warp_rotate_rows<8>(Q, W, m, n, r, r, S.G);
    else if (r <= 16) warp_rotate_rows<16>(Q, W, m, n, r, r, S.G);
    else if (r <= 24) warp_rotate_rows<24>(Q, W, m, n, r, r, S.G);
    else warp_rotate_rows<WJ>(Q, W, m, n, r, r, S.G);
    __syncwarp();
  }
  // G = W^T W (upper triangle by pairs, mirrored)
  for (int o = lane; o < rr * rr; o += 32) {
    const int i = o % rr, j = o / rr;
    S.V[i + j * WJ] = (i == j) ? 1.0 : 0.0;
    if (i > j) continue;
    double sum = 0.0;
    if (i < r && j < r) {
      const double *wi = W + (int64_t)i * n, *wj = W + (int64_t)j * n;
      for (int64_t k = 0; k < n; k++) sum += wi[k] * wj[k];
    }
    S.G[i + j * WJ] = sum;
    S.G[j + i * WJ] = sum;
  }
  __syncwarp();
  // rotations on entries below skip are left out (see k_final)
  double trace = 0.0;
  for (int i = 0; i < r; i++) trace += S.G[i + i * WJ];
  const double skip = 1e-2 * eps * eps * trace / r;
  const int npair = rr / 2;
  int pass_sweeps = 0;
  for (int sweep = 0; sweep < 40; sweep++) {
    bool changed = false;
    for (int step = 0; step < rr - 1; step++) {
      if (lane < npair) {
        const int k = lane;
        int a = (k == 0) ? 0 : 1 + ((k - 1 + step) % (rr - 1));
        int c = 1 + ((rr - 2 - k + step) % (rr - 1));
        if (a > c) { const int tmp = a; a = c; c = tmp; }
        const double app = S.G[a + a * WJ], aqq = S.G[c + c * WJ], apq = S.G[a + c * WJ];
        double co = 1.0, si = 0.0;
        if (apq != 0.0 && fabs(apq) > 1e-15 * sqrt(fabs(app * aqq)) && fabs(apq) > skip) {
          const double zeta = (aqq - app) / (2.0 * apq);
          const double tt = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          co = 1.0 / sqrt(1.0 + tt * tt);
          si = co * tt;
          changed = true;
        }
        S.pa[k] = a;
        S.pc[k] = c;
        S.co[k] = co;
        S.si[k] = si;
      }
      __syncwarp();
      for (int o = lane; o < npair * rr; o += 32) {  // columns (G J) and V J
        const int k = o / rr, i = o % rr;
        const int a = S.pa[k], c = S.pc[k];
        const double co = S.co[k], si = S.si[k];
        const double ga = S.G[i + a * WJ], gc = S.G[i + c * WJ];
        S.G[i + a * WJ] = co * ga - si * gc;
        S.G[i + c * WJ] = si * ga + co * gc;
        const double va = S.V[i + a * WJ], vc = S.V[i + c * WJ];
        S.V[i + a * WJ] = co * va - si * vc;
        S.V[i + c * WJ] = si * va + co * vc;
      }
      __syncwarp();
      for (int o = lane; o < npair * rr; o += 32) {  // rows J^T G
        const int k = o / rr, j = o % rr;
        const int a = S.pa[k], c = S.pc[k];
        const double co = S.co[k], si = S.si[k];
        const double ga = S.G[a + j * WJ], gc = S.G[c + j * WJ];
        S.G[a + j * WJ] = co * ga - si * gc;
        S.G[c + j * WJ] = si * ga + co * gc;
      }
      __syncwarp();
    }
    pass_sweeps = sweep + 1;
    if (!__any_sync(0xffffffffu, changed)) break;
  }
  sweeps_total += pass_sweeps;
  }  // pass
  if (lane == 0) st[b].sweeps = sweeps_total;
  int k = 0;
  if (lane == 0) {
    for (int i = 0; i < rr; i++) S.order[i] = i;
    for (int i = 1; i < rr; i++) {
      const int x = S.order[i];
      const double lx = S.G[x + x * WJ];
      int j = i - 1;
      while (j >= 0 && S.G[S.order[j] + S.order[j] * WJ] < lx) { S.order[j + 1] = S.order[j]; j--; }
      S.order[j + 1] = x;
    }
    double tot = 0.0;
    for (int i = 0; i < rr; i++) tot += fmax(S.G[i + i * WJ], 0.0);
    double tail = 0.0;
    k = rr;
    for (int i = rr - 1; i >= 0; i--) {
      const double nt = tail + fmax(S.G[S.order[i] + S.order[i] * WJ], 0.0);
      if (nt <= eps * eps * tot) { tail = nt; k = i; }
      else break;
    }
    if (k > r) k = r;
    st[b].tail2 = tail;
  }
  k = __shfl_sync(0xffffffffu, k, 0);
  __syncwarp();
  // V_k (r x k, zero below row r) into G's storage, then rows of Q and W rotated in place
  for (int o = lane; o < WJ * k; o += 32) {
    const int i = o % WJ, j = o / WJ;
    S.G[i + j * WJ] = i < r ? S.V[i + S.order[j] * WJ] : 0.0;
  }
  __syncwarp();
  if (r <= 8) warp_rotate_rows<8>(Q, W, m, n, r, k, S.G);
  else if (r <= 16) warp_rotate_rows<16>(Q, W, m, n, r, k, S.G);
  else if (r <= 24) warp_rotate_rows<24>(Q, W, m, n, r, k, S.G);
  else warp_rotate_rows<WJ>(Q, W, m, n, r, k, S.G);
  if (lane == 0) {
    if (st[b].rank != -2) st[b].rank = k;
    else st[b].rank = -(k + 3);
  }
}

// ---------------------------------------------------------------------------------------
// a3-a5 by cross approximation: Algorithm 6 on the sum-expression, one row and one column per
// step, every unfinished far target of the product in the same launches
// ---------------------------------------------------------------------------------------

// used-row flags of target t (m doubles, 0 or 1) in the last column of its Q buffer
__device__ __forceinline__ double *aca_used(double *qw, const TargetDev &t) {
  return qw + t.q_off + (int64_t)(t.rmax - 1) * t.m;
}

// first pivot row i_1 = 0: clear the flags and set e_0 (m entries) as the S^T pass input
template <typename T>
__global__ void __launch_bounds__(NT) k_aca_start(const TargetDev *tg, TargetState *st, double *qw, T *x_base) {
  const int b = blockIdx.x;
  const TargetDev t = tg[b];
  double *used = aca_used(qw, t);
  T *X = x_base + t.x_off;
  for (int64_t i = threadIdx.x; i < t.m; i += NT) {
    used[i] = 0.0;
    X[i] = T(i == 0 ? 1 : 0);
  }
  if (threadIdx.x == 0) {
    st[b].piv_i = 0;
    st[b].piv_j = -1;
    st[b].p_new = 0;
    st[b].hits = 0;
  }
}

// Row step: u_hat = e_i^T S - sum_{s<r} [l_s]_i u_s (Algorithm 6), column pivot j_r = argmax
// |u_hat| (first on ties), u_r = u_hat / [u_hat]_{j_r}, stored as column r of the W buffer; the
// S pass then gets e_{j_r}. A residual row that is exactly zero is marked used and the first
// unused row becomes the pivot row of the next step (no column this step: p_new = 0); a target
// with every row used stops.
template <typename T>
__global__ void __launch_bounds__(NT) k_aca_row(const TargetDev *tg, TargetState *st, const T *y_base, double *qw,
                                                T *x_base) {
  __shared__ double li[JMAX];
  __shared__ double redv[NT / 32];
  __shared__ int64_t redi[NT / 32];
  const int b = blockIdx.x;
  if (st[b].active == 0) return;
  const TargetDev t = tg[b];
  const int r = st[b].r;
  const int64_t m = t.m, n = t.n, i = st[b].piv_i;
  const double *L = qw + t.q_off;
  double *U = qw + t.w_off;
  double *u = U + (int64_t)r * n;
  const T *row = y_base + t.y_off;
  for (int s = threadIdx.x; s < r; s += NT) li[s] = L[i + (int64_t)s * m];
  __syncthreads();
  double bv = -1.0;
  int64_t bj = -1;
  for (int64_t j = threadIdx.x; j < n; j += NT) {
    double v = (double)row[j];
    for (int s = 0; s < r; s++) v -= li[s] * U[j + (int64_t)s * n];
    u[j] = v;
    const double a = fabs(v);
    if (a > bv) { bv = a; bj = j; }
  }
  const int64_t jr = block_argmax(bv, bj, redv, redi);  // ends with a barrier: u is complete
  const double piv = jr >= 0 ? u[jr] : 0.0;
  __syncthreads();  // every thread holds piv before u[jr] is overwritten
  T *X = x_base + t.x_off;
  if (piv != 0.0) {
    const double inv = 1.0 / piv;
    for (int64_t j = threadIdx.x; j < n; j += NT) {
      u[j] = (j == jr) ? 1.0 : u[j] * inv;
      X[j] = T(j == jr ? 1 : 0);
    }
    if (threadIdx.x == 0) {
      st[b].piv_j = (int)jr;
      st[b].p_new = 1;
    }
    return;
  }
  // zero residual row
  double *used = aca_used(qw, t);
  if (threadIdx.x == 0) used[i] = 1.0;
  __syncthreads();
  int64_t cand = m;  // this thread's first unused row (m: none); the block takes the smallest
  for (int64_t k = threadIdx.x; k < m; k += NT)
    if (used[k] == 0.0) { cand = k; break; }
  const int64_t next = block_argmax(-(double)cand, cand < m ? cand : -1, redv, redi);
  if (threadIdx.x == 0) {
    st[b].p_new = 0;
    if (next < 0) st[b].active = 0;
    else st[b].piv_i = (int)next;
  }
}

// Column step: l_r = S e_{j_r} - sum_{s<r} [u_s]_{j_r} l_s (Algorithm 6), stored as column r of
// the Q buffer; ||L_{r+1} U_{r+1}||_F^2 updated from the cross terms; stop once two consecutive
// crosses have met eq. (truncaca), ||l_r|| ||u_r|| <= eps_stop ||L_r U_r||_F (keeping the new
// crosses), or when r + 1 reaches min(m, n) (exact) or the basis capacity (cap: rank marked -2);
// otherwise the next pivot row is argmax |l_r| over the unused rows and its unit vector the next
// S^T input.
template <typename T>
__global__ void __launch_bounds__(NT) k_aca_col(const TargetDev *tg, TargetState *st, const T *y_base, double *qw,
                                                T *x_base, double eps_stop, int32_t *active_count) {
  __shared__ double uj[JMAX], dl[JMAX], du[JMAX];
  __shared__ double red[NT / 32];
  __shared__ double redv[NT / 32];
  __shared__ int64_t redi[NT / 32];
  const int b = blockIdx.x;
  if (st[b].active == 0) return;
  const TargetDev t = tg[b];
  const int64_t m = t.m, n = t.n;
  T *X = x_base + t.x_off;
  if (st[b].p_new == 0) {  // the row step found a zero row: next row step at the new pivot
    const int64_t i = st[b].piv_i;
    for (int64_t k = threadIdx.x; k < m; k += NT) X[k] = T(k == i ? 1 : 0);
    if (threadIdx.x == 0) atomicAdd(active_count, 1);
    return;
  }
  const int r = st[b].r;
  const int64_t i = st[b].piv_i, j = st[b].piv_j;
  double *L = qw + t.q_off;
  const double *U = qw + t.w_off;
  double *l = L + (int64_t)r * m;
  const double *u = U + (int64_t)r * n;
  const T *col = y_base + t.y_off;
  for (int s = threadIdx.x; s < r; s += NT) uj[s] = U[j + (int64_t)s * n];
  __syncthreads();
  double pl = 0.0;
  for (int64_t k = threadIdx.x; k < m; k += NT) {
    double v = (double)col[k];
    for (int s = 0; s < r; s++) v -= uj[s] * L[k + (int64_t)s * m];
    l[k] = v;
    pl += v * v;
  }
  double pu = 0.0;
  for (int64_t k = threadIdx.x; k < n; k += NT) pu += u[k] * u[k];
  const double nl2 = block_sum(pl, red), nu2 = block_sum(pu, red);  // barriers: l is complete
  // cross terms (l_s . l_r)(u_s . u_r), s < r: one warp per s
  {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int s = w; s < r; s += NT / 32) {
      const double *ls = L + (int64_t)s * m, *us = U + (int64_t)s * n;
      double a = 0.0, c = 0.0;
      for (int64_t k = lane; k < m; k += 32) a += ls[k] * l[k];
      for (int64_t k = lane; k < n; k += 32) c += us[k] * u[k];
      a = warp_sum(a);
      c = warp_sum(c);
      if (lane == 0) { dl[s] = a; du[s] = c; }
    }
  }
  double *used = aca_used(qw, t);
  if (threadIdx.x == 0) used[i] = 1.0;
  __syncthreads();
  __shared__ int act_s;
  if (threadIdx.x == 0) {
    double cross = 0.0;
    for (int s = 0; s < r; s++) cross += dl[s] * du[s];
    const double prev = st[b].nrm2;
    st[b].nrm2 = prev + 2.0 * cross + nl2 * nu2;
    const int rn = r + 1;
    st[b].r = rn;
    st[b].nfwd += 1;
    int act = 1;
    const int hits = nl2 * nu2 <= eps_stop * eps_stop * prev ? st[b].hits + 1 : 0;  // eq. (truncaca)
    st[b].hits = hits;
    if (hits >= 2) act = 0;
    if (rn >= min(t.m, t.n)) act = 0;                        // exact
    if (act && rn >= t.rmax - 1) {                           // capacity (last column: flags)
      st[b].rank = -2;
      act = 0;
    }
    act_s = act;
  }
  __syncthreads();
  if (!act_s) {
    if (threadIdx.x == 0) st[b].active = 0;
    return;
  }
  double bv = -1.0;
  int64_t bi = -1;
  for (int64_t k = threadIdx.x; k < m; k += NT)
    if (used[k] == 0.0) {
      const double a = fabs(l[k]);
      if (a > bv) { bv = a; bi = k; }
    }
  const int64_t next = block_argmax(bv, bi, redv, redi);
  if (next < 0) {
    if (threadIdx.x == 0) st[b].active = 0;
    return;
  }
  for (int64_t k = threadIdx.x; k < m; k += NT) X[k] = T(k == next ? 1 : 0);
  if (threadIdx.x == 0) {
    st[b].piv_i = (int)next;
    atomicAdd(active_count, 1);
  }
}

// L = Q R by classical Gram-Schmidt applied twice (FP64, in place in the Q buffer, R in shared
// memory), then W <- U R^T in place: row i of W, column c, is sum_{s >= c} U[i][s] R[c][s], so
// ascending c only overwrites entries no later column reads. A column with an exactly zero
// remainder gets q = 0 and a zero row of R (it adds nothing to L U^T).
__global__ void __launch_bounds__(NT) k_aca_qr(const TargetDev *tg, const TargetState *st, double *qw) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double *R = (double *)smem_raw;  // r x r, R[c][s] at c + s * r
  __shared__ double g[JMAX];
  __shared__ double red[NT / 32];
  const int b = blockIdx.x;
  const int r = st[b].r;
  if (r == 0) return;
  const TargetDev t = tg[b];
  const int64_t m = t.m, n = t.n;
  double *L = qw + t.q_off, *W = qw + t.w_off;
  for (int o = threadIdx.x; o < r * r; o += NT) R[o] = 0.0;
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int c = 0; c < r; c++) {
    double *v = L + (int64_t)c * m;
    for (int pass = 0; pass < 2 && c > 0; pass++) {
      for (int s = w; s < c; s += NT / 32) {
        const double *q = L + (int64_t)s * m;
        double a = 0.0;
        for (int64_t k = lane; k < m; k += 32) a += q[k] * v[k];
        a = warp_sum(a);
        if (lane == 0) g[s] = a;
      }
      __syncthreads();
      for (int64_t k = threadIdx.x; k < m; k += NT) {
        double a = 0.0;
        for (int s = 0; s < c; s++) a += L[k + (int64_t)s * m] * g[s];
        v[k] -= a;
      }
      for (int s = threadIdx.x; s < c; s += NT) R[s + c * r] += g[s];
      __syncthreads();
    }
    double part = 0.0;
    for (int64_t k = threadIdx.x; k < m; k += NT) part += v[k] * v[k];
    const double nrm = sqrt(block_sum(part, red));
    const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
    for (int64_t k = threadIdx.x; k < m; k += NT) v[k] *= inv;
    if (threadIdx.x == 0) R[c + c * r] = nrm;
    __syncthreads();
  }
  for (int64_t k = threadIdx.x; k < n; k += NT)
    for (int c = 0; c < r; c++) {
      double a = 0.0;
      for (int s = c; s < r; s++) a += W[k + (int64_t)s * n] * R[c + s * r];
      W[k + (int64_t)c * n] = a;
    }
}

// ---------------------------------------------------------------------------------------
// a3-a5 by Lanczos bidiagonalization: Algorithm 7 on the sum-expression with full
// reorthogonalization, one S and one S^T pass per step for every unfinished far target
// ---------------------------------------------------------------------------------------

// v <- v - B (B^T v), twice, for the first nb columns of B (ld rows); g holds nb <= JMAX
// coefficients. Every thread of the block must call; ends with a barrier.
__device__ void block_project2(double *v, const double *B, int64_t rows, int nb, double *g) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int pass = 0; pass < 2 && nb > 0; pass++) {
    for (int s = w; s < nb; s += NT / 32) {
      const double *bs = B + (int64_t)s * rows;
      double a = 0.0;
      for (int64_t k = lane; k < rows; k += 32) a += bs[k] * v[k];
      a = warp_sum(a);
      if (lane == 0) g[s] = a;
    }
    __syncthreads();
    for (int64_t k = threadIdx.x; k < rows; k += NT) {
      double a = 0.0;
      for (int s = 0; s < nb; s++) a += B[k + (int64_t)s * rows] * g[s];
      v[k] -= a;
    }
    __syncthreads();
  }
}

// w_1: Gaussian entries (the same counter-based generator as the test matrices, round 0,
// column 0), normalised, into column 0 of the W buffer and as the S pass input
template <typename T>
__global__ void __launch_bounds__(NT) k_lz_start(const TargetDev *tg, TargetState *st, double *qw, T *x_base,
                                                 uint64_t seed) {
  __shared__ double red[NT / 32];
  const int b = blockIdx.x;
  const TargetDev t = tg[b];
  double *w = qw + t.w_off;
  T *X = x_base + t.x_off;
  double part = 0.0;
  for (int64_t i = threadIdx.x; i < t.n; i += NT) {
    const double v = (double)omega(seed, t.leaf, 0, 0, (int)i);
    w[i] = v;
    part += v * v;
  }
  const double nrm = sqrt(block_sum(part, red));
  const double inv = nrm > 0.0 ? 1.0 / nrm : 0.0;
  for (int64_t i = threadIdx.x; i < t.n; i += NT) {
    w[i] *= inv;
    X[i] = T(w[i]);
  }
  if (threadIdx.x == 0) {
    st[b].alpha = 0.0;
    st[b].beta = 0.0;
    st[b].hits = 0;
    if (!(nrm > 0.0)) st[b].active = 0;
  }
}

// q_r = S w_r - beta_{r-1} q_{r-1} (S w_r from the S pass in y_base), projected twice against
// q_1..q_{r-1}, alpha_r = ||q_r||, q_r / alpha_r into column r of the Q buffer and as the S^T
// pass input. alpha_r = 0 (the Krylov space is exhausted) ends the target.
template <typename T>
__global__ void __launch_bounds__(NT) k_lz_q(const TargetDev *tg, TargetState *st, const T *y_base, double *qw,
                                             T *x_base) {
  __shared__ double g[JMAX];
  __shared__ double red[NT / 32];
  const int b = blockIdx.x;
  if (st[b].active == 0) return;
  const TargetDev t = tg[b];
  const int r = st[b].r;
  const int64_t m = t.m;
  double *Q = qw + t.q_off;
  double *q = Q + (int64_t)r * m;
  const T *y = y_base + t.y_off;
  const double beta = st[b].beta;
  for (int64_t k = threadIdx.x; k < m; k += NT) q[k] = (double)y[k] - (r > 0 ? beta * Q[k + (int64_t)(r - 1) * m] : 0.0);
  __syncthreads();
  block_project2(q, Q, m, r, g);
  double part = 0.0;
  for (int64_t k = threadIdx.x; k < m; k += NT) part += q[k] * q[k];
  const double alpha = sqrt(block_sum(part, red));
  if (!(alpha > 0.0) || !isfinite(alpha)) {
    if (threadIdx.x == 0) st[b].active = 0;
    return;
  }
  const double inv = 1.0 / alpha;
  T *X = x_base + t.x_off;
  for (int64_t k = threadIdx.x; k < m; k += NT) {
    q[k] *= inv;
    X[k] = T(q[k]);
  }
  if (threadIdx.x == 0) st[b].alpha = alpha;
}

// w = S^T q_r - alpha_r w_r (S^T q_r from the S^T pass), projected twice against w_1..w_r,
// beta_r = ||w||. The step's increment q_r (alpha_r w_r + beta_r w_{r+1})^T has Frobenius norm
// sqrt(alpha_r^2 + beta_r^2) and the approximation so far sum_{s<r} (alpha_s^2 + beta_s^2):
// eq. (truncaca) at eps_stop, met by two consecutive steps, ends the target, as do r + 1 = min(m, n),
// beta_r = 0 and the basis capacity (rank marked -2). Otherwise w_{r+1} = w / beta_r goes into
// column r + 1 of the W buffer and becomes the next S pass input.
template <typename T>
__global__ void __launch_bounds__(NT) k_lz_w(const TargetDev *tg, TargetState *st, const T *y_base, double *qw,
                                             T *x_base, double eps_stop, int32_t *active_count) {
  __shared__ double g[JMAX];
  __shared__ double red[NT / 32];
  __shared__ int act_s;
  const int b = blockIdx.x;
  if (st[b].active == 0) return;
  const TargetDev t = tg[b];
  const int r = st[b].r;
  const int64_t n = t.n;
  double *W = qw + t.w_off;
  const double *wr = W + (int64_t)r * n;
  double *wn = W + (int64_t)(r + 1) * n;  // r + 1 <= rmax - 1: inside the buffer
  const T *y = y_base + t.y_off;
  const double alpha = st[b].alpha;
  for (int64_t k = threadIdx.x; k < n; k += NT) wn[k] = (double)y[k] - alpha * wr[k];
  __syncthreads();
  block_project2(wn, W, n, r + 1, g);
  double part = 0.0;
  for (int64_t k = threadIdx.x; k < n; k += NT) part += wn[k] * wn[k];
  const double beta = sqrt(block_sum(part, red));
  if (threadIdx.x == 0) {
    const double inc = alpha * alpha + beta * beta;
    const double prev = st[b].nrm2;
    st[b].nrm2 = prev + inc;
    const int hits = inc <= eps_stop * eps_stop * prev ? st[b].hits + 1 : 0;  // eq. (truncaca)
    st[b].hits = hits;
    const int rn = r + 1;
    st[b].r = rn;
    st[b].nfwd += 1;
    int act = hits < 2;
    if (rn >= min(t.m, t.n)) act = 0;                 // exact
    if (!(beta > 0.0) || !isfinite(beta)) act = 0;    // invariant subspace
    if (act && rn >= t.rmax - 1) {                    // capacity
      st[b].rank = -2;
      act = 0;
    }
    act_s = act;
  }
  __syncthreads();
  if (!act_s) {
    if (threadIdx.x == 0) st[b].active = 0;
    return;
  }
  const double inv = 1.0 / beta;
  T *X = x_base + t.x_off;
  for (int64_t k = threadIdx.x; k < n; k += NT) {
    wn[k] *= inv;
    X[k] = T(wn[k]);
  }
  if (threadIdx.x == 0) {
    st[b].beta = beta;
    atomicAdd(active_count, 1);
  }
}

// columns c0 .. c0+p-1 of Q (those below r) as the S^T pass input, zero padded; targets with no
// such column sit the pass out
template <typename T>
__global__ void __launch_bounds__(NT) k_lz_load(const TargetDev *tg, TargetState *st, const double *qw, T *x_base,
                                                int c0, int p) {
  const int b = blockIdx.x;
  const TargetDev t = tg[b];
  const int cnt = min(p, st[b].r - c0);
  __syncthreads();  // every thread has read r before thread 0 may change the state
  if (threadIdx.x == 0) st[b].active = cnt > 0 ? 1 : 0;
  if (cnt <= 0) return;
  const double *Q = qw + t.q_off + (int64_t)c0 * t.m;
  T *X = x_base + t.x_off;
  for (int64_t o = threadIdx.x; o < (int64_t)t.m * p; o += NT) X[o] = o < (int64_t)t.m * cnt ? T(Q[o]) : T(0);
}

// the S^T pass output (n x p) into columns c0 .. c0+p-1 of W, those below r
template <typename T>
__global__ void __launch_bounds__(NT) k_lz_store(const TargetDev *tg, const TargetState *st, const T *y_base,
                                                 double *qw, int c0, int p) {
  const int b = blockIdx.x;
  if (st[b].active == 0) return;
  const TargetDev t = tg[b];
  const int cnt = min(p, st[b].r - c0);
  if (cnt <= 0) return;
  double *W = qw + t.w_off + (int64_t)c0 * t.n;
  const T *y = y_base + t.y_off;
  for (int64_t o = threadIdx.x; o < (int64_t)t.n * cnt; o += NT) W[o] = (double)y[o];
}

template <typename T>
__global__ void __launch_bounds__(NT) k_write_far(const TargetDev *tg, const TargetState *st, const double *qw,
                                                  const LeafDev *leafC, T *dataC) {
  const TargetDev t = tg[blockIdx.x];
  const LeafDev lc = leafC[t.leaf];
  const int k = lc.rank;
  const double *Q = qw + t.q_off, *W = qw + t.w_off;
  for (int64_t o = threadIdx.x; o < (int64_t)t.m * k; o += NT) dataC[lc.off_u + o] = T(Q[o]);
  for (int64_t o = threadIdx.x; o < (int64_t)t.n * k; o += NT) dataC[lc.off_v + o] = T(W[o]);
  (void)st;
}

// index of the first non-finite entry (or -1) of an array, for the opt-in finiteness check
template <typename T>
__global__ void k_find_nonfinite(const T *x, int64_t count, unsigned long long *first) {
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < count; o += (int64_t)gridDim.x * blockDim.x)
    if (!isfinite((double)x[o])) atomicMin(first, (unsigned long long)o);
}

cudaError_t launch_find_nonfinite(int prec, const void *x, int64_t count, unsigned long long *first, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((count + NT - 1) / NT, 152 * 16);
  if (prec == 64) k_find_nonfinite<double><<<blocks, NT, 0, s>>>((const double *)x, count, first);
  else k_find_nonfinite<float><<<blocks, NT, 0, s>>>((const float *)x, count, first);
  return cudaGetLastError();
}

template <typename T>
__global__ void k_convert(const T *src, double *dst, int64_t count) {
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < count; o += (int64_t)gridDim.x * blockDim.x)
    dst[o] = (double)src[o];
}

// ---------------------------------------------------------------------------------------
// launch wrappers
// ---------------------------------------------------------------------------------------

template <typename K>
static cudaError_t set_smem(K kern, size_t bytes) {
  return raise_smem_limit(kern, bytes);
}

int max_dynamic_smem() {
  static int cached[64];  // per device; 0 = not queried yet
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 48 * 1024;
  if (cached[dev] == 0) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess || v <= 0)
      v = 48 * 1024;
    cached[dev] = v;
  }
  return cached[dev];
}

cudaError_t launch_kernel_dense(int prec, int kernel, const double *pts, int dim, const LeafDev *leaves,
                                const int32_t *near_ids, int nnear, void *data, cudaStream_t s) {
  if (nnear == 0) return cudaSuccess;
  if (prec == 64)
    k_kernel_dense<double><<<nnear, NT, 0, s>>>(kernel, pts, dim, leaves, near_ids, (double *)data);
  else
    k_kernel_dense<float><<<nnear, NT, 0, s>>>(kernel, pts, dim, leaves, near_ids, (float *)data);
  return cudaGetLastError();
}

cudaError_t launch_aca(int kernel, const double *pts, int dim, const LeafDev *leaves, const int32_t *far_ids,
                       int nfar, int nsmall, double eps, int kmax, double *scratch, const int64_t *scratch_off,
                       int32_t *ranks, cudaStream_t s) {
  if (nfar == 0) return cudaSuccess;
  if (kmax < 1 || kmax > ACA_KMAX) return cudaErrorInvalidValue;  // the kernel's dot table holds ACA_KMAX
  if (nsmall < 0 || nsmall > nfar) return cudaErrorInvalidValue;
  if (nsmall > 0)
    k_aca_warp<<<(nsmall + NT / 32 - 1) / (NT / 32), NT, 0, s>>>(kernel, pts, dim, leaves, far_ids, nsmall, eps, kmax,
                                                               scratch, scratch_off, ranks);
  if (nfar > nsmall)
    k_aca<<<nfar - nsmall, NT, 0, s>>>(kernel, pts, dim, leaves, far_ids, nsmall, eps, kmax, scratch, scratch_off,
                                       ranks);
  return cudaGetLastError();
}

cudaError_t launch_aca_compact(int prec, const LeafDev *leaves, const int32_t *far_ids, int nfar,
                               const double *scratch, const int64_t *scratch_off, int kmax, void *data,
                               cudaStream_t s) {
  if (nfar == 0) return cudaSuccess;
  if (prec == 64)
    k_aca_compact<double><<<nfar, NT, 0, s>>>(leaves, far_ids, scratch, scratch_off, kmax, (double *)data);
  else
    k_aca_compact<float><<<nfar, NT, 0, s>>>(leaves, far_ids, scratch, scratch_off, kmax, (float *)data);
  return cudaGetLastError();
}

// Far x far products with both ranks <= 32, one warp per job (Algorithm 3, both factors low
// rank): M = V_a^T U_b (ka x kb) with the rho rows staged FF_CH at a time in the warp's shared
// memory and each lane accumulating a 4 x 8 tile of M in registers; then FF_L writes
// L_new = U_a M (lanes over rows, a row of M broadcast per step) and FF_R writes R_new = V_b M^T.
constexpr int FF_CH = 16;  // rows of V_a and U_b staged per step
constexpr int FF_K = 32;   // max rank of either factor

// K: the job's rank bucket (8, 16 or 32, at least both ranks); ranks below K read as zeros
template <typename T, int K>
struct FfSmem {
  T va[FF_CH][K + 1], ub[FF_CH][K + 1];
  T M[K][K + 1];
};

template <typename T, int K>
__global__ void __launch_bounds__(NT) k_ff_warp(const TermJob *jobs, const int32_t *ids, int n, const LeafDev *leafA,
                                                const LeafDev *leafB, const T *dataA, const T *dataB, T *terms) {
  static_assert(K == 8 || K == 16 || K == 32, "rank bucket");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ji = blockIdx.x * (NT / 32) + w;
  if (ji >= n) return;  // whole warps only; no block barrier below
  FfSmem<T, K> &S = ((FfSmem<T, K> *)smem_raw)[w];
  const TermJob jb = jobs[ids[ji]];
  const LeafDev a = leafA[jb.a], b = leafB[jb.b];
  const int ka = a.rank, kb = b.rank, rho = a.n;
  const T *Ua = dataA + a.off_u, *Va = dataA + a.off_v;
  const T *Ub = dataB + b.off_u, *Vb = dataB + b.off_v;
  // M = V_a^T U_b; lane owns rows q0 .. q0 + TQ - 1 and columns c0 .. c0 + TC - 1 of M
  constexpr int TQ = K / 8, TC = K / 4;
  const int q0 = (lane >> 2) * TQ, c0 = (lane & 3) * TC;
  T acc[TQ][TC];
#pragma unroll
  for (int u = 0; u < TQ; u++)
#pragma unroll
    for (int v = 0; v < TC; v++) acc[u][v] = T(0);
  for (int i0 = 0; i0 < rho; i0 += FF_CH) {
    const int ni = min(FF_CH, rho - i0);
    for (int o = lane; o < FF_CH * K; o += 32) {
      const int i = o % FF_CH, q = o / FF_CH;
      S.va[i][q] = (i < ni && q < ka) ? Va[(i0 + i) + (int64_t)q * rho] : T(0);
      S.ub[i][q] = (i < ni && q < kb) ? Ub[(i0 + i) + (int64_t)q * rho] : T(0);
    }
    __syncwarp();
    for (int i = 0; i < ni; i++) {
      T x[TQ], y[TC];
#pragma unroll
      for (int u = 0; u < TQ; u++) x[u] = S.va[i][q0 + u];
#pragma unroll
      for (int v = 0; v < TC; v++) y[v] = S.ub[i][c0 + v];
#pragma unroll
      for (int u = 0; u < TQ; u++)
#pragma unroll
        for (int v = 0; v < TC; v++) acc[u][v] += x[u] * y[v];
    }
    __syncwarp();
  }
#pragma unroll
  for (int u = 0; u < TQ; u++)
#pragma unroll
    for (int v = 0; v < TC; v++) S.M[q0 + u][c0 + v] = acc[u][v];
  __syncwarp();
  T *out = terms + jb.out;
  const int rows = (int)jb.rows;
  if (jb.type == JOB_FF_L) {  // out (rows x kb) = U_a M
    for (int i = lane; i < rows; i += 32) {
      T o[K];
#pragma unroll
      for (int c = 0; c < K; c++) o[c] = T(0);
      for (int q = 0; q < ka; q++) {
        const T u = Ua[i + (int64_t)q * rows];
#pragma unroll
        for (int c = 0; c < K; c++) o[c] += u * S.M[q][c];
      }
#pragma unroll
      for (int c = 0; c < K; c++)
        if (c < kb) out[i + (int64_t)c * rows] = o[c];
    }
  } else {  // FF_R: out (rows x ka) = V_b M^T
    for (int i = lane; i < rows; i += 32) {
      T o[K];
#pragma unroll
      for (int q = 0; q < K; q++) o[q] = T(0);
      for (int c = 0; c < kb; c++) {
        const T v = Vb[i + (int64_t)c * rows];
#pragma unroll
        for (int q = 0; q < K; q++) o[q] += v * S.M[q][c];
      }
#pragma unroll
      for (int q = 0; q < K; q++)
        if (q < ka) out[i + (int64_t)q * rows] = o[q];
    }
  }
}

template <typename T, int K>
static cudaError_t launch_ff_bucket(const TermJob *jobs, const int32_t *ids, int n, const LeafDev *leafA,
                                    const LeafDev *leafB, const void *dataA, const void *dataB, void *terms,
                                    cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const size_t sm = sizeof(FfSmem<T, K>) * (NT / 32);
  cudaError_t e;
  if ((e = set_smem(k_ff_warp<T, K>, sm)) != cudaSuccess) return e;
  k_ff_warp<T, K><<<(n + NT / 32 - 1) / (NT / 32), NT, sm, s>>>(jobs, ids, n, leafA, leafB, (const T *)dataA,
                                                               (const T *)dataB, (T *)terms);
  return cudaGetLastError();
}

cudaError_t launch_ff_warp(int prec, const TermJob *jobs, const int32_t *ids, const int *nbucket,
                           const LeafDev *leafA, const LeafDev *leafB, const void *dataA, const void *dataB,
                           void *terms, cudaStream_t s) {
  cudaError_t e;
  const int n8 = nbucket[0], n16 = nbucket[1], n32 = nbucket[2];
  if (prec == 64) {
    if ((e = launch_ff_bucket<double, 8>(jobs, ids, n8, leafA, leafB, dataA, dataB, terms, s))) return e;
    if ((e = launch_ff_bucket<double, 16>(jobs, ids + n8, n16, leafA, leafB, dataA, dataB, terms, s))) return e;
    return launch_ff_bucket<double, 32>(jobs, ids + n8 + n16, n32, leafA, leafB, dataA, dataB, terms, s);
  }
  if ((e = launch_ff_bucket<float, 8>(jobs, ids, n8, leafA, leafB, dataA, dataB, terms, s))) return e;
  if ((e = launch_ff_bucket<float, 16>(jobs, ids + n8, n16, leafA, leafB, dataA, dataB, terms, s))) return e;
  return launch_ff_bucket<float, 32>(jobs, ids + n8 + n16, n32, leafA, leafB, dataA, dataB, terms, s);
}

cudaError_t launch_term_jobs(int prec, const TermJob *jobs, const int32_t *ids, int njobs, const LeafDev *leafA,
                             const LeafDev *leafB, const BlockDev *blocks, const void *dataA, const void *dataB,
                             void *terms, cudaStream_t s) {
  if (njobs == 0) return cudaSuccess;
  cudaError_t e;
  if (prec == 64) {
    const size_t sm = Smem::bytes<double>();
    if ((e = set_smem(k_term_jobs<double>, sm)) != cudaSuccess) return e;
    k_term_jobs<double><<<njobs, NT, sm, s>>>(jobs, ids, leafA, leafB, blocks, (const double *)dataA,
                                              (const double *)dataB, (double *)terms);
  } else {
    const size_t sm = Smem::bytes<float>();
    if ((e = set_smem(k_term_jobs<float>, sm)) != cudaSuccess) return e;
    k_term_jobs<float><<<njobs, NT, sm, s>>>(jobs, ids, leafA, leafB, blocks, (const float *)dataA,
                                             (const float *)dataB, (float *)terms);
  }
  return cudaGetLastError();
}


// TermDev of every low-rank product from its job: the created block gives the origin and the
// leading dimensions; one factor is a stored factor of A or B, the other the new one.
template <typename T>
__global__ void k_make_terms(const TermJob *jobs, int njobs, const BlockDev *blocks, const LeafDev *leafA,
                             const LeafDev *leafB, const T *dataA, const T *dataB, const T *termbuf, TermDev *terms) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= njobs) return;
  const TermJob jb = jobs[i];
  if (jb.type < 0) return;  // a term another group of the product builds
  const BlockDev bk = blocks[jb.blk];
  TermDev d;
  d.row0 = bk.row;
  d.col0 = bk.col;
  d.ldL = bk.m;
  d.ldR = bk.n;
  d.rank = jb.rank;
  d.pad = 0;
  if (jb.type == JOB_FF_R || jb.type == JOB_FH) {
    d.L = dataA + leafA[jb.a].off_u;
    d.R = termbuf + jb.out;
  } else {
    d.L = termbuf + jb.out;
    d.R = dataB + leafB[jb.b].off_v;
  }
  terms[i] = d;
}

cudaError_t launch_make_terms(int prec, const TermJob *jobs, int njobs, const BlockDev *blocks, const LeafDev *leafA,
                              const LeafDev *leafB, const void *dataA, const void *dataB, const void *termbuf,
                              TermDev *terms, cudaStream_t s) {
  if (njobs == 0) return cudaSuccess;
  const int g = (njobs + 255) / 256;
  if (prec == 64)
    k_make_terms<double><<<g, 256, 0, s>>>(jobs, njobs, blocks, leafA, leafB, (const double *)dataA,
                                           (const double *)dataB, (const double *)termbuf, terms);
  else
    k_make_terms<float><<<g, 256, 0, s>>>(jobs, njobs, blocks, leafA, leafB, (const float *)dataA,
                                          (const float *)dataB, (const float *)termbuf, terms);
  return cudaGetLastError();
}

cudaError_t launch_near_eval(int prec, const TargetDev *tg, int ntg, const int2 *blk_terms, const TermDev *terms,
                             const PairDev *pairs, const BlockDev *blocks, const LeafDev *leafA,
                             const LeafDev *leafB, const void *dataA, const void *dataB, const LeafDev *leafC,
                             void *dataC, int *err, cudaStream_t s) {
  if (ntg == 0) return cudaSuccess;
  if (prec != 64)
    return launch_near_tc(tg, ntg, blk_terms, terms, pairs, blocks, leafA, leafB, (const float *)dataA,
                          (const float *)dataB, leafC, (float *)dataC, err, s);
  k_near_eval<double><<<ntg, NT, 0, s>>>(tg, blk_terms, terms, pairs, blocks, leafA, leafB, (const double *)dataA,
                                         (const double *)dataB, leafC, (double *)dataC);
  return cudaGetLastError();
}

cudaError_t launch_gaussian(int prec, const TargetDev *tg, const TargetState *st, int ntg, int p, uint64_t seed,
                            int round, void *x_base, cudaStream_t s) {
  if (ntg == 0) return cudaSuccess;
  if (prec == 64) k_gaussian<double><<<ntg, NT, 0, s>>>(tg, st, p, seed, round, (double *)x_base);
  else k_gaussian<float><<<ntg, NT, 0, s>>>(tg, st, p, seed, round, (float *)x_base);
  return cudaGetLastError();
}

cudaError_t launch_orth(int prec, const TargetDev *tg, const int32_t *ids_warp, int n_warp, const int32_t *ids_block,
                        int n_block, TargetState *st, int p, double eps, void *y_base, double *qw, void *x_base,
                        int round, cudaStream_t s, int side, int fresh) {
  if (p > OW) return cudaErrorInvalidValue;
  const int gw = (n_warp + NT / 32 - 1) / (NT / 32);
  if (prec == 64) {
    if (n_warp)
      k_orth_warp<double><<<gw, NT, 0, s>>>(tg, ids_warp, n_warp, st, p, eps, (const double *)y_base, qw,
                                            (double *)x_base, round, side, fresh);
    if (n_block)
      k_orth<double><<<n_block, NT, 0, s>>>(tg, ids_block, st, p, eps, (const double *)y_base, qw, (double *)x_base,
                                            round, side, fresh);
  } else {
    if (n_warp)
      k_orth_warp<float><<<gw, NT, 0, s>>>(tg, ids_warp, n_warp, st, p, eps, (const float *)y_base, qw,
                                           (float *)x_base, round, side, fresh);
    if (n_block)
      k_orth<float><<<n_block, NT, 0, s>>>(tg, ids_block, st, p, eps, (const float *)y_base, qw, (float *)x_base,
                                           round, side, fresh);
  }
  return cudaGetLastError();
}

cudaError_t launch_absorb_w(int prec, const TargetDev *tg, TargetState *st, int ntg, int p, double eps_stop,
                            void *y_base, double *qw, int round, int max_rounds, int32_t *active_count,
                            cudaStream_t s, int fixed) {
  if (ntg == 0) return cudaSuccess;
  if (prec == 64)
    k_absorb_w<double><<<ntg, NT, 0, s>>>(tg, st, p, eps_stop, (const double *)y_base, qw, round, max_rounds,
                                          active_count, fixed);
  else
    k_absorb_w<float><<<ntg, NT, 0, s>>>(tg, st, p, eps_stop, (const float *)y_base, qw, round, max_rounds,
                                         active_count, fixed);
  return cudaGetLastError();
}

cudaError_t launch_aca_start(int prec, const TargetDev *tg, TargetState *st, int ntg, double *qw, void *x_base,
                             cudaStream_t s) {
  if (ntg == 0) return cudaSuccess;
  if (prec == 64) k_aca_start<double><<<ntg, NT, 0, s>>>(tg, st, qw, (double *)x_base);
  else k_aca_start<float><<<ntg, NT, 0, s>>>(tg, st, qw, (float *)x_base);
  return cudaGetLastError();
}

cudaError_t launch_aca_row(int prec, const TargetDev *tg, TargetState *st, int ntg, const void *y_base, double *qw,
                           void *x_base, cudaStream_t s) {
  if (ntg == 0) return cudaSuccess;
  if (prec == 64) k_aca_row<double><<<ntg, NT, 0, s>>>(tg, st, (const double *)y_base, qw, (double *)x_base);
  else k_aca_row<float><<<ntg, NT, 0, s>>>(tg, st, (const float *)y_base, qw, (float *)x_base);
  return cudaGetLastError();
}

cudaError_t launch_aca_col(int prec, const TargetDev *tg, TargetState *st, int ntg, const void *y_base, double *qw,
                           void *x_base, double eps_stop, int32_t *active_count, cudaStream_t s) {
  if (ntg == 0) return cudaSuccess;
  if (prec == 64)
    k_aca_col<double><<<ntg, NT, 0, s>>>(tg, st, (const double *)y_base, qw, (double *)x_base, eps_stop,
                                         active_count);
  else
    k_aca_col<float><<<ntg, NT, 0, s>>>(tg, st, (const float *)y_base, qw, (float *)x_base, eps_stop, active_count);
  return cudaGetLastError();
}

cudaError_t launch_lz_start(int prec, const TargetDev *tg, TargetState *st, int ntg, double *qw, void *x_base,
                            uint64_t seed, cudaStream_t s) {
  if (ntg == 0) return cudaSuccess;
  if (prec == 64) k_lz_start<double><<<ntg, NT, 0, s>>>(tg, st, qw, (double *)x_base, seed);
  else k_lz_start<float><<<ntg, NT, 0, s>>>(tg, st, qw, (float *)x_base, seed);
  return cudaGetLastError();
}

cudaError_t launch_lz_q(int prec, const TargetDev *tg, TargetState *st, int ntg, const void *y_base, double *qw,
                        void *x_base, cudaStream_t s) {
  if (ntg == 0) return cudaSuccess;
  if (prec == 64) k_lz_q<double><<<ntg, NT, 0, s>>>(tg, st, (const double *)y_base, qw, (double *)x_base);
  else k_lz_q<float><<<ntg, NT, 0, s>>>(tg, st, (const float *)y_base, qw, (float *)x_base);
  return cudaGetLastError();
}

cudaError_t launch_lz_w(int prec, const TargetDev *tg, TargetState *st, int ntg, const void *y_base, double *qw,
                        void *x_base, double eps_stop, int32_t *active_count, cudaStream_t s) {
  if (ntg == 0) return cudaSuccess;
  if (prec == 64)
    k_lz_w<double><<<ntg, NT, 0, s>>>(tg, st, (const double *)y_base, qw, (double *)x_base, eps_stop, active_count);
  else
    k_lz_w<float><<<ntg, NT, 0, s>>>(tg, st, (const float *)y_base, qw, (float *)x_base, eps_stop, active_count);
  return cudaGetLastError();
}

cudaError_t launch_lz_load(int prec, const TargetDev *tg, TargetState *st, int ntg, const double *qw, void *x_base,
                           int c0, int p, cudaStream_t s) {
  if (ntg == 0) return cudaSuccess;
  if (prec == 64) k_lz_load<double><<<ntg, NT, 0, s>>>(tg, st, qw, (double *)x_base, c0, p);
  else k_lz_load<float><<<ntg, NT, 0, s>>>(tg, st, qw, (float *)x_base, c0, p);
  return cudaGetLastError();
}

cudaError_t launch_lz_store(int prec, const TargetDev *tg, const TargetState *st, int ntg, const void *y_base,
                            double *qw, int c0, int p, cudaStream_t s) {
  if (ntg == 0) return cudaSuccess;
  if (prec == 64) k_lz_store<double><<<ntg, NT, 0, s>>>(tg, st, (const double *)y_base, qw, c0, p);
  else k_lz_store<float><<<ntg, NT, 0, s>>>(tg, st, (const float *)y_base, qw, c0, p);
  return cudaGetLastError();
}

cudaError_t launch_aca_qr(const TargetDev *tg, const TargetState *st, int ntg, double *qw, cudaStream_t s) {
  if (ntg == 0) return cudaSuccess;
  const size_t sm = sizeof(double) * (JMAX - 1) * (JMAX - 1);
  cudaError_t e;
  if ((e = set_smem(k_aca_qr, sm)) != cudaSuccess) return e;
  k_aca_qr<<<ntg, NT, sm, s>>>(tg, st, qw);
  return cudaGetLastError();
}

cudaError_t launch_final(const TargetDev *tg, TargetState *st, const int32_t *ids, int nids, bool warp_kernel,
                         double eps, double *qw, cudaStream_t s) {
  if (nids == 0) return cudaSuccess;
  cudaError_t e;
  if (warp_kernel) {
    const size_t sm = sizeof(WarpFinalSmem) * WF_WARPS;
    if ((e = set_smem(k_final_warp, sm)) != cudaSuccess) return e;
    k_final_warp<<<(nids + WF_WARPS - 1) / WF_WARPS, WF_WARPS * 32, sm, s>>>(tg, st, ids, nids, eps, qw);
  } else {
    const size_t sm = sizeof(double) * (2 * JMAX * JMAX + JMAX) + sizeof(int) * 2 * JMAX;
    if ((e = set_smem(k_final, sm)) != cudaSuccess) return e;
    k_final<<<nids, NT, sm, s>>>(tg, st, ids, eps, qw);
  }
  return cudaGetLastError();
}

cudaError_t launch_write_far(int prec, const TargetDev *tg, const TargetState *st, int ntg, const double *qw,
                             const LeafDev *leafC, void *dataC, cudaStream_t s) {
  if (ntg == 0) return cudaSuccess;
  if (prec == 64)
    k_write_far<double><<<ntg, NT, 0, s>>>(tg, st, qw, leafC, (double *)dataC);
  else
    k_write_far<float><<<ntg, NT, 0, s>>>(tg, st, qw, leafC, (float *)dataC);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// The global error estimator (Sec. 6): a block of `size` columns as ceil(size / 16) row-major
// panels of 16 columns (row stride 17, the layout of the H-matrix times panel kernel), n rows in
// tree order; column c is slot c % 16 of panel c / 16.
// ---------------------------------------------------------------------------------------
constexpr int EP = 16, ESP = 17;
__device__ __forceinline__ int64_t est_at(int64_t n, int64_t i, int c) {
  return (int64_t)(c / EP) * n * ESP + i * ESP + (c % EP);
}

__device__ __forceinline__ uint64_t est_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Gaussian start block: entry (i, c), k = i + c n, from two splitmix64 draws of the counters
// 2k + 1 and 2k + 2 (uniforms in (0, 1] and [0, 1)) by Box-Muller; padding slots zero
__global__ void k_est_gaussian(double *X, int64_t n, int size, uint64_t seed) {
  const int npan = (size + EP - 1) / EP;
  const int64_t total = (int64_t)npan * n * ESP;
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < total; o += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = o / (n * ESP), r = o % (n * ESP);
    const int64_t i = r / ESP;
    const int c = (int)(p * EP + r % ESP);
    double v = 0.0;
    if (r % ESP < EP && c < size) {
      const uint64_t k = (uint64_t)i + (uint64_t)c * (uint64_t)n;
      const double u1 = (double)((est_mix(seed + (2 * k + 1) * 0x9E3779B97F4A7C15ull) >> 11) + 1) * 0x1.0p-53;
      const double u2 = (double)(est_mix(seed + (2 * k + 2) * 0x9E3779B97F4A7C15ull) >> 11) * 0x1.0p-53;
      v = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
    }
    X[o] = v;
  }
}

// Y -= Z over count entries
__global__ void k_est_sub(double *Y, const double *Z, int64_t count) {
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < count; o += (int64_t)gridDim.x * blockDim.x)
    Y[o] -= Z[o];
}

// G (size x size, upper triangle, zeroed beforehand) += X^T X over the rows of this block's chunk
constexpr int EST_ROWS = 16;
__global__ void __launch_bounds__(NT) k_est_gram(const double *X, int64_t n, int size, double *G) {
  __shared__ double xs[EST_ROWS][128];
  const int npairs = size * (size + 1) / 2;
  constexpr int PER = 128 * 129 / 2 / NT + 1;  // pairs per thread for size <= 128
  double acc[PER];
  int16_t pa[PER], pb[PER];  // this thread's pairs (a <= b), row-major over the upper triangle
#pragma unroll
  for (int j = 0; j < PER; j++) {
    acc[j] = 0.0;
    const int e = threadIdx.x + j * NT;
    int a = 0, rem = e;
    if (e < npairs)
      while (rem >= size - a) { rem -= size - a; a++; }
    pa[j] = (int16_t)(e < npairs ? a : -1);
    pb[j] = (int16_t)(e < npairs ? a + rem : -1);
  }
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t i0 = blockIdx.x * chunk, i1 = min(n, i0 + chunk);
  for (int64_t ib = i0; ib < i1; ib += EST_ROWS) {
    const int nr = (int)(i1 - ib < EST_ROWS ? i1 - ib : EST_ROWS);
    __syncthreads();
    for (int o = threadIdx.x; o < EST_ROWS * size; o += NT) {
      const int r = o / size, c = o % size;
      xs[r][c] = r < nr ? X[est_at(n, ib + r, c)] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < PER; j++) {
      if (pa[j] >= 0) {
        const int a = pa[j], b = pb[j];
        double sum = 0.0;
#pragma unroll
        for (int r = 0; r < EST_ROWS; r++) sum += xs[r][a] * xs[r][b];
        acc[j] += sum;
      }
    }
  }
#pragma unroll
  for (int j = 0; j < PER; j++)
    if (pa[j] >= 0) atomicAdd(&G[pa[j] + (int64_t)pb[j] * size], acc[j]);
}

// Cholesky G + 1e-15 trace I = R^T R in place (upper R), one block; a zero Gram sets *zero = 1 and
// leaves R = I (the block is then zero and stays zero)
__global__ void __launch_bounds__(NT) k_est_chol(double *G, int size, int *zero) {
  __shared__ double tr_s;
  if (threadIdx.x == 0) {
    double tr = 0.0;
    for (int a = 0; a < size; a++) tr += G[a + (int64_t)a * size];
    tr_s = tr;
  }
  __syncthreads();
  const double tr = tr_s;
  if (!(tr > 0.0)) {
    for (int o = threadIdx.x; o < size * size; o += NT) G[o] = (o % size == o / size) ? 1.0 : 0.0;
    if (threadIdx.x == 0) *zero = 1;
    return;
  }
  for (int a = threadIdx.x; a < size; a += NT) G[a + (int64_t)a * size] += 1e-15 * tr;
  __syncthreads();
  for (int k = 0; k < size; k++) {
    if (threadIdx.x == 0) G[k + (int64_t)k * size] = sqrt(fmax(G[k + (int64_t)k * size], 1e-300));
    __syncthreads();
    const double rkk = G[k + (int64_t)k * size];
    for (int j = k + 1 + threadIdx.x; j < size; j += NT) G[k + (int64_t)j * size] /= rkk;
    __syncthreads();
    const int m = size - k - 1;
    for (int o = threadIdx.x; o < m * m; o += NT) {
      const int i = k + 1 + o % m, j = k + 1 + o / m;
      if (i <= j) G[i + (int64_t)j * size] -= G[k + (int64_t)i * size] * G[k + (int64_t)j * size];
    }
    __syncthreads();
  }
}

// X <- X R^{-1} row by row (R upper, size x size), one thread per row
__global__ void __launch_bounds__(NT) k_est_trsm(double *X, int64_t n, int size, const double *R) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double row[128];
  for (int j = 0; j < size; j++) {
    double v = X[est_at(n, i, j)];
    for (int k = 0; k < j; k++) v -= row[k] * R[k + (int64_t)j * size];
    row[j] = v / R[j + (int64_t)j * size];
  }
  for (int j = 0; j < size; j++) X[est_at(n, i, j)] = row[j];
}

// *out += sum of squares of the block's entries
__global__ void __launch_bounds__(NT) k_est_norm2(const double *Y, int64_t count, double *out) {
  __shared__ double red[NT / 32];
  double v = 0.0;
  for (int64_t o = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; o < count; o += (int64_t)gridDim.x * blockDim.x)
    v += Y[o] * Y[o];
  v = block_sum(v, red);
  if (threadIdx.x == 0) atomicAdd(out, v);
}

cudaError_t launch_est_gaussian(double *X, int64_t n, int size, uint64_t seed, cudaStream_t s) {
  k_est_gaussian<<<152 * 8, NT, 0, s>>>(X, n, size, seed);
  return cudaGetLastError();
}
cudaError_t launch_est_sub(double *Y, const double *Z, int64_t count, cudaStream_t s) {
  k_est_sub<<<152 * 8, NT, 0, s>>>(Y, Z, count);
  return cudaGetLastError();
}
// X <- X R^{-1} with X^T X = R^T R, twice (Cholesky QR twice); G is size x size scratch
cudaError_t launch_est_orth(double *X, int64_t n, int size, double *G, int *zero, cudaStream_t s) {
  if (size > 128) return cudaErrorInvalidValue;
  for (int pass = 0; pass < 2; pass++) {
    cudaError_t e = cudaMemsetAsync(G, 0, sizeof(double) * size * size, s);
    if (e != cudaSuccess) return e;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(152 * 4, (n + 255) / 256));
    k_est_gram<<<grid, NT, 0, s>>>(X, n, size, G);
    k_est_chol<<<1, NT, 0, s>>>(G, size, zero);
    k_est_trsm<<<(unsigned)((n + NT - 1) / NT), NT, 0, s>>>(X, n, size, G);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  return cudaSuccess;
}
cudaError_t launch_est_norm2(const double *Y, int64_t count, double *out, cudaStream_t s) {
  k_est_norm2<<<152 * 4, NT, 0, s>>>(Y, count, out);
  return cudaGetLastError();
}

cudaError_t launch_convert(int prec, const void *src, double *dst, int64_t count, cudaStream_t s) {
  if (count == 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((count + NT - 1) / NT, 152 * 16);
  if (prec == 64)
    k_convert<double><<<blocks, NT, 0, s>>>((const double *)src, dst, count);
  else
    k_convert<float><<<blocks, NT, 0, s>>>((const float *)src, dst, count);
  return cudaGetLastError();
}

}  // namespace hm
