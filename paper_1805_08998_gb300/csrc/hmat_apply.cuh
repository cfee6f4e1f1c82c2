#pragma once
// hmat_apply.cuh -- the sum-expression application for all far targets (a3: Y = S(b) Omega,
// a6: W = S(b)^T Q), the dominant kernel of the product.
//
// For a target b = tau x sigma with sum-expression S(b) = sum_j L_j R_j^T + sum_rho A|tau x rho
// B|rho x sigma (Sec. 3.3: S v = sum A_j (B_j^T v) + sum H_j (K_j v)), one thread block applies
// every term of b to the p sample columns:
//   * the input panel (Omega or Q, p columns padded to P) and the output panel are staged
//     row-major in shared memory (or, for very large targets, in a global staging area);
//   * each warp takes whole low-rank terms: c = R^T X by lane-per-column reductions into a
//     private scratch, then Out += L c by lane-per-row expansions accumulated with atomics;
//   * H-pairs of two dense leaves (the leaf level) are taken warp per pair, the intermediate
//     B|rho x sigma X kept in the warp's scratch;
//   * H-pairs of inner blocks walk their two subtrees (Algorithm 2), leaves split over warps,
//     with one block barrier between the B side and the A side.
// No block barrier separates two terms, so warps stream the factor data independently.
#include <cstdint>
#include <cuda_runtime.h>

#include "hmat_internal.h"

namespace hm {
namespace apply_detail {

constexpr int AT = 256;
constexpr int NWARP = AT / 32;

template <typename T>
__device__ __forceinline__ void acc_add(T *p, T v, bool atomic) {
  if (atomic) atomicAdd(p, v);
  else *p = v;
}

// out[q*osr + c*osc] (+)= sum_{i < len} M[i + q*ldm] * X[i*SP + c]  for q < r, c < P (only
// c < ncol stored; SP = the panel's row stride). With r <= 32/G, G lanes share column q (rows split
// round-robin) and are combined by shuffles, so narrow ranks still use the whole warp. Default
// strides: row-major panel (osr = SP, osc = 1).
template <typename T, int P, int G, bool ATOMIC, int SP>
__device__ __forceinline__ void warp_tn_g(T *out, const T *__restrict__ M, int64_t ldm, const T *X, int len, int r,
                                          int64_t osr, int64_t osc, int ncol) {
  const int lane = threadIdx.x & 31;
  constexpr int COLS = 32 / G;
  const int g = lane % G;
  for (int q0 = 0; q0 < r; q0 += COLS) {
    const int q = q0 + lane / G;
    T acc[P];
#pragma unroll
    for (int c = 0; c < P; c++) acc[c] = T(0);
    if (q < r) {
      const T *mc = M + (int64_t)q * ldm;
      int i = g;
      for (; i + 7 * G < len; i += 8 * G) {  // eight independent loads in flight per lane
        T mv[8];
#pragma unroll
        for (int u = 0; u < 8; u++) mv[u] = __ldg(mc + i + u * G);
        const T *x = X + i * SP;
#pragma unroll
        for (int c = 0; c < P; c++) {
          T s = acc[c];
#pragma unroll
          for (int u = 0; u < 8; u++) s += mv[u] * x[u * G * SP + c];
          acc[c] = s;
        }
      }
      for (; i + 3 * G < len; i += 4 * G) {
        const T m0 = __ldg(mc + i), m1 = __ldg(mc + i + G), m2 = __ldg(mc + i + 2 * G), m3 = __ldg(mc + i + 3 * G);
        const T *x = X + i * SP;
#pragma unroll
        for (int c = 0; c < P; c++) {
          T s = acc[c];
          s += m0 * x[c];
          s += m1 * x[G * SP + c];
          s += m2 * x[2 * G * SP + c];
          s += m3 * x[3 * G * SP + c];
          acc[c] = s;
        }
      }
      for (; i < len; i += G) {
        const T m0 = __ldg(mc + i);
#pragma unroll
        for (int c = 0; c < P; c++) acc[c] += m0 * X[i * SP + c];
      }
    }
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1)
#pragma unroll
      for (int c = 0; c < P; c++) acc[c] += __shfl_down_sync(0xffffffffu, acc[c], off, G);
    if (q < r && g == 0) {
#pragma unroll
      for (int c = 0; c < P; c++)
        if (c < ncol) acc_add(out + q * osr + c * osc, acc[c], ATOMIC);
    }
  }
}

template <typename T, int P, bool ATOMIC, int SP>
__device__ __forceinline__ void warp_tn(T *out, const T *__restrict__ M, int64_t ldm, const T *X, int len, int r,
                                        int64_t osr = SP, int64_t osc = 1, int ncol = P) {
  if (r <= 4) warp_tn_g<T, P, 8, ATOMIC, SP>(out, M, ldm, X, len, r, osr, osc, ncol);
  else if (r <= 8) warp_tn_g<T, P, 4, ATOMIC, SP>(out, M, ldm, X, len, r, osr, osc, ncol);
  else if (r <= 16) warp_tn_g<T, P, 2, ATOMIC, SP>(out, M, ldm, X, len, r, osr, osc, ncol);
  else warp_tn_g<T, P, 1, ATOMIC, SP>(out, M, ldm, X, len, r, osr, osc, ncol);
}

// out[i*osr + c*osc] (+)= sum_{q < r} M[i + q*ldm] * C[q*SP + c]  for i < rows; lane owns rows.
template <typename T, int P, bool ATOMIC, int SP>
__device__ __forceinline__ void warp_nn(T *out, const T *__restrict__ M, int64_t ldm, const T *C, int rows, int r,
                                        int64_t osr = SP, int64_t osc = 1, int ncol = P) {
  const int lane = threadIdx.x & 31;
  for (int i0 = 0; i0 < rows; i0 += 64) {
    const int ia = i0 + lane, ib = i0 + 32 + lane;
    const bool va = ia < rows, vb = ib < rows;
    T a[P], b[P];
#pragma unroll
    for (int c = 0; c < P; c++) { a[c] = T(0); b[c] = T(0); }
    int q = 0;
    for (; q + 4 <= r; q += 4) {  // eight independent loads in flight per lane
      T xv[4], yv[4];
#pragma unroll
      for (int u = 0; u < 4; u++) {
        const T *mu = M + (int64_t)(q + u) * ldm;
        xv[u] = va ? __ldg(mu + ia) : T(0);
        yv[u] = vb ? __ldg(mu + ib) : T(0);
      }
      const T *c0 = C + q * SP;
#pragma unroll
      for (int c = 0; c < P; c++) {
#pragma unroll
        for (int u = 0; u < 4; u++) {
          const T cv = c0[u * SP + c];
          a[c] += xv[u] * cv;
          b[c] += yv[u] * cv;
        }
      }
    }
    for (; q + 2 <= r; q += 2) {
      const T *m0 = M + (int64_t)q * ldm, *m1 = m0 + ldm;
      const T x0 = va ? __ldg(m0 + ia) : T(0), y0 = vb ? __ldg(m0 + ib) : T(0);
      const T x1 = va ? __ldg(m1 + ia) : T(0), y1 = vb ? __ldg(m1 + ib) : T(0);
      const T *c0 = C + q * SP;
#pragma unroll
      for (int c = 0; c < P; c++) {
        const T u = c0[c], v = c0[SP + c];
        a[c] += x0 * u;
        b[c] += y0 * u;
        a[c] += x1 * v;
        b[c] += y1 * v;
      }
    }
    if (q < r) {
      const T *m0 = M + (int64_t)q * ldm;
      const T x0 = va ? __ldg(m0 + ia) : T(0), y0 = vb ? __ldg(m0 + ib) : T(0);
#pragma unroll
      for (int c = 0; c < P; c++) {
        a[c] += x0 * C[q * SP + c];
        b[c] += y0 * C[q * SP + c];
      }
    }
    if (va)
#pragma unroll
      for (int c = 0; c < P; c++)
        if (c < ncol) acc_add(out + ia * osr + c * osc, a[c], ATOMIC);
    if (vb)
#pragma unroll
      for (int c = 0; c < P; c++)
        if (c < ncol) acc_add(out + ib * osr + c * osc, b[c], ATOMIC);
  }
}

// Sum over the warp of the P per-lane values v[0..P) (P in {8, 16}), halving the values each
// lane carries at every exchange: returns, in every lane, the total of column
// c = (lane >> (5 - log2 P)) & (P - 1); 32 / P consecutive lanes hold the same column.
template <typename T, int P>
__device__ __forceinline__ T warp_reduce_scatter(T (&v)[P], int lane) {
  static_assert(P == 8 || P == 16, "panel width");
  int off = 16;
#pragma unroll
  for (int h = P / 2; h >= 1; h /= 2) {
    const bool hi = (lane & off) != 0;
#pragma unroll
    for (int k = 0; k < h; k++) {
      const T send = hi ? v[k] : v[k + h];
      const T keep = hi ? v[k + h] : v[k];
      v[k] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
    off >>= 1;
  }
  T s = v[0];
#pragma unroll
  for (int o = P == 8 ? 2 : 1; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// cw[q*SP + c] = sum_{i < len} M[i + q*ldm] * X[i][c] for q < r, with the panel X held in
// registers (xr[u][c] = X[lane + 32 u][c], zero beyond len): lanes run along the rows, so every
// load of a column of M is one coalesced request, and each column's P sums are combined by
// warp_reduce_scatter. Columns are taken four at a time to keep several loads in flight.
template <typename T, int P, int RB, int SP>
__device__ __forceinline__ void warp_tn_reg(T *cw, const T *__restrict__ M, int64_t ldm, const T (&xr)[RB][P], int len,
                                            int r) {
  const int lane = threadIdx.x & 31;
  constexpr int LPC = 32 / P;  // lanes holding one column after the reduction
  const int col = (lane / LPC) & (P - 1);
  int q = 0;
  for (; q + 4 <= r; q += 4) {
    T mv[4][RB];
#pragma unroll
    for (int w = 0; w < 4; w++)
#pragma unroll
      for (int u = 0; u < RB; u++) {
        const int i = lane + 32 * u;
        mv[w][u] = i < len ? __ldg(M + (int64_t)(q + w) * ldm + i) : T(0);
      }
#pragma unroll
    for (int w = 0; w < 4; w++) {
      T part[P];
#pragma unroll
      for (int c = 0; c < P; c++) {
        T a = T(0);
#pragma unroll
        for (int u = 0; u < RB; u++) a += mv[w][u] * xr[u][c];
        part[c] = a;
      }
      const T sum = warp_reduce_scatter<T, P>(part, lane);
      if ((lane & (LPC - 1)) == 0) cw[(q + w) * SP + col] = sum;
    }
  }
  for (; q < r; q++) {
    T mv[RB];
#pragma unroll
    for (int u = 0; u < RB; u++) {
      const int i = lane + 32 * u;
      mv[u] = i < len ? __ldg(M + (int64_t)q * ldm + i) : T(0);
    }
    T part[P];
#pragma unroll
    for (int c = 0; c < P; c++) {
      T a = T(0);
#pragma unroll
      for (int u = 0; u < RB; u++) a += mv[u] * xr[u][c];
      part[c] = a;
    }
    const T sum = warp_reduce_scatter<T, P>(part, lane);
    if ((lane & (LPC - 1)) == 0) cw[q * SP + col] = sum;
  }
}

// The same reduction for a panel X of any height kept row-major in shared memory (row stride SP):
// lanes run along the rows (coalesced loads of M), four columns of M share each X row read, and
// each column's P sums are combined by warp_reduce_scatter.
template <typename T, int P, int SP, bool ATOMIC = false>
__device__ __forceinline__ void warp_tn_rows(T *cw, const T *__restrict__ M, int64_t ldm, const T *X, int len,
                                             int r) {
  const int lane = threadIdx.x & 31;
  constexpr int LPC = 32 / P;
  const int col = (lane / LPC) & (P - 1);
  for (int q = 0; q < r; q += 4) {
    const int nq = min(4, r - q);
    T acc[4][P];
#pragma unroll
    for (int w = 0; w < 4; w++)
#pragma unroll
      for (int c = 0; c < P; c++) acc[w][c] = T(0);
#pragma unroll 2
    for (int i = lane; i < len; i += 32) {
      T mv[4];
#pragma unroll
      for (int w = 0; w < 4; w++) mv[w] = w < nq ? __ldg(M + (int64_t)(q + w) * ldm + i) : T(0);
      const T *x = X + i * SP;
#pragma unroll
      for (int c = 0; c < P; c++) {
        const T xv = x[c];
#pragma unroll
        for (int w = 0; w < 4; w++) acc[w][c] += mv[w] * xv;
      }
    }
#pragma unroll
    for (int w = 0; w < 4; w++) {
      if (w >= nq) break;
      const T sum = warp_reduce_scatter<T, P>(acc[w], lane);
      if ((lane & (LPC - 1)) == 0) acc_add(cw + (q + w) * SP + col, sum, ATOMIC);
    }
  }
}

// M^T X into out (rows q of out, stride SP): in FP32 by lanes along the rows (warp_tn_rows) for
// long columns or wide panels, otherwise by lane groups per column (warp_tn): for short columns
// of 8-wide panels the per-column exchange of warp_tn_rows costs more than its coalescing saves.
template <typename T, int P, int SP, bool ATOMIC>
__device__ __forceinline__ void warp_tn_any(T *out, const T *__restrict__ M, int64_t ldm, const T *X, int len,
                                            int r) {
  // FP64: the lane-group form throughout (the FP64 pipe, not the load path, bounds it)
  if (sizeof(T) == 4 && (P >= 16 || len >= 128)) warp_tn_rows<T, P, SP, ATOMIC>(out, M, ldm, X, len, r);
  else warp_tn<T, P, ATOMIC, SP>(out, M, ldm, X, len, r);
}

// One leaf of an H-matrix block with origin (row0, col0):
//   trans = false: Out[rows of leaf] += leaf   * X[cols of leaf]
//   trans = true:  Out[cols of leaf] += leaf^T * X[rows of leaf]
template <typename T, int P, int SP>
__device__ __forceinline__ void warp_leaf(const LeafDev &lf, const T *data, bool trans, int64_t row0, int64_t col0,
                                          const T *X, T *Out, T *cw) {
  const int ro = (int)(lf.row - row0), co = (int)(lf.col - col0);
  if (lf.rank < 0) {
    const T *D = data + lf.off_u;
    if (!trans) warp_nn<T, P, true, SP>(Out + ro * SP, D, lf.m, X + co * SP, lf.m, lf.n);
    else warp_tn_any<T, P, SP, true>(Out + co * SP, D, lf.m, X + ro * SP, lf.m, lf.n);
  } else if (lf.rank > 0) {
    const T *U = data + lf.off_u, *V = data + lf.off_v;
    if (!trans) {
      warp_tn_any<T, P, SP, false>(cw, V, lf.n, X + co * SP, lf.n, lf.rank);
      __syncwarp();
      warp_nn<T, P, true, SP>(Out + ro * SP, U, lf.m, cw, lf.m, lf.rank);
    } else {
      warp_tn_any<T, P, SP, false>(cw, U, lf.m, X + ro * SP, lf.m, lf.rank);
      __syncwarp();
      warp_nn<T, P, true, SP>(Out + co * SP, V, lf.n, cw, lf.n, lf.rank);
    }
    __syncwarp();
  }
}

// acc[rr][c] += sum_{q < r} M[lane + 32 rr + q*ldm] * C[q*SP + c], rows < rows (lane owns rows)
template <typename T, int P, int RB, int SP>
__device__ __forceinline__ void warp_nn_reg(T (&acc)[RB][P], const T *__restrict__ M, int64_t ldm, const T *C, int rows,
                                            int r) {
  const int lane = threadIdx.x & 31;
  int q = 0;
  for (; q + 2 <= r; q += 2) {  // 2 RB independent loads in flight per lane
    const T *mq = M + (int64_t)q * ldm;
    T mv[2][RB];
#pragma unroll
    for (int u = 0; u < 2; u++)
#pragma unroll
      for (int rr = 0; rr < RB; rr++) {
        const int i = lane + 32 * rr;
        mv[u][rr] = i < rows ? __ldg(mq + u * ldm + i) : T(0);
      }
    const T *cq = C + q * SP;
#pragma unroll
    for (int c = 0; c < P; c++) {
      const T c0 = cq[c], c1 = cq[SP + c];
#pragma unroll
      for (int rr = 0; rr < RB; rr++) acc[rr][c] += mv[0][rr] * c0 + mv[1][rr] * c1;
    }
  }
  for (; q < r; q++) {
    const T *mq = M + (int64_t)q * ldm;
    T mv[RB];
#pragma unroll
    for (int rr = 0; rr < RB; rr++) {
      const int i = lane + 32 * rr;
      mv[rr] = i < rows ? __ldg(mq + i) : T(0);
    }
    const T *cq = C + q * SP;
#pragma unroll
    for (int c = 0; c < P; c++) {
      const T cv = cq[c];
#pragma unroll
      for (int rr = 0; rr < RB; rr++) acc[rr][c] += mv[rr] * cv;
    }
  }
}

template <typename T, int P, bool TRANS, bool GSTAGE, int RB>
__global__ void __launch_bounds__(AT) k_apply(ApplyArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  // K thread blocks per target (K > 1 only when RB == 0 and !GSTAGE); block `part` takes every
  // K-th H-pair of inner blocks and, with its warps, every (K NWARP)-th term and leaf pair
  const int K = a.split > 1 ? a.split : 1;
  const int b = a.first + (int)(blockIdx.x / K), part = (int)(blockIdx.x % K);
  if (a.state[b].active == 0) return;  // uniform over the block
  const TargetDev t = a.tg[b];
  const int inlen = TRANS ? t.m : t.n, outlen = TRANS ? t.n : t.m;
  constexpr int SP = apply_row_stride(P);
  T *sm = (T *)smem_raw;
  T *Xs, *Ys, *Zs, *cwall;
  if (GSTAGE) {
    Xs = (T *)a.stage_base + t.stage_off;
    Ys = Xs + (int64_t)inlen * SP;
    Zs = Ys + (int64_t)outlen * SP;
    cwall = sm;
  } else {
    Xs = sm;
    Ys = Xs + a.smem_in * SP;
    Zs = Ys + a.smem_out * SP;  // H-pair intermediate, or (RB > 0) the warps' partial outputs
    cwall = Zs + a.smem_rho * SP;
  }
  const int warp = threadIdx.x >> 5;
  const int vw = part * NWARP + warp, NV = K * NWARP;  // virtual warp over the target's blocks
  T *cw = cwall + warp * a.smem_cw * SP;
  const T *X = (const T *)a.x_base + t.x_off;  // Omega or Q_new, column-major inlen x p
  T *Out = (T *)a.y_base + t.y_off;            // column-major outlen x p
  const int p = a.round == 0 ? t.p0 : a.p;     // this target's columns this round (<= P)
  for (int o = threadIdx.x; o < inlen * P; o += AT) {  // threads along the rows: coalesced reads
    const int c = o / inlen, i = o - c * inlen;
    Xs[i * SP + c] = c < p ? X[i + (int64_t)c * inlen] : T(0);
  }
  for (int o = threadIdx.x; o < outlen * SP; o += AT) Ys[o] = T(0);
  __syncthreads();

  // low-rank terms (those created at the target's block and its ancestors), warp per term.
  // RB > 0 (outputs of at most 32 RB rows): every warp accumulates its terms and leaf pairs in
  // registers and the warps' partial results are summed in a fixed order; RB = 0: shared atomics.
  constexpr int RBX = RB > 0 ? RB : 1;
  T racc[RBX][P];
#pragma unroll
  for (int rr = 0; rr < RBX; rr++)
#pragma unroll
    for (int c = 0; c < P; c++) racc[rr][c] = T(0);
  // FP32 with RB > 0: the input panel is also held in registers, lane owning rows lane + 32 u
  constexpr bool XREG = RB > 0 && sizeof(T) == 4;
  T xr[RBX][P];
  if (XREG) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int u = 0; u < RBX; u++) {
      const int i = lane + 32 * u;
#pragma unroll
      for (int c = 0; c < P; c++) xr[u][c] = i < inlen ? Xs[i * SP + c] : T(0);
    }
  }
  int base = 0;
  for (int blk = t.blk; blk >= 0; blk = a.blocks[blk].parent) {
    const int2 rg = a.blk_terms[blk];
    const int cnt = rg.y - rg.x;
    const int j0 = ((vw - base) % NV + NV) % NV;
    base += cnt;
    for (int j = j0; j < cnt; j += NV) {
      const TermDev tm = a.terms[rg.x + j];
      const T *L = (const T *)tm.L + (t.row - tm.row0);
      const T *R = (const T *)tm.R + (t.col - tm.col0);
      const T *red = TRANS ? L : R;   // the factor contracted with the input panel
      const T *exp = TRANS ? R : L;   // the factor that expands into the output
      const int64_t ldred = TRANS ? tm.ldL : tm.ldR, ldexp = TRANS ? tm.ldR : tm.ldL;
      if (XREG) warp_tn_reg<T, P, RBX, SP>(cw, red, ldred, xr, inlen, tm.rank);
      else warp_tn_any<T, P, SP, false>(cw, red, ldred, Xs, inlen, tm.rank);
      __syncwarp();
      if (RB > 0) warp_nn_reg<T, P, RBX, SP>(racc, exp, ldexp, cw, outlen, tm.rank);
      else warp_nn<T, P, true, SP>(Ys, exp, ldexp, cw, outlen, tm.rank);
      __syncwarp();
    }
  }

  // H-pairs of two dense leaves, warp per pair; the intermediate lives in the warp's scratch
  for (int pi = t.pair_lo + vw; pi < t.pair_mid; pi += NV) {
    const PairDev pr = a.pairs[pi];
    const LeafDev la = a.leafA[a.blocks[pr.blkA].leaf_lo], lb = a.leafB[a.blocks[pr.blkB].leaf_lo];
    const T *DA = (const T *)a.dataA + la.off_u;  // m x rho, ld m
    const T *DB = (const T *)a.dataB + lb.off_u;  // rho x n, ld rho
    const int rho = la.n;
    if (!TRANS) {
      warp_nn<T, P, false, SP>(cw, DB, rho, Xs, rho, lb.n);   // cw = D_B X      (rho x P)
      __syncwarp();
      if (RB > 0) warp_nn_reg<T, P, RBX, SP>(racc, DA, la.m, cw, la.m, rho);
      else warp_nn<T, P, true, SP>(Ys, DA, la.m, cw, la.m, rho);   // Y += D_A cw
    } else {
      if (XREG) warp_tn_reg<T, P, RBX, SP>(cw, DA, la.m, xr, la.m, rho);  // cw = D_A^T Q (rho x P)
      else warp_tn<T, P, false, SP>(cw, DA, la.m, Xs, la.m, rho);
      __syncwarp();
      warp_tn<T, P, true, SP>(Ys, DB, rho, cw, rho, lb.n);    // W += D_B^T cw
    }
    __syncwarp();
  }
  if (RB > 0) {
    // fixed-order sum of the warps' register partials (deterministic), through the scratch
    T *part = Zs;  // NWARP * outlen * SP entries reserved for RB > 0 launches
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int rr = 0; rr < RBX; rr++) {
      const int i = lane + 32 * rr;
      if (i < outlen)
#pragma unroll
        for (int c = 0; c < P; c++) part[(warp * outlen + i) * SP + c] = racc[rr][c];
    }
    __syncthreads();
    for (int o = threadIdx.x; o < outlen * SP; o += AT) {
      T v = Ys[o];
      for (int w2 = 0; w2 < NWARP; w2++) v += part[w2 * outlen * SP + o];
      Ys[o] = v;
    }
    __syncthreads();
  }

  // H-pairs of inner blocks: walk the two subtrees (Algorithm 2), leaves split over warps
  for (int pi = t.pair_mid + part; pi < t.pair_hi; pi += K) {
    const PairDev pr = a.pairs[pi];
    const BlockDev ba = a.blocks[pr.blkA], bb = a.blocks[pr.blkB];
    const int rho = ba.n;
    __syncthreads();
    for (int o = threadIdx.x; o < rho * SP; o += AT) Zs[o] = T(0);
    __syncthreads();
    if (!TRANS) {
      for (int l = bb.leaf_lo + warp; l < bb.leaf_hi; l += NWARP)
        warp_leaf<T, P, SP>(a.leafB[l], (const T *)a.dataB, false, bb.row, bb.col, Xs, Zs, cw);
      __syncthreads();
      for (int l = ba.leaf_lo + warp; l < ba.leaf_hi; l += NWARP)
        warp_leaf<T, P, SP>(a.leafA[l], (const T *)a.dataA, false, ba.row, ba.col, Zs, Ys, cw);
    } else {
      for (int l = ba.leaf_lo + warp; l < ba.leaf_hi; l += NWARP)
        warp_leaf<T, P, SP>(a.leafA[l], (const T *)a.dataA, true, ba.row, ba.col, Xs, Zs, cw);
      __syncthreads();
      for (int l = bb.leaf_lo + warp; l < bb.leaf_hi; l += NWARP)
        warp_leaf<T, P, SP>(a.leafB[l], (const T *)a.dataB, true, bb.row, bb.col, Zs, Ys, cw);
    }
  }
  __syncthreads();
  for (int o = threadIdx.x; o < outlen * p; o += AT) {
    const int c = o / outlen, i = o - c * outlen;
    if (K > 1) atomicAdd(Out + o, Ys[i * SP + c]);
    else Out[o] = Ys[i * SP + c];
  }
}

// ---------------------------------------------------------------------------------------
// a2: low-rank products of Algorithm 3 with an inadmissible factor, batched by H-block.
// A panel = up to P columns of far factors (U_b of B for products A|tau' x rho' U_b, V_a of A
// for B|rho' x sigma'^T V_a) that meet the same H-block; each column's result goes to its own
// term's new factor. The H-block's leaves are read once per panel.
// ---------------------------------------------------------------------------------------

// what a panel multiplies: the H-block, the direction, the input columns and the outputs
struct PanelJob {
  int blk;
  bool trans;
  int64_t src, src_ld;  // first input column (element offset into A's or B's data) and its stride
  int64_t dst, dst_ld;  // first output column (element offset into the term buffer) and its stride
  int ncol;
};

__device__ __forceinline__ PanelJob panel_job(const PanelArgs &a, const PanelDev &pn, int P) {
  const TermJob jb = a.jobs[pn.job];
  PanelJob q;
  q.ncol = min(P, jb.rank - pn.q0);
  q.dst_ld = jb.rows;
  q.dst = jb.out + (int64_t)pn.q0 * jb.rows;
  if (jb.type == JOB_HF) {  // Out = A|tau' x rho' U_b
    const LeafDev lb = a.leafB[jb.b];
    q.blk = jb.a;
    q.trans = false;
    q.src_ld = lb.m;
    q.src = lb.off_u + (int64_t)pn.q0 * lb.m;
  } else {  // FH: Out = B|rho' x sigma'^T V_a
    const LeafDev la = a.leafA[jb.a];
    q.blk = jb.b;
    q.trans = true;
    q.src_ld = la.n;
    q.src = la.off_v + (int64_t)pn.q0 * la.n;
  }
  return q;
}

// the panel's input columns into the row-major staging (row stride SP); threads run along the
// rows of each column, so the global reads are coalesced
template <typename T, int P, int SP>
__device__ __forceinline__ void panel_stage(T *Xs, const PanelJob &q, int inlen, const T *src, int lane0,
                                            int nthreads) {
  for (int o = lane0; o < inlen * P; o += nthreads) {
    const int c = o / inlen, i = o - c * inlen;
    Xs[i * SP + c] = c < q.ncol ? src[q.src + (int64_t)c * q.src_ld + i] : T(0);
  }
}

// one warp per panel whose H-block is a single dense leaf: private input and output panels in
// shared memory, then each output column is written to its own term
template <typename T, int P>
__global__ void __launch_bounds__(AT) k_panel_leaf(PanelArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int pi = blockIdx.x * NWARP + warp;
  if (pi >= a.count) return;  // whole warps only; no block barrier below
  const PanelJob pj = panel_job(a, a.panels[a.first + pi], P);
  const BlockDev bk = a.blocks[pj.blk];
  const bool trans = pj.trans;
  const LeafDev lf = (trans ? a.leafB : a.leafA)[bk.leaf_lo];
  const T *D = (const T *)(trans ? a.dataB : a.dataA) + lf.off_u;
  const T *src = (const T *)(trans ? a.dataA : a.dataB);
  constexpr int SP = panel_row_stride(P);
  T *Xs = (T *)smem_raw + warp * (a.smem_in + a.smem_out) * SP;
  T *Os = Xs + a.smem_in * SP;
  const int inlen = trans ? lf.m : lf.n, outlen = trans ? lf.n : lf.m;
  panel_stage<T, P, SP>(Xs, pj, inlen, src, lane, 32);
  __syncwarp();
  if (!trans) warp_nn<T, P, false, SP>(Os, D, lf.m, Xs, lf.m, lf.n);   // Os = D X
  else warp_tn<T, P, false, SP>(Os, D, lf.m, Xs, lf.m, lf.n);          // Os = D^T X
  __syncwarp();
  T *out = (T *)a.terms;
  for (int c = 0; c < pj.ncol; c++) {
    const int64_t dst = pj.dst + (int64_t)c * pj.dst_ld;
    for (int i = lane; i < outlen; i += 32) out[dst + i] = Os[i * SP + c];
  }
}

// one panel of an inner H-block; leaves split over the block's NW warps, shared-memory atomics
template <typename T, int P, bool GSTAGE, int NW>
__device__ __forceinline__ void panel_body(const PanelArgs &a, int pi, unsigned char *smem_raw) {
  constexpr int NTH = NW * 32;
  const PanelJob pj = panel_job(a, a.panels[a.first + pi], P);
  const BlockDev bk = a.blocks[pj.blk];
  const bool trans = pj.trans;
  const int inlen = trans ? bk.m : bk.n, outlen = trans ? bk.n : bk.m;
  constexpr int SP = panel_row_stride(P);
  T *Xs, *Os, *cwall;
  if (GSTAGE) {
    Xs = (T *)a.stage_base + (int64_t)blockIdx.x * a.stage_stride;
    Os = Xs + (int64_t)inlen * SP;
    cwall = (T *)smem_raw;
  } else {
    Xs = (T *)smem_raw;
    Os = Xs + a.smem_in * SP;
    cwall = Os + a.smem_out * SP;
  }
  const int warp = threadIdx.x >> 5;
  T *cw = cwall + warp * a.smem_cw * SP;
  const T *src = (const T *)(trans ? a.dataA : a.dataB);
  panel_stage<T, P, SP>(Xs, pj, inlen, src, threadIdx.x, NTH);
  for (int o = threadIdx.x; o < outlen * SP; o += NTH) Os[o] = T(0);
  __syncthreads();
  const LeafDev *leaves = trans ? a.leafB : a.leafA;
  const T *data = (const T *)(trans ? a.dataB : a.dataA);
  for (int l = bk.leaf_lo + warp; l < bk.leaf_hi; l += NW)
    warp_leaf<T, P, SP>(leaves[l], data, trans, bk.row, bk.col, Xs, Os, cw);
  __syncthreads();
  T *out = (T *)a.terms;
  for (int o = threadIdx.x; o < outlen * pj.ncol; o += NTH) {
    const int c = o / outlen, i = o - c * outlen;
    out[pj.dst + (int64_t)c * pj.dst_ld + i] = Os[i * SP + c];
  }
}

// shared-memory staging: one block per panel; global staging: a bounded number of blocks loops
// over the panels, block b using staging slot b. NW warps per block: 4 for H-blocks of at most
// 128 rows (at most 4 leaves of 64 rows, so that fewer warps wait idle at the block barriers),
// 16 for H-blocks of more than 512 rows (whose staging lets one block per SM), else 8.
template <typename T, int P, bool GSTAGE, int NW = NWARP>
__global__ void __launch_bounds__(NW * 32) k_panel(PanelArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (!GSTAGE) {
    panel_body<T, P, false, NW>(a, blockIdx.x, smem_raw);
  } else {
    for (int pi = blockIdx.x; pi < a.count; pi += gridDim.x) {
      panel_body<T, P, true, NW>(a, pi, smem_raw);
      __syncthreads();  // the staging slot and shared memory are reused by the next panel
    }
  }
}

// ---------------------------------------------------------------------------------------
// H-matrix times a panel (Alg. 2, all leaves at once): Y += H X for row-major P-column panels X,
// Y of the whole index set (tree order). Warps take leaves; outputs are added atomically.
// ---------------------------------------------------------------------------------------
template <typename T, int P>
__global__ void __launch_bounds__(AT) k_hmatvec(const LeafDev *leaves, int nleaf, const T *data, const T *X, T *Y,
                                                int cw_rows) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int SP = panel_row_stride(P);
  const int warp = threadIdx.x >> 5;
  T *cw = (T *)smem_raw + warp * cw_rows * SP;
  for (int l = blockIdx.x * NWARP + warp; l < nleaf; l += gridDim.x * NWARP)
    warp_leaf<T, P, SP>(leaves[l], data, false, 0, 0, X, Y, cw);
}

}  // namespace apply_detail
}  // namespace hm
