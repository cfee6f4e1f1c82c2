// hmat_internal.h -- data layout and launch interface shared by the library's sources.
//
// Layout in HBM (all device arrays owned by the library):
//   * an H-matrix keeps ONE factor buffer of element type T (double or float). Leaves are
//     numbered in depth-first order of the block tree; far leaf l stores U (m x k) at
//     off_u and V (n x k) at off_v, column-major with leading dimensions m and n; near
//     leaf l stores the dense block (m x n, column-major, ld m) at off_u.
//   * a LeafDev table (one entry per leaf) and a BlockDev table (one entry per block of the
//     tree, with the depth-first leaf range of its subtree) let a kernel walk any inadmissible
//     block's subtree: the subtree of a block is a contiguous range of leaves.
//   * the product's plan: TermDev table (low-rank products L R^T created by the restriction,
//     Algorithm 3), per-target CSR lists of term ids and of H-pairs (block of A, block of B).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace hm {

// Row strides (elements) of the P-column panels kept row-major in shared memory. The
// application kernel keeps P (rows stay 16-byte aligned for vector loads; its small targets
// accumulate in registers); the low-rank product panels use P + 1, so that the lanes of a warp,
// each owning one row of an atomically updated output, fall into distinct banks.
__host__ __device__ constexpr int apply_row_stride(int P) { return P; }
__host__ __device__ constexpr int panel_row_stride(int P) { return P + 1; }
// thread blocks (and global staging slots) of a launch of panels staged in global memory
constexpr int PANEL_GSTAGE_SLOTS = 152 * 4;

// Largest dynamic shared memory a block of the current device may opt into. Every kernel's
// limit is raised to this one value (not to what a launch needs), so that products launched from
// several host threads at once never lower each other's limits between set-up and launch.
int max_dynamic_smem();

// Raise kern's dynamic shared-memory limit to the device maximum less its static shared memory,
// after checking that `bytes` fits under it (cudaErrorInvalidValue otherwise).
template <typename K>
cudaError_t raise_smem_limit(K kern, size_t bytes) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kern);
  if (e != cudaSuccess) return e;
  const int limit = max_dynamic_smem() - (int)fa.sharedSizeBytes;
  if ((long long)bytes > (long long)limit) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, limit);
}

// learned rank proposal: 12 features -> 64 -> 64 -> 1
constexpr int RANK_FEATURES = 12;
constexpr int RANK_PARAMS = 64 * 12 + 64 + 64 * 64 + 64 + 64 + 1;

struct LeafDev {
  int64_t row, col;     // permuted begin of tau and sigma
  int32_t m, n, rank;   // rank < 0: dense leaf
  int32_t level;
  int64_t off_u, off_v; // element offsets into the factor buffer (dense: off_u)
};

struct BlockDev {
  int64_t row, col;     // permuted begin of tau, sigma
  int32_t m, n;
  int32_t leaf_lo, leaf_hi;  // depth-first leaf range of the subtree
  int32_t parent, pad;       // parent block (-1 at the root)
};

// A low-rank term L R^T of a sum-expression, on the block tau' x sigma' where it was created.
// Restricted to tau x sigma (inside tau' x sigma') by index shift: L + (tau.begin - row0),
// R + (sigma.begin - col0) (Sec. 3.2: restriction of low-rank matrices is an index shift).
struct TermDev {
  const void *L, *R;
  int64_t ldL, ldR;
  int64_t row0, col0;
  int32_t rank, pad;
};

// Work item of the low-rank products (a2).
enum TermJobType : int32_t {
  JOB_FF_R = 0,   // far x far, ka <= kb: R_new = V_b (V_a^T U_b)^T   (n' x ka)
  JOB_FF_L = 1,   // far x far, ka >  kb: L_new = U_a (V_a^T U_b)     (m' x kb)
  JOB_FH = 2,     // far x inadmissible:  R_new = B|rho' x sigma'^T V_a (n' x ka)
  JOB_HF = 3      // inadmissible x far:  L_new = A|tau' x rho' U_b   (m' x kb)
};
struct TermJob {
  int32_t type;
  int32_t a;      // leaf of A (FF, FH) or block of the tree (HF)
  int32_t b;      // leaf of B (FF, HF) or block of the tree (FH)
  int32_t rank;   // width of the new factor
  int64_t out;    // element offset of the new factor in the term buffer
  int64_t rows;   // rows of the new factor
  int32_t blk;    // block tau' x sigma' where the term was created
  int32_t pad;
};

// a2 panels: up to panel_width() columns of one product with an inadmissible factor:
// HF jobs: Out = A|tau' x rho' U_b (columns of U_b), FH jobs: Out = B|rho' x sigma'^T V_a.
struct PanelDev {
  int32_t job;           // index into the TermJob table
  int32_t q0;            // first column of the job's new factor in this panel
};
struct PanelArgs {
  int first, count;
  int smem_in, smem_out, smem_cw;
  int gstage;
  int64_t stage_stride;  // elements of global staging per panel (gstage)
  void *stage_base;
  const PanelDev *panels;
  const TermJob *jobs;
  const BlockDev *blocks;
  const LeafDev *leafA, *leafB;
  const void *dataA, *dataB;
  void *terms;
};

struct PairDev {
  int32_t blkA, blkB;   // tau x rho (in A) and rho x sigma (in B), same level as the target
};

struct TargetDev {
  int64_t row, col;     // permuted begin of tau, sigma
  int32_t m, n;
  int32_t blk, nterms;  // the target's block; its low-rank terms are those created at blk and
                        // its ancestors (ranges blk_terms[.] along the parent links)
  int32_t pair_lo, pair_mid, pair_hi;  // [lo, mid): pairs of two dense leaves; [mid, hi): inner blocks
  int32_t leaf;         // leaf id in the block tree
  int32_t rmax;         // basis capacity (columns of Q and W)
  int32_t p0;           // columns of the first round (its last p are a verification block when p0 > p)
  int64_t q_off, w_off; // FP64 basis Q (m x rmax) and W (n x rmax)
  int64_t y_off, x_off; // per-round sample buffers (max(m,n) x p each), element type T
  int64_t stage_off;    // global staging panels (targets too large for shared memory)
};

// Per-target state of the adaptive range finder.
struct TargetState {
  int32_t r;            // columns in Q so far
  int32_t active;       // 1 while sampling continues
  int32_t p_new;        // columns kept in the current round
  int32_t rank;         // final rank
  int32_t nfwd;         // rounds in which the target was sampled
  int32_t sweeps;       // Jacobi sweeps of the core truncation
  int32_t piv_i, piv_j; // cross approximation: pivot row and column of the current step
  int32_t hits, pad;    // cross approximation: consecutive crosses that met eq. (truncaca)
  double nrm2;          // ||W||_F^2 over all columns so far (= ||Q Q^T S||_F^2)
  double est2;          // ||Y||_F^2 / p of the first round (scale for dropping)
  double tail2;         // discarded energy in the final truncation
  double alpha, beta;   // Lanczos bidiagonalization: the latest alpha_r and beta_r
};

struct ApplyArgs {
  int first, count;      // targets [first, first + count) of tg form this launch
  int smem_in, smem_out, smem_rho, smem_cw;  // staged rows: input, output, H-pair intermediate,
                                             // per-warp scratch
  int gstage;            // 1: stage panels in global memory (stage_base + stage_off)
  void *stage_base;
  const TargetDev *tg;
  const int2 *blk_terms;  // per block: [lo, hi) of the terms created at it
  const TermDev *terms;
  const PairDev *pairs;
  const BlockDev *blocks;
  const LeafDev *leafA, *leafB;
  const void *dataA, *dataB;
  TargetState *state;
  void *y_base;          // per-target In/Out regions (element type T), offsets in TargetDev
  void *x_base;
  int p;                 // columns this round (the first round: each target's p0 instead)
  int split;             // thread blocks per target (> 1 only for shared-atomic launches without
                         // global staging): each takes a share of the target's terms and
                         // H-pairs and adds its partial output to Out, which starts at zero
  int round;
};

// ---- launch wrappers (hmat_kernels.cu); all return cudaError_t of the launch ----
cudaError_t launch_kernel_dense(int prec, int kernel, const double *pts, int dim,
                                const LeafDev *leaves, const int32_t *near_ids, int nnear,
                                void *data, cudaStream_t s);
// far_ids[0 .. nsmall) must be leaves of at most 64 x 64 (one warp each), the rest any size
// (one block each)
cudaError_t launch_aca(int kernel, const double *pts, int dim, const LeafDev *leaves,
                       const int32_t *far_ids, int nfar, int nsmall, double eps, int kmax,
                       double *scratch, const int64_t *scratch_off, int32_t *ranks,
                       cudaStream_t s);
cudaError_t launch_aca_compact(int prec, const LeafDev *leaves, const int32_t *far_ids, int nfar,
                               const double *scratch, const int64_t *scratch_off, int kmax,
                               void *data, cudaStream_t s);
// far x far products ids[0..n) with both ranks <= 32, one warp per job (the others: launch_term_jobs)
// far x far products one warp each: ids lists nbucket[0] jobs with both ranks <= 8, then
// nbucket[1] with both <= 16, then nbucket[2] with both <= 32
cudaError_t launch_ff_warp(int prec, const TermJob *jobs, const int32_t *ids, const int *nbucket,
                           const LeafDev *leafA, const LeafDev *leafB, const void *dataA, const void *dataB,
                           void *terms, cudaStream_t s);
cudaError_t launch_term_jobs(int prec, const TermJob *jobs, const int32_t *ids, int njobs, const LeafDev *leafA,
                             const LeafDev *leafB, const BlockDev *blocks, const void *dataA,
                             const void *dataB, void *terms, cudaStream_t s);
cudaError_t launch_make_terms(int prec, const TermJob *jobs, int njobs, const BlockDev *blocks,
                              const LeafDev *leafA, const LeafDev *leafB, const void *dataA,
                              const void *dataB, const void *termbuf, TermDev *terms, cudaStream_t s);
// a8: FP64 on the FP64 pipe; FP32 on the tensor cores (3 x TF32), which set *err when one of
// their bounded waits gives up
cudaError_t launch_near_eval(int prec, const TargetDev *tg, int ntg, const int2 *blk_terms,
                             const TermDev *terms, const PairDev *pairs, const BlockDev *blocks,
                             const LeafDev *leafA, const LeafDev *leafB, const void *dataA,
                             const void *dataB, const LeafDev *leafC, void *dataC, int *err, cudaStream_t s);
// one block: a bounded wait on an mbarrier that nothing arrives on (the near field's failure path)
cudaError_t launch_tc_wait_check(int polls, int *gave_up, cudaStream_t s);
cudaError_t launch_near_tc(const TargetDev *tg, int ntg, const int2 *blk_terms, const TermDev *terms,
                           const PairDev *pairs, const BlockDev *blocks, const LeafDev *leafA, const LeafDev *leafB,
                           const float *dataA, const float *dataB, const LeafDev *leafC, float *dataC, int *err,
                           cudaStream_t s);
cudaError_t launch_apply(int prec, bool trans, const ApplyArgs &a, cudaStream_t s);
size_t apply_smem_bytes(int prec, int P, const ApplyArgs &a);
int apply_rows_per_lane(int dmax);
cudaError_t launch_panels(int prec, const PanelArgs &a, bool leaf_kind, cudaStream_t s);
int panel_width();
// Y += H X (FP64) for row-major panels of panel_width() columns and row stride
// panel_row_stride(panel_width()) over the whole index set in tree order; cw_rows >= max rank
cudaError_t launch_hmatvec(const LeafDev *leaves, int nleaf, const double *data, const double *X, double *Y,
                           int cw_rows, cudaStream_t s);
int apply_panel_width(int p);
// Gaussian test matrices Omega (n x p per active target, into x_base; round 0: p0 columns)
cudaError_t launch_gaussian(int prec, const TargetDev *tg, const TargetState *st, int ntg, int p, uint64_t seed,
                            int round, void *x_base, cudaStream_t s);
// a4 for targets ids_warp (at most 64 rows: one warp each) and ids_block (one block each); side 1
// orthonormalises the column-side block (n rows, basis in the W buffer), fresh ignores the basis
cudaError_t launch_orth(int prec, const TargetDev *tg, const int32_t *ids_warp, int n_warp, const int32_t *ids_block,
                        int n_block, TargetState *st, int p, double eps, void *y_base, double *qw, void *x_base,
                        int round, cudaStream_t s, int side = 0, int fresh = 0);
cudaError_t launch_absorb_w(int prec, const TargetDev *tg, TargetState *st, int ntg, int p,
                            double eps_stop, void *y_base, double *qw, int round, int max_rounds,
                            int32_t *active_count, cudaStream_t s, int fixed = 0);
// Adaptive cross approximation of the sum-expressions (Algorithm 6), one step per call pair.
// L_k (m x k) lives in the Q buffer, U_k^T (n x k, the rows u_r as columns) in the W buffer;
// column rmax - 1 of the Q buffer holds the used-row flags. launch_aca_start sets the first
// pivot row's unit vector e_i as the input of the S^T pass; launch_aca_row takes e_i^T S from
// y_base, forms u_r, picks the column pivot and sets e_j as the input of the S pass;
// launch_aca_col takes S e_j, forms l_r, applies eq. (truncaca) at eps_stop (the target stops
// after two consecutive crosses meet it), picks the next row pivot and counts the targets still
// active into *active_count.
cudaError_t launch_aca_start(int prec, const TargetDev *tg, TargetState *st, int ntg, double *qw, void *x_base,
                             cudaStream_t s);
cudaError_t launch_aca_row(int prec, const TargetDev *tg, TargetState *st, int ntg, const void *y_base, double *qw,
                           void *x_base, cudaStream_t s);
cudaError_t launch_aca_col(int prec, const TargetDev *tg, TargetState *st, int ntg, const void *y_base, double *qw,
                           void *x_base, double eps_stop, int32_t *active_count, cudaStream_t s);
// Golub-Kahan-Lanczos bidiagonalization of the sum-expressions (Algorithm 7) with full
// reorthogonalization, one step per call pair: q_r (column r of the Q buffer) from S w_r and
// w_{r+1} (column r + 1 of the W buffer) from S^T q_r. launch_lz_start draws w_1 (Gaussian,
// normalised; the S pass input); launch_lz_q forms q_r = S w_r - beta_{r-1} q_{r-1}, projects it
// twice against q_1..q_{r-1}, normalises (alpha_r) and sets it as the S^T input; launch_lz_w
// forms S^T q_r - alpha_r w_r, projects it twice against w_1..w_r, normalises (beta_r), applies
// eq. (truncaca) to alpha_r^2 + beta_r^2 at eps_stop (two consecutive steps) and counts the
// targets still active. launch_lz_load / launch_lz_store move columns c0 .. c0+p-1 of Q into the
// S^T pass input and its output into W (the projection W = S^T Q that ends the compression).
cudaError_t launch_lz_start(int prec, const TargetDev *tg, TargetState *st, int ntg, double *qw, void *x_base,
                            uint64_t seed, cudaStream_t s);
cudaError_t launch_lz_q(int prec, const TargetDev *tg, TargetState *st, int ntg, const void *y_base, double *qw,
                        void *x_base, cudaStream_t s);
cudaError_t launch_lz_w(int prec, const TargetDev *tg, TargetState *st, int ntg, const void *y_base, double *qw,
                        void *x_base, double eps_stop, int32_t *active_count, cudaStream_t s);
cudaError_t launch_lz_load(int prec, const TargetDev *tg, TargetState *st, int ntg, const double *qw, void *x_base,
                           int c0, int p, cudaStream_t s);
cudaError_t launch_lz_store(int prec, const TargetDev *tg, const TargetState *st, int ntg, const void *y_base,
                            double *qw, int c0, int p, cudaStream_t s);
// L = Q R (classical Gram-Schmidt twice, FP64) in place in the Q buffer and W <- U R^T in place,
// so that L U^T = Q W^T with orthonormal Q: the input of the core truncation
cudaError_t launch_aca_qr(const TargetDev *tg, const TargetState *st, int ntg, double *qw, cudaStream_t s);
// core truncation of the targets listed in ids: one warp per target (bases of at most 32
// columns) or one block per target (up to 96 columns)
cudaError_t launch_final(const TargetDev *tg, TargetState *st, const int32_t *ids, int nids, bool warp_kernel,
                         double eps, double *qw, cudaStream_t s);
cudaError_t launch_write_far(int prec, const TargetDev *tg, const TargetState *st, int ntg,
                             const double *qw, const LeafDev *leafC, void *dataC, cudaStream_t s);
cudaError_t launch_convert(int prec, const void *src, double *dst, int64_t count, cudaStream_t s);
// the global error estimator's device steps, on blocks of size <= 128 columns held as row-major
// panels of 16 columns (row stride 17) in tree order: the Gaussian start, Y -= Z, Cholesky QR
// twice (G: size x size scratch; *zero set when the block is zero) and the sum of squares into *out
cudaError_t launch_est_gaussian(double *X, int64_t n, int size, uint64_t seed, cudaStream_t s);
cudaError_t launch_est_sub(double *Y, const double *Z, int64_t count, cudaStream_t s);
cudaError_t launch_est_orth(double *X, int64_t n, int size, double *G, int *zero, cudaStream_t s);
cudaError_t launch_est_norm2(const double *Y, int64_t count, double *out, cudaStream_t s);
// atomicMin of the index of every non-finite entry into *first (initialise to ~0ull)
cudaError_t launch_find_nonfinite(int prec, const void *x, int64_t count, unsigned long long *first, cudaStream_t s);

// learned rank proposal (hmat_rank.cu); w16 holds RANK_PARAMS FP16 weights
cudaError_t launch_mlp_forward(const void *w16, const float *x, int count, float *out, cudaStream_t s);
cudaError_t launch_mlp_grad(const void *w16, const float *x, const float *y, int count, float *grad, float *loss,
                            cudaStream_t s);
cudaError_t launch_to_half(const float *w, void *w16, cudaStream_t s);
cudaError_t mlp_train(float *w, void *w16, const float *x, const float *y, int count, int epochs, float lr,
                      cudaStream_t s, float *final_loss);
// Gradient and loss of the network on count <= RANKGRAD_NOALLOC_MAX samples given on the host
// (raw features, raw ranks), normalised on the device, with every device buffer inside one
// fixed-size __device__ array of hmat_rank.cu: no device allocation. Synchronises s.
constexpr int RANKGRAD_NOALLOC_MAX = 16384;
cudaError_t mlp_grad_noalloc(const void *w16, const float *mean, const float *dev, const float *features,
                             const float *ranks, int count, float *grad, float *loss, cudaStream_t s);

}  // namespace hm
