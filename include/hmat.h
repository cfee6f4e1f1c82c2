/*
 * hmat.h -- C-ABI of the GB300 H-matrix product library (libhmat.so).
 *
 * The library computes the product of two hierarchical (H-) matrices on one block-cluster
 * tree and compresses every admissible target block to its eps-best low-rank approximation,
 * following Doelz, Harbrecht, Multerer, "On the best approximation of the hierarchical
 * matrix product": the product L = HK is written as the sum-expression S(I,I) = HK
 * (Sec. 3.1), restricted block by block (Algorithm 3) and, at every leaf, either truncated
 * to low rank (far leaves, operator T of Algorithm 4, realised by the blocked adaptive
 * randomized range finder of Algorithm 8 with the stop test eq. (truncaca), or on request by
 * cross approximation, Algorithm 6, or Lanczos bidiagonalization, Algorithm 7) or evaluated
 * densely (near leaves, evaluate() of Algorithm 4).
 *
 * Conventions for every entry point:
 *   - Every call returns an hmat_status; nothing aborts or throws across the ABI. On error an
 *     output handle is set to NULL and no partial object leaks; hmat_last_error() returns a
 *     thread-local message describing the last failure on the calling thread.
 *   - Host buffers are owned by the caller. Device memory is owned by the library and is
 *     taken from the allocator set with hmat_set_allocator (default: the CUDA stream-ordered
 *     pool, cudaMallocAsync/cudaFreeAsync, on the given stream). Three small kinds of buffer
 *     are taken with plain cudaMalloc instead: a block tree's point and block tables
 *     (n * dim * 8 + 32 bytes per block, shared by every handle on that tree, so they may
 *     outlive the stream they were made on), a rank model's weights (about 30 KB) and the
 *     optimizer state of hmat_rankmodel_train (freed before it returns).
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream). Work is
 *     enqueued on it; calls that read results back to the host synchronise it (stated per call).
 *   - Index conventions: points are given in their ORIGINAL order; internally the library
 *     permutes them along its cluster tree. Leaf ranges (hmat_leaf) are in PERMUTED order;
 *     hmat_permutation gives perm[i] = original index of permuted position i.
 *   - Matrices on the host are column-major.
 *   - An hmat_t is immutable once created and may be read from several threads at once.
 */
#ifndef HMAT_H
#define HMAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hmat_s *hmat_t;
typedef struct hmat_rankmodel_s *hmat_rankmodel_t;  /* learned rank proposal (an MLP) */

/* Number of features per far block fed to the rank proposal, and of the MLP's parameters
 * (12 -> 64 -> 64 -> 1, ReLU; layout W1[64][12], b1[64], W2[64][64], b2[64], w3[64], b3). */
#define HMAT_RANK_FEATURES 12
#define HMAT_RANK_PARAMS 5057

typedef enum {
  HMAT_OK = 0,
  HMAT_EINVAL = 1,     /* invalid argument (bad size, NULL pointer, eps <= 0, NaN points) */
  HMAT_ENOMEM = 2,     /* a device or host allocation failed */
  HMAT_ECUDA = 3,      /* a CUDA runtime call or kernel launch failed */
  HMAT_ENOTCONV = 4,   /* some far block hit max_rank / max_rounds before the stop test held;
                          the result is complete and usable, see hmat_stats.not_converged */
  HMAT_ETIMEOUT = 5,   /* a bounded device wait gave up (the tensor-core near field of an FP32 product) */
  HMAT_EMISMATCH = 6   /* the two factors of a product are not on the same block tree */
} hmat_status;

/* Kernel functions k(x, y) used to assemble test matrices (r = |x - y|). */
typedef enum {
  HMAT_K_EXP = 0,      /* exp(-r)            (Sec. 6.1 uses this kernel) */
  HMAT_K_INVQ = 1,     /* 1 / (1 + r^2) */
  HMAT_K_POLY2 = 2     /* (1 + x.y)^2, separable, rank <= (d+1)(d+2)/2: a closed-form check */
} hmat_kernel;

/* Seeded point distributions (splitmix64 stream; see hmat_points). */
typedef enum {
  HMAT_PTS_CUBE = 0,   /* uniform in [0,1]^dim, dim in {1,2,3} */
  HMAT_PTS_SPHERE = 1  /* uniform on the unit sphere S^2, dim = 3 */
} hmat_ptdist;

typedef enum {
  HMAT_MODE_F64 = 0,   /* every contraction in FP64 ("plain" path) */
  HMAT_MODE_MIXED = 1  /* contractions in the factors' precision (FP32 for factor_prec = 32),
                          orthogonalisation (Gram, Cholesky) and the core eigen-solve in FP64 */
} hmat_mode;

/* Compressor of the far blocks' sum-expressions (Sec. 4). Both end with the same truncation of
 * the compressed block to its eps-rank (Algorithm 5); they differ in how the low-rank factors are
 * found from products of the sum-expression with vectors. */
typedef enum {
  HMAT_COMP_RANDOMIZED = 0,  /* blocked adaptive randomized range finder (Algorithm 8) */
  HMAT_COMP_ACA = 1,         /* adaptive cross approximation (Algorithm 6): one row e_i^T S and
                                one column S e_j per step, partial pivoting, stopped when
                                two consecutive crosses meet eq. (truncaca) at
                                max(eps/8, 4 u), u the unit roundoff of the passes */
  HMAT_COMP_LANCZOS = 2      /* Golub-Kahan-Lanczos bidiagonalization (Algorithm 7) from a
                                Gaussian start vector (opts->seed), full reorthogonalization,
                                one S w and one S^T q per step, stopped like ACA; the
                                coefficient factor is then S^T Q (the bidiagonal B_k with one
                                step of lookahead) */
} hmat_compressor;

typedef struct {
  int leaf_size;       /* n_min: leaf clusters hold at most this many points (2..64; all leaves
                          sit on one level, and n_min >= 2 keeps every cluster non-empty as
                          Def. 2.2 requires; the device kernels stage whole leaves in shared
                          memory and are laid out for at most 64 points) */
  double eta;          /* admissibility: max(diam tau, diam sigma) <= eta * dist(tau, sigma) */
  double aca_eps;      /* ACA stop tolerance for far leaves (Algorithm 6, eq. (truncaca)) */
  int factor_prec;     /* 64: store factors in FP64; 32: store factors in FP32 */
  int aca_kmax;        /* rank cap of ACA (0 = default 128) */
} hmat_build_opts;

typedef struct {
  double eps;          /* relative Frobenius tolerance per far block (> 0) */
  int mode;            /* hmat_mode */
  int rank_proposal;   /* first-round width of each far block: 0 = block_width columns;
                          1 = learned (rank_model must be set): predicted rank + block_width;
                          2 = heuristic: max of A's and B's ranks on the block + block_width.
                          With 1 or 2 the first round holds a verification block (its last
                          block_width/2 kept columns) and eq. (truncaca) is tested within it; the
                          adaptive rounds continue whenever that test fails. Widths <= 16. */
  int max_rank;        /* cap on the sampled basis per block (0 = default 96) */
  int max_rounds;      /* cap on adaptive rounds (0 = default max_rank / block_width + 1) */
  int block_width;     /* columns added per adaptive round (0 = default 8; <= 16) */
  uint64_t seed;       /* seed of the Gaussian test matrices (counter-based, splitmix64) */
  hmat_rankmodel_t rank_model;  /* used when rank_proposal == 1 (NULL otherwise) */
  int fixed_rank;      /* 0: eps-rank truncation (the default). k in 1..16: every far block of C
                          gets rank at most k by Algorithm 9 (k Gaussian samples, power_iters
                          subspace iterations, no eps test; eps then only sets the threshold
                          below which sample directions are dropped as zero) */
  int power_iters;     /* subspace iterations q of the fixed-rank mode (0..4; -1 = default 1) */
  int compressor;      /* hmat_compressor (HMAT_COMP_ACA and HMAT_COMP_LANCZOS need fixed_rank = 0
                          and rank_proposal = 0; their rank is capped at max_rank - 1 per block,
                          HMAT_ENOTCONV beyond) */
} hmat_mult_opts;

typedef struct {
  int epochs;          /* full-batch training steps (0 = default 1500) */
  float lr;            /* Adam learning rate (0 = default 3e-3) */
  uint64_t seed;       /* initial weights */
} hmat_train_opts;

typedef struct {
  int64_t row_begin, row_size;   /* permuted row range of tau */
  int64_t col_begin, col_size;   /* permuted column range of sigma */
  int level;                     /* level of tau x sigma in the block tree (root = 0) */
  int far;                       /* 1: admissible leaf (low-rank U V^T), 0: near leaf (dense) */
  int rank;                      /* far: rank of U V^T; near: -1 */
} hmat_leaf;

typedef struct {
  int64_t n;                     /* #I */
  int depth;                     /* depth of the cluster tree */
  int csp;                       /* C_sp: max number of blocks sharing one row cluster */
  int64_t n_far, n_near;         /* number of far / near leaves */
  int64_t storage_bytes;         /* bytes of the stored factors and dense leaves */
  int factor_prec;               /* 32 or 64 */
  int max_rank;                  /* largest far-leaf rank */
  /* filled by hmat_multiply on its output handle (zero elsewhere): */
  int64_t n_terms;               /* low-rank products created by the restriction (a2) */
  int64_t n_lr_refs;             /* sum over leaves of their low-rank term counts */
  int64_t n_hpairs;              /* sum over leaves of their H-pair counts */
  int rounds;                    /* adaptive rounds run (cross approximation / Lanczos: steps) */
  int64_t not_converged;         /* far blocks that hit max_rank or max_rounds */
  double flops_apply;            /* algorithmic flops of the sum-expression applications */
  double flops_terms;            /* algorithmic flops of the low-rank products (a2) */
  double flops_near;             /* algorithmic flops of the near-field evaluation */
  double bytes_apply;            /* algorithmic bytes read by the sum-expression applications */
  double ms_plan, ms_terms, ms_near, ms_sample, ms_final;  /* device/host phase times */
  double ms_apply;               /* summed device time of the sum-expression application kernels
                                    (CUDA events on the call's stream around each launch) */
  int64_t apply_launches;        /* number of those launches */
  double bytes_apply_use;        /* algorithmic bytes of those launches: every factor element of
                                    every target's sum-expression read once per launch, plus the
                                    In/Out panels ((m + n) * p elements per target) */
  int64_t launches;              /* kernels this call launched (all of them are the library's) */
  int64_t n_ff_jobs;             /* low-rank products with two far factors */
  int64_t n_panels;              /* panels of products with one inadmissible factor */
  int64_t first_round_cols;      /* columns sampled in the first round, summed over far blocks */
  int64_t done_in_first_round;   /* far blocks whose stop test held in the first round */
  int64_t sample_passes;         /* sum over far blocks of the rounds each one took part in
                                    (cross approximation: crosses; Lanczos: steps) */
  int64_t groups;                /* subtree groups the product ran in (1: one pass) */
  double bytes_apply_unique;     /* the minimum bytes of the same launches: per pass, every stored
                                    factor element that an active target's sum-expression
                                    references counted once (the rows of a term's factors in the
                                    union of its active targets' clusters; an H-pair block once),
                                    plus the In/Out panels */
  int64_t apply_gstage_targets;  /* far targets whose application panels were staged in global
                                    memory (too large for shared memory) */
  int64_t apply_split_targets;   /* far targets whose application was split over several thread
                                    blocks (partial outputs added atomically) */
  int apply_max_split;           /* the largest such split (thread blocks per target) */
  double bytes_terms_use;        /* algorithmic bytes of the low-rank products (a2): every panel
                                    reads its H-block's stored elements once plus its input and
                                    output columns; every far x far product reads its four factors
                                    and writes the new one */
  double ms_near_kernel;         /* device time of the near-field kernel (a8), from CUDA events on
                                    the second stream it runs on, concurrently with the sampling */
} hmat_stats_t;

/* Synthetic inputs (the paper's experiments, Sec. 6.1, use Galerkin matrices on the unit sphere;
 * seeded point sets in a cube or on the sphere stand in for them). Fill xyz (n*dim doubles,
 * row-major, caller-owned) with the seeded points of the given distribution: splitmix64 stream
 * of `seed`, u = (z >> 11) * 2^-53; cube: point i uses draws dim*i .. dim*i+dim-1; sphere: draws
 * 2i, 2i+1 -> z = 2u1 - 1, phi = 2 pi u2, (sqrt(1-z^2) cos phi, sqrt(1-z^2) sin phi, z).
 * EINVAL on a bad dim/n, an unknown distribution or NULL xyz. */
hmat_status hmat_points(hmat_ptdist dist, int dim, int64_t n, uint64_t seed, double *xyz);

/* Build the H-matrix of kernel `kernel` on the points xyz (n x dim, row-major, original
 * order, host, caller-owned): cluster tree by cardinality-balanced bisection (Def. 2.2),
 * block tree by Algorithm 1 with eta-admissibility (Def. 2.3), near leaves evaluated densely,
 * far leaves by ACA (Algorithm 6) on the GPU. If tree_from is not NULL its cluster and block
 * tree are reused (xyz must then hold the same points; only kernel and factors differ), which
 * is how two factors of a product are put on one block tree (Sec. 3). Synchronises `stream`
 * once (to size the far-leaf storage). EINVAL on bad sizes (n must be below 2^31), NaN/Inf
 * points, an unknown kernel or bad opts; EMISMATCH if tree_from was built on other points. */
hmat_status hmat_build(const double *xyz, int64_t n, int dim, hmat_kernel kernel,
                       const hmat_build_opts *opts, const hmat_t tree_from, void *stream,
                       hmat_t *out);

/* The structure hmat_build and hmat_multiply would use on these points, computed on the host
 * alone (no device memory, no stream, no GPU needed): the cluster tree by cardinality-balanced
 * bisection (Def. 2.2), the block tree by Algorithm 1 with eta-admissibility (Def. 2.3), and
 * the symbolic restriction of S(I,I) = HK down the whole block tree (Algorithm 3, as Algorithm 4
 * recurses). xyz: n x dim, row-major, original order, host. Outputs, host, caller-owned, each
 * may be NULL:
 *   perm[n]            perm[i] = original index of permuted position i (as hmat_permutation);
 *   *n_leaves          leaves of the block tree;
 *   leaves[max_leaves] the first min(max_leaves, *n_leaves) leaves in depth-first order, as
 *                      hmat_leaf_info gives them before factors exist (far: rank 0, near: -1);
 *   n_lowrank[max_leaves], n_hpairs[max_leaves]  per leaf, the low-rank terms and H-pairs of
 *                      its sum-expression (as hmat_sumexpr_counts);
 *   *csp               C_sp, the largest number of blocks sharing one row cluster.
 * leaf_size may be 2..128 here (hmat_build takes 2..64).
 * EINVAL on NULL xyz, n < 1, dim outside 1..3, leaf_size outside 2..128, eta <= 0 or a
 * non-finite coordinate. Memory: a block tree with few admissible blocks (coincident points, or
 * eta near 0) keeps every block inadmissible down to the leaves, and its plan then holds about
 * (n / leaf_size)^3 H-pairs (8 bytes each), as the dense product it describes would need; the
 * same holds for hmat_multiply on such inputs. */
hmat_status hmat_plan_host(const double *xyz, int64_t n, int dim, int leaf_size, double eta, int64_t *perm,
                           int64_t *n_leaves, hmat_leaf *leaves, int64_t *n_lowrank, int64_t *n_hpairs,
                           int64_t max_leaves, int *csp);

/* C ~= A B with every far block of C the eps-approximation of its sum-expression
 * (Algorithm 4 with the truncation operator of Algorithm 8 + eq. (truncaca), then an FP64
 * eigen-truncation of the sampled core to relative Frobenius error eps) and every near
 * block evaluated exactly. A and B must share one block tree (EMISMATCH otherwise) and one
 * factor precision. C lives on the same tree with A's factor precision. Synchronises
 * `stream` at the end of every adaptive round and at the end. Returns HMAT_ENOTCONV (with a
 * valid C) when some block hit the rank or round cap. With opts->compressor = HMAT_COMP_ACA the
 * far blocks are compressed by adaptive cross approximation (Algorithm 6; a round is then one
 * cross, a row and a column of every unfinished block) and the cross factors L U are truncated
 * to the eps-rank by a QR of L and the same FP64 eigen-truncation; with HMAT_COMP_LANCZOS by
 * Lanczos bidiagonalization (Algorithm 7), then the same truncation of Q (S^T Q)^T. Host memory:
 * the product's host tables (restriction plan, job and panel lists) are kept per calling thread
 * after the call, so that the next product on that thread reuses their pages; they are released
 * when the thread exits. */
hmat_status hmat_multiply(const hmat_t A, const hmat_t B, const hmat_mult_opts *opts,
                          void *stream, hmat_t *C);

/* Device memory of a product. hmat_multiply plans for the new factors of the low-rank products,
 * the sampling buffers and the near field; when their estimate exceeds 45 % of the free device
 * memory (or HMAT_MEMORY_BUDGET_GB gigabytes, if that environment variable is set), the block
 * tree is cut at a level and its subtrees run in groups that fit: each group builds the terms
 * created in its subtrees and those created above the cut (rebuilt per group), runs its own
 * target blocks, and C is assembled from the groups. */

/* y = H x for ncols right-hand sides (Alg. 2 over all leaves, on the device, in FP64): x and y are
 * n x ncols column-major host arrays in the ORIGINAL point order (caller-owned). Synchronises. */
hmat_status hmat_matvec(const hmat_t H, const double *x, double *y, int64_t ncols, void *stream);

/* Estimate of the relative Frobenius error ||C - A B||_F / ||A B||_F of a product (the paper's
 * check of its products, Sec. 6: `iters` subspace iterations on a block of `size` Gaussian
 * vectors (splitmix64 stream of `seed`), the operator applied as C v - A (B v)). The same
 * iteration on C estimates the denominator. Every step runs on the device (the H-matrix
 * products, C v - A (B v), Cholesky QR twice of the block, the norms); only the two norms are
 * read back. size must be 1..128 (the paper uses 100). A, B, C on one block tree.
 * Synchronises. */
hmat_status hmat_product_error(const hmat_t A, const hmat_t B, const hmat_t C, int iters, int size, uint64_t seed,
                               double *rel_err);

/* Check, on the current device, that the library's bounded tensor-core waits give up and
 * report: one thread block allocates tensor memory, waits on an mbarrier that nothing arrives on
 * for `polls` polls (1..2^22; the tensor-core near field gives up after 2^18, about a second on
 * GB300), frees the tensor memory and reports. Returns HMAT_ETIMEOUT when the wait gave up (the expected result; the CUDA context
 * stays usable), HMAT_OK if it completed (it cannot), HMAT_EINVAL for polls out of range and
 * HMAT_ECUDA on a CUDA error. A test hook for the failure path of the FP32 near field; the paper
 * has no counterpart. Synchronises. */
hmat_status hmat_check_bounded_wait(int polls);

/* count independent products C[i] = A[i] B[i] (each pair on one block tree; the trees of
 * different pairs may differ) with the same options, in one call: the products are planned on
 * host threads and run on up to 8 streams of their own, largest first, so that the GPU works on
 * several products at once; every stream first waits for the work already queued on `stream`,
 * and `stream` then waits for all of them. Outputs are caller-owned handles (release each with
 * hmat_destroy). Status: the first failing product's status, with every C[i] NULL, except
 * HMAT_ENOTCONV, which leaves all outputs valid. The paper treats one product at a time (Sec. 4);
 * this is the batched form of the same call. */
hmat_status hmat_multiply_batched(const hmat_t *A, const hmat_t *B, int count, const hmat_mult_opts *opts,
                                  void *stream, hmat_t *C);

/* Dense copy of the whole matrix (every leaf of the block tree expanded as in the definition of
 * H(B, k), Sec. 2: U V^T on far leaves, the stored block on near leaves) in ORIGINAL point order
 * into the host buffer out (column-major, leading dimension ld >= n). Synchronises `stream` of
 * the handle's last use. Intended for checking small problems. */
hmat_status hmat_to_dense(const hmat_t h, double *out, int64_t ld);

/* Number of leaves of the block tree (far + near), numbered in depth-first order. */
hmat_status hmat_leaf_count(const hmat_t h, int64_t *n_leaves);

/* Geometry, kind and rank of leaf i (0 <= i < leaf count): tau x sigma, its level, far (in F, a
 * low-rank matrix of R(tau x sigma, k), Sec. 2) or near (in N, dense). */
hmat_status hmat_leaf_info(const hmat_t h, int64_t i, hmat_leaf *info);

/* Copy leaf i to the host as FP64: far leaf -> U (row_size x rank) into U and V
 * (col_size x rank) into V; near leaf -> the dense block (row_size x col_size) into U,
 * V unused. Column-major, caller-owned. Synchronises. */
hmat_status hmat_leaf_get(const hmat_t h, int64_t i, double *U, double *V);

/* perm[i] = original index of permuted position i (n entries, caller-owned). */
hmat_status hmat_permutation(const hmat_t h, int64_t *perm);

/* Size in bytes of h's packed factor buffer (all leaves; element type float or double as
 * hmat_stats.factor_prec says; leaf offsets follow the depth-first leaf order: for each leaf,
 * far: U (row_size x rank) then V (col_size x rank); near: the dense block). */
hmat_status hmat_data_bytes(const hmat_t h, int64_t *bytes);

/* Copy h's packed factor buffer to the host buffer out (capacity `bytes`, caller-owned;
 * EINVAL if smaller than hmat_data_bytes). Pinned host memory makes it one DMA. Synchronises. */
hmat_status hmat_data_get(const hmat_t h, void *out, int64_t bytes);

/* Structure and, for products, work statistics of h: the counts of Sec. 2 (#F, #N, depth, C_sp)
 * and the algorithmic flops and bytes of the product's steps (the quantities of Lemmas 5.1-5.3
 * and Thm. 5.4 as the product actually ran them), with device times per phase. */
hmat_status hmat_stats(const hmat_t h, hmat_stats_t *stats);

/* Per leaf: number of low-rank terms and of H-pairs in the sum-expression S(leaf) that the
 * restriction of Algorithm 3 builds from S(I,I) = AB (Algorithm 4); arrays of leaf-count
 * entries, caller-owned. Needs only the block tree of A (B must share it). */
hmat_status hmat_sumexpr_counts(const hmat_t A, const hmat_t B, int64_t *n_lowrank, int64_t *n_hpairs);

/* Features of the far blocks of the product A B for the rank proposal, in depth-first leaf order
 * (n_far x HMAT_RANK_FEATURES, row-major, caller-owned): log2 of the block's rows and columns,
 * its level, diam(tau)/dist and diam(sigma)/dist, log2(1 + #low-rank terms), log2(1 + #H-pairs),
 * the largest and log2(1 + sum of) the terms' ranks, the ranks of A and B on the block, and
 * -log10(eps). If C (the product) is given, ranks[i] = C's rank on the block. *n_far: in the
 * capacity of the arrays (rows), out the number of far blocks (EINVAL if the capacity is
 * too small; pass features = NULL to query the count). Host-only. */
hmat_status hmat_rank_features(const hmat_t A, const hmat_t B, double eps, const hmat_t C, float *features,
                               float *ranks, int64_t *n_far);

/* The learned rank proposal (no counterpart in the paper, whose Algorithm 8 keeps drawing samples
 * until its stop test holds, with no prior guess of the rank): a small network predicts a far
 * block's eps-rank from its features, and the product uses the prediction only to size the first
 * sampling round; the stop test and the final truncation still decide rank and error.
 *
 * Train a rank model on the GPU on (features, ranks) samples (host arrays, count rows): features
 * are standardised with the sample mean and deviation, the target is log2(1 + rank), the loss
 * the mean squared error, optimised by Adam over full batches; forward and backward run in the
 * library's kernels (FP16 weights, FP32 accumulation). Synchronises. */
hmat_status hmat_rankmodel_train(const float *features, const float *ranks, int64_t count,
                                 const hmat_train_opts *opts, void *stream, hmat_rankmodel_t *out);

/* Predicted ranks (2^y - 1 of the network's output y) for count feature rows. Synchronises. */
hmat_status hmat_rankmodel_predict(const hmat_rankmodel_t m, const float *features, int64_t count, float *ranks);

/* Copy the model out: weights (HMAT_RANK_PARAMS floats, the FP16 values the forward pass uses,
 * widened), feature mean and deviation (HMAT_RANK_FEATURES each), final training loss. Any output
 * may be NULL. */
hmat_status hmat_rankmodel_get(const hmat_rankmodel_t m, float *weights, float *mean, float *dev, float *loss);

/* A model from given weights (rounded to FP16) and normalisation. */
hmat_status hmat_rankmodel_create(const float *weights, const float *mean, const float *dev, hmat_rankmodel_t *out);

/* Gradient of the training loss with respect to the weights at the model's current weights, and
 * the loss, on the given samples (as one training step computes them). Synchronises. */
hmat_status hmat_rankmodel_grad(const hmat_rankmodel_t m, const float *features, const float *ranks, int64_t count,
                                float *grad, float *loss);

/* The same gradient and loss as hmat_rankmodel_grad (the same FP32 standardisation, the targets
 * evaluated in FP64 and rounded to FP32; the sums differ only in the order of their atomic
 * accumulation), computed without allocating any device memory (the paper has no counterpart
 * of this call; it is a library convenience). It is for
 * callers that must not allocate: code that runs under a fixed device-memory budget or beside
 * an allocator it must not re-enter (a custom allocator hook that itself fine-tunes the model,
 * a serving loop whose memory is reserved up front), where a stray allocation can fail or
 * stall. Every device buffer of the call is part of one fixed array compiled into the library,
 * HMAT_RANKGRAD_NOALLOC_MAX * (HMAT_RANK_FEATURES + 1) + HMAT_RANK_PARAMS + 1 floats (about
 * 0.87 MB) per device:
 *   - count must be 1 .. HMAT_RANKGRAD_NOALLOC_MAX; more samples -> HMAT_EINVAL, nothing runs;
 *   - features (count x HMAT_RANK_FEATURES, row-major) and ranks (count) are raw host values,
 *     standardised on the device with the model's mean and deviation; grad
 *     (HMAT_RANK_PARAMS) and *loss are host outputs; loss may be NULL;
 *   - the gradient and loss accumulators in the array are set to zero by every call before
 *     it accumulates, so no state carries over between calls;
 *   - every call looks up the array's address on the current device (cudaGetSymbolAddress,
 *     which allocates nothing) and sets the network kernel's shared-memory limit; the first
 *     call on a device also loads the library's kernels there, so make one call before any
 *     stream capture begins;
 *   - calls on one device share the array: two calls that overlap in time (other threads,
 *     other streams) race on it and may return wrong results; serialise them;
 *   - runs on stream (NULL = the default stream) and synchronises it before returning;
 *   - m must live on the current device. */
#define HMAT_RANKGRAD_NOALLOC_MAX 16384
hmat_status hmat_rankmodel_grad_noalloc(const hmat_rankmodel_t m, const float *features, const float *ranks,
                                        int64_t count, float *grad, float *loss, void *stream);

void hmat_rankmodel_destroy(hmat_rankmodel_t m);

/* Handle management and errors (library conventions; no counterpart in the paper).
 * Release h and its device memory (NULL is a no-op). A handle's device memory is freed in stream
 * order on the stream of the call that made it (hmat_build, hmat_multiply; for
 * hmat_multiply_batched, the caller's stream), so that stream must still exist when the handle is
 * destroyed: destroy handles before their stream. */
void hmat_destroy(hmat_t h);

/* Message of the last failed call on this thread ("" if none). */
const char *hmat_last_error(void);

/* Route the library's device allocations through alloc/free (both non-NULL), or restore the
 * default stream-ordered CUDA pool (both NULL). alloc(bytes, stream, ctx) returns a device
 * pointer or NULL; free(ptr, ctx) releases it. Covers every buffer of builds, products,
 * matrix-vector products and error estimates (factors, plan tables, sampling buffers); not the
 * cudaMalloc buffers listed under the conventions above. A buffer is released through the
 * free function set when it is released, so change the allocator only while no handle made
 * under the previous one is alive. Not thread-safe against concurrent calls. */
hmat_status hmat_set_allocator(void *(*alloc)(size_t bytes, void *stream, void *ctx),
                               void (*free_fn)(void *ptr, void *ctx), void *ctx);

#ifdef __cplusplus
}
#endif

#endif /* HMAT_H */
