/*
 * hmat_oracle.c -- plain, slow FP64 CPU oracle for the H-matrix product with
 * blockwise eps-best truncation (Doelz, Harbrecht, Multerer, "On the best
 * approximation of the hierarchical matrix product").
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load this file's library. The CUDA library never
 * links, includes or calls it, and it shares no code with the CUDA library.
 *
 * What it computes, each part citing the passage it follows:
 *   - cluster tree by cardinality-balanced bisection (Def. 2.2; the paper leaves the
 *     construction open, the reading used is stated at or_tree_build);
 *   - eta-admissibility on bounding boxes (Def. 2.3; concrete form left open by the paper);
 *   - block-cluster tree (Algorithm 1), far leaves F and near leaves N;
 *   - kernel-matrix assembly: near leaves dense, far leaves by adaptive cross
 *     approximation (Algorithm 6) stopped by eq. (truncaca);
 *   - the dense product of the stored H-matrices, D_C = D_A * D_B (Sec. 3.1, L = HK);
 *   - per target block: SVD (one-sided Jacobi) and the eps-rank, the smallest k whose
 *     relative Frobenius truncation error is at most eps (Sec. 6, definition of the
 *     eps-rank); the best rank-k approximation (Eckart-Young);
 *   - the exact product block C|tau x sigma = A|tau x I * B|I x sigma for sampled
 *     blocks of large products (the definition of a block of a matrix product);
 *   - the sum-expression of every leaf of the product's block tree, built by the
 *     restriction of Algorithm 3 recursively from S(I,I) = HK (Algorithm 4), counted
 *     per leaf (low-rank terms by origin, H-pairs).
 *
 * Everything is FP64. Built with -ffp-contract=off so a*b+c is never fused: the
 * admissibility and tree decisions are then the plain IEEE results of the formulas.
 * Parity pins: see tests/test_oracle.py (brute force, closed forms, Eckart-Young,
 * rank monotonicity, library SVD at tiny sizes).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXDIM 3

/* ------------------------------------------------------------------ */
/* Cluster tree (Def. 2.2)                                              */
/* ------------------------------------------------------------------ */

typedef struct {
  int level;
  int64_t begin, size;           /* contiguous range in the permuted order */
  int child[2];                  /* -1 for a leaf */
  double lo[OR_MAXDIM], hi[OR_MAXDIM]; /* tight bounding box */
} or_cluster;

typedef struct {
  int tau, sigma;                /* cluster ids */
  int kind;                      /* 0 = inadmissible non-leaf, 1 = far leaf (F), 2 = near leaf (N) */
  int level;
  int child[4];
  int nchild;
  int leaf;                      /* DFS leaf index, -1 for non-leaves */
} or_block;

typedef struct {
  int64_t n;
  int dim, leaf_size, depth;
  double eta;
  double *pts;                   /* permuted copy, n*dim row-major */
  int64_t *perm;                 /* perm[i] = original index of permuted position i */
  or_cluster *cl;
  int ncl;
  or_block *bl;
  int nbl, cap_bl;
  int *leaf_block;               /* leaf index -> block id */
  int nleaf;
} or_tree;

/* sort key: coordinate, then original index (fully deterministic) */
static const double *g_sort_pts;
static int g_sort_dim, g_sort_axis;
static const int64_t *g_sort_orig;
static int cmp_axis(const void *a, const void *b) {
  int64_t i = *(const int64_t *)a, j = *(const int64_t *)b;
  double xi = g_sort_pts[g_sort_orig[i] * g_sort_dim + g_sort_axis];
  double xj = g_sort_pts[g_sort_orig[j] * g_sort_dim + g_sort_axis];
  if (xi < xj) return -1;
  if (xi > xj) return 1;
  int64_t oi = g_sort_orig[i], oj = g_sort_orig[j];
  return (oi < oj) ? -1 : (oi > oj) ? 1 : 0;
}

static void bbox(const or_tree *t, const double *orig_pts, int64_t begin, int64_t size,
                 double *lo, double *hi) {
  for (int d = 0; d < t->dim; d++) { lo[d] = INFINITY; hi[d] = -INFINITY; }
  for (int64_t i = begin; i < begin + size; i++) {
    const double *p = orig_pts + t->perm[i] * t->dim;
    for (int d = 0; d < t->dim; d++) {
      if (p[d] < lo[d]) lo[d] = p[d];
      if (p[d] > hi[d]) hi[d] = p[d];
    }
  }
}

static int build_cluster(or_tree *t, const double *orig_pts, int64_t begin, int64_t size, int level) {
  int id = t->ncl++;
  or_cluster *c = &t->cl[id];
  c->level = level; c->begin = begin; c->size = size;
  c->child[0] = c->child[1] = -1;
  bbox(t, orig_pts, begin, size, c->lo, c->hi);
  if (level < t->depth) {
    int axis = 0;
    double best = c->hi[0] - c->lo[0];
    for (int d = 1; d < t->dim; d++) {
      double e = c->hi[d] - c->lo[d];
      if (e > best) { best = e; axis = d; }
    }
    /* sort the positions begin..begin+size-1 by (coordinate on axis, original index) */
    int64_t *pos = (int64_t *)malloc(sizeof(int64_t) * size);
    for (int64_t i = 0; i < size; i++) pos[i] = begin + i;
    g_sort_pts = orig_pts; g_sort_dim = t->dim; g_sort_axis = axis; g_sort_orig = t->perm;
    qsort(pos, size, sizeof(int64_t), cmp_axis);
    int64_t *tmp = (int64_t *)malloc(sizeof(int64_t) * size);
    for (int64_t i = 0; i < size; i++) tmp[i] = t->perm[pos[i]];
    memcpy(t->perm + begin, tmp, sizeof(int64_t) * size);
    free(tmp); free(pos);
    int64_t h = size / 2;
    int c0 = build_cluster(t, orig_pts, begin, h, level + 1);
    int c1 = build_cluster(t, orig_pts, begin + h, size - h, level + 1);
    t->cl[id].child[0] = c0;
    t->cl[id].child[1] = c1;
  }
  return id;
}

/* Def. 2.3 with the eta-criterion: max(diam tau, diam sigma) <= eta * dist(tau, sigma),
 * diam = bounding-box diagonal, dist = Euclidean distance between the boxes; a pair at
 * distance zero is never admissible. */
static int admissible(const or_tree *t, const or_cluster *a, const or_cluster *b) {
  double da = 0.0, db = 0.0, dd = 0.0;
  for (int d = 0; d < t->dim; d++) {
    double ea = a->hi[d] - a->lo[d];
    double eb = b->hi[d] - b->lo[d];
    da += ea * ea;
    db += eb * eb;
    double g1 = b->lo[d] - a->hi[d];
    double g2 = a->lo[d] - b->hi[d];
    double g = g1 > g2 ? g1 : g2;
    if (g < 0.0) g = 0.0;
    dd += g * g;
  }
  da = sqrt(da); db = sqrt(db); dd = sqrt(dd);
  if (!(dd > 0.0)) return 0;
  double m = da > db ? da : db;
  return m <= t->eta * dd;
}

static int push_block(or_tree *t) {
  if (t->nbl == t->cap_bl) {
    t->cap_bl = t->cap_bl ? 2 * t->cap_bl : 1024;
    t->bl = (or_block *)realloc(t->bl, sizeof(or_block) * t->cap_bl);
  }
  return t->nbl++;
}

/* Algorithm 1 (BuildBlockClusterTree); children in the order tau'-major (tau'_0 x sigma'_0,
 * tau'_0 x sigma'_1, tau'_1 x sigma'_0, tau'_1 x sigma'_1); leaves numbered in DFS order. */
static int build_block(or_tree *t, int tau, int sigma) {
  int id = push_block(t);
  or_block *b = &t->bl[id];
  b->tau = tau; b->sigma = sigma; b->level = t->cl[tau].level;
  b->nchild = 0; b->leaf = -1;
  for (int i = 0; i < 4; i++) b->child[i] = -1;
  const or_cluster *ct = &t->cl[tau], *cs = &t->cl[sigma];
  if (admissible(t, ct, cs)) {
    t->bl[id].kind = 1;
    t->bl[id].leaf = t->nleaf++;
  } else if (ct->child[0] >= 0 && cs->child[0] >= 0) {
    t->bl[id].kind = 0;
    int k = 0;
    for (int i = 0; i < 2; i++)
      for (int j = 0; j < 2; j++) {
        int c = build_block(t, t->cl[tau].child[i], t->cl[sigma].child[j]);
        t->bl[id].child[k++] = c;
      }
    t->bl[id].nchild = 4;
  } else {
    t->bl[id].kind = 2;
    t->bl[id].leaf = t->nleaf++;
  }
  return id;
}

/* Cluster tree reading of Def. 2.2: every cluster above the depth D is split in two,
 * D = smallest d >= 0 with ceil(n / 2^d) <= leaf_size, so all leaves sit on level D and
 * hold at most leaf_size points. Split axis = longest bounding-box side (first on ties);
 * the points are ordered by (coordinate, original index) and the first floor(size/2) form
 * the first child. leaf_size >= 2 is required: the clusters of level d hold floor(n / 2^d)
 * or ceil(n / 2^d) points, so those of level D - 1 hold at least leaf_size and their halves
 * at least floor(leaf_size / 2); with leaf_size = 1 a one-point cluster above level D would
 * split into an empty and a one-point child, and Def. 2.2 (iii) wants every cluster
 * non-empty. */
void *or_tree_build(const double *pts, int64_t n, int dim, int leaf_size, double eta) {
  if (n < 1 || dim < 1 || dim > OR_MAXDIM || leaf_size < 2 || !(eta > 0.0)) return NULL;
  or_tree *t = (or_tree *)calloc(1, sizeof(or_tree));
  t->n = n; t->dim = dim; t->leaf_size = leaf_size; t->eta = eta;
  int depth = 0;
  while ((n + ((int64_t)1 << depth) - 1) / ((int64_t)1 << depth) > leaf_size) depth++;
  t->depth = depth;
  t->perm = (int64_t *)malloc(sizeof(int64_t) * n);
  for (int64_t i = 0; i < n; i++) t->perm[i] = i;
  t->cl = (or_cluster *)calloc(((size_t)2 << depth), sizeof(or_cluster));
  build_cluster(t, pts, 0, n, 0);
  t->pts = (double *)malloc(sizeof(double) * n * dim);
  for (int64_t i = 0; i < n; i++)
    for (int d = 0; d < dim; d++) t->pts[i * dim + d] = pts[t->perm[i] * dim + d];
  build_block(t, 0, 0);
  t->leaf_block = (int *)malloc(sizeof(int) * (t->nleaf > 0 ? t->nleaf : 1));
  for (int b = 0; b < t->nbl; b++)
    if (t->bl[b].leaf >= 0) t->leaf_block[t->bl[b].leaf] = b;
  return t;
}

void or_tree_free(void *h) {
  or_tree *t = (or_tree *)h;
  if (!t) return;
  free(t->pts); free(t->perm); free(t->cl); free(t->bl); free(t->leaf_block); free(t);
}

void or_tree_counts(const void *h, int64_t *out) {
  const or_tree *t = (const or_tree *)h;
  out[0] = t->ncl; out[1] = t->nbl; out[2] = t->nleaf; out[3] = t->depth;
}

void or_tree_export(const void *h, int64_t *perm, int64_t *cl_info /* ncl x 5 */,
                    int64_t *bl_info /* nbl x 6: tau, sigma, kind, level, leaf, nchild */,
                    int64_t *bl_child /* nbl x 4 */) {
  const or_tree *t = (const or_tree *)h;
  if (perm) memcpy(perm, t->perm, sizeof(int64_t) * t->n);
  if (cl_info)
    for (int c = 0; c < t->ncl; c++) {
      cl_info[c * 5 + 0] = t->cl[c].level;
      cl_info[c * 5 + 1] = t->cl[c].begin;
      cl_info[c * 5 + 2] = t->cl[c].size;
      cl_info[c * 5 + 3] = t->cl[c].child[0];
      cl_info[c * 5 + 4] = t->cl[c].child[1];
    }
  if (bl_info)
    for (int b = 0; b < t->nbl; b++) {
      bl_info[b * 6 + 0] = t->bl[b].tau;
      bl_info[b * 6 + 1] = t->bl[b].sigma;
      bl_info[b * 6 + 2] = t->bl[b].kind;
      bl_info[b * 6 + 3] = t->bl[b].level;
      bl_info[b * 6 + 4] = t->bl[b].leaf;
      bl_info[b * 6 + 5] = t->bl[b].nchild;
    }
  if (bl_child)
    for (int b = 0; b < t->nbl; b++)
      for (int i = 0; i < 4; i++) bl_child[b * 4 + i] = t->bl[b].child[i];
}

/* ------------------------------------------------------------------ */
/* Kernels and H-matrix assembly                                       */
/* ------------------------------------------------------------------ */

/* kernel 0: exp(-|x-y|); kernel 1: 1/(1+|x-y|^2); kernel 2: (1 + x.y)^2, a separable
 * kernel of global rank <= (d+1)(d+2)/2 used as a closed-form check */
static double kernel_eval(int kernel, const double *x, const double *y, int dim) {
  if (kernel == 2) {
    double ip = 0.0;
    for (int d = 0; d < dim; d++) ip += x[d] * y[d];
    return (1.0 + ip) * (1.0 + ip);
  }
  double r2 = 0.0;
  for (int d = 0; d < dim; d++) {
    double e = x[d] - y[d];
    r2 += e * e;
  }
  if (kernel == 0) return exp(-sqrt(r2));
  return 1.0 / (1.0 + r2);
}

typedef struct {
  const or_tree *t;
  int nleaf;                  /* t->nleaf, kept so that freeing never reads the tree, which a
                                 garbage collector may have freed first */
  int kernel;
  int prec32;                 /* factors rounded to float after assembly */
  int *rank;                  /* per leaf; -1 for near leaves */
  double **U, **V;            /* far: U (m x k), V (n x k), column-major */
  double **D;                 /* near: m x n column-major */
} or_hmat;

static double round_prec(double v, int prec32) { return prec32 ? (double)(float)v : v; }

/* Algorithm 6 (ACA) on the block tau x sigma given entry-wise. Reading of the parts the
 * paper leaves open: the first pivot row is the block's first row; each later pivot row is
 * the unused row where |l_r| is largest; the column pivot is the largest |u_hat_r| (first
 * on ties); a residual row that is entirely zero is marked used and the next unused row in
 * order is tried. Stop by eq. (truncaca): ||l_{k+1}|| ||u_{k+1}|| <= eps ||L_k U_k||_F,
 * keeping the last term; also stop at rank min(m, n) or when every row is used. */
static int aca_block(const or_tree *t, int kernel, int64_t r0, int64_t m, int64_t c0, int64_t n,
                     double eps, int kmax, double **Uout, double **Vout) {
  int cap = kmax < (int)(m < n ? m : n) ? kmax : (int)(m < n ? m : n);
  double *L = (double *)malloc(sizeof(double) * m * (cap > 0 ? cap : 1));
  double *R = (double *)malloc(sizeof(double) * n * (cap > 0 ? cap : 1));
  char *used = (char *)calloc(m, 1);
  double *row = (double *)malloc(sizeof(double) * n);
  double *col = (double *)malloc(sizeof(double) * m);
  const int dim = t->dim;
  double norm2 = 0.0;  /* ||L_k U_k||_F^2 */
  int k = 0;
  int64_t i_piv = 0;
  while (k < cap) {
    /* find a pivot row with a nonzero residual row */
    int found = 0;
    int64_t j_piv = 0;
    while (!found) {
      if (i_piv < 0 || used[i_piv]) {
        i_piv = -1;
        for (int64_t i = 0; i < m; i++) if (!used[i]) { i_piv = i; break; }
        if (i_piv < 0) break;
      }
      const double *x = t->pts + (r0 + i_piv) * dim;
      for (int64_t j = 0; j < n; j++) {
        double v = kernel_eval(kernel, x, t->pts + (c0 + j) * dim, dim);
        for (int q = 0; q < k; q++) v -= L[q * m + i_piv] * R[q * n + j];
        row[j] = v;
      }
      used[i_piv] = 1;
      double best = 0.0;
      for (int64_t j = 0; j < n; j++)
        if (fabs(row[j]) > best) { best = fabs(row[j]); j_piv = j; }
      if (best > 0.0) found = 1;
      else i_piv = -1;
    }
    if (!found) break;
    double piv = row[j_piv];
    for (int64_t j = 0; j < n; j++) R[k * n + j] = row[j] / piv;
    const double *y = t->pts + (c0 + j_piv) * dim;
    for (int64_t i = 0; i < m; i++) {
      double v = kernel_eval(kernel, t->pts + (r0 + i) * dim, y, dim);
      for (int q = 0; q < k; q++) v -= R[q * n + j_piv] * L[q * m + i];
      col[i] = v;
    }
    memcpy(L + k * m, col, sizeof(double) * m);
    double nl = 0.0, nu = 0.0;
    for (int64_t i = 0; i < m; i++) nl += L[k * m + i] * L[k * m + i];
    for (int64_t j = 0; j < n; j++) nu += R[k * n + j] * R[k * n + j];
    double cross = 0.0;
    for (int q = 0; q < k; q++) {
      double a = 0.0, b = 0.0;
      for (int64_t i = 0; i < m; i++) a += L[q * m + i] * L[k * m + i];
      for (int64_t j = 0; j < n; j++) b += R[q * n + j] * R[k * n + j];
      cross += a * b;
    }
    double prev = norm2;
    norm2 = prev + 2.0 * cross + nl * nu;
    k++;
    if (sqrt(nl) * sqrt(nu) <= eps * sqrt(prev)) break;
    /* next pivot row: largest |l_k| among unused rows */
    double best = -1.0;
    i_piv = -1;
    for (int64_t i = 0; i < m; i++)
      if (!used[i] && fabs(L[(k - 1) * m + i]) > best) { best = fabs(L[(k - 1) * m + i]); i_piv = i; }
    if (i_piv < 0) break;
  }
  *Uout = (double *)malloc(sizeof(double) * m * (k > 0 ? k : 1));
  *Vout = (double *)malloc(sizeof(double) * n * (k > 0 ? k : 1));
  memcpy(*Uout, L, sizeof(double) * m * k);
  memcpy(*Vout, R, sizeof(double) * n * k);
  free(L); free(R); free(used); free(row); free(col);
  return k;
}

void *or_hmat_build(const void *tree, int kernel, double aca_eps, int aca_kmax, int prec32) {
  const or_tree *t = (const or_tree *)tree;
  or_hmat *h = (or_hmat *)calloc(1, sizeof(or_hmat));
  h->t = t; h->nleaf = t->nleaf; h->kernel = kernel; h->prec32 = prec32;
  h->rank = (int *)malloc(sizeof(int) * t->nleaf);
  h->U = (double **)calloc(t->nleaf, sizeof(double *));
  h->V = (double **)calloc(t->nleaf, sizeof(double *));
  h->D = (double **)calloc(t->nleaf, sizeof(double *));
#pragma omp parallel for schedule(dynamic, 4)
  for (int l = 0; l < t->nleaf; l++) {
    const or_block *b = &t->bl[t->leaf_block[l]];
    const or_cluster *ct = &t->cl[b->tau], *cs = &t->cl[b->sigma];
    int64_t m = ct->size, n = cs->size;
    if (b->kind == 2) {
      double *D = (double *)malloc(sizeof(double) * m * n);
      for (int64_t j = 0; j < n; j++)
        for (int64_t i = 0; i < m; i++)
          D[j * m + i] = round_prec(kernel_eval(kernel, t->pts + (ct->begin + i) * t->dim,
                                                t->pts + (cs->begin + j) * t->dim, t->dim), prec32);
      h->D[l] = D;
      h->rank[l] = -1;
    } else {
      double *U, *V;
      int k = aca_block(t, kernel, ct->begin, m, cs->begin, n, aca_eps, aca_kmax, &U, &V);
      for (int64_t i = 0; i < m * k; i++) U[i] = round_prec(U[i], prec32);
      for (int64_t i = 0; i < n * k; i++) V[i] = round_prec(V[i], prec32);
      h->U[l] = U; h->V[l] = V; h->rank[l] = k;
    }
  }
  return h;
}

void or_hmat_free(void *hh) {
  or_hmat *h = (or_hmat *)hh;
  if (!h) return;
  for (int l = 0; l < h->nleaf; l++) { free(h->U[l]); free(h->V[l]); free(h->D[l]); }
  free(h->U); free(h->V); free(h->D); free(h->rank); free(h);
}

void or_hmat_ranks(const void *hh, int64_t *ranks) {
  const or_hmat *h = (const or_hmat *)hh;
  for (int l = 0; l < h->t->nleaf; l++) ranks[l] = h->rank[l];
}

/* copy a leaf's factors (far: U then V, column-major) or dense block (near) */
void or_hmat_leaf(const void *hh, int leaf, double *U, double *V) {
  const or_hmat *h = (const or_hmat *)hh;
  const or_tree *t = h->t;
  const or_block *b = &t->bl[t->leaf_block[leaf]];
  int64_t m = t->cl[b->tau].size, n = t->cl[b->sigma].size;
  if (b->kind == 2) { memcpy(U, h->D[leaf], sizeof(double) * m * n); return; }
  int k = h->rank[leaf];
  memcpy(U, h->U[leaf], sizeof(double) * m * k);
  memcpy(V, h->V[leaf], sizeof(double) * n * k);
}

/* value of the stored H-matrix at permuted position (i, j) of one leaf */
static double leaf_entry(const or_hmat *h, int leaf, int64_t i, int64_t j) {
  const or_tree *t = h->t;
  const or_block *b = &t->bl[t->leaf_block[leaf]];
  int64_t m = t->cl[b->tau].size, n = t->cl[b->sigma].size;
  if (b->kind == 2) return h->D[leaf][j * m + i];
  double v = 0.0;
  for (int q = 0; q < h->rank[leaf]; q++) v += h->U[leaf][q * m + i] * h->V[leaf][q * n + j];
  return v;
}

/* Dense sub-block [r0, r0+mr) x [c0, c0+nc) of the stored H-matrix, permuted order,
 * column-major with leading dimension ld, by walking the block tree (eq. (blockHMat)). */
static void dense_rec(const or_hmat *h, int b, int64_t r0, int64_t mr, int64_t c0, int64_t nc,
                      double *out, int64_t ld) {
  const or_tree *t = h->t;
  const or_block *bk = &t->bl[b];
  const or_cluster *ct = &t->cl[bk->tau], *cs = &t->cl[bk->sigma];
  int64_t a0 = ct->begin > r0 ? ct->begin : r0;
  int64_t a1 = (ct->begin + ct->size) < (r0 + mr) ? (ct->begin + ct->size) : (r0 + mr);
  int64_t b0 = cs->begin > c0 ? cs->begin : c0;
  int64_t b1 = (cs->begin + cs->size) < (c0 + nc) ? (cs->begin + cs->size) : (c0 + nc);
  if (a0 >= a1 || b0 >= b1) return;
  if (bk->kind == 0) {
    for (int c = 0; c < bk->nchild; c++) dense_rec(h, bk->child[c], r0, mr, c0, nc, out, ld);
    return;
  }
  if (bk->kind == 2) {
    for (int64_t j = b0; j < b1; j++)
      for (int64_t i = a0; i < a1; i++)
        out[(j - c0) * ld + (i - r0)] = leaf_entry(h, bk->leaf, i - ct->begin, j - cs->begin);
    return;
  }
  /* far leaf: the same sums as leaf_entry (over q in ascending order), column by column */
  const int64_t m = ct->size, n = cs->size;
  const double *U = h->U[bk->leaf], *V = h->V[bk->leaf];
  for (int64_t j = b0; j < b1; j++) {
    double *o = out + (j - c0) * ld - r0;
    for (int64_t i = a0; i < a1; i++) o[i] = 0.0;
    for (int q = 0; q < h->rank[bk->leaf]; q++) {
      const double vj = V[q * n + (j - cs->begin)];
      const double *u = U + q * m - ct->begin;
      for (int64_t i = a0; i < a1; i++) o[i] += u[i] * vj;
    }
  }
}

/* The window is cut along its longer side into parts filled on separate threads; every entry
 * is the same leaf_entry value either way. */
void or_hmat_dense_sub(const void *hh, int64_t r0, int64_t mr, int64_t c0, int64_t nc,
                       double *out, int64_t ld) {
  const or_hmat *h = (const or_hmat *)hh;
  for (int64_t j = 0; j < nc; j++)
    for (int64_t i = 0; i < mr; i++) out[j * ld + i] = 0.0;
  int by_cols = nc >= mr;
  int64_t len = by_cols ? nc : mr;
  int64_t parts = len >= 1024 ? 64 : 1;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t q = 0; q < parts; q++) {
    int64_t lo = len * q / parts, hi = len * (q + 1) / parts;
    if (by_cols)
      dense_rec(h, 0, r0, mr, c0 + lo, hi - lo, out + lo * ld, ld);
    else
      dense_rec(h, 0, r0 + lo, hi - lo, c0, nc, out + lo, ld);
  }
}

/* ------------------------------------------------------------------ */
/* Dense product and block products                                    */
/* ------------------------------------------------------------------ */

/* C = A * B, all n x n column-major; every C(i,j) sums k = 0..n-1 in ascending order. */
void or_matmul(const double *A, const double *B, double *C, int64_t m, int64_t kk, int64_t n) {
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n; j++) {
    double *c = C + j * m;
    for (int64_t i = 0; i < m; i++) c[i] = 0.0;
    for (int64_t k = 0; k < kk; k++) {
      double bkj = B[j * kk + k];
      const double *a = A + k * m;
      for (int64_t i = 0; i < m; i++) c[i] += a[i] * bkj;
    }
  }
}

/* C|tau x sigma = A|tau x I * B|I x sigma for the permuted ranges [r0, r0+m) and
 * [c0, c0+n), the inner index taken in chunks of `chunk` rows of B. */
void or_block_product(const void *ha, const void *hb, int64_t r0, int64_t m, int64_t c0, int64_t n,
                      int64_t chunk, double *out) {
  const or_hmat *A = (const or_hmat *)ha;
  int64_t N = A->t->n;
  for (int64_t i = 0; i < m * n; i++) out[i] = 0.0;
  double *Ab = (double *)malloc(sizeof(double) * m * chunk);
  double *Bb = (double *)malloc(sizeof(double) * chunk * n);
  for (int64_t k0 = 0; k0 < N; k0 += chunk) {
    int64_t kc = (N - k0) < chunk ? (N - k0) : chunk;
    or_hmat_dense_sub(ha, r0, m, k0, kc, Ab, m);
    or_hmat_dense_sub(hb, k0, kc, c0, n, Bb, kc);
#pragma omp parallel for schedule(static)
    for (int64_t j = 0; j < n; j++)
      for (int64_t k = 0; k < kc; k++) {
        double bkj = Bb[j * kc + k];
        for (int64_t i = 0; i < m; i++) out[j * m + i] += Ab[k * m + i] * bkj;
      }
  }
  free(Ab); free(Bb);
}

/* ------------------------------------------------------------------ */
/* SVD (one-sided Jacobi, Hestenes) and eps-rank                       */
/* ------------------------------------------------------------------ */

/* Singular values (descending) and, if U/V non-NULL, vectors of the m x n column-major M.
 * U is m x p, V is n x p, p = min(m, n). Returns the number of sweeps, or -1 if it did
 * not converge in 80 sweeps. */
int or_svd(const double *M, int64_t m, int64_t n, double *s, double *U, double *V) {
  int trans = m < n;
  int64_t r = trans ? n : m, c = trans ? m : n; /* work on W (r x c), r >= c */
  double *W = (double *)malloc(sizeof(double) * r * c);
  double *X = (double *)calloc(c * c, sizeof(double));
  for (int64_t j = 0; j < c; j++)
    for (int64_t i = 0; i < r; i++) W[j * r + i] = trans ? M[i * m + j] : M[j * m + i];
  for (int64_t j = 0; j < c; j++) X[j * c + j] = 1.0;
  int sweep, conv = 0;
  for (sweep = 0; sweep < 80 && !conv; sweep++) {
    conv = 1;
    for (int64_t p = 0; p < c - 1; p++)
      for (int64_t q = p + 1; q < c; q++) {
        double a = 0.0, b = 0.0, g = 0.0;
        double *wp = W + p * r, *wq = W + q * r;
        for (int64_t i = 0; i < r; i++) { a += wp[i] * wp[i]; b += wq[i] * wq[i]; g += wp[i] * wq[i]; }
        if (g == 0.0 || fabs(g) <= 1e-15 * sqrt(a * b)) continue;
        conv = 0;
        double zeta = (b - a) / (2.0 * g);
        double tt = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        double cs = 1.0 / sqrt(1.0 + tt * tt), sn = cs * tt;
        for (int64_t i = 0; i < r; i++) {
          double x = wp[i], y = wq[i];
          wp[i] = cs * x - sn * y;
          wq[i] = sn * x + cs * y;
        }
        double *xp = X + p * c, *xq = X + q * c;
        for (int64_t i = 0; i < c; i++) {
          double x = xp[i], y = xq[i];
          xp[i] = cs * x - sn * y;
          xq[i] = sn * x + cs * y;
        }
      }
  }
  /* singular values = column norms; order descending */
  double *nrm = (double *)malloc(sizeof(double) * c);
  int64_t *ord = (int64_t *)malloc(sizeof(int64_t) * c);
  for (int64_t j = 0; j < c; j++) {
    double v = 0.0;
    for (int64_t i = 0; i < r; i++) v += W[j * r + i] * W[j * r + i];
    nrm[j] = sqrt(v);
    ord[j] = j;
  }
  for (int64_t a = 1; a < c; a++) { /* insertion sort, stable, descending */
    int64_t x = ord[a], b = a - 1;
    while (b >= 0 && nrm[ord[b]] < nrm[x]) { ord[b + 1] = ord[b]; b--; }
    ord[b + 1] = x;
  }
  for (int64_t j = 0; j < c; j++) s[j] = nrm[ord[j]];
  if (U && V) {
    /* left vectors of W: columns of W / norm; right vectors: X */
    double *Lw = trans ? V : U;   /* r x c */
    double *Rw = trans ? U : V;   /* c x c */
    for (int64_t jj = 0; jj < c; jj++) {
      int64_t j = ord[jj];
      double inv = nrm[j] > 0.0 ? 1.0 / nrm[j] : 0.0;
      for (int64_t i = 0; i < r; i++) Lw[jj * r + i] = W[j * r + i] * inv;
      for (int64_t i = 0; i < c; i++) Rw[jj * c + i] = X[j * c + i];
    }
  }
  free(W); free(X); free(nrm); free(ord);
  return conv ? sweep : -1;
}

/* smallest k with sqrt(sum_{i>=k} s_i^2) <= eps * sqrt(sum_i s_i^2); s descending.
 * A zero block has rank 0. */
int64_t or_eps_rank(const double *s, int64_t p, double eps) {
  double tot = 0.0;
  for (int64_t i = 0; i < p; i++) tot += s[i] * s[i];
  if (tot == 0.0) return 0;
  double tail = 0.0;
  int64_t k = p;
  /* walk from the end, accumulating the tail while it stays within eps */
  for (int64_t i = p - 1; i >= 0; i--) {
    double nt = tail + s[i] * s[i];
    if (sqrt(nt) <= eps * sqrt(tot)) { tail = nt; k = i; }
    else break;
  }
  return k;
}

/* Singular values of an m x n column-major M whose numerical rank is far below min(m, n)
 * (the large far blocks of a product). Householder QR with column pivoting (Businger and
 * Golub 1965; Golub and Van Loan, "Matrix Computations", Sec. 5.4.1): at step j the remaining
 * column of largest norm is swapped into place and reflected onto e_j; the column norms are
 * recomputed exactly at every step. The factorisation stops at the first step whose remaining
 * (m - j) x (n - j) block has Frobenius norm <= tol * ||M||_F. The singular values of the k
 * leading rows of R are those of M P Q-rotated with the remaining block set to zero; they come
 * from the one-sided Jacobi SVD above. Writes them (descending) to s (room for min(m, n)),
 * returns k and sets *resid to the remaining block's Frobenius norm, which bounds the dropped
 * energy: sum_{i >= k} s_i(M)^2 <= resid^2 (the best rank-k error is at most that of Q R_k P^T). */
int64_t or_svd_values_qrcp(const double *M, int64_t m, int64_t n, double tol, double *s, double *resid) {
  int64_t p = m < n ? m : n;
  double *A = (double *)malloc(sizeof(double) * (m * n > 0 ? m * n : 1));
  double *cn = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
  double *v = (double *)malloc(sizeof(double) * (m > 0 ? m : 1));
  double fro2 = 0.0;
  for (int64_t i = 0; i < m * n; i++) { A[i] = M[i]; fro2 += M[i] * M[i]; }
  double rem = 0.0;
  int64_t k = 0;
  for (int64_t j = 0; j < p; j++) {
#pragma omp parallel for schedule(static)
    for (int64_t c = j; c < n; c++) {
      double t = 0.0;
      for (int64_t r = j; r < m; r++) t += A[c * m + r] * A[c * m + r];
      cn[c] = t;
    }
    rem = 0.0;
    int64_t piv = j;
    for (int64_t c = j; c < n; c++) {
      rem += cn[c];
      if (cn[c] > cn[piv]) piv = c;
    }
    if (sqrt(rem) <= tol * sqrt(fro2)) break;
    if (piv != j)
      for (int64_t r = 0; r < m; r++) { double t = A[j * m + r]; A[j * m + r] = A[piv * m + r]; A[piv * m + r] = t; }
    /* reflector H = I - 2 v v^T / (v^T v) with H x = alpha e_1, x = A[j:m, j] */
    double nx = 0.0;
    for (int64_t r = j; r < m; r++) nx += A[j * m + r] * A[j * m + r];
    nx = sqrt(nx);
    double x0 = A[j * m + j];
    double alpha = x0 >= 0.0 ? -nx : nx;
    v[j] = x0 - alpha;
    double vtv = v[j] * v[j];
    for (int64_t r = j + 1; r < m; r++) { v[r] = A[j * m + r]; vtv += v[r] * v[r]; }
    if (vtv > 0.0) {
#pragma omp parallel for schedule(static)
      for (int64_t c = j + 1; c < n; c++) {
        double d = 0.0;
        for (int64_t r = j; r < m; r++) d += v[r] * A[c * m + r];
        double f = 2.0 * d / vtv;
        for (int64_t r = j; r < m; r++) A[c * m + r] -= f * v[r];
      }
    }
    A[j * m + j] = alpha;
    for (int64_t r = j + 1; r < m; r++) A[j * m + r] = 0.0;
    k = j + 1;
    rem = 0.0;
  }
  *resid = sqrt(rem);
  if (k > 0) {
    double *R = (double *)malloc(sizeof(double) * k * n);
    for (int64_t c = 0; c < n; c++)
      for (int64_t r = 0; r < k; r++) R[c * k + r] = r <= c ? A[c * m + r] : 0.0;
    or_svd(R, k, n, s, NULL, NULL);
    free(R);
  }
  free(A); free(cn); free(v);
  return k;
}

/* ------------------------------------------------------------------ */
/* Sum-expressions by Algorithm 3 / Algorithm 4                        */
/* ------------------------------------------------------------------ */

typedef struct { int *tau_rho_sigma; int n, cap; } triple_list;

static int find_block(const or_tree *t, int parent_block, int tau, int sigma);

/* block id of tau x sigma, or -1 if it is not in the block tree. The block tree is
 * searched from the root along the ancestors of tau and sigma. */
static int lookup(const or_tree *t, int tau, int sigma) {
  return find_block(t, 0, tau, sigma);
}

static int contains(const or_cluster *a, const or_cluster *b) {
  return a->begin <= b->begin && b->begin + b->size <= a->begin + a->size;
}

static int find_block(const or_tree *t, int b, int tau, int sigma) {
  const or_block *bk = &t->bl[b];
  if (bk->tau == tau && bk->sigma == sigma) return b;
  if (bk->kind != 0) return -1;
  for (int c = 0; c < bk->nchild; c++) {
    const or_block *ch = &t->bl[bk->child[c]];
    if (contains(&t->cl[ch->tau], &t->cl[tau]) && contains(&t->cl[ch->sigma], &t->cl[sigma]) &&
        t->cl[ch->tau].level <= t->cl[tau].level)
      return find_block(t, bk->child[c], tau, sigma);
  }
  return -1;
}

/* Statistics of S(tau', sigma') for every leaf, following Algorithm 4 from
 * S(I, I) = S_H(I, I) = {(A|IxI, B|IxI)} and Algorithm 3 at every step:
 *   out_lr[leaf]  = number of low-rank terms in S_R(leaf)
 *   out_h[leaf]   = number of H-pairs in S_H(leaf)
 *   out_lr_at[leaf * (depth+1) + l] = low-rank terms created at level l
 * The pairs are kept as (tau, rho, sigma) cluster triples. */
static void restrict_rec(const or_tree *t, int b, const int *pairs, int np, int nlr_in,
                         const int *lr_at_in, int64_t *out_lr, int64_t *out_h, int64_t *out_lr_at) {
  const or_block *bk = &t->bl[b];
  int D = t->depth;
  if (bk->kind != 0) {
    out_lr[bk->leaf] = nlr_in;
    out_h[bk->leaf] = np;
    for (int l = 0; l <= D; l++) out_lr_at[(int64_t)bk->leaf * (D + 1) + l] = lr_at_in[l];
    return;
  }
  for (int c = 0; c < bk->nchild; c++) {
    const or_block *ch = &t->bl[bk->child[c]];
    int tp = ch->tau, sp = ch->sigma;
    int lvl = ch->level;
    int *np_pairs = (int *)malloc(sizeof(int) * (np * 2 + 1));
    int nnew = 0, nlr = nlr_in;
    int *lr_at = (int *)malloc(sizeof(int) * (D + 1));
    memcpy(lr_at, lr_at_in, sizeof(int) * (D + 1));
    for (int q = 0; q < np; q++) {
      int rho = pairs[q];
      const or_cluster *cr = &t->cl[rho];
      for (int rc = 0; rc < 2; rc++) {
        int rp = cr->child[rc];
        if (rp < 0) continue;
        int b1 = lookup(t, tp, rp), b2 = lookup(t, rp, sp);
        if (b1 < 0 || b2 < 0) continue; /* cannot happen in a level-conserving tree */
        if (t->bl[b1].kind == 1 || t->bl[b2].kind == 1) { nlr++; lr_at[lvl]++; }
        else np_pairs[nnew++] = rp;
      }
    }
    restrict_rec(t, bk->child[c], np_pairs, nnew, nlr, lr_at, out_lr, out_h, out_lr_at);
    free(np_pairs); free(lr_at);
  }
}

/* Dense value of S(leaf) = S_R(leaf) + S_H(leaf), built along the path from the root by
 * Algorithm 3: at every step the new low-rank products A|tau' x rho' * B|rho' x sigma'
 * (one factor far) are restricted to the leaf and added, and at the leaf the H-pairs are
 * multiplied out (the evaluate() of Algorithm 4 applied to every term). Used to pin that
 * the sum-expression of each leaf equals the product block. out is m x n column-major. */
static void add_product(const or_hmat *A, const or_hmat *B, int64_t r0, int64_t m, int64_t k0,
                        int64_t kc, int64_t c0, int64_t n, double *out) {
  double *Ab = (double *)malloc(sizeof(double) * m * kc);
  double *Bb = (double *)malloc(sizeof(double) * kc * n);
  or_hmat_dense_sub(A, r0, m, k0, kc, Ab, m);
  or_hmat_dense_sub(B, k0, kc, c0, n, Bb, kc);
  for (int64_t j = 0; j < n; j++)
    for (int64_t k = 0; k < kc; k++) {
      double bkj = Bb[j * kc + k];
      for (int64_t i = 0; i < m; i++) out[j * m + i] += Ab[k * m + i] * bkj;
    }
  free(Ab); free(Bb);
}

int or_sumexpr_eval(const void *ha, const void *hb, int leaf, double *out) {
  const or_hmat *A = (const or_hmat *)ha, *B = (const or_hmat *)hb;
  const or_tree *t = A->t;
  int target = t->leaf_block[leaf];
  const or_cluster *T = &t->cl[t->bl[target].tau], *S = &t->cl[t->bl[target].sigma];
  int64_t m = T->size, n = S->size;
  for (int64_t i = 0; i < m * n; i++) out[i] = 0.0;
  int *pairs = (int *)malloc(sizeof(int) * 1);
  int np = 1, nterms = 0;
  pairs[0] = 0;
  int b = 0;
  while (t->bl[b].kind == 0) {
    int next = -1;
    for (int c = 0; c < t->bl[b].nchild; c++) {
      const or_block *ch = &t->bl[t->bl[b].child[c]];
      if (contains(&t->cl[ch->tau], T) && contains(&t->cl[ch->sigma], S)) next = t->bl[b].child[c];
    }
    if (next < 0) { free(pairs); return -1; }
    int tp = t->bl[next].tau, sp = t->bl[next].sigma;
    int *np_pairs = (int *)malloc(sizeof(int) * (2 * np + 1));
    int nnew = 0;
    for (int q = 0; q < np; q++) {
      const or_cluster *cr = &t->cl[pairs[q]];
      for (int rc = 0; rc < 2; rc++) {
        int rp = cr->child[rc];
        if (rp < 0) continue;
        int b1 = lookup(t, tp, rp), b2 = lookup(t, rp, sp);
        if (b1 < 0 || b2 < 0) continue;
        if (t->bl[b1].kind == 1 || t->bl[b2].kind == 1) {
          /* low-rank product computed at this level, restricted to the leaf by index shift */
          add_product(A, B, T->begin, m, t->cl[rp].begin, t->cl[rp].size, S->begin, n, out);
          nterms++;
        } else {
          np_pairs[nnew++] = rp;
        }
      }
    }
    free(pairs);
    pairs = np_pairs; np = nnew; b = next;
  }
  for (int q = 0; q < np; q++)
    add_product(A, B, T->begin, m, t->cl[pairs[q]].begin, t->cl[pairs[q]].size, S->begin, n, out);
  free(pairs);
  return nterms;
}

void or_sumexpr_counts(const void *tree, int64_t *out_lr, int64_t *out_h, int64_t *out_lr_at) {
  const or_tree *t = (const or_tree *)tree;
  int root_pair = 0; /* rho = I */
  int *lr0 = (int *)calloc(t->depth + 1, sizeof(int));
  restrict_rec(t, 0, &root_pair, 1, 0, lr0, out_lr, out_h, out_lr_at);
  free(lr0);
}

int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void or_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
