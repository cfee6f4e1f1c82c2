// hmat_tree.cpp -- cluster tree (Def. 2.2), admissibility (Def. 2.3), block-cluster tree
// (Algorithm 1) and the symbolic sum-expression plan (Algorithm 3 applied from S(I,I) = HK,
// Algorithm 4). Host code; compiled without floating-point contraction so the tree decisions
// are the plain IEEE values of their formulas.
#include "hmat_tree.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <limits>
#include <stdexcept>
#include <thread>
#include <utility>
#include <cuda_runtime.h>

namespace hm {

Tree::~Tree() {
  if (d_pts) cudaFree(d_pts);
  if (d_blocks) cudaFree(d_blocks);
}

namespace {

struct Builder {
  Tree &t;
  void bbox(int64_t begin, int64_t size, double *lo, double *hi) {
    for (int d = 0; d < t.dim; d++) { lo[d] = INFINITY; hi[d] = -INFINITY; }
    for (int64_t i = begin; i < begin + size; i++) {
      const double *p = &t.orig[t.perm[i] * t.dim];
      for (int d = 0; d < t.dim; d++) {
        if (p[d] < lo[d]) lo[d] = p[d];
        if (p[d] > hi[d]) hi[d] = p[d];
      }
    }
  }
  // Every cluster above depth D splits in two (D = smallest d with ceil(n/2^d) <= leaf_size):
  // axis = longest bounding-box side (first on ties), points ordered by (coordinate, original
  // index), first child = the first floor(size/2) of them. Only the last split orders its
  // points completely (that order is the one inside the leaves); a split above it only selects
  // the floor(size/2) smallest keys, since each child orders its own points again by its own
  // axis and its bounding box does not depend on their order. The keys are a strict total order,
  // so the selected sets, and hence the permutation, equal those of a full sort at every level.
  //
  // The tree is complete, so a cluster's depth-first (preorder) id follows from its parent's: the
  // first child is id + 1, the second id + 2^(D - level) (after the first child's 2^(D - level) - 1
  // clusters). Clusters therefore fill their own slots and their own ranges of the permutation,
  // and disjoint subtrees are built on different threads with the same result as one thread.
  using Keys = std::vector<std::pair<double, int64_t>>;
  // fills cluster id; above depth D also orders its points for the split and records its
  // children's ids; returns the size of the first child (0 at a leaf)
  int64_t make(int id, int64_t begin, int64_t size, int level, Keys &keys) {
    Cluster c;
    c.level = level;
    c.begin = begin;
    c.size = size;
    bbox(begin, size, c.lo, c.hi);
    int64_t h = 0;
    if (level < t.depth) {
      int axis = 0;
      double best = c.hi[0] - c.lo[0];
      for (int d = 1; d < t.dim; d++) {
        const double e = c.hi[d] - c.lo[d];
        if (e > best) { best = e; axis = d; }
      }
      const double *P = t.orig.data();
      const int dim = t.dim;
      keys.resize(size);
      for (int64_t i = 0; i < size; i++) {
        const int64_t q = t.perm[begin + i];
        keys[i] = {P[q * dim + axis], q};
      }
      auto less = [](const std::pair<double, int64_t> &a, const std::pair<double, int64_t> &b) {
        if (a.first < b.first) return true;
        if (a.first > b.first) return false;
        return a.second < b.second;
      };
      h = size / 2;
      if (level + 1 < t.depth) std::nth_element(keys.begin(), keys.begin() + h, keys.end(), less);
      else std::sort(keys.begin(), keys.end(), less);
      for (int64_t i = 0; i < size; i++) t.perm[begin + i] = keys[i].second;
      c.child[0] = id + 1;
      c.child[1] = id + (1 << (t.depth - level));
    }
    t.cl[id] = c;
    return h;
  }
  void subtree(int id, int64_t begin, int64_t size, int level, Keys &keys) {
    const int64_t h = make(id, begin, size, level, keys);
    if (level < t.depth) {
      subtree(id + 1, begin, h, level + 1, keys);
      subtree(id + (1 << (t.depth - level)), begin + h, size - h, level + 1, keys);
    }
  }
  // the whole cluster tree: the top levels one level at a time (the clusters of a level in
  // parallel), then the subtrees below them in parallel
  void clusters() {
    t.cl.assign(((size_t)2 << t.depth) - 1, Cluster{});
    struct Item {
      int id;
      int64_t begin, size;
    };
    std::vector<Item> cur{Item{0, 0, t.n}};
    const int top = std::min(t.depth, 4);
    for (int level = 0; level < top; level++) {
      std::vector<int64_t> h(cur.size());
      parallel_for(cur.size(), [&](size_t i) {
        Keys keys;
        h[i] = make(cur[i].id, cur[i].begin, cur[i].size, level, keys);
      });
      std::vector<Item> nxt;
      for (size_t i = 0; i < cur.size(); i++) {
        nxt.push_back(Item{cur[i].id + 1, cur[i].begin, h[i]});
        nxt.push_back(Item{cur[i].id + (1 << (t.depth - level)), cur[i].begin + h[i], cur[i].size - h[i]});
      }
      cur.swap(nxt);
    }
    parallel_for(cur.size(), [&](size_t i) {
      Keys keys;
      subtree(cur[i].id, cur[i].begin, cur[i].size, top, keys);
    });
  }
  // eta-admissibility: max(diam tau, diam sigma) <= eta * dist(tau, sigma) with bounding-box
  // diagonals and the Euclidean distance of the boxes; distance zero is never admissible.
  bool admissible(const Cluster &a, const Cluster &b) const {
    double da = 0.0, db = 0.0, dd = 0.0;
    for (int d = 0; d < t.dim; d++) {
      const double ea = a.hi[d] - a.lo[d];
      const double eb = b.hi[d] - b.lo[d];
      da += ea * ea;
      db += eb * eb;
      const double g1 = b.lo[d] - a.hi[d];
      const double g2 = a.lo[d] - b.hi[d];
      double g = g1 > g2 ? g1 : g2;
      if (g < 0.0) g = 0.0;
      dd += g * g;
    }
    da = std::sqrt(da);
    db = std::sqrt(db);
    dd = std::sqrt(dd);
    if (!(dd > 0.0)) return false;
    const double mx = da > db ? da : db;
    return mx <= t.eta * dd;
  }
  int nleaf = 0;
  // Algorithm 1; children tau'-major; leaves numbered depth-first.
  int block(int tau, int sigma) {
    const int id = (int)t.bl.size();
    t.bl.emplace_back();
    Block b;
    b.tau = tau;
    b.sigma = sigma;
    b.level = t.cl[tau].level;
    b.leaf_lo = nleaf;
    const Cluster &ct = t.cl[tau], &cs = t.cl[sigma];
    if (admissible(ct, cs)) {
      b.kind = BK_FAR;
      b.leaf = nleaf++;
    } else if (ct.child[0] >= 0 && cs.child[0] >= 0) {
      b.kind = BK_INNER;
      t.bl[id] = b;
      int k = 0;
      for (int i = 0; i < 2; i++)
        for (int j = 0; j < 2; j++) {
          const int c = block(t.cl[tau].child[i], t.cl[sigma].child[j]);
          t.bl[c].parent = id;
          t.bl[id].child[k++] = c;
        }
      t.bl[id].nchild = 4;
      t.bl[id].leaf_hi = nleaf;
      return id;
    } else {
      b.kind = BK_NEAR;
      b.leaf = nleaf++;
    }
    b.leaf_hi = nleaf;
    t.bl[id] = b;
    return id;
  }
};

}  // namespace

std::shared_ptr<Tree> build_tree(const double *xyz, int64_t n, int dim, int leaf_size, double eta) {
  // leaf_size >= 2 keeps every cluster non-empty (Def. 2.2): a cluster of level depth - 1 holds
  // at least leaf_size points, so each half holds at least leaf_size / 2 >= 1
  if (!xyz || n < 1 || dim < 1 || dim > 3 || leaf_size < 2 || !(eta > 0.0)) return nullptr;
  auto t = std::make_shared<Tree>();
  t->n = n;
  t->dim = dim;
  t->leaf_size = leaf_size;
  t->eta = eta;
  t->orig.assign(xyz, xyz + n * dim);
  int depth = 0;
  while ((n + ((int64_t)1 << depth) - 1) / ((int64_t)1 << depth) > leaf_size) depth++;
  t->depth = depth;
  t->perm.resize(n);
  for (int64_t i = 0; i < n; i++) t->perm[i] = i;
  Builder bd{*t};
  bd.clusters();
  t->pts.resize(n * dim);
  for (int64_t i = 0; i < n; i++)
    for (int d = 0; d < dim; d++) t->pts[i * dim + d] = t->orig[t->perm[i] * dim + d];
  bd.block(0, 0);
  t->leaf_block.assign(bd.nleaf, -1);
  std::vector<int> per_row(t->cl.size(), 0);
  for (size_t b = 0; b < t->bl.size(); b++) {
    if (t->bl[b].leaf >= 0) t->leaf_block[t->bl[b].leaf] = (int)b;
    per_row[t->bl[b].tau]++;
  }
  t->csp = *std::max_element(per_row.begin(), per_row.end());
  return t;
}

// ----------------------------------------------------------------------------------------
// Plan: Algorithm 3 from S(I,I) = S_H(I,I) = {(A|IxI, B|IxI)} down the whole block tree.
// A pair is carried as the two block ids (tau x rho in A, rho x sigma in B); since the tree is
// level-conserving, the blocks tau' x rho' and rho' x sigma' of a child are children of these.
// ----------------------------------------------------------------------------------------

namespace {

// Read-only copies of the block tree for the planner's hot loop.
struct PlanTree {
  const Tree &t;
  const std::vector<int32_t> &rA, &rB;
  std::vector<int32_t> child;  // 4 per block, tau'-major
  std::vector<int8_t> kind;
  std::vector<int32_t> leaf;
  std::vector<int8_t> level;
  PlanTree(const Tree &tt, const std::vector<int32_t> &a, const std::vector<int32_t> &b) : t(tt), rA(a), rB(b) {
    const size_t nb = t.bl.size();
    child.resize(nb * 4);
    kind.resize(nb);
    leaf.resize(nb);
    level.resize(nb);
    for (size_t i = 0; i < nb; i++) {
      const Block &bk = t.bl[i];
      for (int c = 0; c < 4; c++) child[i * 4 + c] = bk.child[c];
      kind[i] = (int8_t)bk.kind;
      leaf[i] = bk.leaf;
      level[i] = (int8_t)bk.level;
    }
  }
};

struct Task {
  int block;
  std::vector<PairDev> pairs;
};

// One depth-first walk of Algorithm 3 below a block. Terms and leaf pairs go to local vectors;
// the per-block arrays of the plan are written at the indices of this walk's blocks only, so
// walks of disjoint subtrees can run on different threads.
struct Planner {
  const PlanTree *ptp = nullptr;
  Plan *planp = nullptr;
  int stop_level = -1;               // >= 0: record a Task instead of descending below this level
  std::vector<Task> *tasks = nullptr;
  std::vector<PlanTerm> terms;
  std::vector<int32_t> blocks;       // blocks whose term range this walk set (local indices)
  std::vector<PairDev> leaf_pairs;
  std::vector<int64_t> leaf_rec;     // (leaf, local offset, count) triples
  std::vector<PairDev> pool;         // pairs of the blocks on the current path, innermost last

  void reset(const PlanTree *t, Plan *p, int stop, std::vector<Task> *tk) {
    ptp = t;
    planp = p;
    stop_level = stop;
    tasks = tk;
    terms.clear();
    blocks.clear();
    leaf_pairs.clear();
    leaf_rec.clear();
    pool.clear();
  }

  // pairs of block b are pool[p0, p1)
  void visit(int b, size_t p0, size_t p1) {
    const PlanTree &pt = *ptp;
    Plan &plan = *planp;
    if (pt.kind[b] != BK_INNER) {
      leaf_rec.push_back(pt.leaf[b]);
      leaf_rec.push_back((int64_t)leaf_pairs.size());
      leaf_rec.push_back((int64_t)(p1 - p0));
      leaf_pairs.insert(leaf_pairs.end(), pool.begin() + p0, pool.begin() + p1);
      return;
    }
    if (stop_level >= 0 && pt.level[b] == stop_level) {
      tasks->push_back(Task{b, std::vector<PairDev>(pool.begin() + p0, pool.begin() + p1)});
      return;
    }
    for (int c = 0; c < 4; c++) {
      const int cb = pt.child[(size_t)b * 4 + c];
      const int ti = c >> 1, si = c & 1;  // tau'-major order of the children
      plan.blk_term_lo[cb] = (int32_t)terms.size();
      int64_t rsum = 0;
      const size_t q0 = pool.size();
      for (size_t q = p0; q < p1; q++) {
        const PairDev pr = pool[q];
        const int32_t *ca = &pt.child[(size_t)pr.blkA * 4], *cbb = &pt.child[(size_t)pr.blkB * 4];
        for (int ri = 0; ri < 2; ri++) {
          const int a2 = ca[ti * 2 + ri];   // tau' x rho'
          const int b2 = cbb[ri * 2 + si];  // rho' x sigma'
          const int kx = pt.kind[a2], ky = pt.kind[b2];
          if (kx == BK_FAR || ky == BK_FAR) {
            PlanTerm tm;
            tm.block = cb;
            if (kx == BK_FAR && ky == BK_FAR) {
              const int ka = pt.rA[pt.leaf[a2]], kb = pt.rB[pt.leaf[b2]];
              tm.type = ka <= kb ? JOB_FF_R : JOB_FF_L;
              tm.a = pt.leaf[a2];
              tm.b = pt.leaf[b2];
              tm.rank = ka <= kb ? ka : kb;
            } else if (kx == BK_FAR) {
              tm.type = JOB_FH;
              tm.a = pt.leaf[a2];
              tm.b = b2;
              tm.rank = pt.rA[pt.leaf[a2]];
            } else {
              tm.type = JOB_HF;
              tm.a = a2;
              tm.b = pt.leaf[b2];
              tm.rank = pt.rB[pt.leaf[b2]];
            }
            rsum += tm.rank;
            terms.push_back(tm);
          } else {
            pool.push_back(PairDev{a2, b2});
          }
        }
      }
      plan.blk_term_hi[cb] = (int32_t)terms.size();
      blocks.push_back(cb);
      plan.nterm_cum[cb] = plan.nterm_cum[b] + (plan.blk_term_hi[cb] - plan.blk_term_lo[cb]);
      plan.rank_cum[cb] = plan.rank_cum[b] + rsum;
      const size_t q1 = pool.size();
      visit(cb, q0, q1);
      pool.resize(q0);
    }
  }
};

}  // namespace

void build_plan(const Tree &t, const std::vector<int32_t> &rankA, const std::vector<int32_t> &rankB, Plan &plan) {
  const size_t nleaf = t.leaf_block.size(), nb = t.bl.size();
  plan.blk_term_lo.assign(nb, 0);
  plan.blk_term_hi.assign(nb, 0);
  plan.nterm_cum.assign(nb, 0);
  plan.rank_cum.assign(nb, 0);
  PlanTree pt(t, rankA, rankB);
  // serial walk down to split_level, then one walk per remaining subtree on a thread pool. The
  // walks' buffers are kept between calls (thread-local), so their memory is already mapped.
  static thread_local std::vector<Planner> walks_tl;
  static thread_local std::vector<Task> tasks_tl;
  std::vector<Planner> &walks = walks_tl;  // the calling thread's buffers, shared with the workers
  std::vector<Task> &tasks = tasks_tl;
  const int split_level = t.depth >= 6 ? 3 : -1;
  tasks.clear();
  if (walks.empty()) walks.resize(1);
  walks[0].reset(&pt, &plan, split_level, &tasks);
  walks[0].pool.push_back(PairDev{0, 0});  // S(I, I) = S_H(I, I) = {(A|I x I, B|I x I)}
  walks[0].visit(0, 0, 1);
  const size_t ntask = tasks.size();
  if (walks.size() < 1 + ntask) walks.resize(1 + ntask);
  for (size_t i = 0; i < ntask; i++) walks[1 + i].reset(&pt, &plan, -1, nullptr);
  const size_t nwalk = 1 + ntask;
  if (ntask > 0)
    parallel_for(ntask, [&](size_t i) {
      Planner &w = walks[1 + i];
      w.pool.assign(tasks[i].pairs.begin(), tasks[i].pairs.end());
      w.visit(tasks[i].block, 0, tasks[i].pairs.size());
    });
  // merge: terms concatenated walk by walk (block ranges shifted), leaf pairs laid out in leaf order
  std::vector<size_t> toff(nwalk + 1, 0);
  size_t npairs = 0;
  for (size_t i = 0; i < nwalk; i++) {
    toff[i + 1] = toff[i] + walks[i].terms.size();
    npairs += walks[i].leaf_pairs.size();
  }
  // term indices are 32-bit in the plan and in the device tables
  if (toff[nwalk] > (size_t)std::numeric_limits<int32_t>::max())
    throw std::length_error("restriction plan: more than 2^31 - 1 low-rank terms");
  plan.terms.resize(toff[nwalk]);
  std::vector<const PairDev *> src(nleaf, nullptr);
  std::vector<int64_t> cnt(nleaf, 0);
  for (size_t i = 0; i < nwalk; i++) {
    const Planner &w = walks[i];
    for (size_t k = 0; k + 2 < w.leaf_rec.size(); k += 3) {
      const int64_t lf = w.leaf_rec[k];
      src[lf] = w.leaf_pairs.data() + w.leaf_rec[k + 1];
      cnt[lf] = w.leaf_rec[k + 2];
    }
  }
  plan.leaf_pair_off.assign(nleaf + 1, 0);
  for (size_t l = 0; l < nleaf; l++) plan.leaf_pair_off[l + 1] = plan.leaf_pair_off[l] + cnt[l];
  plan.leaf_pairs.resize(npairs);
  parallel_for(nwalk, [&](size_t i) {
    const Planner &w = walks[i];
    std::copy(w.terms.begin(), w.terms.end(), plan.terms.begin() + toff[i]);
    const int32_t off = (int32_t)toff[i];
    for (int32_t b : w.blocks) {
      plan.blk_term_lo[b] += off;
      plan.blk_term_hi[b] += off;
    }
    for (size_t k = 0; k + 2 < w.leaf_rec.size(); k += 3) {
      const int64_t lf = w.leaf_rec[k];
      std::copy(src[lf], src[lf] + cnt[lf], plan.leaf_pairs.begin() + plan.leaf_pair_off[lf]);
    }
  });
}

}  // namespace hm
