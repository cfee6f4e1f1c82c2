// hmat_tree.h -- host-side cluster tree, block-cluster tree and sum-expression plan.
#pragma once
#include <algorithm>
#include <atomic>
#include <cstdint>
#include <exception>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "hmat_internal.h"

namespace hm {

// Runs fn(0 .. count-1) on up to 16 host threads, the calling thread included. If fn throws on
// any thread, no thread takes a new index, and the first exception is rethrown on the calling
// thread once all threads have joined: no exception leaves a worker thread (that would end the
// process). If the system refuses a new thread, the threads already started do the work.
template <typename F>
void parallel_for(size_t count, F &&fn) {
  const unsigned hw = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
  std::atomic<size_t> next{0};
  std::exception_ptr err;
  std::mutex mu;
  auto worker = [&]() {
    try {
      for (size_t i = next++; i < count; i = next++) fn(i);
    } catch (...) {
      std::lock_guard<std::mutex> lk(mu);
      if (!err) err = std::current_exception();
      next = count;
    }
  };
  const size_t nt = std::min<size_t>(hw, count);
  std::vector<std::thread> th;
  th.reserve(nt);
  for (size_t k = 1; k < nt; k++) {
    try {
      th.emplace_back(worker);
    } catch (...) {
      break;
    }
  }
  worker();
  for (auto &x : th) x.join();
  if (err) std::rethrow_exception(err);
}

struct Cluster {
  int level = 0;
  int64_t begin = 0, size = 0;
  int child[2] = {-1, -1};
  double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
};

enum BlockKind : int { BK_INNER = 0, BK_FAR = 1, BK_NEAR = 2 };

struct Block {
  int tau = -1, sigma = -1, kind = BK_INNER, level = 0;
  int parent = -1;
  int child[4] = {-1, -1, -1, -1};
  int nchild = 0;
  int leaf = -1;               // depth-first leaf number (leaves only)
  int32_t leaf_lo = 0, leaf_hi = 0;
};

struct Tree {
  int64_t n = 0;
  int dim = 0, leaf_size = 0, depth = 0;
  double eta = 0;
  std::vector<double> orig;    // points in original order (n x dim)
  std::vector<double> pts;     // points in permuted order
  std::vector<int64_t> perm;   // perm[i] = original index of permuted position i
  std::vector<Cluster> cl;
  std::vector<Block> bl;
  std::vector<int> leaf_block; // leaf -> block
  int csp = 0;
  // device copies (owned)
  double *d_pts = nullptr;
  BlockDev *d_blocks = nullptr;
  ~Tree();
};

// Def. 2.2 / Def. 2.3 / Algorithm 1. Returns nullptr on invalid input.
std::shared_ptr<Tree> build_tree(const double *xyz, int64_t n, int dim, int leaf_size, double eta);

// Symbolic restriction (Algorithm 3) over the whole block tree, from S(I,I) = HK.
struct PlanTerm {
  int32_t type;        // TermJobType
  int32_t a, b;        // see TermJob
  int32_t rank;
  int block;           // block tau' x sigma' where the term was created
};

// The low-rank terms of S_R(b) are the terms created (by the restriction into b) at b and at
// every ancestor of b; the planner stores the terms created at a block contiguously, so a
// target's terms are the ranges of the blocks on its path to the root.
struct Plan {
  std::vector<PlanTerm> terms;          // grouped by creating block
  std::vector<int32_t> blk_term_lo, blk_term_hi;  // per block: its created terms
  std::vector<int32_t> nterm_cum;       // per block: number of terms of S_R(block)
  std::vector<int64_t> rank_cum;        // per block: sum of their ranks
  std::vector<int64_t> leaf_pair_off;   // nleaf + 1
  std::vector<PairDev> leaf_pairs;      // S_H(leaf)
};

// rankA/rankB: per leaf ranks of the two factors (-1 for dense leaves).
void build_plan(const Tree &t, const std::vector<int32_t> &rankA, const std::vector<int32_t> &rankB, Plan &plan);

}  // namespace hm
