// hmat_api.cpp -- the C-ABI of libhmat.so: handles, allocation, and the orchestration of the
// product (Algorithm 4 driven level-free: all far targets of the whole tree are truncated
// together by the blocked adaptive range finder, all near targets evaluated together).
#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <memory>
#include <mutex>
#include <stdexcept>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/hmat.h"
#include "hmat_internal.h"
#include "hmat_tree.h"

using namespace hm;

// ------------------------------------------------------------------ errors

namespace {

thread_local std::string g_last_error;

struct HErr {
  hmat_status st;
  std::string msg;
};

[[noreturn]] void fail(hmat_status st, const std::string &msg) { throw HErr{st, msg}; }

void ck(cudaError_t e, const char *what) {
  if (e != cudaSuccess) fail(HMAT_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

template <typename F>
hmat_status guard(F &&f) {
  try {
    f();
    g_last_error.clear();
    return HMAT_OK;
  } catch (const HErr &e) {
    g_last_error = e.msg;
    return e.st;
  } catch (const std::bad_alloc &) {
    g_last_error = "host allocation failed";
    return HMAT_ENOMEM;
  } catch (const std::exception &e) {
    g_last_error = e.what();
    return HMAT_EINVAL;
  } catch (...) {  // nothing crosses the C-ABI
    g_last_error = "unknown exception";
    return HMAT_EINVAL;
  }
}

// ------------------------------------------------------------------ allocation

void *(*g_alloc)(size_t, void *, void *) = nullptr;
void (*g_free)(void *, void *) = nullptr;
void *g_ctx = nullptr;
// per device: the default pool's release threshold has been raised (set once; threads of a batched
// product may race to set it, which is harmless, so the flag only has to be race-free itself)
constexpr int kMaxDevices = 64;
std::atomic<bool> g_pool_set[kMaxDevices];

void keep_pool_memory() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return;
  if (g_pool_set[dev].load(std::memory_order_acquire)) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = std::numeric_limits<uint64_t>::max();
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  g_pool_set[dev].store(true, std::memory_order_release);
}

void *dev_alloc(size_t bytes, cudaStream_t s) {
  if (bytes == 0) bytes = 16;
  if (g_alloc) {
    void *p = g_alloc(bytes, (void *)s, g_ctx);
    if (!p) fail(HMAT_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed (custom allocator)");
    return p;
  }
  keep_pool_memory();
  void *p = nullptr;
  cudaError_t e = cudaMallocAsync(&p, bytes, s);
  if (e != cudaSuccess || !p) {
    cudaGetLastError();
    fail(HMAT_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed: " + cudaGetErrorString(e));
  }
  return p;
}

void dev_free(void *p, cudaStream_t s) {
  if (!p) return;
  if (g_free) g_free(p, g_ctx);
  else cudaFreeAsync(p, s);
}

struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
  cudaStream_t s = nullptr;
  DevBuf() = default;
  DevBuf(size_t b, cudaStream_t st) : bytes(b), s(st) { p = dev_alloc(b, st); }
  DevBuf(const DevBuf &) = delete;
  DevBuf &operator=(const DevBuf &) = delete;
  DevBuf(DevBuf &&o) noexcept : p(o.p), bytes(o.bytes), s(o.s) { o.p = nullptr; }
  DevBuf &operator=(DevBuf &&o) noexcept {
    if (this != &o) {
      release();
      p = o.p; bytes = o.bytes; s = o.s;
      o.p = nullptr;
    }
    return *this;
  }
  ~DevBuf() { release(); }
  void release() {
    if (p) dev_free(p, s);
    p = nullptr;
  }
  template <typename T>
  T *as() const { return (T *)p; }
};

template <typename T>
DevBuf upload(const std::vector<T> &v, cudaStream_t s) {
  DevBuf b(sizeof(T) * std::max<size_t>(v.size(), 1), s);
  if (!v.empty()) ck(cudaMemcpyAsync(b.p, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, s), "upload");
  return b;
}

// An enum parameter arrives from C or ctypes as a plain int that may lie outside the enumeration,
// and reading such a value as the C++ enum type is undefined; its bits are read as an int instead,
// so that the range check is well defined.
template <typename E>
int enum_bits(const E &e) {
  static_assert(sizeof(E) == sizeof(int), "enum parameters are int-sized");
  int v;
  std::memcpy(&v, &e, sizeof v);
  return v;
}

double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

}  // namespace

// ------------------------------------------------------------------ handle

struct hmat_s {
  std::shared_ptr<Tree> tree;
  int prec = 64;                   // element type of the factor buffer
  int kernel = -1;                 // -1 for products
  std::vector<LeafDev> leaves;     // host copy
  DevBuf d_leaves;
  DevBuf d_data;
  int64_t data_elems = 0;
  hmat_stats_t stats{};
  cudaStream_t stream = nullptr;
};

namespace {

size_t esize(int prec) { return prec == 64 ? sizeof(double) : sizeof(float); }

// storage (elements) of every block's subtree, bottom-up
std::vector<double> block_storage(const Tree &t, const std::vector<LeafDev> &lv) {
  std::vector<double> st(t.bl.size(), 0.0);
  for (int b = (int)t.bl.size() - 1; b >= 0; b--) {  // children have larger ids than parents
    const Block &bk = t.bl[b];
    if (bk.kind == BK_INNER) {
      double s = 0;
      for (int c = 0; c < bk.nchild; c++) s += st[bk.child[c]];
      st[b] = s;
    } else {
      const LeafDev &l = lv[bk.leaf];
      st[b] = l.rank < 0 ? (double)l.m * l.n : (double)l.rank * (l.m + l.n);
    }
  }
  return st;
}

// Unique elements of the sum-expression applications, summed over the passes of a product (the
// algorithmic minimum of what a pass must read and write): in each pass, every stored factor
// element that an active target's sum-expression references counts once, plus the targets' In
// and Out panels ((m + n) * pcols elements each).
//  - A low-rank term created at block beta reaches the targets below beta by index shift, so a
//    pass reads the rows of its factors that lie in the union of the row clusters (column
//    clusters) of the active targets below beta.
//  - A factor of an input leaf that several terms share (U of A's leaf, V of B's leaf) counts the
//    union over all of them once.
//  - The H-pair blocks of A and of B count their stored elements once per pass; a block inside
//    another referenced block adds nothing.
// Unions of clusters are bitsets over the leaf clusters (every leaf of the cluster tree sits on
// level depth), built bottom-up over the block tree: children are tau-major and have larger ids
// than their parents. Target i is active in passes 0 .. 2 max(1, rounds_of[i]) - 1, the count
// bytes_apply_use uses; the S and S^T passes of a round share their active set.
double apply_unique_elems(const Tree &t, const Plan &plan, const std::vector<LeafDev> &lA,
                          const std::vector<LeafDev> &lB, const std::vector<double> &storA,
                          const std::vector<double> &storB, const std::vector<TargetDev> &tg,
                          const std::vector<PairDev> &pairs, const std::vector<int32_t> &rounds_of, int pcols,
                          double *parts = nullptr) {
  const size_t nf = tg.size(), ncl = t.cl.size(), nblk = t.bl.size();
  if (nf == 0) return 0.0;
  const int D = t.depth;
  const size_t nlc = (size_t)1 << D;
  std::vector<int32_t> lc0(ncl, 0);  // first leaf cluster of every cluster (parents precede children)
  std::vector<int64_t> lcs(nlc, 0);
  for (size_t c = 0; c < ncl; c++) {
    const Cluster &k = t.cl[c];
    if (k.child[0] >= 0) {
      lc0[k.child[0]] = lc0[c];
      lc0[k.child[1]] = lc0[c] + (int32_t)(((int64_t)1 << (D - k.level)) / 2);
    } else {
      lcs[lc0[c]] = k.size;
    }
  }
  std::vector<int64_t> pre(nlc + 1, 0);  // prefix sums of the leaf clusters' sizes
  for (size_t i = 0; i < nlc; i++) pre[i + 1] = pre[i] + lcs[i];
  auto nbits = [&](int level) { return (int64_t)1 << (D - level); };
  auto nwords = [&](int level) { return (size_t)std::max<int64_t>(1, nbits(level) / 64); };
  // points in the set bits of a bitset over the leaf clusters first .. first + nbits(level) - 1
  auto points = [&](const uint64_t *w, int level, int32_t first) {
    const int64_t nb = nbits(level);
    int64_t sum = 0;
    for (int64_t i0 = 0; i0 < nb; i0 += 64) {
      uint64_t x = w[i0 >> 6];
      if (nb >= 64 && x == ~0ull) {
        sum += pre[first + i0 + 64] - pre[first + i0];
        continue;
      }
      while (x) {
        const int b = __builtin_ctzll(x);
        if (i0 + b < nb) sum += lcs[first + i0 + b];
        x &= x - 1;
      }
    }
    return sum;
  };
  auto fill = [&](uint64_t *w, int level) {
    const int64_t nb = nbits(level);
    if (nb >= 64) std::fill(w, w + nb / 64, ~0ull);
    else w[0] = (1ull << nb) - 1;
  };
  // OR the bitset of a child (half the bits) into half `half` of its parent's bitset
  auto or_half = [&](uint64_t *dst, int dlevel, const uint64_t *src, int half) {
    const int64_t sb = nbits(dlevel) / 2;
    if (sb >= 64) {
      const size_t sw = (size_t)sb / 64;
      for (size_t w = 0; w < sw; w++) dst[half * sw + w] |= src[w];
    } else {
      dst[0] |= (src[0] & ((1ull << sb) - 1)) << (half * sb);
    }
  };
  std::vector<size_t> bo(nblk + 1, 0);
  for (size_t b = 0; b < nblk; b++) bo[b + 1] = bo[b] + nwords(t.bl[b].level);
  std::vector<uint64_t> rows(bo[nblk]), cols(bo[nblk]);
  auto leaf_words = [&](const std::vector<LeafDev> &lv, std::vector<size_t> &off) {
    off.assign(lv.size() + 1, 0);
    for (size_t l = 0; l < lv.size(); l++) off[l + 1] = off[l] + nwords(t.bl[t.leaf_block[l]].level);
  };
  std::vector<size_t> oa, ob;
  leaf_words(lA, oa);
  leaf_words(lB, ob);
  std::vector<uint64_t> objA(oa.back()), objB(ob.back());
  std::vector<int32_t> touchA, touchB, listA, listB;
  std::vector<int32_t> markA(lA.size(), -1), markB(lB.size(), -1), stampA(nblk, -1), stampB(nblk, -1);
  int rmax = 0;
  for (size_t i = 0; i < nf; i++) rmax = std::max(rmax, std::max(1, rounds_of[i]));
  double total = 0.0, tot_panels = 0.0, tot_pairs = 0.0;
  for (int j = 0; j < rmax; j++) {
    std::fill(rows.begin(), rows.end(), 0ull);
    std::fill(cols.begin(), cols.end(), 0ull);
    double u = 0.0, u_panels = 0.0, u_pairs = 0.0;
    listA.clear();
    listB.clear();
    for (size_t i = 0; i < nf; i++) {
      if (std::max(1, rounds_of[i]) <= j) continue;
      const TargetDev &d = tg[i];
      const int lev = t.bl[d.blk].level;
      fill(&rows[bo[d.blk]], lev);
      fill(&cols[bo[d.blk]], lev);
      u_panels += (double)(d.m + d.n) * pcols;
      for (int32_t q = d.pair_lo; q < d.pair_hi; q++) {
        const PairDev &pr = pairs[q];
        if (stampA[pr.blkA] != j) { stampA[pr.blkA] = j; listA.push_back(pr.blkA); }
        if (stampB[pr.blkB] != j) { stampB[pr.blkB] = j; listB.push_back(pr.blkB); }
      }
    }
    for (int b = (int)nblk - 1; b >= 0; b--) {
      const Block &bk = t.bl[b];
      if (bk.kind != BK_INNER) continue;
      for (int k = 0; k < bk.nchild; k++) {
        const int c = bk.child[k];
        or_half(&rows[bo[b]], bk.level, &rows[bo[c]], k / 2);
        or_half(&cols[bo[b]], bk.level, &cols[bo[c]], k % 2);
      }
    }
    touchA.clear();
    touchB.clear();
    for (size_t b = 0; b < nblk; b++) {
      if (plan.blk_term_lo[b] == plan.blk_term_hi[b]) continue;
      const Block &bk = t.bl[b];
      const uint64_t *rw = &rows[bo[b]], *cw = &cols[bo[b]];
      bool any = false;
      for (size_t w = 0; w < nwords(bk.level) && !any; w++) any = rw[w] != 0;
      if (!any) continue;
      const size_t nw = nwords(bk.level);
      const double prow = (double)points(rw, bk.level, lc0[bk.tau]);
      const double pcol = (double)points(cw, bk.level, lc0[bk.sigma]);
      for (int32_t q = plan.blk_term_lo[b]; q < plan.blk_term_hi[b]; q++) {
        const PlanTerm &pt = plan.terms[q];
        if (pt.type == JOB_FF_R || pt.type == JOB_FH) {  // L = U of A's leaf a (rows tau), R new
          uint64_t *o = &objA[oa[pt.a]];
          if (markA[pt.a] != j) { markA[pt.a] = j; std::fill(o, o + nw, 0ull); touchA.push_back(pt.a); }
          for (size_t w = 0; w < nw; w++) o[w] |= rw[w];
          u += (double)pt.rank * pcol;
        } else {  // L new, R = V of B's leaf b (rows sigma)
          uint64_t *o = &objB[ob[pt.b]];
          if (markB[pt.b] != j) { markB[pt.b] = j; std::fill(o, o + nw, 0ull); touchB.push_back(pt.b); }
          for (size_t w = 0; w < nw; w++) o[w] |= cw[w];
          u += (double)pt.rank * prow;
        }
      }
    }
    for (int32_t a : touchA) {
      const Block &bk = t.bl[t.leaf_block[a]];
      u += (double)lA[a].rank * points(&objA[oa[a]], bk.level, lc0[bk.tau]);
    }
    for (int32_t b : touchB) {
      const Block &bk = t.bl[t.leaf_block[b]];
      u += (double)lB[b].rank * points(&objB[ob[b]], bk.level, lc0[bk.sigma]);
    }
    // H-pair blocks: only those with no referenced ancestor
    for (int side = 0; side < 2; side++) {
      const std::vector<int32_t> &lst = side ? listB : listA;
      const std::vector<int32_t> &stp = side ? stampB : stampA;
      const std::vector<double> &stor = side ? storB : storA;
      for (int32_t b : lst) {
        bool inside = false;
        for (int p = t.bl[b].parent; p >= 0 && !inside; p = t.bl[p].parent) inside = stp[p] == j;
        if (!inside) u_pairs += stor[b];
      }
    }
    total += 2.0 * (u + u_panels + u_pairs);
    tot_panels += 2.0 * u_panels;
    tot_pairs += 2.0 * u_pairs;
  }
  if (parts) {  // (low-rank terms, H-pair blocks, panels)
    parts[0] = total - tot_pairs - tot_panels;
    parts[1] = tot_pairs;
    parts[2] = tot_panels;
  }
  return total;
}

void ensure_tree_device(Tree &t, cudaStream_t s) {
  if (t.d_pts) return;
  ck(cudaMalloc(&t.d_pts, sizeof(double) * t.pts.size()), "cudaMalloc points");
  ck(cudaMemcpyAsync(t.d_pts, t.pts.data(), sizeof(double) * t.pts.size(), cudaMemcpyHostToDevice, s), "points");
  std::vector<BlockDev> bd(t.bl.size());
  for (size_t b = 0; b < t.bl.size(); b++) {
    const Block &bk = t.bl[b];
    bd[b].row = t.cl[bk.tau].begin;
    bd[b].col = t.cl[bk.sigma].begin;
    bd[b].m = (int32_t)t.cl[bk.tau].size;
    bd[b].n = (int32_t)t.cl[bk.sigma].size;
    bd[b].leaf_lo = bk.leaf_lo;
    bd[b].leaf_hi = bk.leaf_hi;
    bd[b].parent = bk.parent;
    bd[b].pad = 0;
  }
  ck(cudaMalloc(&t.d_blocks, sizeof(BlockDev) * bd.size()), "cudaMalloc blocks");
  ck(cudaMemcpyAsync(t.d_blocks, bd.data(), sizeof(BlockDev) * bd.size(), cudaMemcpyHostToDevice, s), "blocks");
  ck(cudaStreamSynchronize(s), "tree upload");
}

std::vector<LeafDev> base_leaves(const Tree &t) {
  std::vector<LeafDev> lv(t.leaf_block.size());
  for (size_t l = 0; l < lv.size(); l++) {
    const Block &bk = t.bl[t.leaf_block[l]];
    lv[l].row = t.cl[bk.tau].begin;
    lv[l].col = t.cl[bk.sigma].begin;
    lv[l].m = (int32_t)t.cl[bk.tau].size;
    lv[l].n = (int32_t)t.cl[bk.sigma].size;
    lv[l].rank = bk.kind == BK_NEAR ? -1 : 0;
    lv[l].level = bk.level;
    lv[l].off_u = lv[l].off_v = 0;
  }
  return lv;
}

void fill_structure_stats(hmat_s *h) {
  const Tree &t = *h->tree;
  hmat_stats_t &s = h->stats;
  s.n = t.n;
  s.depth = t.depth;
  s.csp = t.csp;
  s.n_far = s.n_near = 0;
  s.max_rank = 0;
  for (const LeafDev &l : h->leaves) {
    if (l.rank < 0) s.n_near++;
    else {
      s.n_far++;
      s.max_rank = std::max(s.max_rank, (int)l.rank);
    }
  }
  s.storage_bytes = h->data_elems * (int64_t)esize(h->prec);
  s.factor_prec = h->prec;
}

bool same_points(const Tree &t, const double *xyz, int64_t n, int dim) {
  return t.n == n && t.dim == dim && std::memcmp(t.orig.data(), xyz, sizeof(double) * n * dim) == 0;
}

}  // namespace

// ------------------------------------------------------------------ rank proposal

static_assert(HMAT_RANKGRAD_NOALLOC_MAX == RANKGRAD_NOALLOC_MAX, "scratch capacity");

struct hmat_rankmodel_s {
  float *w = nullptr;   // FP32 master weights (device)
  void *w16 = nullptr;  // FP16 weights used by the forward pass (device)
  float mean[RANK_FEATURES], dev[RANK_FEATURES];
  float loss = 0.f;
  ~hmat_rankmodel_s() {
    if (w) cudaFree(w);
    if (w16) cudaFree(w16);
  }
};

namespace {

// per block: the largest rank among the terms of S_R(block) (created at it or an ancestor);
// parents precede children in the block numbering
std::vector<int32_t> chain_max_rank(const Tree &t, const Plan &plan) {
  std::vector<int32_t> mx(t.bl.size(), 0);
  for (size_t b = 0; b < t.bl.size(); b++) {
    int32_t v = t.bl[b].parent >= 0 ? mx[t.bl[b].parent] : 0;
    for (int32_t i = plan.blk_term_lo[b]; i < plan.blk_term_hi[b]; i++) v = std::max(v, plan.terms[i].rank);
    mx[b] = v;
  }
  return mx;
}

double box_diam(const Cluster &c, int dim) {
  double s = 0.0;
  for (int d = 0; d < dim; d++) s += (c.hi[d] - c.lo[d]) * (c.hi[d] - c.lo[d]);
  return std::sqrt(s);
}

double box_dist(const Cluster &a, const Cluster &b, int dim) {
  double s = 0.0;
  for (int d = 0; d < dim; d++) {
    const double g = std::max(0.0, std::max(b.lo[d] - a.hi[d], a.lo[d] - b.hi[d]));
    s += g * g;
  }
  return std::sqrt(s);
}

// the HMAT_RANK_FEATURES features of far leaf l (see hmat_rank_features)
void far_features(const Tree &t, const Plan &plan, const std::vector<int32_t> &mxr, const std::vector<LeafDev> &LA,
                  const std::vector<LeafDev> &LB, double eps, int l, float *f) {
  const int b = t.leaf_block[l];
  const Block &bk = t.bl[b];
  const Cluster &ct = t.cl[bk.tau], &cs = t.cl[bk.sigma];
  const double dist = std::max(box_dist(ct, cs, t.dim), 1e-300);
  f[0] = (float)std::log2((double)ct.size);
  f[1] = (float)std::log2((double)cs.size);
  f[2] = (float)bk.level;
  f[3] = (float)(box_diam(ct, t.dim) / dist);
  f[4] = (float)(box_diam(cs, t.dim) / dist);
  f[5] = (float)std::log2(1.0 + plan.nterm_cum[b]);
  f[6] = (float)std::log2(1.0 + (double)(plan.leaf_pair_off[l + 1] - plan.leaf_pair_off[l]));
  f[7] = (float)mxr[b];
  f[8] = (float)std::log2(1.0 + (double)plan.rank_cum[b]);
  f[9] = (float)std::max(0, (int)LA[l].rank);
  f[10] = (float)std::max(0, (int)LB[l].rank);
  f[11] = (float)(-std::log10(eps));
}

void normalise(const hmat_rankmodel_s *m, const float *in, int64_t count, std::vector<float> &out) {
  out.resize((size_t)count * RANK_FEATURES);
  for (int64_t i = 0; i < count; i++)
    for (int k = 0; k < RANK_FEATURES; k++)
      out[i * RANK_FEATURES + k] = (in[i * RANK_FEATURES + k] - m->mean[k]) / m->dev[k];
}

}  // namespace

// ------------------------------------------------------------------ C-ABI

extern "C" {

const char *hmat_last_error(void) { return g_last_error.c_str(); }

hmat_status hmat_set_allocator(void *(*alloc)(size_t, void *, void *), void (*free_fn)(void *, void *), void *ctx) {
  return guard([&] {
    if ((alloc == nullptr) != (free_fn == nullptr)) fail(HMAT_EINVAL, "alloc and free must both be set or both NULL");
    g_alloc = alloc;
    g_free = free_fn;
    g_ctx = alloc ? ctx : nullptr;
  });
}

hmat_status hmat_points(hmat_ptdist dist_in, int dim, int64_t n, uint64_t seed, double *xyz) {
  const int dist = enum_bits(dist_in);
  return guard([&] {
    if (n < 0 || (n > 0 && !xyz)) fail(HMAT_EINVAL, "bad n or NULL xyz");
    auto draw = [&](uint64_t c) {  // c-th output of the splitmix64 stream
      uint64_t z = seed + (c + 1) * 0x9E3779B97F4A7C15ull;
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      z = z ^ (z >> 31);
      return (double)(z >> 11) * 0x1.0p-53;
    };
    if (dist == HMAT_PTS_CUBE) {
      if (dim < 1 || dim > 3) fail(HMAT_EINVAL, "cube points need dim in 1..3");
      for (int64_t i = 0; i < n * dim; i++) xyz[i] = draw((uint64_t)i);
    } else if (dist == HMAT_PTS_SPHERE) {
      if (dim != 3) fail(HMAT_EINVAL, "sphere points need dim 3");
      const double two_pi = 2.0 * 3.14159265358979323846;
      for (int64_t i = 0; i < n; i++) {
        const double z = 2.0 * draw(2 * (uint64_t)i) - 1.0;
        const double phi = two_pi * draw(2 * (uint64_t)i + 1);
        const double s = std::sqrt(1.0 - z * z);
        xyz[3 * i] = s * std::cos(phi);
        xyz[3 * i + 1] = s * std::sin(phi);
        xyz[3 * i + 2] = z;
      }
    } else {
      fail(HMAT_EINVAL, "unknown point distribution");
    }
  });
}

// HMAT_TRACE=1: print the host-side phases of a build or a product with their wall times to stderr.
struct Trace {
  bool on;
  double t0, last;
  Trace() : on(false), t0(now_ms()), last(t0) {
    const char *e = std::getenv("HMAT_TRACE");
    on = e && e[0] == '1';
  }
  void mark(const char *what) {
    if (!on) return;
    const double t = now_ms();
    std::fprintf(stderr, "hmat trace: %-28s %8.2f ms (total %8.2f)\n", what, t - last, t - t0);
    last = t;
  }
};

hmat_status hmat_build(const double *xyz, int64_t n, int dim, hmat_kernel kernel_in, const hmat_build_opts *opts,
                       const hmat_t tree_from, void *stream, hmat_t *out) {
  if (out) *out = nullptr;
  return guard([&] {
    if (!out || !xyz || !opts) fail(HMAT_EINVAL, "NULL argument");
    if (n < 1 || dim < 1 || dim > 3) fail(HMAT_EINVAL, "need n >= 1 and dim in 1..3");
    // block sizes are 32-bit in the device tables
    if (n > (int64_t)std::numeric_limits<int32_t>::max()) fail(HMAT_EINVAL, "n must be below 2^31");
    const int kernel = enum_bits(kernel_in);
    if (kernel < HMAT_K_EXP || kernel > HMAT_K_POLY2) fail(HMAT_EINVAL, "unknown kernel");
    if (opts->factor_prec != 32 && opts->factor_prec != 64) fail(HMAT_EINVAL, "factor_prec must be 32 or 64");
    // the device kernels stage whole leaves in shared memory, per warp; their layouts are sized
    // for leaves of at most 64 points (an FP64 dense leaf of 107 or more points per warp would not
    // fit the low-rank product kernel's shared memory at all)
    if (opts->leaf_size < 2 || opts->leaf_size > 64) fail(HMAT_EINVAL, "leaf_size must be in 2..64");
    if (!(opts->eta > 0.0) || !(opts->aca_eps > 0.0)) fail(HMAT_EINVAL, "eta and aca_eps must be > 0");
    const int kmax = opts->aca_kmax > 0 ? opts->aca_kmax : 128;
    if (kmax > 128) fail(HMAT_EINVAL, "aca_kmax must be <= 128");
    for (int64_t i = 0; i < n * dim; i++)
      if (!std::isfinite(xyz[i])) fail(HMAT_EINVAL, "non-finite point coordinate");
    cudaStream_t s = (cudaStream_t)stream;
    Trace tr;
    auto h = std::make_unique<hmat_s>();
    h->stream = s;
    if (tree_from) {
      if (!same_points(*tree_from->tree, xyz, n, dim) || tree_from->tree->leaf_size != opts->leaf_size ||
          tree_from->tree->eta != opts->eta)
        fail(HMAT_EMISMATCH, "tree_from was built on other points or tree options");
      h->tree = tree_from->tree;
    } else {
      h->tree = build_tree(xyz, n, dim, opts->leaf_size, opts->eta);
      if (!h->tree) fail(HMAT_EINVAL, "tree construction failed");
    }
    Tree &t = *h->tree;
    ensure_tree_device(t, s);
    tr.mark("build: tree on the device");
    h->prec = opts->factor_prec;
    h->kernel = kernel;
    h->leaves = base_leaves(t);
    std::vector<LeafDev> &lv = h->leaves;
    std::vector<int32_t> near_ids, far_ids;
    for (size_t l = 0; l < lv.size(); l++) (lv[l].rank < 0 ? near_ids : far_ids).push_back((int32_t)l);
    // ACA in batches of FP64 scratch (sized below); each batch is compacted into an exact-size
    // buffer, and the final factor buffer [near leaves | far leaves] is assembled once every rank
    // is known.
    struct BatchOut {
      DevBuf buf;
      int64_t elems;
      std::vector<int32_t> ids;
    };
    std::vector<BatchOut> batches;
    {
      DevBuf d_lv0 = upload(lv, s);
      size_t pos = 0;
      // FP64 scratch per batch: up to 2^29 elements (4 GiB) and an eighth of the free device
      // memory; fewer, larger batches mean fewer launches and synchronisations (a build at
      // N = 32768 went from 7 batches and 40 ms to 2 and 35 ms)
      size_t fr = 0, tot_mem = 0;
      ck(cudaMemGetInfo(&fr, &tot_mem), "memory info");
      const size_t cap_elems = std::max<size_t>((size_t)1 << 24, std::min<size_t>((size_t)1 << 29, fr / 64));
      while (pos < far_ids.size()) {
        std::vector<int64_t> soff;
        std::vector<int32_t> ids;
        size_t tot = 0;
        while (pos < far_ids.size()) {
          const LeafDev &l = lv[far_ids[pos]];
          const size_t need = (size_t)(l.m + l.n) * kmax + l.m;
          if (!ids.empty() && tot + need > cap_elems) break;
          soff.push_back((int64_t)tot);
          ids.push_back(far_ids[pos]);
          tot += need;
          pos++;
        }
        DevBuf scratch(sizeof(double) * tot, s), d_soff = upload(soff, s), d_ids = upload(ids, s);
        // the ACA runs leaves of at most 64 x 64 one warp each, the others one block each: its
        // launch lists the small ones first (the factor layout keeps the batch's own order)
        std::vector<int32_t> order;
        for (size_t i = 0; i < ids.size(); i++)
          if (lv[ids[i]].m <= 64 && lv[ids[i]].n <= 64) order.push_back((int32_t)i);
        const int nsmall = (int)order.size();
        for (size_t i = 0; i < ids.size(); i++)
          if (!(lv[ids[i]].m <= 64 && lv[ids[i]].n <= 64)) order.push_back((int32_t)i);
        std::vector<int32_t> ids_l(ids.size());
        std::vector<int64_t> soff_l(ids.size());
        for (size_t i = 0; i < ids.size(); i++) {
          ids_l[i] = ids[order[i]];
          soff_l[i] = soff[order[i]];
        }
        DevBuf d_ids_l = upload(ids_l, s), d_soff_l = upload(soff_l, s);
        DevBuf d_rk(sizeof(int32_t) * ids.size(), s);
        ck(launch_aca(kernel, t.d_pts, dim, d_lv0.as<LeafDev>(), d_ids_l.as<int32_t>(), (int)ids.size(), nsmall,
                      opts->aca_eps, kmax, scratch.as<double>(), d_soff_l.as<int64_t>(), d_rk.as<int32_t>(), s),
           "ACA launch");
        std::vector<int32_t> rk_l(ids.size()), rk(ids.size());
        ck(cudaMemcpyAsync(rk_l.data(), d_rk.p, sizeof(int32_t) * ids.size(), cudaMemcpyDeviceToHost, s), "ranks");
        ck(cudaStreamSynchronize(s), "ACA");
        for (size_t i = 0; i < ids.size(); i++) rk[order[i]] = rk_l[i];
        // batch-relative offsets
        std::vector<LeafDev> blv = lv;
        int64_t e = 0;
        for (size_t i = 0; i < ids.size(); i++) {
          LeafDev &l = blv[ids[i]];
          l.rank = rk[i];
          l.off_u = e;
          l.off_v = e + (int64_t)l.m * l.rank;
          e = l.off_v + (int64_t)l.n * l.rank;
          lv[ids[i]].rank = rk[i];
          lv[ids[i]].off_u = l.off_u;  // relative for now
        }
        BatchOut bo;
        bo.elems = e;
        bo.ids = ids;
        bo.buf = DevBuf(esize(h->prec) * (size_t)std::max<int64_t>(e, 1), s);
        DevBuf d_blv = upload(blv, s);
        ck(launch_aca_compact(h->prec, d_blv.as<LeafDev>(), d_ids.as<int32_t>(), (int)ids.size(), scratch.as<double>(),
                              d_soff.as<int64_t>(), kmax, bo.buf.p, s),
           "ACA compaction");
        ck(cudaStreamSynchronize(s), "ACA compaction");
        if (tr.on) std::fprintf(stderr, "hmat trace: build: ACA batch of %zu far leaves, %zu scratch elems\n", ids.size(), tot);
        tr.mark("build: ACA batch");
        batches.push_back(std::move(bo));
      }
    }
    int64_t off = 0;
    for (int32_t id : near_ids) {
      lv[id].off_u = off;
      off += (int64_t)lv[id].m * lv[id].n;
    }
    std::vector<int64_t> batch_base;
    for (BatchOut &bo : batches) {
      batch_base.push_back(off);
      for (int32_t id : bo.ids) {
        LeafDev &l = lv[id];
        l.off_u += off;
        l.off_v = l.off_u + (int64_t)l.m * l.rank;
      }
      off += bo.elems;
    }
    h->data_elems = off;
    h->d_data = DevBuf(esize(h->prec) * (size_t)std::max<int64_t>(off, 1), s);
    for (size_t i = 0; i < batches.size(); i++)
      if (batches[i].elems)
        ck(cudaMemcpyAsync((char *)h->d_data.p + esize(h->prec) * batch_base[i], batches[i].buf.p,
                           esize(h->prec) * batches[i].elems, cudaMemcpyDeviceToDevice, s),
           "assemble factors");
    h->d_leaves = upload(lv, s);
    DevBuf d_near = upload(near_ids, s);
    ck(launch_kernel_dense(h->prec, kernel, t.d_pts, dim, h->d_leaves.as<LeafDev>(), d_near.as<int32_t>(),
                           (int)near_ids.size(), h->d_data.p, s),
       "dense leaves");
    ck(cudaStreamSynchronize(s), "build");
    tr.mark("build: assembled, dense leaves");
    fill_structure_stats(h.get());
    *out = h.release();
  });
}

void hmat_destroy(hmat_t h) {
  if (!h) return;
  delete h;
}

hmat_status hmat_leaf_count(const hmat_t h, int64_t *n_leaves) {
  return guard([&] {
    if (!h || !n_leaves) fail(HMAT_EINVAL, "NULL argument");
    *n_leaves = (int64_t)h->leaves.size();
  });
}

hmat_status hmat_leaf_info(const hmat_t h, int64_t i, hmat_leaf *info) {
  return guard([&] {
    if (!h || !info) fail(HMAT_EINVAL, "NULL argument");
    if (i < 0 || i >= (int64_t)h->leaves.size()) fail(HMAT_EINVAL, "leaf index out of range");
    const LeafDev &l = h->leaves[i];
    info->row_begin = l.row;
    info->row_size = l.m;
    info->col_begin = l.col;
    info->col_size = l.n;
    info->level = l.level;
    info->far = l.rank >= 0 ? 1 : 0;
    info->rank = l.rank;
  });
}

hmat_status hmat_leaf_get(const hmat_t h, int64_t i, double *U, double *V) {
  return guard([&] {
    if (!h || !U) fail(HMAT_EINVAL, "NULL argument");
    if (i < 0 || i >= (int64_t)h->leaves.size()) fail(HMAT_EINVAL, "leaf index out of range");
    const LeafDev &l = h->leaves[i];
    if (l.rank >= 0 && !V && l.rank > 0) fail(HMAT_EINVAL, "V is NULL for a far leaf");
    const int64_t nu = l.rank < 0 ? (int64_t)l.m * l.n : (int64_t)l.m * l.rank;
    const int64_t nv = l.rank < 0 ? 0 : (int64_t)l.n * l.rank;
    cudaStream_t s = h->stream;
    if (nu + nv == 0) return;
    DevBuf tmp(sizeof(double) * (nu + nv), s);
    const char *base = (const char *)h->d_data.p;
    ck(launch_convert(h->prec, base + esize(h->prec) * l.off_u, tmp.as<double>(), nu, s), "convert");
    if (nv) ck(launch_convert(h->prec, base + esize(h->prec) * l.off_v, tmp.as<double>() + nu, nv, s), "convert");
    ck(cudaMemcpyAsync(U, tmp.p, sizeof(double) * nu, cudaMemcpyDeviceToHost, s), "leaf U");
    if (nv) ck(cudaMemcpyAsync(V, tmp.as<double>() + nu, sizeof(double) * nv, cudaMemcpyDeviceToHost, s), "leaf V");
    ck(cudaStreamSynchronize(s), "leaf get");
  });
}

hmat_status hmat_to_dense(const hmat_t h, double *out, int64_t ld) {
  return guard([&] {
    if (!h || !out) fail(HMAT_EINVAL, "NULL argument");
    const Tree &t = *h->tree;
    if (ld < t.n) fail(HMAT_EINVAL, "ld < n");
    cudaStream_t s = h->stream;
    DevBuf tmp(sizeof(double) * std::max<int64_t>(h->data_elems, 1), s);
    ck(launch_convert(h->prec, h->d_data.p, tmp.as<double>(), h->data_elems, s), "convert");
    std::vector<double> data(h->data_elems);
    ck(cudaMemcpyAsync(data.data(), tmp.p, sizeof(double) * h->data_elems, cudaMemcpyDeviceToHost, s), "to host");
    ck(cudaStreamSynchronize(s), "to dense");
    for (const LeafDev &l : h->leaves) {
      for (int64_t j = 0; j < l.n; j++) {
        const int64_t oj = t.perm[l.col + j];
        for (int64_t i = 0; i < l.m; i++) {
          const int64_t oi = t.perm[l.row + i];
          double v;
          if (l.rank < 0) v = data[l.off_u + i + j * l.m];
          else {
            v = 0.0;
            for (int q = 0; q < l.rank; q++) v += data[l.off_u + i + (int64_t)q * l.m] * data[l.off_v + j + (int64_t)q * l.n];
          }
          out[oi + oj * ld] = v;
        }
      }
    }
  });
}

}  // extern "C"

namespace {

// FP64 products of an H-matrix with panels of panel_width() columns (row-major, tree order)
struct DevMatvec {
  const hmat_s *h;
  DevBuf wide;
  const double *data = nullptr;
  int cw_rows = 1;
  DevMatvec(const hmat_s *hh, cudaStream_t s) : h(hh) {
    if (h->prec == 64) {
      data = h->d_data.as<double>();
    } else {
      wide = DevBuf(sizeof(double) * std::max<int64_t>(h->data_elems, 1), s);
      ck(launch_convert(h->prec, h->d_data.p, wide.as<double>(), h->data_elems, s), "widen");
      data = wide.as<double>();
    }
    for (const LeafDev &l : h->leaves) cw_rows = std::max(cw_rows, (int)l.rank);
  }
  // Y = H X
  void apply(const double *X, double *Y, cudaStream_t s) const {
    const int64_t n = h->tree->n;
    ck(cudaMemsetAsync(Y, 0, sizeof(double) * n * panel_row_stride(panel_width()), s), "memset");
    ck(launch_hmatvec(h->d_leaves.as<LeafDev>(), (int)h->leaves.size(), data, X, Y, cw_rows, s), "matvec");
  }
};

// columns c0 .. c0+P-1 of the column-major n x ncols x (original order) as a padded row-major panel
// in tree order, and back
void to_panel(const Tree &t, const double *x, int64_t ncols, int64_t c0, std::vector<double> &pan) {
  const int P = panel_width(), SP = panel_row_stride(P);
  pan.assign((size_t)t.n * SP, 0.0);
  for (int c = 0; c < P && c0 + c < ncols; c++)
    for (int64_t i = 0; i < t.n; i++) pan[i * SP + c] = x[t.perm[i] + (c0 + c) * t.n];
}
void from_panel(const Tree &t, const std::vector<double> &pan, int64_t ncols, int64_t c0, double *y) {
  const int P = panel_width(), SP = panel_row_stride(P);
  for (int c = 0; c < P && c0 + c < ncols; c++)
    for (int64_t i = 0; i < t.n; i++) y[t.perm[i] + (c0 + c) * t.n] = pan[i * SP + c];
}

}  // namespace

extern "C" {

hmat_status hmat_matvec(const hmat_t H, const double *x, double *y, int64_t ncols, void *stream) {
  return guard([&] {
    if (!H || !x || !y || ncols < 0) fail(HMAT_EINVAL, "NULL argument or negative ncols");
    const Tree &t = *H->tree;
    cudaStream_t s = (cudaStream_t)stream;
    DevMatvec mv(H, s);
    const int P = panel_width();
    const size_t pan_elems = (size_t)t.n * panel_row_stride(P);
    DevBuf dx(sizeof(double) * std::max<size_t>(pan_elems, 1), s), dy(sizeof(double) * std::max<size_t>(pan_elems, 1), s);
    std::vector<double> pan;
    for (int64_t c0 = 0; c0 < ncols; c0 += P) {
      to_panel(t, x, ncols, c0, pan);
      ck(cudaMemcpyAsync(dx.p, pan.data(), sizeof(double) * pan_elems, cudaMemcpyHostToDevice, s), "upload");
      mv.apply(dx.as<double>(), dy.as<double>(), s);
      ck(cudaMemcpyAsync(pan.data(), dy.p, sizeof(double) * pan_elems, cudaMemcpyDeviceToHost, s), "download");
      ck(cudaStreamSynchronize(s), "matvec");
      from_panel(t, pan, ncols, c0, y);
    }
  });
}

hmat_status hmat_check_bounded_wait(int polls) {
  return guard([&] {
    if (polls < 1 || polls > (1 << 22)) fail(HMAT_EINVAL, "polls must be in 1..2^22");
    DevBuf d(sizeof(int), nullptr);
    ck(cudaMemsetAsync(d.p, 0, sizeof(int), nullptr), "memset");
    ck(launch_tc_wait_check(polls, d.as<int>(), nullptr), "bounded wait");
    int gave_up = 0;
    ck(cudaMemcpy(&gave_up, d.p, sizeof(int), cudaMemcpyDeviceToHost), "bounded wait");
    if (gave_up) fail(HMAT_ETIMEOUT, "the bounded wait gave up (expected)");
  });
}

hmat_status hmat_product_error(const hmat_t A, const hmat_t B, const hmat_t C, int iters, int size, uint64_t seed,
                               double *rel_err) {
  return guard([&] {
    if (!A || !B || !C || !rel_err || iters < 0 || size < 1) fail(HMAT_EINVAL, "NULL argument or bad iters/size");
    if (size > 128) fail(HMAT_EINVAL, "size must be at most 128");
    if (A->tree != C->tree && !same_points(*A->tree, C->tree->orig.data(), C->tree->n, C->tree->dim))
      fail(HMAT_EMISMATCH, "A and C are not on one block tree");
    if (A->tree != B->tree && !same_points(*A->tree, B->tree->orig.data(), B->tree->n, B->tree->dim))
      fail(HMAT_EMISMATCH, "A and B are not on one block tree");
    const Tree &t = *A->tree;
    const int64_t n = t.n;
    cudaStream_t s = C->stream;
    DevMatvec ma(A, s), mb(B, s), mc(C, s);
    // the n x size blocks as row-major panels of panel_width() columns, all on the device
    const int P = panel_width(), SP = panel_row_stride(P);
    const int npan = (size + P - 1) / P;
    const int64_t pan = n * SP, blk = (int64_t)npan * pan;
    DevBuf dX(sizeof(double) * blk, s), dY(sizeof(double) * blk, s);
    DevBuf d2(sizeof(double) * pan, s), d3(sizeof(double) * pan, s);
    DevBuf dG(sizeof(double) * size * size, s), dzero(sizeof(int) * 2, s), dsum(sizeof(double) * 2, s);
    ck(cudaMemsetAsync(dzero.p, 0, sizeof(int) * 2, s), "memset");
    ck(cudaMemsetAsync(dsum.p, 0, sizeof(double) * 2, s), "memset");
    double *X = dX.as<double>(), *Y = dY.as<double>();
    // Y = E X with E = C - A B (which = 0), or Y = C X (which = 1), panel by panel
    auto apply = [&](int which, const double *Xb, double *Yb) {
      for (int q = 0; q < npan; q++) {
        mc.apply(Xb + q * pan, Yb + q * pan, s);
        if (which == 0) {
          mb.apply(Xb + q * pan, d2.as<double>(), s);
          ma.apply(d2.as<double>(), d3.as<double>(), s);
          ck(launch_est_sub(Yb + q * pan, d3.as<double>(), pan, s), "difference");
        }
      }
    };
    // block power iteration on a Gaussian start, orthonormalised by Cholesky QR twice at every
    // step, then the squared Frobenius norm of the operator on the final block
    for (int which = 0; which < 2; which++) {
      ck(launch_est_gaussian(X, n, size, seed, s), "start block");
      ck(launch_est_orth(X, n, size, dG.as<double>(), dzero.as<int>() + which, s), "orthonormalise");
      for (int it = 0; it < iters; it++) {
        apply(which, X, Y);
        ck(launch_est_orth(Y, n, size, dG.as<double>(), dzero.as<int>() + which, s), "orthonormalise");
        std::swap(X, Y);
      }
      apply(which, X, Y);
      ck(launch_est_norm2(Y, blk, dsum.as<double>() + which, s), "norm");
    }
    double sums[2] = {0.0, 0.0};
    ck(cudaMemcpyAsync(sums, dsum.p, sizeof(sums), cudaMemcpyDeviceToHost, s), "norms");
    ck(cudaStreamSynchronize(s), "error estimate");
    const double e = std::sqrt(sums[0]), c = std::sqrt(sums[1]);
    *rel_err = c > 0.0 ? e / c : e;
  });
}

hmat_status hmat_permutation(const hmat_t h, int64_t *perm) {
  return guard([&] {
    if (!h || !perm) fail(HMAT_EINVAL, "NULL argument");
    std::memcpy(perm, h->tree->perm.data(), sizeof(int64_t) * h->tree->n);
  });
}

hmat_status hmat_data_bytes(const hmat_t h, int64_t *bytes) {
  return guard([&] {
    if (!h || !bytes) fail(HMAT_EINVAL, "NULL argument");
    *bytes = h->data_elems * (int64_t)esize(h->prec);
  });
}

hmat_status hmat_data_get(const hmat_t h, void *out, int64_t bytes) {
  return guard([&] {
    if (!h || !out) fail(HMAT_EINVAL, "NULL argument");
    const int64_t need = h->data_elems * (int64_t)esize(h->prec);
    if (bytes < need) fail(HMAT_EINVAL, "output buffer smaller than hmat_data_bytes");
    if (need == 0) return;
    ck(cudaMemcpyAsync(out, h->d_data.p, (size_t)need, cudaMemcpyDeviceToHost, h->stream), "data get");
    ck(cudaStreamSynchronize(h->stream), "data get");
  });
}

hmat_status hmat_stats(const hmat_t h, hmat_stats_t *stats) {
  return guard([&] {
    if (!h || !stats) fail(HMAT_EINVAL, "NULL argument");
    *stats = h->stats;
  });
}

hmat_status hmat_rank_features(const hmat_t A, const hmat_t B, double eps, const hmat_t C, float *features,
                               float *ranks, int64_t *n_far) {
  return guard([&] {
    if (!A || !B || !n_far) fail(HMAT_EINVAL, "NULL argument");
    if (!(eps > 0.0)) fail(HMAT_EINVAL, "eps must be > 0");
    if (A->tree != B->tree && !same_points(*A->tree, B->tree->orig.data(), B->tree->n, B->tree->dim))
      fail(HMAT_EMISMATCH, "A and B are not on one block tree");
    const Tree &t = *A->tree;
    int64_t nfar = 0;
    for (const LeafDev &l : A->leaves) nfar += l.rank >= 0 ? 1 : 0;
    if (!features) {
      *n_far = nfar;
      return;
    }
    if (*n_far < nfar) fail(HMAT_EINVAL, "feature array smaller than the number of far blocks");
    if (C && C->leaves.size() != A->leaves.size()) fail(HMAT_EMISMATCH, "C is not on the tree of A and B");
    std::vector<int32_t> ra(A->leaves.size()), rb(B->leaves.size());
    for (size_t l = 0; l < ra.size(); l++) { ra[l] = A->leaves[l].rank; rb[l] = B->leaves[l].rank; }
    Plan plan;
    build_plan(t, ra, rb, plan);
    const std::vector<int32_t> mxr = chain_max_rank(t, plan);
    int64_t i = 0;
    for (size_t l = 0; l < A->leaves.size(); l++) {
      if (A->leaves[l].rank < 0) continue;
      far_features(t, plan, mxr, A->leaves, B->leaves, eps, (int)l, features + i * RANK_FEATURES);
      if (ranks) ranks[i] = C ? (float)std::max(0, (int)C->leaves[l].rank) : 0.f;
      i++;
    }
    *n_far = nfar;
  });
}

hmat_status hmat_rankmodel_create(const float *weights, const float *mean, const float *dev, hmat_rankmodel_t *out) {
  if (out) *out = nullptr;
  return guard([&] {
    if (!weights || !mean || !dev || !out) fail(HMAT_EINVAL, "NULL argument");
    auto m = std::make_unique<hmat_rankmodel_s>();
    for (int k = 0; k < RANK_FEATURES; k++) {
      if (!(dev[k] > 0.f)) fail(HMAT_EINVAL, "feature deviations must be > 0");
      m->mean[k] = mean[k];
      m->dev[k] = dev[k];
    }
    ck(cudaMalloc(&m->w, sizeof(float) * RANK_PARAMS), "model");
    ck(cudaMalloc(&m->w16, 2 * RANK_PARAMS), "model");
    ck(cudaMemcpy(m->w, weights, sizeof(float) * RANK_PARAMS, cudaMemcpyHostToDevice), "model");
    ck(launch_to_half(m->w, m->w16, nullptr), "model");
    ck(cudaDeviceSynchronize(), "model");
    *out = m.release();
  });
}

hmat_status hmat_rankmodel_train(const float *features, const float *ranks, int64_t count,
                                 const hmat_train_opts *opts, void *stream, hmat_rankmodel_t *out) {
  if (out) *out = nullptr;
  return guard([&] {
    if (!features || !ranks || !out || count < 1) fail(HMAT_EINVAL, "NULL argument or no samples");
    const int epochs = opts && opts->epochs > 0 ? opts->epochs : 1500;
    const float lr = opts && opts->lr > 0.f ? opts->lr : 3e-3f;
    const uint64_t seed = opts ? opts->seed : 0;
    cudaStream_t s = (cudaStream_t)stream;
    auto m = std::make_unique<hmat_rankmodel_s>();
    for (int k = 0; k < RANK_FEATURES; k++) {
      double mu = 0.0, sq = 0.0;
      for (int64_t i = 0; i < count; i++) mu += features[i * RANK_FEATURES + k];
      mu /= (double)count;
      for (int64_t i = 0; i < count; i++) {
        const double d = features[i * RANK_FEATURES + k] - mu;
        sq += d * d;
      }
      m->mean[k] = (float)mu;
      m->dev[k] = (float)std::max(std::sqrt(sq / (double)count), 1e-3);
    }
    std::vector<float> xn, y(count);
    normalise(m.get(), features, count, xn);
    double ymean = 0.0;
    for (int64_t i = 0; i < count; i++) {
      y[i] = (float)std::log2(1.0 + std::max(0.f, ranks[i]));
      ymean += y[i];
    }
    ymean /= (double)count;
    // He-uniform initial weights from a splitmix64 stream, zero biases, output bias = mean target
    std::vector<float> w(RANK_PARAMS, 0.f);
    uint64_t c = 0;
    auto uni = [&]() {
      uint64_t z = seed + (++c) * 0x9E3779B97F4A7C15ull;
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      z ^= z >> 31;
      return (double)(z >> 11) * 0x1.0p-53 * 2.0 - 1.0;
    };
    const int F = RANK_FEATURES, Hh = 64;
    for (int i = 0; i < Hh * F; i++) w[i] = (float)(uni() * std::sqrt(6.0 / F));
    for (int i = 0; i < Hh * Hh; i++) w[Hh * F + Hh + i] = (float)(uni() * std::sqrt(6.0 / Hh));
    for (int i = 0; i < Hh; i++) w[Hh * F + Hh + Hh * Hh + Hh + i] = (float)(uni() * std::sqrt(6.0 / Hh) * 0.1);
    w[RANK_PARAMS - 1] = (float)ymean;
    ck(cudaMalloc(&m->w, sizeof(float) * RANK_PARAMS), "model");
    ck(cudaMalloc(&m->w16, 2 * RANK_PARAMS), "model");
    DevBuf dx(sizeof(float) * xn.size(), s), dy(sizeof(float) * count, s);
    ck(cudaMemcpyAsync(m->w, w.data(), sizeof(float) * RANK_PARAMS, cudaMemcpyHostToDevice, s), "model");
    ck(cudaMemcpyAsync(dx.p, xn.data(), sizeof(float) * xn.size(), cudaMemcpyHostToDevice, s), "samples");
    ck(cudaMemcpyAsync(dy.p, y.data(), sizeof(float) * count, cudaMemcpyHostToDevice, s), "samples");
    ck(mlp_train(m->w, m->w16, dx.as<float>(), dy.as<float>(), (int)count, epochs, lr, s, &m->loss), "training");
    ck(cudaStreamSynchronize(s), "training");
    *out = m.release();
  });
}

hmat_status hmat_rankmodel_predict(const hmat_rankmodel_t m, const float *features, int64_t count, float *ranks) {
  return guard([&] {
    if (!m || !features || !ranks) fail(HMAT_EINVAL, "NULL argument");
    if (count == 0) return;
    std::vector<float> xn;
    normalise(m, features, count, xn);
    DevBuf dx(sizeof(float) * xn.size(), nullptr), dout(sizeof(float) * count, nullptr);
    ck(cudaMemcpyAsync(dx.p, xn.data(), sizeof(float) * xn.size(), cudaMemcpyHostToDevice, nullptr), "samples");
    ck(launch_mlp_forward(m->w16, dx.as<float>(), (int)count, dout.as<float>(), nullptr), "forward");
    std::vector<float> y(count);
    ck(cudaMemcpyAsync(y.data(), dout.p, sizeof(float) * count, cudaMemcpyDeviceToHost, nullptr), "forward");
    ck(cudaStreamSynchronize(nullptr), "forward");
    for (int64_t i = 0; i < count; i++) ranks[i] = std::max(0.f, std::exp2(y[i]) - 1.f);
  });
}

hmat_status hmat_rankmodel_get(const hmat_rankmodel_t m, float *weights, float *mean, float *dev, float *loss) {
  return guard([&] {
    if (!m) fail(HMAT_EINVAL, "NULL model");
    if (weights) {
      std::vector<uint16_t> h(RANK_PARAMS);
      ck(cudaMemcpy(h.data(), m->w16, 2 * RANK_PARAMS, cudaMemcpyDeviceToHost), "weights");
      for (int i = 0; i < RANK_PARAMS; i++) {  // IEEE binary16 -> float
        const uint32_t hb = h[i], sign = (hb >> 15) & 1, ex = (hb >> 10) & 31, man = hb & 1023;
        float v;
        if (ex == 0) v = std::ldexp((float)man, -24);
        else if (ex == 31) v = man ? NAN : INFINITY;
        else v = std::ldexp((float)(man | 1024), (int)ex - 25);
        weights[i] = sign ? -v : v;
      }
    }
    if (mean) std::memcpy(mean, m->mean, sizeof(m->mean));
    if (dev) std::memcpy(dev, m->dev, sizeof(m->dev));
    if (loss) *loss = m->loss;
  });
}

hmat_status hmat_rankmodel_grad(const hmat_rankmodel_t m, const float *features, const float *ranks, int64_t count,
                                float *grad, float *loss) {
  return guard([&] {
    if (!m || !features || !ranks || !grad || count < 1) fail(HMAT_EINVAL, "NULL argument or no samples");
    std::vector<float> xn, y(count);
    normalise(m, features, count, xn);
    for (int64_t i = 0; i < count; i++) y[i] = (float)std::log2(1.0 + std::max(0.f, ranks[i]));
    DevBuf dx(sizeof(float) * xn.size(), nullptr), dy(sizeof(float) * count, nullptr);
    DevBuf dg(sizeof(float) * RANK_PARAMS, nullptr), dl(sizeof(float), nullptr);
    ck(cudaMemcpyAsync(dx.p, xn.data(), sizeof(float) * xn.size(), cudaMemcpyHostToDevice, nullptr), "samples");
    ck(cudaMemcpyAsync(dy.p, y.data(), sizeof(float) * count, cudaMemcpyHostToDevice, nullptr), "samples");
    ck(launch_mlp_grad(m->w16, dx.as<float>(), dy.as<float>(), (int)count, dg.as<float>(), dl.as<float>(), nullptr),
       "gradient");
    float l = 0.f;
    ck(cudaMemcpyAsync(grad, dg.p, sizeof(float) * RANK_PARAMS, cudaMemcpyDeviceToHost, nullptr), "gradient");
    ck(cudaMemcpyAsync(&l, dl.p, sizeof(float), cudaMemcpyDeviceToHost, nullptr), "gradient");
    ck(cudaStreamSynchronize(nullptr), "gradient");
    if (loss) *loss = l;
  });
}

hmat_status hmat_rankmodel_grad_noalloc(const hmat_rankmodel_t m, const float *features, const float *ranks,
                                        int64_t count, float *grad, float *loss, void *stream) {
  return guard([&] {
    if (!m || !features || !ranks || !grad || count < 1) fail(HMAT_EINVAL, "NULL argument or no samples");
    if (count > HMAT_RANKGRAD_NOALLOC_MAX)
      fail(HMAT_EINVAL, "count exceeds HMAT_RANKGRAD_NOALLOC_MAX (16384 samples), the capacity of the fixed scratch");
    ck(mlp_grad_noalloc(m->w16, m->mean, m->dev, features, ranks, (int)count, grad, loss, (cudaStream_t)stream),
       "gradient (fixed scratch)");
  });
}

void hmat_rankmodel_destroy(hmat_rankmodel_t m) { delete m; }

hmat_status hmat_plan_host(const double *xyz, int64_t n, int dim, int leaf_size, double eta, int64_t *perm,
                           int64_t *n_leaves, hmat_leaf *leaves, int64_t *n_lowrank, int64_t *n_hpairs,
                           int64_t max_leaves, int *csp) {
  return guard([&] {
    if (!xyz) fail(HMAT_EINVAL, "NULL argument");
    if (n < 1 || dim < 1 || dim > 3) fail(HMAT_EINVAL, "need n >= 1 and dim in 1..3");
    if (leaf_size < 2 || leaf_size > 128) fail(HMAT_EINVAL, "leaf_size must be in 2..128");
    if (!(eta > 0.0)) fail(HMAT_EINVAL, "eta must be > 0");
    if (max_leaves < 0) fail(HMAT_EINVAL, "max_leaves must be >= 0");
    for (int64_t i = 0; i < n * dim; i++)
      if (!std::isfinite(xyz[i])) fail(HMAT_EINVAL, "non-finite point coordinate");
    std::shared_ptr<Tree> tp = build_tree(xyz, n, dim, leaf_size, eta);
    if (!tp) fail(HMAT_EINVAL, "tree construction failed");
    const Tree &t = *tp;
    const std::vector<LeafDev> lv = base_leaves(t);
    const int64_t nl = (int64_t)lv.size();
    if (perm) std::copy(t.perm.begin(), t.perm.end(), perm);
    if (n_leaves) *n_leaves = nl;
    if (csp) *csp = t.csp;
    const int64_t k = std::min(max_leaves, nl);
    if (leaves)
      for (int64_t l = 0; l < k; l++) {
        leaves[l].row_begin = lv[l].row;
        leaves[l].row_size = lv[l].m;
        leaves[l].col_begin = lv[l].col;
        leaves[l].col_size = lv[l].n;
        leaves[l].level = lv[l].level;
        leaves[l].far = lv[l].rank >= 0 ? 1 : 0;
        leaves[l].rank = lv[l].rank;
      }
    if ((n_lowrank || n_hpairs) && k > 0) {
      std::vector<int32_t> rk(lv.size());
      for (size_t l = 0; l < lv.size(); l++) rk[l] = lv[l].rank;  // the counts do not depend on ranks
      Plan plan;
      build_plan(t, rk, rk, plan);
      for (int64_t l = 0; l < k; l++) {
        if (n_lowrank) n_lowrank[l] = plan.nterm_cum[t.leaf_block[l]];
        if (n_hpairs) n_hpairs[l] = plan.leaf_pair_off[l + 1] - plan.leaf_pair_off[l];
      }
    }
  });
}

hmat_status hmat_sumexpr_counts(const hmat_t A, const hmat_t B, int64_t *n_lowrank, int64_t *n_hpairs) {
  return guard([&] {
    if (!A || !B || !n_lowrank || !n_hpairs) fail(HMAT_EINVAL, "NULL argument");
    if (A->tree != B->tree && !same_points(*A->tree, B->tree->orig.data(), B->tree->n, B->tree->dim))
      fail(HMAT_EMISMATCH, "A and B are not on one block tree");
    const Tree &t = *A->tree;
    std::vector<int32_t> ra(A->leaves.size()), rb(B->leaves.size());
    for (size_t l = 0; l < ra.size(); l++) { ra[l] = A->leaves[l].rank; rb[l] = B->leaves[l].rank; }
    Plan plan;
    build_plan(t, ra, rb, plan);
    for (size_t l = 0; l + 1 < plan.leaf_pair_off.size(); l++) {
      n_lowrank[l] = plan.nterm_cum[t.leaf_block[l]];
      n_hpairs[l] = plan.leaf_pair_off[l + 1] - plan.leaf_pair_off[l];
    }
  });
}

}  // extern "C"

// ------------------------------------------------------------------ the product

namespace {

// Device-memory admission for products run side by side (hmat_multiply_batched): a product
// reserves its estimated bytes before its first large allocation and returns them when it ends;
// a product that does not fit waits until enough have ended, and runs alone if it exceeds the
// whole budget.
struct MemGate {
  std::mutex m;
  std::condition_variable cv;
  int64_t budget = 0, used = 0;
  int running = 0;
  void acquire(int64_t b) {
    std::unique_lock<std::mutex> lk(m);
    cv.wait(lk, [&] { return running == 0 || used + b <= budget; });
    used += b;
    running++;
  }
  void release(int64_t b) {
    {
      std::lock_guard<std::mutex> lk(m);
      used -= b;
      running--;
    }
    cv.notify_all();
  }
};

struct Product {
  const hmat_s *A, *B;
  const hmat_mult_opts *o;
  cudaStream_t s;
  int cprec;              // compute / output precision
  std::unique_ptr<hmat_s> C;
  MemGate *gate = nullptr;  // set by the batched call
  int64_t gate_bytes = 0;

  void run();
  ~Product() {
    if (gate && gate_bytes) gate->release(gate_bytes);
  }
};

// HMAT_CHECK_FINITE=1: after each phase of a product, scan its outputs for NaN/Inf and report
// the first bad entry on stderr (a debugging aid; off by default).
bool check_finite_enabled() {
  const char *e = std::getenv("HMAT_CHECK_FINITE");
  return e && e[0] == '1';
}

void check_finite(int prec, const void *x, int64_t count, const char *what, cudaStream_t s) {
  if (!check_finite_enabled() || count == 0) return;
  DevBuf d(sizeof(unsigned long long), s);
  ck(cudaMemsetAsync(d.p, 0xff, sizeof(unsigned long long), s), "check");
  ck(launch_find_nonfinite(prec, x, count, d.as<unsigned long long>(), s), "check");
  unsigned long long h = 0;
  ck(cudaMemcpyAsync(&h, d.p, sizeof(h), cudaMemcpyDeviceToHost, s), "check");
  ck(cudaStreamSynchronize(s), "check");
  if (h != ~0ull) std::fprintf(stderr, "hmat: non-finite value after %s at element %llu of %lld\n", what, h, (long long)count);
}


void Product::run() {
  const Tree &t = *A->tree;
  const double t_plan0 = now_ms();
  Trace tr;
  C = std::make_unique<hmat_s>();
  C->tree = A->tree;
  C->stream = s;
  C->prec = cprec;
  C->kernel = -1;
  hmat_stats_t &S = C->stats;
  const size_t es = esize(cprec);
  const int p = o->block_width > 0 ? o->block_width : 8;
  if (p > 16) fail(HMAT_EINVAL, "block_width must be <= 16");
  int max_rank = o->max_rank > 0 ? o->max_rank : 96;
  if (max_rank > 96) fail(HMAT_EINVAL, "max_rank must be <= 96");
  if (max_rank < p) max_rank = p;
  const int max_rounds = o->max_rounds > 0 ? o->max_rounds : max_rank / p + 1;
  if (o->rank_proposal < 0 || o->rank_proposal > 2) fail(HMAT_EINVAL, "rank_proposal must be 0, 1 or 2");
  const int fixed_k = o->fixed_rank;
  if (fixed_k < 0 || fixed_k > 16) fail(HMAT_EINVAL, "fixed_rank must be 0 (eps-rank) or 1..16");
  const int power_q = o->power_iters < 0 ? 1 : o->power_iters;
  if (power_q > 4) fail(HMAT_EINVAL, "power_iters must be -1 (default) or 0..4");
  if (o->rank_proposal == 1 && !o->rank_model) fail(HMAT_EINVAL, "rank_proposal 1 needs a rank_model");
  if (o->compressor != HMAT_COMP_RANDOMIZED && o->compressor != HMAT_COMP_ACA && o->compressor != HMAT_COMP_LANCZOS)
    fail(HMAT_EINVAL, "compressor must be 0 (randomized), 1 (cross approximation) or 2 (Lanczos)");
  const bool aca = o->compressor == HMAT_COMP_ACA, lanczos = o->compressor == HMAT_COMP_LANCZOS;
  const bool single = aca || lanczos;  // one matrix-vector product per pass
  if (single && (fixed_k != 0 || o->rank_proposal != 0))
    fail(HMAT_EINVAL, "the cross approximation and Lanczos compressors take neither fixed_rank nor rank_proposal");

  // factors in compute precision
  DevBuf convA, convB;
  const void *dataA = A->d_data.p, *dataB = B->d_data.p;
  if (A->prec != cprec) {
    convA = DevBuf(sizeof(double) * std::max<int64_t>(A->data_elems, 1), s);
    ck(launch_convert(A->prec, A->d_data.p, convA.as<double>(), A->data_elems, s), "widen A");
    dataA = convA.p;
  }
  if (B->prec != cprec) {
    if (B == A) dataB = dataA;
    else {
      convB = DevBuf(sizeof(double) * std::max<int64_t>(B->data_elems, 1), s);
      ck(launch_convert(B->prec, B->d_data.p, convB.as<double>(), B->data_elems, s), "widen B");
      dataB = convB.p;
    }
  }

  // ---- a1: symbolic restriction (Algorithm 3) over the tree
  std::vector<int32_t> ra(A->leaves.size()), rb(B->leaves.size());
  for (size_t l = 0; l < ra.size(); l++) { ra[l] = A->leaves[l].rank; rb[l] = B->leaves[l].rank; }
  // host tables of the product are kept between calls (thread-local), so their memory is mapped
  static thread_local Plan plan_tl;
  static thread_local std::vector<TermJob> jobs_tl;
  Plan &plan = plan_tl;
  build_plan(t, ra, rb, plan);
  tr.mark("plan (Algorithm 3)");
  const std::vector<double> storA = block_storage(t, A->leaves), storB = block_storage(t, B->leaves);
  const size_t smem_cap = 200 * 1024;  // shared memory a launch may ask for per block

  // ---- groups. A product whose device memory (the new factors of the low-rank products, the
  // sampling buffers, the near field) would exceed a budget runs in groups: the blocks at a cut
  // level lc are packed, in depth-first order, into groups that fit; a group builds the terms
  // created in its subtrees and at every block above lc (needed by all groups), and runs its
  // own targets. Leaves above lc belong to the first group.
  const size_t nleaf = t.leaf_block.size(), nblk = t.bl.size();
  std::vector<int> blk_group(nblk, -1), leaf_group(nleaf, 0);
  int ngroups = 1;
  {
    const int p_est = std::max(p, 16);
    std::vector<double> mem(nblk, 0.0);  // bytes of the terms created at each block and its leaf
    parallel_for(64, [&](size_t c) {      // blocks split in 64 ranges; each block's terms are contiguous
      for (size_t b = nblk * c / 64; b < nblk * (c + 1) / 64; b++)
        for (int32_t i = plan.blk_term_lo[b]; i < plan.blk_term_hi[b]; i++) {
          const PlanTerm &pt = plan.terms[i];
          const Block &cb = t.bl[b];
          const int64_t rows =
              (pt.type == JOB_FF_L || pt.type == JOB_HF) ? t.cl[cb.tau].size : t.cl[cb.sigma].size;
          mem[b] += (double)es * rows * pt.rank;
        }
    });
    for (size_t l = 0; l < nleaf; l++) {
      const LeafDev &lf = A->leaves[l];
      const double mx = std::max(lf.m, lf.n);
      mem[t.leaf_block[l]] += lf.rank >= 0
                                  ? 8.0 * (lf.m + lf.n) * max_rank + (double)es * 5.0 * mx * p_est
                                  : (double)es * 2.0 * lf.m * lf.n;
    }
    double total = 0.0;
    for (double x : mem) total += x;
    size_t fr = 0, tot = 0;
    ck(cudaMemGetInfo(&fr, &tot), "memory info");
    const double budget = 0.45 * (double)fr;
    const char *ge = std::getenv("HMAT_MEMORY_BUDGET_GB");  // a caller's own limit
    const double budget_used = (ge && std::atof(ge) > 0.0) ? std::atof(ge) * 1e9 : budget;
    if (total > budget_used && t.depth >= 2) {
      std::vector<double> sub(nblk, 0.0);  // subtree bytes (children follow their parent)
      for (size_t b = nblk; b-- > 0;) {
        sub[b] += mem[b];
        if (t.bl[b].parent >= 0) sub[t.bl[b].parent] += sub[b];
      }
      for (int lc = 1; lc < t.depth; lc++) {
        double shared = 0.0, biggest = 0.0;
        for (size_t b = 0; b < nblk; b++) {
          if (t.bl[b].level < lc) shared += mem[b];
          else if (t.bl[b].level == lc) biggest = std::max(biggest, sub[b]);
        }
        if (shared + biggest > budget_used && lc + 1 < t.depth) continue;
        // pack the blocks of level lc in depth-first order
        ngroups = 0;
        double cur = 0.0;
        bool open = false;
        for (size_t b = 0; b < nblk; b++) {
          if (t.bl[b].level != lc) continue;
          if (!open || cur + sub[b] + shared > budget_used) {
            ngroups++;
            cur = 0.0;
            open = true;
          }
          cur += sub[b];
          const int gid = ngroups - 1;
          // the subtree of b: ids b .. b + size - 1 (depth-first numbering), leaves leaf_lo .. leaf_hi
          std::vector<int> stack{(int)b};
          while (!stack.empty()) {
            const int x = stack.back();
            stack.pop_back();
            blk_group[x] = gid;
            for (int c = 0; c < t.bl[x].nchild; c++) stack.push_back(t.bl[x].child[c]);
          }
          for (int32_t l = t.bl[b].leaf_lo; l < t.bl[b].leaf_hi; l++) leaf_group[l] = gid;
        }
        if (ngroups == 0) ngroups = 1;
        break;
      }
    }
    if (tr.on)
      std::fprintf(stderr, "hmat trace: memory estimate %.2f GB, budget %.2f GB, %d group(s)\n", total / 1e9,
                   budget_used / 1e9, ngroups);
  }
  S.n_terms = (int64_t)plan.terms.size();
  S.n_hpairs = (int64_t)plan.leaf_pairs.size();
  C->leaves = base_leaves(t);
  struct GroupOut {
    DevBuf data;
    int64_t elems = 0;
  };
  std::vector<GroupOut> gouts(ngroups);
  auto in_group = [&](int blk, int grp) { return blk_group[blk] < 0 || blk_group[blk] == grp; };

  auto run_group = [&](const int grp) {
  const double t_g0 = now_ms();
  if (gate && gate_bytes) {  // the previous group's reservation
    gate->release(gate_bytes);
    gate_bytes = 0;
  }

  // jobs of the low-rank products (a2), their storage, and the panels of products with an
  // inadmissible factor: 0 = the H-block is one dense leaf (warp per panel), 1 = inner block with
  // shared-memory staging, 2 = inner block with global staging
  const int PW = panel_width();
  int pcw_rows = 1;
  for (const LeafDev &l : A->leaves) pcw_rows = std::max(pcw_rows, (int)l.rank);
  for (const LeafDev &l : B->leaves) pcw_rows = std::max(pcw_rows, (int)l.rank);
  const size_t pcw_bytes = (size_t)8 * pcw_rows * panel_row_stride(PW) * es;
  const size_t nterm = plan.terms.size();
  std::vector<TermJob> &jobs = jobs_tl;
  jobs.resize(nterm);
  std::vector<int32_t> ff_ids;
  // panel kinds: 0 = one dense leaf; 1..NB = inner block in shared memory, by size bucket
  // (at most 64 << (kind - 1) rows and columns); NB + 1 = inner block, global staging
  constexpr int NB = 10;
  static thread_local std::vector<PanelDev> pk_tl[NB + 2];
  std::vector<PanelDev> *pk = pk_tl;
  for (int k = 0; k < NB + 2; k++) pk[k].clear();
  int pdim[NB + 2] = {0};
  int64_t term_elems = 0;
  double flops_terms = 0, elems_terms_use = 0;
  double kind_flops[NB + 2] = {0}, kind_cols[NB + 2] = {0};
  {
    // two passes over chunks of the terms on a thread pool, with the serial order preserved:
    // (1) per chunk: storage, flops, far x far count, panels per kind; (2) fill at the offsets
    struct Chunk {
      int64_t elems = 0, nff = 0;
      double flops = 0, elems_use = 0;
      int64_t npk[NB + 2] = {0};
      int pd[NB + 2] = {0};
      double fk[NB + 2] = {0}, ck[NB + 2] = {0};  // per kind: flops, columns (for the trace)
    };
    const size_t nch = std::max<size_t>(1, std::min<size_t>(64, nterm / 4096 + 1));
    std::vector<Chunk> ch(nch);
    auto range = [&](size_t c) { return std::make_pair(nterm * c / nch, nterm * (c + 1) / nch); };
    auto kind_of = [&](const PlanTerm &pt, int &dmx) {
      const int hb = pt.type == JOB_HF ? pt.a : pt.b;  // the inadmissible H-block
      const Block &bk = t.bl[hb];
      const int dm = (int)t.cl[bk.tau].size, dn = (int)t.cl[bk.sigma].size;
      dmx = std::max(dm, dn);
      if (bk.kind == BK_NEAR) return 0;
      int bkt = 1;
      while ((64 << (bkt - 1)) < dmx && bkt < NB) bkt++;
      const int cap = 64 << (bkt - 1);
      if (cap >= dmx && (size_t)(2 * cap) * panel_row_stride(PW) * es + pcw_bytes <= smem_cap) return bkt;
      return NB + 1;
    };
    auto rows_of = [&](const PlanTerm &pt) -> int64_t {
      const Block &cb = t.bl[pt.block];
      return (pt.type == JOB_FF_L || pt.type == JOB_HF) ? t.cl[cb.tau].size : t.cl[cb.sigma].size;
    };
    parallel_for(nch, [&](size_t c) {
      Chunk &k = ch[c];
      const auto r = range(c);
      for (size_t i = r.first; i < r.second; i++) {
        const PlanTerm &pt = plan.terms[i];
        if (!in_group(pt.block, grp)) continue;
        const int64_t rows = rows_of(pt);
        k.elems += rows * pt.rank;
        if (pt.type == JOB_FF_R || pt.type == JOB_FF_L) {
          const LeafDev &la = A->leaves[pt.a], &lb = B->leaves[pt.b];
          k.flops += 2.0 * la.n * la.rank * lb.rank + 2.0 * rows * la.rank * lb.rank;
          // V_a and U_b (rho' rows), the far factor that is kept (rows of the new one), the new factor
          k.elems_use += (double)la.n * la.rank + (double)lb.m * lb.rank +
                         (double)rows * (pt.type == JOB_FF_R ? lb.rank : la.rank) + (double)rows * pt.rank;
          k.nff++;
        } else {
          const int hb = pt.type == JOB_HF ? pt.a : pt.b;
          k.flops += 2.0 * (pt.type == JOB_HF ? storA[hb] : storB[hb]) * pt.rank;
          // every panel reads the H-block once, plus its input columns and its output columns
          const int64_t inrows = pt.type == JOB_HF ? t.cl[t.bl[hb].sigma].size : t.cl[t.bl[hb].tau].size;
          k.elems_use += (double)((pt.rank + PW - 1) / PW) * (pt.type == JOB_HF ? storA[hb] : storB[hb]) +
                         (double)(inrows + rows) * pt.rank;
          int dmx;
          const int kind = kind_of(pt, dmx);
          k.npk[kind] += (pt.rank + PW - 1) / PW;
          k.pd[kind] = std::max(k.pd[kind], dmx);
          k.fk[kind] += 2.0 * (pt.type == JOB_HF ? storA[hb] : storB[hb]) * pt.rank;
          k.ck[kind] += pt.rank;
        }
      }
    });
    std::vector<int64_t> eoff(nch + 1, 0), foff(nch + 1, 0);
    std::vector<std::array<int64_t, NB + 2>> poff(nch + 1);
    poff[0].fill(0);
    for (size_t c = 0; c < nch; c++) {
      eoff[c + 1] = eoff[c] + ch[c].elems;
      foff[c + 1] = foff[c] + ch[c].nff;
      flops_terms += ch[c].flops;
      elems_terms_use += ch[c].elems_use;
      for (int k = 0; k < NB + 2; k++) {
        poff[c + 1][k] = poff[c][k] + ch[c].npk[k];
        pdim[k] = std::max(pdim[k], ch[c].pd[k]);
        kind_flops[k] += ch[c].fk[k];
        kind_cols[k] += ch[c].ck[k];
      }
    }
    term_elems = eoff[nch];
    ff_ids.resize(foff[nch]);
    for (int k = 0; k < NB + 2; k++) pk[k].resize(poff[nch][k]);
    parallel_for(nch, [&](size_t c) {
      const auto r = range(c);
      int64_t e = eoff[c], f = foff[c];
      std::array<int64_t, NB + 2> q = poff[c];
      for (size_t i = r.first; i < r.second; i++) {
        const PlanTerm &pt = plan.terms[i];
        TermJob &j = jobs[i];
        if (!in_group(pt.block, grp)) {
          j.type = -1;  // skipped by the term-table kernel
          continue;
        }
        j.type = pt.type;
        j.a = pt.a;
        j.b = pt.b;
        j.rank = pt.rank;
        j.rows = rows_of(pt);
        j.out = e;
        j.blk = pt.block;
        j.pad = 0;
        e += j.rows * j.rank;
        if (pt.type == JOB_FF_R || pt.type == JOB_FF_L) {
          ff_ids[f++] = (int32_t)i;
        } else {
          int dmx;
          const int kind = kind_of(pt, dmx);
          for (int q0 = 0; q0 < pt.rank; q0 += PW) pk[kind][q[kind]++] = PanelDev{(int32_t)i, q0};
        }
      }
    });
  }
  tr.mark("jobs and panels");
  S.flops_terms += flops_terms;
  S.bytes_terms_use += (double)es * elems_terms_use;
  std::vector<int2> blk_terms(t.bl.size());
  for (size_t b = 0; b < t.bl.size(); b++) blk_terms[b] = make_int2(plan.blk_term_lo[b], plan.blk_term_hi[b]);

  tr.mark("block term ranges");
  static thread_local std::vector<PanelDev> panels_tl;
  std::vector<PanelDev> &panels = panels_tl;
  panels.clear();
  int pfirst[NB + 2];
  for (int k = 0; k < NB + 2; k++) {
    pfirst[k] = (int)panels.size();
    panels.insert(panels.end(), pk[k].begin(), pk[k].end());
  }
  tr.mark("panel tables");
  S.ms_plan += now_ms() - (grp == 0 ? t_plan0 : t_g0);

  cudaEvent_t ev[6];
  for (auto &e : ev) ck(cudaEventCreate(&e), "event");
  struct EvGuard {
    cudaEvent_t *e;
    ~EvGuard() { for (int i = 0; i < 6; i++) cudaEventDestroy(e[i]); }
  } evg{ev};

  // FP32 far x far products with both ranks <= 32 and at most 2048 inner rows run one warp per
  // job (listed first), the others (and all FP64 ones) one block per job.
  // The warp jobs are listed by rank bucket (both ranks <= 8, <= 16, <= 32), each run by a
  // kernel sized for its bucket; the order within a bucket is the plan's.
  int n_ff_warp = 0;
  int ff_bucket[3] = {0, 0, 0};
  if (cprec == 32) {
    std::vector<int32_t> bk[3], big;
    for (int32_t i : ff_ids) {
      const LeafDev &la = A->leaves[jobs[i].a], &lb = B->leaves[jobs[i].b];
      const int r = std::max(la.rank, lb.rank);
      if (r <= 32 && la.n <= 2048) bk[r <= 8 ? 0 : r <= 16 ? 1 : 2].push_back(i);
      else big.push_back(i);
    }
    for (int b = 0; b < 3; b++) {
      std::copy(bk[b].begin(), bk[b].end(), ff_ids.begin() + n_ff_warp);
      n_ff_warp += (int)bk[b].size();
      ff_bucket[b] = (int)bk[b].size();
    }
    std::copy(big.begin(), big.end(), ff_ids.begin() + n_ff_warp);
  }
  // ---- a2: low-rank products. Far x far products (small) run one job per warp or block;
  // products with an inadmissible factor run as panels of up to panel_width() columns.
  ck(cudaEventRecord(ev[0], s), "event");
  if (tr.on)
    std::fprintf(stderr, "hmat trace: buffers: terms %lld elems, panel staging %lld x %lld\n", (long long)term_elems,
                 (long long)std::min<int64_t>((int64_t)pk[NB + 1].size(), PANEL_GSTAGE_SLOTS),
                 (long long)(2 * pdim[NB + 1] * panel_row_stride(PW)));
  if (gate) {  // reserve this product's device memory: terms, sampling buffers, near field
    int64_t est = (int64_t)es * term_elems;
    for (size_t li = 0; li < A->leaves.size(); li++) {
      const LeafDev &l = A->leaves[li];
      if (leaf_group[li] != grp) continue;
      if (l.rank >= 0) {
        const int64_t mx = std::max(l.m, l.n);
        est += (int64_t)sizeof(double) * (l.m + l.n) * 96 + (int64_t)es * (2 * mx * 16 + 3 * mx * 16);
      } else {
        est += (int64_t)es * l.m * l.n;
      }
    }
    gate_bytes = est + (est >> 3);
    gate->acquire(gate_bytes);
  }
  DevBuf d_termbuf(es * std::max<int64_t>(term_elems, 1), s);
  DevBuf d_jobs = upload(jobs, s), d_ffids = upload(ff_ids, s), d_panels = upload(panels, s);
  DevBuf d_blkterms = upload(blk_terms, s);
  DevBuf d_terms(sizeof(TermDev) * std::max<size_t>(nterm, 1), s);
  ck(launch_make_terms(cprec, d_jobs.as<TermJob>(), (int)nterm, t.d_blocks, A->d_leaves.as<LeafDev>(),
                       B->d_leaves.as<LeafDev>(), dataA, dataB, d_termbuf.p, d_terms.as<TermDev>(), s),
     "term table");
  std::vector<std::pair<int, std::array<cudaEvent_t, 2>>> a2ev;  // HMAT_TRACE only: -1 = far x far
  struct A2EvGuard {  // events not yet read when the product fails
    std::vector<std::pair<int, std::array<cudaEvent_t, 2>>> &v;
    ~A2EvGuard() {
      for (auto &e : v)
        for (cudaEvent_t x : e.second)
          if (x) cudaEventDestroy(x);
    }
  } a2evg{a2ev};
  auto a2mark = [&](int kind, int which) {
    if (!tr.on) return;
    if (which == 0) {
      a2ev.push_back({kind, {nullptr, nullptr}});
      cudaEventCreate(&a2ev.back().second[0]);
      cudaEventCreate(&a2ev.back().second[1]);
    }
    cudaEventRecord(a2ev.back().second[which], s);
  };
  a2mark(-1, 0);
  ck(launch_ff_warp(cprec, d_jobs.as<TermJob>(), d_ffids.as<int32_t>(), ff_bucket, A->d_leaves.as<LeafDev>(),
                    B->d_leaves.as<LeafDev>(), dataA, dataB, d_termbuf.p, s),
     "far x far products (warp)");
  ck(launch_term_jobs(cprec, d_jobs.as<TermJob>(), d_ffids.as<int32_t>() + n_ff_warp, (int)ff_ids.size() - n_ff_warp,
                      A->d_leaves.as<LeafDev>(), B->d_leaves.as<LeafDev>(), t.d_blocks, dataA, dataB, d_termbuf.p, s),
     "far x far products");
  a2mark(-1, 1);
  int64_t launches = 1 + (ff_bucket[0] > 0 ? 1 : 0) + (ff_bucket[1] > 0 ? 1 : 0) + (ff_bucket[2] > 0 ? 1 : 0) +
                     ((int)ff_ids.size() > n_ff_warp ? 1 : 0);
  const int64_t pstride = (int64_t)2 * pdim[NB + 1] * panel_row_stride(PW);
  // one staging slot per thread block of the global-staging launch (it loops over its panels)
  const int64_t pslots = std::min<int64_t>((int64_t)pk[NB + 1].size(), PANEL_GSTAGE_SLOTS);
  DevBuf d_pstage(es * std::max<int64_t>(pstride * pslots, 1), s);
  for (int k = 0; k < NB + 2; k++) {
    if (pk[k].empty()) continue;
    PanelArgs pa{};
    pa.first = pfirst[k];
    pa.count = (int)pk[k].size();
    pa.smem_in = pa.smem_out = pdim[k];
    pa.smem_cw = pcw_rows;
    pa.gstage = k == NB + 1 ? 1 : 0;
    pa.stage_stride = pstride;
    pa.stage_base = d_pstage.p;
    pa.panels = d_panels.as<PanelDev>();
    pa.jobs = d_jobs.as<TermJob>();
    pa.blocks = t.d_blocks;
    pa.leafA = A->d_leaves.as<LeafDev>();
    pa.leafB = B->d_leaves.as<LeafDev>();
    pa.dataA = dataA;
    pa.dataB = dataB;
    pa.terms = d_termbuf.p;
    a2mark(k, 0);
    ck(launch_panels(cprec, pa, k == 0, s), "low-rank products (panels)");
    a2mark(k, 1);
    launches++;
  }
  S.n_ff_jobs += (int64_t)ff_ids.size();
  S.n_panels += (int64_t)panels.size();
  check_finite(cprec, d_termbuf.p, term_elems, "low-rank products", s);
  tr.mark("a2 launched");
  // (trace) the a2 launches' device times, read once the product has synchronised, so that the
  // trace does not serialise the host work below behind them
  auto a2_report = [&]() {
    if (!tr.on) return;
    for (auto &e : a2ev) {
      float x = 0.f;
      cudaEventElapsedTime(&x, e.second[0], e.second[1]);
      if (e.first < 0)
        std::fprintf(stderr, "hmat trace: a2 far x far: %zu jobs, %8.3f ms\n", ff_ids.size(), x);
      else
        std::fprintf(stderr, "hmat trace: a2 panel kind %2d: %8zu panels (columns used %4.1f%%), H-block dim <= %6d, "
                     "%.3g flops, %8.3f ms\n", e.first, pk[e.first].size(),
                     100.0 * kind_cols[e.first] / std::max<double>(1.0, (double)pk[e.first].size() * PW), pdim[e.first],
                     kind_flops[e.first], x);
      cudaEventDestroy(e.second[0]);
      cudaEventDestroy(e.second[1]);
    }
    a2ev.clear();
  };
  ck(cudaEventRecord(ev[1], s), "event");

  // host work below overlaps the low-rank products on the GPU
  // ---- targets
  struct Tgt {
    int leaf;
    double cost;
  };
  std::vector<Tgt> far, nearv;
  std::vector<double> elems_b(t.leaf_block.size(), 0.0);
  int64_t lr_refs = 0;
  for (size_t l = 0; l < t.leaf_block.size(); l++) {
    if (leaf_group[l] != grp) continue;
    const LeafDev &lc = A->leaves[l];
    const int b = t.leaf_block[l];
    double e = (double)plan.rank_cum[b] * (lc.m + lc.n);
    lr_refs += plan.nterm_cum[b];
    for (int64_t q = plan.leaf_pair_off[l]; q < plan.leaf_pair_off[l + 1]; q++)
      e += storA[plan.leaf_pairs[q].blkA] + storB[plan.leaf_pairs[q].blkB];
    elems_b[l] = e;
    (lc.rank < 0 ? nearv : far).push_back(Tgt{(int)l, e});
  }
  S.n_lr_refs += lr_refs;
  // Columns of each far target's first round: p, or a proposed rank + p (at most PROP_MAX),
  // the last p/2 of which form the verification block of the in-round stop test.
  constexpr int PROP_MAX = 16;
  std::vector<int> p0v(t.leaf_block.size(), p);
  if (o->rank_proposal != 0 && !far.empty() && p < PROP_MAX) {
    std::vector<float> khat(far.size(), 0.f);
    if (o->rank_proposal == 2) {
      for (size_t i = 0; i < far.size(); i++)
        khat[i] = (float)std::max(A->leaves[far[i].leaf].rank, B->leaves[far[i].leaf].rank);
    } else {
      const hmat_rankmodel_s *m = o->rank_model;
      const std::vector<int32_t> mxr = chain_max_rank(t, plan);
      std::vector<float> f(far.size() * RANK_FEATURES), fn;
      const size_t nch = (far.size() + 255) / 256;
      parallel_for(nch, [&](size_t c) {
        for (size_t i = c * 256; i < std::min(far.size(), c * 256 + 256); i++)
          far_features(t, plan, mxr, A->leaves, B->leaves, o->eps, far[i].leaf, f.data() + i * RANK_FEATURES);
      });
      normalise(m, f.data(), (int64_t)far.size(), fn);
      DevBuf dx = upload(fn, s), dy(sizeof(float) * far.size(), s);
      ck(launch_mlp_forward(m->w16, dx.as<float>(), (int)far.size(), dy.as<float>(), s), "rank proposal");
      launches++;
      ck(cudaMemcpyAsync(khat.data(), dy.p, sizeof(float) * far.size(), cudaMemcpyDeviceToHost, s), "rank proposal");
      ck(cudaStreamSynchronize(s), "rank proposal");
      for (float &k : khat) k = std::max(0.f, std::exp2(k) - 1.f);
    }
    for (size_t i = 0; i < far.size(); i++) {
      const LeafDev &lc = A->leaves[far[i].leaf];
      const int mn = (int)std::min(lc.m, lc.n);
      const int k = std::min((int)std::ceil(khat[i] - 0.25f), mn);
      p0v[far[i].leaf] = std::max(p, std::min(PROP_MAX, k + p));
    }
    tr.mark("rank proposal");
  }
  if (fixed_k > 0)  // Algorithm 9: k samples for every far block
    for (const Tgt &g : far) p0v[g.leaf] = fixed_k;
  int pmax = fixed_k > 0 ? fixed_k : p;
  for (const Tgt &g : far) pmax = std::max(pmax, p0v[g.leaf]);
  // Size classes of the application kernel: 0 = panels staged in global memory (targets too
  // large for shared memory); class c >= 1 = targets of at most 32 << (c - 1) rows, columns
  // and H-pair rows, staged in shared memory sized for that bound. Far targets are ordered by
  // class, then by decreasing cost, so every class is one contiguous launch.
  constexpr int NCLS = 12;
  const int P = apply_panel_width(pmax);
  int cw_rows = std::max(t.leaf_size, pcw_rows);
  for (const PlanTerm &pt : plan.terms) cw_rows = std::max(cw_rows, (int)pt.rank);
  const size_t cw_bytes = (size_t)8 * cw_rows * apply_row_stride(P) * es;
  std::vector<int> rho_inner(t.leaf_block.size(), 0), klass(t.leaf_block.size(), 1);
  auto is_leaf_pair = [&](const PairDev &pr) {
    return t.bl[pr.blkA].kind == BK_NEAR && t.bl[pr.blkB].kind == BK_NEAR;
  };
  for (const Tgt &g : far) {
    const int l = g.leaf;
    int rho = 0;
    for (int64_t q = plan.leaf_pair_off[l]; q < plan.leaf_pair_off[l + 1]; q++)
      if (!is_leaf_pair(plan.leaf_pairs[q]))
        rho = std::max(rho, (int)t.cl[t.bl[plan.leaf_pairs[q].blkA].sigma].size);
    rho_inner[l] = rho;
    const LeafDev &lc = A->leaves[l];
    const int dmax = std::max(std::max((int)lc.m, (int)lc.n), rho);
    int c = 1;
    while ((32 << (c - 1)) < dmax && c < NCLS - 1) c++;
    const int cap = 32 << (c - 1);
    const int rb = apply_rows_per_lane(cap);
    const size_t zrows = rb > 0 ? std::max(cap, 8 * cap) : cap;
    if (cap < dmax || (size_t)(2 * cap + zrows) * apply_row_stride(P) * es + cw_bytes > smem_cap) c = 0;
    klass[l] = c;
  }
  // within a class, depth-first leaf order: neighbouring targets share the low-rank terms of
  // their common ancestors and the blocks of their H-pairs, which then stay in L2
  std::stable_sort(far.begin(), far.end(), [&](const Tgt &a, const Tgt &b) {
    if (klass[a.leaf] != klass[b.leaf]) return klass[a.leaf] < klass[b.leaf];
    return a.leaf < b.leaf;
  });

  tr.mark("target classes + sort");
  if (tr.on) {  // per class: targets, low-rank and H-pair elements, term and inner-pair counts
    double lr[NCLS] = {}, lp[NCLS] = {}, ip[NCLS] = {};
    int64_t cnt[NCLS] = {}, nt[NCLS] = {}, nip[NCLS] = {};
    for (const Tgt &g : far) {
      const int l = g.leaf, c = klass[l], b = t.leaf_block[l];
      const LeafDev &lc = A->leaves[l];
      cnt[c]++;
      nt[c] += plan.nterm_cum[b];
      lr[c] += (double)plan.rank_cum[b] * (lc.m + lc.n);
      for (int64_t q = plan.leaf_pair_off[l]; q < plan.leaf_pair_off[l + 1]; q++) {
        const PairDev &pr = plan.leaf_pairs[q];
        const double e = storA[pr.blkA] + storB[pr.blkB];
        if (is_leaf_pair(pr)) lp[c] += e;
        else { ip[c] += e; nip[c]++; }
      }
    }
    for (int c = 0; c < NCLS; c++)
      if (cnt[c])
        std::fprintf(stderr, "hmat trace: class %2d: %7lld targets, %9lld terms, %.3g lr elems, %.3g leaf-pair elems, "
                     "%.3g inner-pair elems (%lld pairs)\n", c, (long long)cnt[c], (long long)nt[c], lr[c], lp[c], ip[c],
                     (long long)nip[c]);
  }
  auto make_targets = [&](const std::vector<Tgt> &tv, std::vector<TargetDev> &tg, std::vector<PairDev> &tpairs) {
    tg.resize(tv.size());
    for (size_t i = 0; i < tv.size(); i++) {
      const int l = tv[i].leaf;
      const LeafDev &lc = A->leaves[l];
      TargetDev &d = tg[i];
      std::memset(&d, 0, sizeof(d));
      d.row = lc.row;
      d.col = lc.col;
      d.m = lc.m;
      d.n = lc.n;
      d.leaf = l;
      d.p0 = p0v[l];
      d.blk = t.leaf_block[l];
      d.nterms = plan.nterm_cum[d.blk];
      d.pair_lo = (int32_t)tpairs.size();
      for (int64_t q = plan.leaf_pair_off[l]; q < plan.leaf_pair_off[l + 1]; q++)
        if (is_leaf_pair(plan.leaf_pairs[q])) tpairs.push_back(plan.leaf_pairs[q]);
      d.pair_mid = (int32_t)tpairs.size();
      for (int64_t q = plan.leaf_pair_off[l]; q < plan.leaf_pair_off[l + 1]; q++)
        if (!is_leaf_pair(plan.leaf_pairs[q])) tpairs.push_back(plan.leaf_pairs[q]);
      d.pair_hi = (int32_t)tpairs.size();
    }
  };
  std::vector<TargetDev> ftg, ntg;
  std::vector<PairDev> fpairs, npairs;
  make_targets(far, ftg, fpairs);
  make_targets(nearv, ntg, npairs);
  tr.mark("target tables");
  // scratch offsets for far targets and the per-class launch parameters
  int64_t qw_elems = 0, xy_elems = 0, stage_elems = 0;
  struct ClassLaunch {
    int first = 0, count = 0, dmax = 0, rho = 0, split = 1;
    int64_t inner_pairs = 0, y_lo = 0, y_hi = 0;
  } cls[NCLS];
  for (int c = 0; c < NCLS; c++) cls[c].first = -1;
  for (size_t i = 0; i < ftg.size(); i++) {
    TargetDev &d = ftg[i];
    const int mn = std::min(d.m, d.n);
    d.rmax = std::min(max_rank, ((mn + p + p - 1) / p) * p);
    if (d.rmax < pmax) d.rmax = pmax;
    d.q_off = qw_elems;
    qw_elems += (int64_t)d.m * d.rmax;
    d.w_off = qw_elems;
    qw_elems += (int64_t)d.n * d.rmax;
    const int64_t mx = std::max(d.m, d.n);
    d.x_off = xy_elems;
    d.y_off = xy_elems;  // separate buffers x and y share the same offsets
    xy_elems += mx * pmax;
    const int c = klass[d.leaf];
    ClassLaunch &cl = cls[c];
    if (cl.first < 0) cl.first = (int)i;
    cl.count++;
    cl.dmax = std::max(cl.dmax, (int)mx);
    cl.rho = std::max(cl.rho, rho_inner[d.leaf]);
    cl.inner_pairs += d.pair_hi - d.pair_mid;
    if (cl.count == 1) cl.y_lo = d.y_off;
    cl.y_hi = d.y_off + mx * pmax;
    if (c == 0) {
      d.stage_off = stage_elems;
      stage_elems += ((int64_t)d.m + d.n + rho_inner[d.leaf]) * apply_row_stride(P);
    }
  }

  // Big targets (shared-atomic launches, panels in shared memory) have few thread blocks each
  // with a long serial chain of H-pairs: their H-pairs and terms are split over K blocks per
  // target (about two H-pairs of inner blocks per block, at most 8), which add their partial
  // outputs into a zeroed output.
  for (int c = 1; c < NCLS; c++) {
    ClassLaunch &cl = cls[c];
    if (cl.count == 0 || apply_rows_per_lane(cl.dmax) > 0) continue;
    const double ppt = (double)cl.inner_pairs / cl.count;
    cl.split = std::max(1, std::min(8, (int)std::ceil(ppt / 2.0)));
  }
  for (int c = 0; c < NCLS; c++) {
    if (cls[c].count == 0) continue;
    if (c == 0) {
      S.apply_gstage_targets += cls[c].count;
    } else if (cls[c].split > 1) {
      S.apply_split_targets += cls[c].count;
      S.apply_max_split = std::max(S.apply_max_split, cls[c].split);
    }
  }

  // ---- a8 on a second stream, concurrent with the far-field rounds: C's buffer starts with the
  // near leaves (their offsets are known now); they are evaluated into a staging buffer that is
  // copied into C once the far ranks are known.
  int64_t near_elems = 0;  // offsets local to this group's output buffer
  for (const TargetDev &d : ntg) {
    LeafDev &l = C->leaves[d.leaf];
    l.off_u = near_elems;
    near_elems += (int64_t)l.m * l.n;
  }
  struct StreamGuard {
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ~StreamGuard() {
      if (e0) cudaEventDestroy(e0);
      if (e1) cudaEventDestroy(e1);
      if (st) cudaStreamDestroy(st);
    }
  } s2;
  ck(cudaStreamCreateWithFlags(&s2.st, cudaStreamNonBlocking), "stream");
  ck(cudaEventCreateWithFlags(&s2.e0, cudaEventDisableTiming), "event");
  ck(cudaEventCreateWithFlags(&s2.e1, cudaEventDisableTiming), "event");
  // the near field's tables go up on the second stream (idle, so the copies do not wait for the
  // products), then that stream waits for the products
  if (tr.on)
    std::fprintf(stderr, "hmat trace: buffers: near %lld, qw %lld, xy %lld, stage %lld elems\n", (long long)near_elems,
                 (long long)qw_elems, (long long)xy_elems, (long long)stage_elems);
  DevBuf d_near(es * std::max<int64_t>(near_elems, 1), s2.st);
  DevBuf d_near_leaves = upload(C->leaves, s2.st);
  DevBuf d_ntg = upload(ntg, s2.st), d_npairs = upload(npairs, s2.st);
  DevBuf d_nerr(sizeof(int), s2.st);
  ck(cudaMemsetAsync(d_nerr.p, 0, sizeof(int), s2.st), "memset");
  // the near field's own device time, on its stream
  struct NearEvents {
    cudaEvent_t e[2] = {nullptr, nullptr};
    ~NearEvents() {
      for (cudaEvent_t x : e)
        if (x) cudaEventDestroy(x);
    }
  } ne;
  ck(cudaEventCreate(&ne.e[0]), "event");
  ck(cudaEventCreate(&ne.e[1]), "event");
  // the near field needs the low-rank products: its stream waits for them, then runs beside the
  // sampling rounds
  {
    ck(cudaEventRecord(s2.e0, s), "event");
    ck(cudaStreamWaitEvent(s2.st, s2.e0, 0), "stream wait");
    ck(cudaEventRecord(ne.e[0], s2.st), "event");
    ck(launch_near_eval(cprec, d_ntg.as<TargetDev>(), (int)ntg.size(), d_blkterms.as<int2>(), d_terms.as<TermDev>(),
                        d_npairs.as<PairDev>(), t.d_blocks, A->d_leaves.as<LeafDev>(), B->d_leaves.as<LeafDev>(),
                        dataA, dataB, d_near_leaves.as<LeafDev>(), d_near.p, d_nerr.as<int>(), s2.st),
       "near field");
    ck(cudaEventRecord(ne.e[1], s2.st), "event");
    ck(cudaEventRecord(s2.e1, s2.st), "event");
    tr.mark("near field launched");
  }
  // ---- a3..a7: adaptive randomized truncation of all far targets
  const int nf = (int)ftg.size();
  DevBuf d_ftg = upload(ftg, s), d_fpairs = upload(fpairs, s);
  DevBuf d_qw(sizeof(double) * std::max<int64_t>(qw_elems, 1), s);
  DevBuf d_x(es * std::max<int64_t>(xy_elems, 1), s), d_y(es * std::max<int64_t>(xy_elems, 1), s);
  DevBuf d_stage(es * std::max<int64_t>(stage_elems, 1), s);
  if (check_finite_enabled()) {  // the finiteness check scans whole buffers: start them at zero
    ck(cudaMemsetAsync(d_qw.p, 0, sizeof(double) * std::max<int64_t>(qw_elems, 1), s), "memset");
    ck(cudaMemsetAsync(d_x.p, 0, es * std::max<int64_t>(xy_elems, 1), s), "memset");
    ck(cudaMemsetAsync(d_y.p, 0, es * std::max<int64_t>(xy_elems, 1), s), "memset");
  }
  std::vector<TargetState> st0(nf);
  for (auto &x : st0) {
    std::memset(&x, 0, sizeof(x));
    x.active = 1;
  }
  DevBuf d_st = upload(st0, s);
  // a4 runs one warp per target of at most 64 rows, one block per larger target
  std::vector<int32_t> orth_w, orth_b, orth_wn, orth_bn;
  for (int i = 0; i < nf; i++) {
    (ftg[i].m <= 64 ? orth_w : orth_b).push_back(i);
    (ftg[i].n <= 64 ? orth_wn : orth_bn).push_back(i);  // the column side (fixed-rank mode)
  }
  DevBuf d_orth_w = upload(orth_w, s), d_orth_b = upload(orth_b, s);
  DevBuf d_orth_wn = upload(orth_wn, s), d_orth_bn = upload(orth_bn, s);
  DevBuf d_cnt(sizeof(int32_t), s);
  ApplyArgs aa{};
  aa.tg = d_ftg.as<TargetDev>();
  aa.blk_terms = d_blkterms.as<int2>();
  aa.terms = d_terms.as<TermDev>();
  aa.pairs = d_fpairs.as<PairDev>();
  aa.blocks = t.d_blocks;
  aa.leafA = A->d_leaves.as<LeafDev>();
  aa.leafB = B->d_leaves.as<LeafDev>();
  aa.dataA = dataA;
  aa.dataB = dataB;
  aa.state = d_st.as<TargetState>();
  aa.x_base = d_x.p;
  aa.y_base = d_y.p;
  aa.stage_base = d_stage.p;
  aa.p = p;
  const double eps = o->eps;
  const double eps_stop = 0.5 * eps;
  // stop tolerance of the one-vector compressors: eps / 8, but not below four rounding units of
  // the precision the passes run in (their increments cannot be resolved below it)
  const double eps_stop_1v = std::max(0.125 * eps, 4.0 * (cprec == 64 ? 0x1.0p-53 : 0x1.0p-24));
  const double eps_trunc = fixed_k > 0 ? 0.0 : eps;  // fixed rank: keep every sampled direction
  int rounds = 0;
  // events around every application pass (S and S^T), read after the stream synchronises
  std::vector<cudaEvent_t> aev;
  struct AevGuard {
    std::vector<cudaEvent_t> &v;
    ~AevGuard() { for (auto e : v) cudaEventDestroy(e); }
  } aevg{aev};
  struct ClassTiming {
    int c;
    bool trans;
    cudaEvent_t e0, e1;
  };
  std::vector<ClassTiming> ctim;  // per-class launch events (HMAT_TRACE only)
  std::vector<std::pair<int, std::array<cudaEvent_t, 2>>> kev;  // gaussian / orth / stop test
  auto kmark = [&](int which_kernel, int edge) {
    if (!tr.on) return;
    if (edge == 0) {
      kev.push_back({which_kernel, {nullptr, nullptr}});
      cudaEventCreate(&kev.back().second[0]);
      cudaEventCreate(&kev.back().second[1]);
    }
    cudaEventRecord(kev.back().second[edge], s);
  };
  auto timed_apply = [&](bool trans) {
    cudaEvent_t e0, e1;
    ck(cudaEventCreate(&e0), "event");
    aev.push_back(e0);
    ck(cudaEventCreate(&e1), "event");
    aev.push_back(e1);
    ck(cudaEventRecord(e0, s), "event");
    for (int c = 0; c < NCLS; c++) {
      if (cls[c].count == 0) continue;
      ApplyArgs ac = aa;
      ac.first = cls[c].first;
      ac.count = cls[c].count;
      ac.smem_in = ac.smem_out = cls[c].dmax;
      ac.smem_rho = cls[c].rho;
      // register-accumulating launches also keep every warp's partial output in this region
      if (c > 0 && apply_rows_per_lane(cls[c].dmax) > 0) ac.smem_rho = std::max(ac.smem_rho, 8 * cls[c].dmax);
      ac.smem_cw = cw_rows;
      ac.gstage = c == 0 ? 1 : 0;
      ac.split = cls[c].split;
      if (ac.split > 1)
        ck(cudaMemsetAsync((char *)d_y.p + es * cls[c].y_lo, 0, es * (cls[c].y_hi - cls[c].y_lo), s), "memset");
      ClassTiming ct{c, trans, nullptr, nullptr};
      if (tr.on) {
        cudaEventCreate(&ct.e0);
        cudaEventCreate(&ct.e1);
        cudaEventRecord(ct.e0, s);
      }
      ck(launch_apply(cprec, trans, ac, s), trans ? "apply S^T" : "apply S");
      if (tr.on) {
        cudaEventRecord(ct.e1, s);
        ctim.push_back(ct);
      }
      launches++;
    }
    ck(cudaEventRecord(e1, s), "event");
  };
  if (fixed_k > 0 && nf > 0) {
    // Algorithm 9: L = S Omega, orthonormalised; q times U = S^T L, orthonormalised, and
    // L = S U, orthonormalised; finally W = S^T L. Every orthonormalisation is of the new block
    // alone.
    rounds = 1;
    aa.p = pmax;
    aa.round = 0;
    ck(launch_gaussian(cprec, aa.tg, aa.state, nf, pmax, o->seed, 0, d_x.p, s), "gaussian");
    timed_apply(false);
    auto orth_side = [&](int side) {
      const std::vector<int32_t> &w = side ? orth_wn : orth_w, &bl = side ? orth_bn : orth_b;
      const DevBuf &dw = side ? d_orth_wn : d_orth_w, &db = side ? d_orth_bn : d_orth_b;
      ck(launch_orth(cprec, aa.tg, dw.as<int32_t>(), (int)w.size(), db.as<int32_t>(), (int)bl.size(), aa.state, pmax,
                     eps, d_y.p, d_qw.as<double>(), d_x.p, 0, s, side, 1),
         "orth");
      launches += (w.empty() ? 0 : 1) + (bl.empty() ? 0 : 1);
    };
    orth_side(0);
    for (int it = 0; it < power_q; it++) {
      timed_apply(true);
      orth_side(1);
      timed_apply(false);
      orth_side(0);
    }
    timed_apply(true);
    ck(cudaMemsetAsync(d_cnt.p, 0, sizeof(int32_t), s), "memset");
    ck(launch_absorb_w(cprec, aa.tg, aa.state, nf, p, eps_stop, d_y.p, d_qw.as<double>(), 0, 1, d_cnt.as<int32_t>(),
                       s, 1),
       "fixed rank");
    launches += 2;
    ck(cudaStreamSynchronize(s), "fixed rank");
  }
  if (aca && nf > 0) {
    // Algorithm 6 on every far target at once: each step is one S^T pass (the pivot rows
    // e_i^T S) and one S pass (the pivot columns S e_j), single columns, with the pivoting, the
    // residual updates and eq. (truncaca) on the device between them. A step adds one cross or
    // marks one zero row used, so the steps are bounded by the basis capacity plus the rows.
    aa.p = 1;
    aa.round = 1;  // every target takes aa.p columns
    ck(launch_aca_start(cprec, aa.tg, aa.state, nf, d_qw.as<double>(), d_x.p, s), "cross approximation");
    launches++;
    int max_steps = 0;
    for (const TargetDev &d : ftg) max_steps = std::max(max_steps, d.rmax + d.m);
    for (int step = 0; step < max_steps; step++) {
      rounds++;
      timed_apply(true);
      ck(launch_aca_row(cprec, aa.tg, aa.state, nf, d_y.p, d_qw.as<double>(), d_x.p, s), "cross approximation row");
      timed_apply(false);
      ck(cudaMemsetAsync(d_cnt.p, 0, sizeof(int32_t), s), "memset");
      ck(launch_aca_col(cprec, aa.tg, aa.state, nf, d_y.p, d_qw.as<double>(), d_x.p, eps_stop_1v,
                        d_cnt.as<int32_t>(), s),
         "cross approximation column");
      launches += 2;
      int32_t act = 0;
      ck(cudaMemcpyAsync(&act, d_cnt.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "count");
      ck(cudaStreamSynchronize(s), "cross approximation step");
      if (act == 0) break;
    }
    ck(launch_aca_qr(aa.tg, aa.state, nf, d_qw.as<double>(), s), "cross approximation QR");
    launches++;
  }
  if (lanczos && nf > 0) {
    // Algorithm 7 on every far target at once: each step is one S pass (q_r from w_r) and one
    // S^T pass (w_{r+1} from q_r), single columns, with the recurrence, the reorthogonalization
    // and eq. (truncaca) on the device between them; at most r_max - 1 steps. Then
    // W = S^T Q in p-column passes, the input of the core truncation.
    aa.p = 1;
    aa.round = 1;
    ck(launch_lz_start(cprec, aa.tg, aa.state, nf, d_qw.as<double>(), d_x.p, o->seed, s), "Lanczos start");
    launches++;
    int max_steps = 0;
    for (const TargetDev &d : ftg) max_steps = std::max(max_steps, d.rmax);
    for (int step = 0; step < max_steps; step++) {
      rounds++;
      timed_apply(false);
      ck(launch_lz_q(cprec, aa.tg, aa.state, nf, d_y.p, d_qw.as<double>(), d_x.p, s), "Lanczos q");
      timed_apply(true);
      ck(cudaMemsetAsync(d_cnt.p, 0, sizeof(int32_t), s), "memset");
      ck(launch_lz_w(cprec, aa.tg, aa.state, nf, d_y.p, d_qw.as<double>(), d_x.p, eps_stop_1v, d_cnt.as<int32_t>(),
                     s),
         "Lanczos w");
      launches += 2;
      int32_t act = 0;
      ck(cudaMemcpyAsync(&act, d_cnt.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "count");
      ck(cudaStreamSynchronize(s), "Lanczos step");
      if (act == 0) break;
    }
    std::vector<TargetState> sl(nf);
    ck(cudaMemcpyAsync(sl.data(), d_st.p, sizeof(TargetState) * nf, cudaMemcpyDeviceToHost, s), "states");
    ck(cudaStreamSynchronize(s), "states");
    int rtop = 0;
    for (const TargetState &x : sl) rtop = std::max(rtop, x.r);
    aa.p = p;
    for (int c0 = 0; c0 < rtop; c0 += p) {
      ck(launch_lz_load(cprec, aa.tg, aa.state, nf, d_qw.as<double>(), d_x.p, c0, p, s), "projection input");
      timed_apply(true);
      ck(launch_lz_store(cprec, aa.tg, aa.state, nf, d_y.p, d_qw.as<double>(), c0, p, s), "projection");
      launches += 2;
    }
  }
  double host_t = now_ms();
  int32_t act_prev = nf;
  for (int round = 0; round < max_rounds && nf > 0 && fixed_k == 0 && !single; round++) {
    rounds++;
    const int pr = round == 0 ? pmax : p;  // widest panel this round (round 0: each target's p0)
    aa.p = pr;
    aa.round = round;
    cudaEvent_t rev[2] = {nullptr, nullptr};  // (trace) the round's span on the device
    if (tr.on) {
      std::fprintf(stderr, "hmat trace: round %d: %d active targets, host %.3f ms since the last round's result\n",
                   round, act_prev, now_ms() - host_t);
      cudaEventCreate(&rev[0]);
      cudaEventCreate(&rev[1]);
      cudaEventRecord(rev[0], s);
    }
    kmark(0, 0);
    ck(launch_gaussian(cprec, aa.tg, aa.state, nf, pr, o->seed, round, d_x.p, s), "gaussian");
    kmark(0, 1);
    timed_apply(false);
    check_finite(cprec, d_y.p, xy_elems, "apply S", s);
    kmark(1, 0);
    ck(launch_orth(cprec, aa.tg, d_orth_w.as<int32_t>(), (int)orth_w.size(), d_orth_b.as<int32_t>(),
                   (int)orth_b.size(), aa.state, pr, eps, d_y.p, d_qw.as<double>(), d_x.p, round, s),
       "orth");
    kmark(1, 1);
    check_finite(64, d_qw.p, qw_elems, "orthogonalisation", s);
    timed_apply(true);
    check_finite(cprec, d_y.p, xy_elems, "apply S^T", s);
    launches += 2 + (orth_w.empty() ? 0 : 1) + (orth_b.empty() ? 0 : 1);
    kmark(2, 0);
    ck(cudaMemsetAsync(d_cnt.p, 0, sizeof(int32_t), s), "memset");
    ck(launch_absorb_w(cprec, aa.tg, aa.state, nf, p, eps_stop, d_y.p, d_qw.as<double>(), round, max_rounds,
                       d_cnt.as<int32_t>(), s),
       "stop test");
    kmark(2, 1);
    if (tr.on) cudaEventRecord(rev[1], s);
    int32_t act = 0;
    ck(cudaMemcpyAsync(&act, d_cnt.p, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "count");
    ck(cudaStreamSynchronize(s), "round");
    host_t = now_ms();
    act_prev = act;
    if (tr.on) {
      float x = 0.f;
      cudaEventElapsedTime(&x, rev[0], rev[1]);
      std::fprintf(stderr, "hmat trace: round %d: %.3f ms on the device\n", round, x);
      cudaEventDestroy(rev[0]);
      cudaEventDestroy(rev[1]);
    }
    if (act == 0) break;
  }
  tr.mark("sampling rounds done");
  if (tr.on) {
    double tc[NCLS][2] = {};
    cudaStreamSynchronize(s);
    for (ClassTiming &ct : ctim) {
      float x = 0.f;
      cudaEventElapsedTime(&x, ct.e0, ct.e1);
      tc[ct.c][ct.trans ? 1 : 0] += x;
      cudaEventDestroy(ct.e0);
      cudaEventDestroy(ct.e1);
    }
    double tk[3] = {};
    for (auto &e : kev) {
      float x = 0.f;
      cudaEventElapsedTime(&x, e.second[0], e.second[1]);
      tk[e.first] += x;
      cudaEventDestroy(e.second[0]);
      cudaEventDestroy(e.second[1]);
    }
    std::fprintf(stderr, "hmat trace: rounds: gaussian %.3f ms, orthogonalisation %.3f ms, stop test %.3f ms\n", tk[0],
                 tk[1], tk[2]);
    for (int c = 0; c < NCLS; c++)
      if (cls[c].count)
        std::fprintf(stderr, "hmat trace: class %2d apply: S %8.3f ms, S^T %8.3f ms (all rounds), %d blocks/target\n",
                     c, tc[c][0], tc[c][1], cls[c].split);
  }
  ck(cudaEventRecord(ev[2], s), "event");
  std::vector<TargetState> st(nf);
  if (nf) ck(cudaMemcpyAsync(st.data(), d_st.p, sizeof(TargetState) * nf, cudaMemcpyDeviceToHost, s), "states");
  ck(cudaStreamSynchronize(s), "states");
  std::vector<int32_t> rounds_of(nf);
  for (int i = 0; i < nf; i++) {
    S.first_round_cols += ftg[i].p0;
    if (st[i].nfwd <= 1 && st[i].rank != -2) S.done_in_first_round++;
    S.sample_passes += st[i].nfwd;
    rounds_of[i] = st[i].nfwd;
  }
  // The unique bytes of the passes (a statistic), counted on a host thread while the device
  // truncates and writes C; joined before the group's statistics are summed (or on unwinding).
  double uniq_elems = 0.0;
  struct Joiner {
    std::thread th;
    ~Joiner() {
      if (th.joinable()) th.join();
    }
  } uniq_thread;
  uniq_thread.th = std::thread([&]() {
    try {
      uniq_elems = apply_unique_elems(t, plan, A->leaves, B->leaves, storA, storB, ftg, fpairs, rounds_of,
                                      single ? 1 : p);
    } catch (...) {
      uniq_elems = 0.0;
    }
  });
  {
    std::vector<int32_t> ids_small, ids_big;
    for (int i = 0; i < nf; i++) (st[i].r <= 32 ? ids_small : ids_big).push_back(i);
    DevBuf d_ids_small = upload(ids_small, s), d_ids_big = upload(ids_big, s);
    cudaEvent_t fe[3] = {nullptr, nullptr, nullptr};
    if (tr.on)
      for (auto &e : fe) {
        cudaEventCreate(&e);
      }
    if (tr.on) cudaEventRecord(fe[0], s);
    ck(launch_final(aa.tg, aa.state, d_ids_small.as<int32_t>(), (int)ids_small.size(), true, eps_trunc,
                    d_qw.as<double>(), s),
       "final truncation (warp)");
    if (tr.on) cudaEventRecord(fe[1], s);
    ck(launch_final(aa.tg, aa.state, d_ids_big.as<int32_t>(), (int)ids_big.size(), false, eps_trunc,
                    d_qw.as<double>(), s),
       "final truncation (block)");
    if (tr.on) {
      cudaEventRecord(fe[2], s);
      cudaStreamSynchronize(s);
      float x0 = 0.f, x1 = 0.f;
      cudaEventElapsedTime(&x0, fe[0], fe[1]);
      cudaEventElapsedTime(&x1, fe[1], fe[2]);
      std::vector<TargetState> sf(nf);
      if (nf) cudaMemcpy(sf.data(), d_st.p, sizeof(TargetState) * nf, cudaMemcpyDeviceToHost);
      int64_t rsum = 0, swsum = 0;
      int swmax = 0;
      for (int i = 0; i < nf; i++) {
        rsum += sf[i].r;
        swsum += sf[i].sweeps;
        swmax = std::max(swmax, sf[i].sweeps);
      }
      std::fprintf(stderr, "hmat trace: final: %zu blocks (r <= 32) %.3f ms, %zu blocks %.3f ms, mean r %.1f, "
                   "sweeps mean %.2f max %d\n", ids_small.size(), x0, ids_big.size(), x1, nf ? (double)rsum / nf : 0.0,
                   nf ? (double)swsum / nf : 0.0, swmax);
      for (auto &e : fe) cudaEventDestroy(e);
    }
    launches += (ids_small.empty() ? 0 : 1) + (ids_big.empty() ? 0 : 1);
    if (tr.on) {  // each size class on its own: what separate launches of the classes must read
      double parts[3] = {0, 0, 0};
      const double uniq = (double)es * apply_unique_elems(t, plan, A->leaves, B->leaves, storA, storB, ftg,
                                                          fpairs, rounds_of, single ? 1 : p, parts);
      double sum = 0.0;
      for (int c = 0; c < NCLS; c++) {
        if (cls[c].count == 0) continue;
        const std::vector<TargetDev> sub(ftg.begin() + cls[c].first, ftg.begin() + cls[c].first + cls[c].count);
        const std::vector<int32_t> sr(rounds_of.begin() + cls[c].first,
                                      rounds_of.begin() + cls[c].first + cls[c].count);
        const double u = (double)es * apply_unique_elems(t, plan, A->leaves, B->leaves, storA, storB, sub, fpairs,
                                                         sr, single ? 1 : p);
        sum += u;
        std::fprintf(stderr, "hmat trace: class %2d unique bytes over its passes %.4g GB\n", c, u * 1e-9);
      }
      std::fprintf(stderr, "hmat trace: unique bytes over all passes %.4g GB (classes on their own: %.4g GB); "
                   "terms %.4g GB, H-pair blocks %.4g GB, panels %.4g GB\n", uniq * 1e-9, sum * 1e-9,
                   es * parts[0] * 1e-9, es * parts[1] * 1e-9, es * parts[2] * 1e-9);
    }
    if (nf) ck(cudaMemcpyAsync(st.data(), d_st.p, sizeof(TargetState) * nf, cudaMemcpyDeviceToHost, s), "states");
    ck(cudaStreamSynchronize(s), "final");
  }
  ck(cudaEventRecord(ev[3], s), "event");

  tr.mark("core truncation done");
  // ---- C: far leaves after the near ones, write far factors (a9), join the near field (a8)
  int64_t off = near_elems;
  int64_t notconv = 0;
  for (size_t i = 0; i < ftg.size(); i++) {
    int k = st[i].rank;
    if (k < -2) { notconv++; k = -(k + 3); }
    LeafDev &l = C->leaves[ftg[i].leaf];
    l.rank = k;
    l.off_u = off;
    l.off_v = off + (int64_t)l.m * k;
    off = l.off_v + (int64_t)l.n * k;
  }
  GroupOut &go = gouts[grp];
  go.elems = off;
  go.data = DevBuf(es * std::max<int64_t>(off, 1), s);
  DevBuf d_gleaves = upload(C->leaves, s);
  ck(launch_write_far(cprec, aa.tg, aa.state, nf, d_qw.as<double>(), d_gleaves.as<LeafDev>(), go.data.p, s),
     "write far");
  ck(cudaStreamWaitEvent(s, s2.e1, 0), "stream wait");
  if (near_elems > 0)
    ck(cudaMemcpyAsync(go.data.p, d_near.p, es * near_elems, cudaMemcpyDeviceToDevice, s), "near copy");
  launches += (nf > 0 ? 1 : 0) + (ntg.empty() ? 0 : 1);
  ck(cudaEventRecord(ev[4], s), "event");
  int near_err = 0;
  ck(cudaMemcpyAsync(&near_err, d_nerr.p, sizeof(int), cudaMemcpyDeviceToHost, s), "near status");
  ck(cudaStreamSynchronize(s), "product");
  a2_report();
  {
    float nms = 0;
    cudaEventElapsedTime(&nms, ne.e[0], ne.e[1]);
    S.ms_near_kernel += nms;
    if (tr.on)
      std::fprintf(stderr, "hmat trace: near field kernel: %zu leaves, %.3f ms (on its own stream)\n", ntg.size(),
                   nms);
  }
  if (near_err) fail(HMAT_ETIMEOUT, "near field: a bounded tensor-core wait gave up");
  tr.mark("C written, synchronised");
  double ms_apply = 0;
  for (size_t i = 0; i + 1 < aev.size(); i += 2) {
    float x = 0;
    cudaEventElapsedTime(&x, aev[i], aev[i + 1]);
    ms_apply += x;
  }
  S.ms_apply += ms_apply;
  S.apply_launches += (int64_t)aev.size() / 2;
  S.launches += launches;

  float ms = 0;
  cudaEventElapsedTime(&ms, ev[0], ev[1]);
  S.ms_terms += ms;
  cudaEventElapsedTime(&ms, ev[1], ev[2]);
  S.ms_sample += ms;
  cudaEventElapsedTime(&ms, ev[2], ev[3]);
  S.ms_final += ms;
  cudaEventElapsedTime(&ms, ev[3], ev[4]);
  S.ms_near += ms;
  S.rounds = std::max(S.rounds, rounds);
  S.not_converged += notconv;
  double fa = 0, ba = 0, fn = 0, bu = 0;
  for (size_t i = 0; i < ftg.size(); i++) {
    const double e = elems_b[ftg[i].leaf];
    const int cols = st[i].r;  // columns that went through both passes
    fa += 2.0 * e * 2.0 * cols;
    ba += e * (single ? 2.0 * cols + (lanczos ? (cols + p - 1) / p : 0) : 2.0 * ((cols + p - 1) / p)) * es;
    const double launches_b = 2.0 * std::max(1, st[i].nfwd);
    bu += launches_b * (e + (double)(ftg[i].m + ftg[i].n) * (single ? 1 : p)) * es;
  }
  for (const TargetDev &d : ntg) {
    const double kk = (double)plan.rank_cum[d.blk];
    double rr = 0;
    for (int q = d.pair_lo; q < d.pair_hi; q++) rr += t.cl[t.bl[npairs[q].blkA].sigma].size;
    fn += 2.0 * d.m * d.n * (kk + rr);
  }
  uniq_thread.th.join();
  S.bytes_apply_unique += (double)es * uniq_elems;
  S.bytes_apply_use += bu;
  S.flops_apply += fa;
  S.bytes_apply += ba;
  S.flops_near += fn;
  };  // run_group

  for (int g = 0; g < ngroups; g++) run_group(g);
  S.groups = ngroups;
  // ---- C: one buffer; with several groups, the groups' buffers one after another
  if (ngroups == 1) {
    C->d_data = std::move(gouts[0].data);
    C->data_elems = gouts[0].elems;
  } else {
    std::vector<int64_t> base(ngroups + 1, 0);
    for (int g = 0; g < ngroups; g++) base[g + 1] = base[g] + gouts[g].elems;
    C->data_elems = base[ngroups];
    C->d_data = DevBuf(es * std::max<int64_t>(base[ngroups], 1), s);
    for (int g = 0; g < ngroups; g++)
      if (gouts[g].elems > 0)
        ck(cudaMemcpyAsync((char *)C->d_data.p + es * base[g], gouts[g].data.p, es * gouts[g].elems,
                           cudaMemcpyDeviceToDevice, s),
           "group copy");
    for (size_t l = 0; l < C->leaves.size(); l++) {
      C->leaves[l].off_u += base[leaf_group[l]];
      C->leaves[l].off_v += base[leaf_group[l]];
    }
    ck(cudaStreamSynchronize(s), "group copy");
    gouts.clear();
  }
  C->d_leaves = upload(C->leaves, s);
  ck(cudaStreamSynchronize(s), "product");
  fill_structure_stats(C.get());
}

}  // namespace

namespace {

void check_pair(const hmat_s *A, const hmat_s *B, const hmat_mult_opts *opts) {
  if (!A || !B || !opts) fail(HMAT_EINVAL, "NULL argument");
  if (!(opts->eps > 0.0) || !std::isfinite(opts->eps)) fail(HMAT_EINVAL, "eps must be a positive number");
  if (opts->mode != HMAT_MODE_F64 && opts->mode != HMAT_MODE_MIXED) fail(HMAT_EINVAL, "unknown mode");
  if (A->tree != B->tree) {
    const Tree &ta = *A->tree, &tb = *B->tree;
    if (!same_points(ta, tb.orig.data(), tb.n, tb.dim) || ta.leaf_size != tb.leaf_size || ta.eta != tb.eta)
      fail(HMAT_EMISMATCH, "A and B are not on one block tree");
  }
  if (A->prec != B->prec) fail(HMAT_EINVAL, "A and B must have the same factor precision");
}

}  // namespace

extern "C" hmat_status hmat_multiply_batched(const hmat_t *A, const hmat_t *B, int count, const hmat_mult_opts *opts,
                                             void *stream, hmat_t *C) {
  if (C && count > 0)
    for (int i = 0; i < count; i++) C[i] = nullptr;
  return guard([&] {
    if (!A || !B || !C || !opts || count < 0) fail(HMAT_EINVAL, "NULL argument or negative count");
    for (int i = 0; i < count; i++) check_pair(A[i], B[i], opts);
    if (count == 0) return;
    // products on NS worker threads, each with its own stream that first waits for the caller's
    // stream; the largest products start first; the caller's stream waits for all of them
    const int NS = std::min(count, 8);
    std::vector<int> order(count);
    for (int i = 0; i < count; i++) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return A[x]->tree->n > A[y]->tree->n; });
    cudaStream_t caller = (cudaStream_t)stream;
    cudaEvent_t start;
    ck(cudaEventCreateWithFlags(&start, cudaEventDisableTiming), "event");
    std::vector<cudaStream_t> ws(NS, nullptr);
    std::vector<cudaEvent_t> done(NS, nullptr);
    struct Cleanup {
      cudaEvent_t &start;
      std::vector<cudaStream_t> &ws;
      std::vector<cudaEvent_t> &done;
      ~Cleanup() {
        for (auto e : done) if (e) cudaEventDestroy(e);
        for (auto st : ws) if (st) cudaStreamDestroy(st);
        if (start) cudaEventDestroy(start);
      }
    } cleanup{start, ws, done};
    ck(cudaEventRecord(start, caller), "event");
    for (int w = 0; w < NS; w++) {
      ck(cudaStreamCreateWithFlags(&ws[w], cudaStreamNonBlocking), "stream");
      ck(cudaEventCreateWithFlags(&done[w], cudaEventDisableTiming), "event");
      ck(cudaStreamWaitEvent(ws[w], start, 0), "stream wait");
    }
    MemGate gate;
    {
      size_t fr = 0, tot = 0;
      ck(cudaMemGetInfo(&fr, &tot), "memory info");
      gate.budget = (int64_t)(0.8 * (double)fr);
    }
    std::vector<std::unique_ptr<hmat_s>> out(count);
    std::vector<hmat_status> st(count, HMAT_OK);
    std::vector<std::string> msg(count);
    std::atomic<int> next{0};
    int dev = 0;
    ck(cudaGetDevice(&dev), "device");
    auto worker = [&](int w) {
      cudaSetDevice(dev);
      for (int k = next++; k < count; k = next++) {
        const int i = order[k];
        try {
          Product pr;
          pr.A = A[i];
          pr.B = B[i];
          pr.o = opts;
          pr.s = ws[w];
          pr.cprec = opts->mode == HMAT_MODE_F64 ? 64 : A[i]->prec;
          pr.gate = &gate;
          pr.run();
          out[i] = std::move(pr.C);
        } catch (const HErr &f) {
          st[i] = f.st;
          msg[i] = f.msg;
        } catch (const std::bad_alloc &) {
          st[i] = HMAT_ENOMEM;
          msg[i] = "host allocation failed";
        } catch (const std::exception &e) {
          st[i] = HMAT_EINVAL;
          msg[i] = e.what();
        } catch (...) {
          st[i] = HMAT_EINVAL;
          msg[i] = "unknown exception";
        }
      }
    };
    std::vector<std::thread> th;
    th.reserve(NS);
    for (int w = 1; w < NS; w++) {
      try {
        th.emplace_back(worker, w);
      } catch (...) {
        break;  // no thread to be had: the threads already started take the remaining products
      }
    }
    worker(0);
    for (auto &x : th) x.join();
    for (int w = 0; w < NS; w++) {
      ck(cudaEventRecord(done[w], ws[w]), "event");
      ck(cudaStreamWaitEvent(caller, done[w], 0), "stream wait");
    }
    // the outputs belong to the caller's stream from here on (the worker streams end with this
    // call); the caller's stream already waits for the work that produced them
    for (auto &h : out)
      if (h) {
        h->stream = caller;
        h->d_data.s = caller;
        h->d_leaves.s = caller;
      }
    for (int i = 0; i < count; i++)
      if (st[i] != HMAT_OK) fail(st[i], "product " + std::to_string(i) + ": " + msg[i]);
    bool nc = false;
    for (int i = 0; i < count; i++) {
      nc |= out[i]->stats.not_converged > 0;
      C[i] = out[i].release();
    }
    if (nc) fail(HMAT_ENOTCONV, "some far blocks hit max_rank or max_rounds");
  });
}

extern "C" hmat_status hmat_multiply(const hmat_t A, const hmat_t B, const hmat_mult_opts *opts, void *stream,
                                     hmat_t *C) {
  if (C) *C = nullptr;
  return guard([&] {
    if (!C) fail(HMAT_EINVAL, "NULL argument");
    check_pair(A, B, opts);
    Product pr;
    pr.A = A;
    pr.B = B;
    pr.o = opts;
    pr.s = (cudaStream_t)stream;
    pr.cprec = opts->mode == HMAT_MODE_F64 ? 64 : A->prec;
    pr.run();
    const bool nc = pr.C->stats.not_converged > 0;
    *C = pr.C.release();
    if (nc) fail(HMAT_ENOTCONV, "some far blocks hit max_rank or max_rounds");
  });
}
