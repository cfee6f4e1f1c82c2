// hmat_near_tc.cu -- a8 in FP32 on the tensor cores: every near leaf of C evaluated as S(b)
// applied to the identity (Algorithm 4, evaluate()), i.e. the sum of its low-rank terms L R^T
// (Algorithm 3's restriction, Lemma 5.3) and of its products of two dense leaves.
//
// One thread block of four warps per near leaf, in output tiles of 64 x 64 (M = N = 64). Each
// contribution (a term, K = its rank; a leaf pair, K = the inner leaf's size) is staged in chunks
// of 32 along K into shared memory, split into a TF32 part and its FP32 remainder, and multiplied
// by three kind::tf32 MMAs per K = 8 (hi hi, hi lo, lo hi) into an FP32 accumulator in TMEM.
// Groups of up to FOLD_GROUP consecutive contributions accumulate in one TMEM accumulator; when a
// group's last chunk is done its tile is read back (tcgen05.ld) and added to the block with a
// compensated (Neumaier) sum, so the error grows with the size of a group (a few roundings) and
// not with the number of contributions. Two shared-memory stages and two TMEM accumulators let
// the staging of the next chunk and the read-back of the last group run while the tensor cores
// work.
#include "hmat_internal.h"
#include "hmat_tc.cuh"

namespace hm {
namespace {

constexpr int NTC = 128;                  // threads per block: four warps
constexpr int TM = 64;                    // tile rows (MMA M) and columns (MMA N)
constexpr int KC = 32;                    // K per staged chunk
constexpr int TILE_ELEMS = TM * KC;       // one operand part (A or B, TF32 part or remainder)
constexpr int STAGE_ELEMS = 4 * TILE_ELEMS;
constexpr uint32_t LBO = 128;             // bytes between core matrices along K
constexpr uint32_t SBO = (KC / 4) * 128;  // bytes between groups of 8 rows
constexpr uint32_t TMEM_COLS = 2 * TM;    // two accumulators of 64 columns
constexpr int WAIT_POLLS = 1 << 18;       // bounded mbarrier waits: about 1 s on GB300
constexpr uint32_t IDESC = tc::idesc_tf32(TM, TM);
constexpr int FOLD_GROUP = 4;             // contributions summed in TMEM between two folds
static_assert(NTC == 128 && KC == 32 && TM == 64, "stage_chunk's thread-to-element map assumes these sizes");

// one contribution restricted to the output tile: A(i, k) = A[i + k a_k] (i < mt),
// B(j, k) = B[j b_j + k b_k] (j < nt), k < K
struct Contrib {
  const float *A, *B;
  int64_t a_k, b_j, b_k;
  int K;
};

// walks the contributions of one output tile in a fixed order, the same in every thread: the terms
// created at the target's block and at each of its ancestors, then its pairs of dense leaves
struct Walk {
  const TargetDev &t;
  const int2 *blk_terms;
  const TermDev *terms;
  const PairDev *pairs;
  const BlockDev *blocks;
  const LeafDev *leafA, *leafB;
  const float *dataA, *dataB;
  int i0, j0;
  int blk, ti, te, pi;

  __device__ void start() {
    blk = t.blk;
    const int2 r = blk_terms[blk];
    ti = r.x;
    te = r.y;
    pi = t.pair_lo;
  }
  __device__ bool next(Contrib &c) {
    while (blk >= 0) {
      if (ti < te) {
        const TermDev tm = terms[ti++];
        if (tm.rank <= 0) continue;
        c.A = (const float *)tm.L + (t.row - tm.row0) + i0;
        c.a_k = tm.ldL;
        c.B = (const float *)tm.R + (t.col - tm.col0) + j0;
        c.b_j = 1;
        c.b_k = tm.ldR;
        c.K = tm.rank;
        return true;
      }
      blk = blocks[blk].parent;
      if (blk >= 0) {
        const int2 r = blk_terms[blk];
        ti = r.x;
        te = r.y;
      }
    }
    while (pi < t.pair_hi) {
      const PairDev pr = pairs[pi++];
      const LeafDev la = leafA[blocks[pr.blkA].leaf_lo], lb = leafB[blocks[pr.blkB].leaf_lo];
      if (la.n <= 0) continue;
      c.A = dataA + la.off_u + i0;  // m x rho, ld m
      c.a_k = la.m;
      c.B = dataB + lb.off_u + (int64_t)j0 * lb.m;  // rho x n, ld rho: B(j, k) = DB[k + j rho]
      c.b_j = lb.m;
      c.b_k = 1;
      c.K = la.n;
      return true;
    }
    return false;
  }
};

// chunk [k0, k0 + KC) of a contribution into one stage. Element e of each part sits at byte 4 e,
// e = g (8 KC) + hk 32 + r 4 + kq for row 8 g + r and k = 4 hk + kq (the core-matrix layout).
// With e = tid + 128 (2 g + half), thread tid always takes rows r + 8 g (g = 0..7) at
// k = kt + 16 half, where r = (tid / 4) % 8 and kt = 4 (tid / 32) + tid % 4: its addresses are
// fixed offsets from two pointers. Zero outside the tile and for k >= K; the columns at and
// beyond the MMAs' last K = 8 step are not written (no MMA reads them).
__device__ __forceinline__ void stage_chunk(float *st, const Contrib &c, int k0, int mt, int nt) {
  const int tid = threadIdx.x;
  const int r = (tid >> 2) & 7, kt = 4 * (tid >> 5) + (tid & 3);
  const int kc = min(KC, c.K - k0);
  const float *pa = c.A + r + (int64_t)(k0 + kt) * c.a_k;
  const float *pb = c.B + r * c.b_j + (int64_t)(k0 + kt) * c.b_k;
  const int64_t bg = 8 * c.b_j;
#pragma unroll
  for (int half = 0; half < 2; half++) {
    if (half == 1 && kc <= 16) break;  // k >= 16 is beyond the last K = 8 step
    const bool kok = kt + 16 * half < kc;
    const float *qa = pa + (half ? 16 * c.a_k : 0), *qb = pb + (half ? 16 * c.b_k : 0);
    float a[8], b[8];
#pragma unroll
    for (int g = 0; g < 8; g++) {
      a[g] = (kok && 8 * g + r < mt) ? __ldg(qa + 8 * g) : 0.f;
      b[g] = (kok && 8 * g + r < nt) ? __ldg(qb + g * bg) : 0.f;
    }
#pragma unroll
    for (int g = 0; g < 8; g++) {
      const int e = tid + 128 * (2 * g + half);
      const float ah = tc::tf32_hi(a[g]), bh = tc::tf32_hi(b[g]);
      st[e] = ah;
      st[TILE_ELEMS + e] = a[g] - ah;
      st[2 * TILE_ELEMS + e] = bh;
      st[3 * TILE_ELEMS + e] = b[g] - bh;
    }
  }
}

__global__ void __launch_bounds__(NTC, 2)
    k_near_tc(const TargetDev *tg, const int2 *blk_terms, const TermDev *terms, const PairDev *pairs,
              const BlockDev *blocks, const LeafDev *leafA, const LeafDev *leafB, const float *dataA,
              const float *dataB, const LeafDev *leafC, float *dataC, int *err) {
  extern __shared__ __align__(1024) float stages[];  // 2 x STAGE_ELEMS
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tslot;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const TargetDev t = tg[blockIdx.x];
  float *C = dataC + leafC[t.leaf].off_u;

  if (threadIdx.x == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
  }
  tc::fence_smem_to_async();
  if (warp == 0) tc::tmem_alloc(&tslot, TMEM_COLS);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tslot;

  // once one block's wait has given up, the blocks that start later skip their work (one decision
  // for the whole block: its threads may read the flag at different times)
  bool failed = __syncthreads_or(*(volatile int *)err != 0) != 0;
  uint32_t u = 0;  // chunks issued so far (all tiles): stage u & 1, mbarrier phase (u >> 1) & 1
  Walk wk{t, blk_terms, terms, pairs, blocks, leafA, leafB, dataA, dataB, 0, 0, 0, 0, 0, 0};
  const int row = 16 * warp + lane;  // the tile row this thread reads back (lanes < 16)
  for (int i0 = 0; i0 < t.m && !failed; i0 += TM)
    for (int j0 = 0; j0 < t.n && !failed; j0 += TM) {
      const int mt = min(TM, t.m - i0), nt = min(TM, t.n - j0);
      float acc[TM], cmp[TM];
#pragma unroll
      for (int j = 0; j < TM; j++) {
        acc[j] = 0.f;
        cmp[j] = 0.f;
      }
      wk.i0 = i0;
      wk.j0 = j0;
      wk.start();
      Contrib cur;
      bool more = wk.next(cur);
      int h = 0;               // chunk of the current contribution
      int cg = 0;              // contributions of the current group done
      uint32_t gi = 0;         // groups begun in this tile: accumulator gi & 1
      bool have_prev = false;  // a chunk in flight from the previous step
      bool prev_last = false;  // ... that ends its group
      uint32_t prev_acc = 0;
      while (more || have_prev) {
        const uint32_t s = u & 1;
        if (more) {
          // stage s was last read by the chunk two steps back, whose completion the previous step
          // waited for
          stage_chunk(stages + s * STAGE_ELEMS, cur, h * KC, mt, nt);
          tc::fence_smem_to_async();
        }
        tc::fence_before_sync();
        __syncthreads();  // staging complete; the previous step's TMEM reads complete
        tc::fence_after_sync();
        if (more && threadIdx.x == 0) {
          const float *st = stages + s * STAGE_ELEMS;
          const uint32_t a_hi = tc::smem_addr(st), a_lo = tc::smem_addr(st + TILE_ELEMS);
          const uint32_t b_hi = tc::smem_addr(st + 2 * TILE_ELEMS), b_lo = tc::smem_addr(st + 3 * TILE_ELEMS);
          const uint32_t d = tmem + (gi & 1) * TM;
          const int kc = min(KC, cur.K - h * KC);
          for (int kk = 0; kk * 8 < kc; kk++) {
            const uint32_t off = kk * 2 * LBO;  // two core matrices along K per K = 8
            const uint32_t first = (cg == 0 && h == 0 && kk == 0) ? 0u : 1u;  // a group starts from zero
            tc::mma_tf32(d, tc::desc_kmajor(a_lo + off, LBO, SBO), tc::desc_kmajor(b_hi + off, LBO, SBO), IDESC, first);
            tc::mma_tf32(d, tc::desc_kmajor(a_hi + off, LBO, SBO), tc::desc_kmajor(b_lo + off, LBO, SBO), IDESC, 1);
            tc::mma_tf32(d, tc::desc_kmajor(a_hi + off, LBO, SBO), tc::desc_kmajor(b_hi + off, LBO, SBO), IDESC, 1);
          }
          tc::commit(&mbar[s]);
        }
        if (have_prev) {
          const uint32_t sp = (u - 1) & 1, par = ((u - 1) >> 1) & 1;
          const bool ok = tc::mbar_wait(&mbar[sp], par, WAIT_POLLS);
          if (__syncthreads_or(!ok)) {
            failed = true;
            break;
          }
          tc::fence_after_sync();
          if (prev_last) {
            const uint32_t base = tmem + prev_acc * TM + ((uint32_t)(warp * 32) << 16);
#pragma unroll
            for (int q = 0; q < TM / 16; q++) {
              float v[16];
              tc::tmem_ld16(base + q * 16, v);
#pragma unroll
              for (int c = 0; c < 16; c++) {
                const float x = v[c], s0 = acc[q * 16 + c], s1 = s0 + x;
                cmp[q * 16 + c] += fabsf(s0) >= fabsf(x) ? (s0 - s1) + x : (x - s1) + s0;
                acc[q * 16 + c] = s1;
              }
            }
          }
        }
        have_prev = more;
        if (more) {
          prev_acc = gi & 1;
          u++;
          h++;
          prev_last = false;
          if (h * KC >= cur.K) {  // the contribution is done
            h = 0;
            more = wk.next(cur);
            if (++cg == FOLD_GROUP || !more) {  // ... and so is its group
              prev_last = true;
              cg = 0;
              gi++;
            }
          }
        }
      }
      if (!failed && lane < 16 && row < mt) {
#pragma unroll
        for (int j = 0; j < TM; j++)
          if (j < nt) C[(i0 + row) + (int64_t)(j0 + j) * t.m] = acc[j] + cmp[j];
      }
    }
  // A block whose wait gave up may still have MMAs in flight when it frees its TMEM below; their
  // results are lost with the product, which then reports HMAT_ETIMEOUT and returns no output.
  if (failed && threadIdx.x == 0) atomicOr(err, 1);  // (already set when the block skipped its work)
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_free(tmem, TMEM_COLS);
}

// The failure path of the waits above on its own: TMEM held, a wait on an mbarrier that nothing
// arrives on, then the same exit (TMEM freed). *gave_up = 1 when the wait gave up.
__global__ void __launch_bounds__(NTC) k_tc_wait_check(int polls, int *gave_up) {
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tslot;
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) tc::mbar_init(&mbar, 1);
  tc::fence_smem_to_async();
  if (warp == 0) tc::tmem_alloc(&tslot, 32);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = tslot;
  const bool ok = tc::mbar_wait(&mbar, 0, polls);
  const bool failed = __syncthreads_or(!ok) != 0;
  if (threadIdx.x == 0) *gave_up = failed ? 1 : 0;
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_free(tmem, 32);
}

}  // namespace

cudaError_t launch_tc_wait_check(int polls, int *gave_up, cudaStream_t s) {
  k_tc_wait_check<<<1, NTC, 0, s>>>(polls, gave_up);
  return cudaGetLastError();
}

cudaError_t launch_near_tc(const TargetDev *tg, int ntg, const int2 *blk_terms, const TermDev *terms,
                           const PairDev *pairs, const BlockDev *blocks, const LeafDev *leafA, const LeafDev *leafB,
                           const float *dataA, const float *dataB, const LeafDev *leafC, float *dataC, int *err,
                           cudaStream_t s) {
  if (ntg == 0) return cudaSuccess;
  const size_t smem = sizeof(float) * 2 * STAGE_ELEMS;
  cudaError_t e = raise_smem_limit(k_near_tc, smem);
  if (e != cudaSuccess) return e;
  k_near_tc<<<ntg, NTC, smem, s>>>(tg, blk_terms, terms, pairs, blocks, leafA, leafB, dataA, dataB, leafC, dataC, err);
  return cudaGetLastError();
}

}  // namespace hm
