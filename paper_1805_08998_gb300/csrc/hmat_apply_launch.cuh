// hmat_apply_launch.cuh -- launch helpers of the application and panel kernels, instantiated per
// element type and direction (hmat_apply_f32.cu / hmat_apply_f32_trans.cu, hmat_apply_f64.cu /
// hmat_apply_f64_trans.cu) so that the four translation units compile in parallel.
#pragma once
#include "hmat_apply.cuh"

namespace hm {
namespace apply_detail {

constexpr int PANEL_P = 16;

template <typename T, int P, bool TRANS, bool GSTAGE, int RB>
static cudaError_t launch_one(const ApplyArgs &a, size_t smem, cudaStream_t s) {
  cudaError_t e = raise_smem_limit(k_apply<T, P, TRANS, GSTAGE, RB>, smem);
  if (e != cudaSuccess) return e;
  const int K = (RB == 0 && !GSTAGE && a.split > 1) ? a.split : 1;
  ApplyArgs b = a;
  b.split = K;
  k_apply<T, P, TRANS, GSTAGE, RB><<<(unsigned)a.count * K, AT, smem, s>>>(b);
  return cudaGetLastError();
}

// register blocking of the launch (rows per lane; 0: shared atomics), from its largest output
inline int rows_per_lane(int dmax) { return dmax <= 64 ? 2 : dmax <= 128 ? 4 : 0; }

template <typename T, int P, bool TRANS>
static cudaError_t launch_rb(const ApplyArgs &a, size_t smem, cudaStream_t s) {
  if (a.gstage) return launch_one<T, P, TRANS, true, 0>(a, smem, s);
  switch (rows_per_lane(a.smem_out)) {
    case 2: return launch_one<T, P, TRANS, false, 2>(a, smem, s);
    case 4: return launch_one<T, P, TRANS, false, 4>(a, smem, s);
    default: return launch_one<T, P, TRANS, false, 0>(a, smem, s);
  }
}

inline size_t smem_bytes(size_t es, int P, const ApplyArgs &a) {
  const size_t SP = apply_row_stride(P);
  const size_t cw = (size_t)NWARP * a.smem_cw * SP * es;
  return a.gstage ? cw : (size_t)(a.smem_in + a.smem_out + a.smem_rho) * SP * es + cw;
}

// one direction of the application: TRANS = false for S X (a3), true for S^T X (a6)
template <typename T, bool TRANS>
static cudaError_t launch_apply_dir(int P, const ApplyArgs &a, cudaStream_t s) {
  const size_t smem = smem_bytes(sizeof(T), P, a);
  return P == 8 ? launch_rb<T, 8, TRANS>(a, smem, s) : launch_rb<T, 16, TRANS>(a, smem, s);
}

template <typename T>
static cudaError_t launch_panels_t(const PanelArgs &a, bool leaf_kind, cudaStream_t s) {
  constexpr int P = PANEL_P;
  constexpr size_t SP = panel_row_stride(P);
  const size_t es = sizeof(T);
  cudaError_t e;
  if (leaf_kind) {
    const size_t smem = (size_t)NWARP * (a.smem_in + a.smem_out) * SP * es;
    if ((e = raise_smem_limit(k_panel_leaf<T, P>, smem)))
      return e;
    k_panel_leaf<T, P><<<(a.count + NWARP - 1) / NWARP, AT, smem, s>>>(a);
    return cudaGetLastError();
  }
  const size_t cw = (size_t)NWARP * a.smem_cw * SP * es;
  const size_t smem = a.gstage ? cw : (size_t)(a.smem_in + a.smem_out) * SP * es + cw;
  if (a.gstage) {
    if ((e = raise_smem_limit(k_panel<T, P, true>, smem)))
      return e;
    k_panel<T, P, true><<<std::min(a.count, PANEL_GSTAGE_SLOTS), AT, smem, s>>>(a);
  } else if (a.smem_in <= 128 && a.smem_out <= 128) {  // small H-blocks: four warps per panel
    const size_t smem4 = (size_t)(a.smem_in + a.smem_out) * SP * es + (size_t)4 * a.smem_cw * SP * es;
    if ((e = raise_smem_limit(k_panel<T, P, false, 4>, smem4)))
      return e;
    k_panel<T, P, false, 4><<<a.count, 128, smem4, s>>>(a);
  } else if (a.smem_in > 512 && (size_t)(a.smem_in + a.smem_out) * SP * es + (size_t)16 * a.smem_cw * SP * es <=
                                      (size_t)max_dynamic_smem()) {
    // H-blocks of more than 512 rows: one block fits an SM, so it runs sixteen warps
    const size_t smem16 = (size_t)(a.smem_in + a.smem_out) * SP * es + (size_t)16 * a.smem_cw * SP * es;
    if ((e = raise_smem_limit(k_panel<T, P, false, 16>, smem16)))
      return e;
    k_panel<T, P, false, 16><<<a.count, 512, smem16, s>>>(a);
  } else {
    if ((e = raise_smem_limit(k_panel<T, P, false>, smem)))
      return e;
    k_panel<T, P, false><<<a.count, AT, smem, s>>>(a);
  }
  return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_hmatvec_t(const LeafDev *leaves, int nleaf, const T *data, const T *X, T *Y, int cw_rows,
                                    cudaStream_t s) {
  constexpr int P = PANEL_P;
  const size_t smem = (size_t)NWARP * cw_rows * panel_row_stride(P) * sizeof(T);
  cudaError_t e = raise_smem_limit(k_hmatvec<T, P>, smem);
  if (e != cudaSuccess) return e;
  const int grid = std::max(1, std::min((nleaf + NWARP - 1) / NWARP, 152 * 16));
  k_hmatvec<T, P><<<grid, AT, smem, s>>>(leaves, nleaf, data, X, Y, cw_rows);
  return cudaGetLastError();
}

}  // namespace apply_detail
}  // namespace hm
