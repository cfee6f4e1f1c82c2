// hmat_apply.cu -- dispatch of the application kernel (a3/a6) and of the low-rank product panels
// (a2) to their FP32 / FP64 instantiations; the kernels are in hmat_apply.cuh.
#include "hmat_internal.h"

namespace hm {

cudaError_t launch_apply_f32(int P, bool trans, const ApplyArgs &a, cudaStream_t s);
cudaError_t launch_apply_f64(int P, bool trans, const ApplyArgs &a, cudaStream_t s);
cudaError_t launch_panels_f32(const PanelArgs &a, bool leaf_kind, cudaStream_t s);
cudaError_t launch_panels_f64(const PanelArgs &a, bool leaf_kind, cudaStream_t s);

int apply_panel_width(int p) { return p <= 8 ? 8 : 16; }
int apply_rows_per_lane(int dmax) { return dmax <= 64 ? 2 : dmax <= 128 ? 4 : 0; }
int panel_width() { return 16; }

size_t apply_smem_bytes(int prec, int P, const ApplyArgs &a) {
  const size_t es = prec == 64 ? 8 : 4;
  const size_t SP = apply_row_stride(P);
  const size_t cw = (size_t)8 * a.smem_cw * SP * es;
  return a.gstage ? cw : (size_t)(a.smem_in + a.smem_out + a.smem_rho) * SP * es + cw;
}

cudaError_t launch_apply(int prec, bool trans, const ApplyArgs &a, cudaStream_t s) {
  if (a.count == 0) return cudaSuccess;
  const int P = apply_panel_width(a.p);
  return prec == 64 ? launch_apply_f64(P, trans, a, s) : launch_apply_f32(P, trans, a, s);
}

cudaError_t launch_panels(int prec, const PanelArgs &a, bool leaf_kind, cudaStream_t s) {
  if (a.count == 0) return cudaSuccess;
  return prec == 64 ? launch_panels_f64(a, leaf_kind, s) : launch_panels_f32(a, leaf_kind, s);
}

}  // namespace hm
