// hmat_apply_f64.cu -- the application and panel kernels instantiated for double elements.
#include "hmat_apply_launch.cuh"

namespace hm {

// the transposed direction is instantiated in hmat_apply_f64_trans.cu
cudaError_t launch_apply_f64_trans(int P, const ApplyArgs &a, cudaStream_t s);

cudaError_t launch_apply_f64(int P, bool trans, const ApplyArgs &a, cudaStream_t s) {
  return trans ? launch_apply_f64_trans(P, a, s) : apply_detail::launch_apply_dir<double, false>(P, a, s);
}

cudaError_t launch_panels_f64(const PanelArgs &a, bool leaf_kind, cudaStream_t s) {
  return apply_detail::launch_panels_t<double>(a, leaf_kind, s);
}

cudaError_t launch_hmatvec(const LeafDev *leaves, int nleaf, const double *data, const double *X, double *Y,
                           int cw_rows, cudaStream_t s) {
  return apply_detail::launch_hmatvec_t<double>(leaves, nleaf, data, X, Y, cw_rows, s);
}

}  // namespace hm
