// hmat_apply_f32.cu -- the application and panel kernels instantiated for float elements.
#include "hmat_apply_launch.cuh"

namespace hm {

// the transposed direction is instantiated in hmat_apply_f32_trans.cu
cudaError_t launch_apply_f32_trans(int P, const ApplyArgs &a, cudaStream_t s);

cudaError_t launch_apply_f32(int P, bool trans, const ApplyArgs &a, cudaStream_t s) {
  return trans ? launch_apply_f32_trans(P, a, s) : apply_detail::launch_apply_dir<float, false>(P, a, s);
}

cudaError_t launch_panels_f32(const PanelArgs &a, bool leaf_kind, cudaStream_t s) {
  return apply_detail::launch_panels_t<float>(a, leaf_kind, s);
}

}  // namespace hm
