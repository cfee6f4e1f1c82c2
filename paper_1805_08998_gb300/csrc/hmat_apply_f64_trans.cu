// hmat_apply_f64_trans.cu -- the application kernel for double elements in the transposed
// direction (W = S^T Q, the projection pass), in a translation unit of its own so that it compiles
// in parallel with the other direction.
#include "hmat_apply_launch.cuh"

namespace hm {

cudaError_t launch_apply_f64_trans(int P, const ApplyArgs &a, cudaStream_t s) {
  return apply_detail::launch_apply_dir<double, true>(P, a, s);
}

}  // namespace hm
