// tcw_persist_f32.cu -- group-kernel variants for fp32 maps.
#include "tcw_persist.cuh"

namespace tcw {

cudaError_t launch_group_f32(const GroupParams& p, bool record, int grid, cudaStream_t st) {
  return launch_group_r<float, false>(p, record, grid, st);
}

cudaError_t prepare_group_f32(int n_det, int lanes) { return prepare_r<float, false>(n_det, lanes); }

}  // namespace tcw
