// tcw_persist_f16.cu -- group-kernel variants for fp16 maps.
#include "tcw_persist.cuh"

namespace tcw {

cudaError_t launch_group_f16(const GroupParams& p, bool record, int grid, cudaStream_t st) {
  return launch_group_r<__half, false>(p, record, grid, st);
}

cudaError_t prepare_group_f16(int n_det, int lanes) { return prepare_r<__half, false>(n_det, lanes); }

}  // namespace tcw
