// tcw_persist_pw.cu -- group-kernel variants for fp32 windows built by the producer (number count, two-bin lookups).
#include "tcw_persist.cuh"

namespace tcw {

cudaError_t launch_group_pw(const GroupParams& p, bool record, int grid, cudaStream_t st) {
  return launch_group_r<float, true>(p, record, grid, st);
}

cudaError_t prepare_group_pw(int n_det, int lanes) { return prepare_r<float, true>(n_det, lanes); }

}  // namespace tcw
