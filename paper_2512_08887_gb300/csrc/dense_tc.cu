// Dense stage-2 apply on the tensor cores (placeholder until the tcgen05 kernel lands).
#include "common.cuh"

namespace fbst {

int build_dense_tc_operand(fbst_plan_s*, cudaStream_t) { return FBST_ERR_UNSUPPORTED; }

int launch_stage2_dense_tc(const fbst_plan_s*, const float2*, float2*, int, cudaStream_t) {
  return FBST_ERR_UNSUPPORTED;
}

}  // namespace fbst
