// FP32 state and arithmetic, memory variables stored as bfloat16.
#include "fw_launch.cuh"

namespace fwgb {
cudaError_t sweeps_bf16(const fw_medium *m, cudaStream_t s, int which)
{
    return launch_sweeps<float, float, __nv_bfloat16>(m, s, which);
}
bool vel_maps_bf16(EncodeTiledFn encode, fw_medium *m) { return build_vel_maps_t<float, float, __nv_bfloat16>(encode, m); }
}  // namespace fwgb
