// FP32 state and arithmetic, memory variables stored as binary16 in scaled
// units (the scale is folded into the class table).
#include "fw_launch.cuh"

namespace fwgb {
cudaError_t sweeps_f16(const fw_medium *m, cudaStream_t s, int which) { return launch_sweeps<float, float, __half>(m, s, which); }
bool vel_maps_f16(EncodeTiledFn encode, fw_medium *m) { return build_vel_maps_t<float, float, __half>(encode, m); }
}  // namespace fwgb
