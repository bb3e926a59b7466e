// FP32 state and FP32 memory variables.
#include "fw_launch.cuh"

namespace fwgb {
cudaError_t sweeps_f32(const fw_medium *m, cudaStream_t s, int which) { return launch_sweeps<float, float, float>(m, s, which); }
cudaError_t io_f32(const fw_medium *m, int j, cudaStream_t s) { return launch_io<float, float>(m, j, s); }
cudaError_t image_step_f32(const fw_medium *m, const StepImages &im, const int *zero, int it, cudaStream_t s)
{
    return launch_image_step<float, float>(m, im, zero, it, s);
}
__global__ void k_advance(int *d_it, int n) { *d_it += n; }
bool vel_maps_f32(EncodeTiledFn encode, fw_medium *m) { return build_vel_maps_t<float, float, float>(encode, m); }
}  // namespace fwgb
