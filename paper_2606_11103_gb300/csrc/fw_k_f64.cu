// FP64 state and arithmetic: the verification build of the same kernels.
#include "fw_launch.cuh"

namespace fwgb {
cudaError_t sweeps_f64(const fw_medium *m, cudaStream_t s, int which) { return launch_sweeps<double, double, double>(m, s, which); }
cudaError_t io_f64(const fw_medium *m, int j, cudaStream_t s) { return launch_io<double, double>(m, j, s); }
cudaError_t image_step_f64(const fw_medium *m, const StepImages &im, const int *zero, int it, cudaStream_t s)
{
    return launch_image_step<double, double>(m, im, zero, it, s);
}
}  // namespace fwgb
