// FP32-storage step kernels, N = 3, with the double-float per-site part once
// per site (a unit of its own so that the build compiles it in parallel).
#include "rlbm_launch.cuh"
namespace rlbmk {
cudaError_t launch_f32_dd_n3(int P, bool two_d, bool full, dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              const KernelArgs &a)
{
    return launch_dd_n<3>(P, two_d, full, grid, block, smem, st, a);
}
} // namespace rlbmk
