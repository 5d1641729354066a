// Per-tile step kernel for quadrature orders N = 4, 5: FP32 storage and per-population
// arithmetic, FP64 per-site arithmetic.
#include "rlbm_launch.cuh"
namespace rlbmk {
cudaError_t launch_f32_n45(int mode, int N, int P, bool two_d, bool full, dim3 grid, dim3 block,
                           size_t smem, cudaStream_t st, const KernelArgs &a)
{
    return launch_t_hi<float, float, double>(mode, N, P, two_d, full, grid, block, smem, st, a);
}
} // namespace rlbmk
