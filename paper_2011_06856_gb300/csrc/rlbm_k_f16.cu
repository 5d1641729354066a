// FP16 deviation storage h = f / w - 1/(2 pi), FP32 arithmetic.
#include "rlbm_launch.cuh"
namespace rlbmk {
cudaError_t launch_f16(int mode, int N, int P, bool two_d, bool full, dim3 grid, dim3 block, size_t smem,
                       cudaStream_t st, const KernelArgs &a)
{
    if (N >= 4) return launch_f16_n45(mode, N, P, two_d, full, grid, block, smem, st, a);
    return launch_t<__half, float, float>(mode, N, P, two_d, full, grid, block, smem, st, a);
}
} // namespace rlbmk
