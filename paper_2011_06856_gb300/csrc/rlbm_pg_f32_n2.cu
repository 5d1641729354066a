// Two-sites-per-lane step kernel with several population groups per warp:
// FP32 storage, double-float per-site part, N = 2.
#include "rlbm_pair.cuh"
namespace rlbmk {
cudaError_t launch_pair_groups_f32_n2(int PP, bool two_d, dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                      const KernelArgs &a)
{
    return launch_pair_groups_n<2>(PP, two_d, grid, block, smem, st, a);
}
} // namespace rlbmk
