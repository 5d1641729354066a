// Two-sites-per-lane step kernel, float storage, FP32 arithmetic.
#include "rlbm_pair.cuh"
namespace rlbmk {
cudaError_t launch_pair_f32(int N, int PP, bool two_d, bool bulk, dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, const KernelArgs &a)
{
    return launch_pair_t<float>(N, PP, two_d, bulk, grid, block, smem, st, a);
}
cudaError_t launch_pair_groups_f32(int N, int PP, bool two_d, dim3 grid, dim3 block, size_t smem,
                                   cudaStream_t st, const KernelArgs &a)
{
    return launch_pair_groups(N, PP, two_d, grid, block, smem, st, a);
}
} // namespace rlbmk
