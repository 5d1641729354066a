// Persistent TMA-staged step kernel, f16 storage.
#include "rlbm_tma_launch.cuh"
namespace rlbmk {
cudaError_t launch_tma_f16(int N, int P, bool two_d, bool full, bool site_fp64, int grid, dim3 block,
                           size_t smem, cudaStream_t st, const TmaArgs &a, int *bps)
{
    (void)site_fp64;
    return tma_t<__half, float, float>(N, P, two_d, full, grid, block, smem, st, a, bps);
}
} // namespace rlbmk
