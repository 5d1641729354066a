// Persistent TMA-staged step kernel, f32 storage (FP64 per-site part).
#include "rlbm_tma_launch.cuh"
namespace rlbmk {
cudaError_t launch_tma_f32(int N, int P, bool two_d, bool full, bool site_fp64, int grid, dim3 block,
                           size_t smem, cudaStream_t st, const TmaArgs &a, int *bps)
{
    // FP64 per-site arithmetic only (site_fp64_for)
    if (!site_fp64) return cudaErrorInvalidValue;
    return tma_t<float, float, double>(N, P, two_d, full, grid, block, smem, st, a, bps);
}
} // namespace rlbmk
