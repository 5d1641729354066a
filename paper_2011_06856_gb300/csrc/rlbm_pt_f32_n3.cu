// Tile-staged two-sites-per-lane step kernel instances: FP32 storage, double-float per-site part, N = 3.
#include "rlbm_pair_tma.cuh"
namespace rlbmk {
cudaError_t launch_pair_tma_f32_n3(int PP, bool two_d, dim3 block, size_t smem, cudaStream_t st,
                                  const PairTmaArgs &ta, int *bps)
{
    return launch_pair_tma_n<float, 3>(PP, two_d, block, smem, st, ta, bps);
}
} // namespace rlbmk
