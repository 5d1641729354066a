// Tile-staged two-sites-per-lane step kernel instances: FP32 storage, double-float per-site part, N = 2.
#include "rlbm_pair_tma.cuh"
namespace rlbmk {
cudaError_t launch_pair_tma_f32_n2(int PP, bool two_d, dim3 block, size_t smem, cudaStream_t st,
                                  const PairTmaArgs &ta, int *bps)
{
    return launch_pair_tma_n<float, 2>(PP, two_d, block, smem, st, ta, bps);
}
} // namespace rlbmk
