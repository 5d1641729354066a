// Tile-staged two-sites-per-lane step kernel instances: FP16 storage, FP32 accumulation, Landau frame refined in double-float where T^ab is near-degenerate, N = 3.
#include "rlbm_pair_tma.cuh"
namespace rlbmk {
cudaError_t launch_pair_tma_f16_n3(int PP, bool two_d, dim3 block, size_t smem, cudaStream_t st,
                                  const PairTmaArgs &ta, int *bps)
{
    return launch_pair_tma_n<__half, 3>(PP, two_d, block, smem, st, ta, bps);
}
} // namespace rlbmk
