// Tile-staged two-sites-per-lane step kernel instances: FP16 storage, FP32 accumulation, double-float Landau frame, N = 2.
#include "rlbm_pair_tma.cuh"
namespace rlbmk {
cudaError_t launch_pair_tma_f16_n2(int PP, bool two_d, dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                  const PairTmaArgs &ta)
{
    return launch_pair_tma_n<__half, 2>(PP, two_d, grid, block, smem, st, ta);
}
} // namespace rlbmk
