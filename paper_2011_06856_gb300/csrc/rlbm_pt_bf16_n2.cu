// Tile-staged two-sites-per-lane step kernel instances: BF16 storage, FP32 accumulation, Landau frame refined in double-float where T^ab is near-degenerate, N = 2.
#include "rlbm_pair_tma.cuh"
namespace rlbmk {
cudaError_t launch_pair_tma_bf16_n2(int PP, bool two_d, dim3 block, size_t smem, cudaStream_t st,
                                  const PairTmaArgs &ta, int *bps)
{
    return launch_pair_tma_n<__nv_bfloat16, 2>(PP, two_d, block, smem, st, ta, bps);
}
} // namespace rlbmk
