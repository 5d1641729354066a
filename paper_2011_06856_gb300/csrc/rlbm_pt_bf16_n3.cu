// Tile-staged two-sites-per-lane step kernel instances: BF16 storage, FP32 accumulation, double-float Landau frame, N = 3.
#include "rlbm_pair_tma.cuh"
namespace rlbmk {
cudaError_t launch_pair_tma_bf16_n3(int PP, bool two_d, dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                  const PairTmaArgs &ta)
{
    return launch_pair_tma_n<__nv_bfloat16, 3>(PP, two_d, grid, block, smem, st, ta);
}
} // namespace rlbmk
