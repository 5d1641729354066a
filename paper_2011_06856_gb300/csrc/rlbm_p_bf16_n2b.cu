// Two-sites-per-lane step kernel instances: BF16 storage, FP32 accumulation, Landau frame refined in double-float where T^ab is near-degenerate, N = 2, bulk-staged first pass.
#include "rlbm_pair.cuh"
namespace rlbmk {
cudaError_t launch_pair_bf16_n2b(int PP, bool two_d, dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                   const KernelArgs &a)
{
    return launch_pair_nb<__nv_bfloat16, 2, true>(PP, two_d, grid, block, smem, st, a);
}
} // namespace rlbmk
