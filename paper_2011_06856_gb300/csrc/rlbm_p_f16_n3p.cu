// Two-sites-per-lane step kernel instances: FP16 storage, FP32 accumulation, Landau frame refined in double-float where T^ab is near-degenerate, N = 3, plain loads.
#include "rlbm_pair.cuh"
namespace rlbmk {
cudaError_t launch_pair_f16_n3p(int PP, bool two_d, dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                   const KernelArgs &a)
{
    return launch_pair_nb<__half, 3, false>(PP, two_d, grid, block, smem, st, a);
}
} // namespace rlbmk
