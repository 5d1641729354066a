// Two-sites-per-lane step kernel instances: FP32 storage, double-float per-site part, N = 2, plain loads.
#include "rlbm_pair.cuh"
namespace rlbmk {
cudaError_t launch_pair_f32_n2p(int PP, bool two_d, dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                   const KernelArgs &a)
{
    return launch_pair_nb<float, 2, false>(PP, two_d, grid, block, smem, st, a);
}
} // namespace rlbmk
