// Per-tile step kernel with a quantum statistic (Fermi-Dirac or Bose-Einstein), FP64 storage.
#include "rlbm_launch.cuh"
namespace rlbmk {
cudaError_t launch_quant_f64(int mode, int N, int P, bool two_d, bool full, dim3 grid, dim3 block,
                             size_t smem, cudaStream_t st, const KernelArgs &a)
{
    return launch_tq<double, double, double>(mode, N, P, two_d, full, grid, block, smem, st, a);
}
} // namespace rlbmk
