// FP32 storage and per-population arithmetic; the per-site part (moment
// folding, Landau frame, equilibrium coefficients) in FP32 or FP64.
#include "rlbm_launch.cuh"
namespace rlbmk {
cudaError_t launch_f32(int mode, int N, int P, bool two_d, bool full, bool site_fp64, dim3 grid, dim3 block,
                       size_t smem, cudaStream_t st, const KernelArgs &a)
{
    if (N >= 4) { // FP64 per-site arithmetic only
        if (!site_fp64) return cudaErrorInvalidValue;
        return launch_f32_n45(mode, N, P, two_d, full, grid, block, smem, st, a);
    }
    if (site_fp64)
        return launch_t<float, float, double>(mode, N, P, two_d, full, grid, block, smem, st, a);
    return launch_t<float, float, float>(mode, N, P, two_d, full, grid, block, smem, st, a);
}
cudaError_t launch_lattice_f32(bool two_d, dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                               const KernelArgs &a)
{
    return launch_lattice_t<float, float, float>(two_d, grid, block, smem, st, a);
}
} // namespace rlbmk
