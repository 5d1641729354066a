// FP64 storage, FP64 arithmetic throughout.
#include "rlbm_launch.cuh"
namespace rlbmk {
cudaError_t launch_f64(int mode, int N, int P, bool two_d, bool full, dim3 grid, dim3 block, size_t smem,
                       cudaStream_t st, const KernelArgs &a)
{
    if (N >= 4) return launch_f64_n45(mode, N, P, two_d, full, grid, block, smem, st, a);
    return launch_t<double, double, double>(mode, N, P, two_d, full, grid, block, smem, st, a);
}
cudaError_t launch_lattice_f64(bool two_d, dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                               const KernelArgs &a)
{
    return launch_lattice_t<double, double, double>(two_d, grid, block, smem, st, a);
}
} // namespace rlbmk
