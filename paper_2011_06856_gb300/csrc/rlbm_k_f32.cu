// FP32 storage and per-population arithmetic.  The per-site part (moment
// folding, Landau frame, equilibrium coefficients) needs FP64-class accuracy:
// in FP32 it would bias the conserved moments by about 4e-7 per step
// (site_fp64_for).  Steps with N = 2, 3 carry it in double-float on the FP32
// pipes, once per site (launch_f32_dd); the init and moments passes, and N = 4,
// 5, carry it in FP64.
#include "rlbm_launch.cuh"
namespace rlbmk {
cudaError_t launch_f32(int mode, int N, int P, bool two_d, bool full, bool site_fp64, dim3 grid, dim3 block,
                       size_t smem, cudaStream_t st, const KernelArgs &a)
{
    if (!site_fp64) return cudaErrorInvalidValue; // FP64 per-site arithmetic only
    if (N >= 4) return launch_f32_n45(mode, N, P, two_d, full, grid, block, smem, st, a);
    return launch_t<float, float, double>(mode, N, P, two_d, full, grid, block, smem, st, a);
}
cudaError_t launch_f32_dd(int N, int P, bool two_d, bool full, dim3 grid, dim3 block, size_t smem,
                          cudaStream_t st, const KernelArgs &a)
{
    switch (N) {
    case 2: return launch_f32_dd_n2(P, two_d, full, grid, block, smem, st, a);
    case 3: return launch_f32_dd_n3(P, two_d, full, grid, block, smem, st, a);
    default: return cudaErrorInvalidValue;
    }
}
cudaError_t launch_lattice_f32(bool two_d, dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                               const KernelArgs &a)
{
    return launch_lattice_t<float, float, float>(two_d, grid, block, smem, st, a);
}
} // namespace rlbmk
