// Batched persistent kernel instances (FP64 and FP32 storage, N = 2, 3; the
// per-site part in FP64 for FP64 storage, in double-float for FP32).
#include "rlbm_batch.cuh"

namespace rlbmk {

template <class St, class R, class LR, int N>
static cudaError_t launch_b(const BatchArgs &b, int grid, cudaStream_t st, int *bps)
{
    void (*k)(const BatchArgs) = rlbm_batch_kernel<St, R, LR, N>;
    const dim3 block(32, kBatchWarps);
    if (bps) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k, 32 * kBatchWarps, 0);
        if (e != cudaSuccess || grid <= 0) return e;
    }
    // cooperative: every CTA is resident, so the grid barrier cannot deadlock
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, b);
}

cudaError_t launch_batch(int prec, int N, const BatchArgs &b, int grid, cudaStream_t st, int *bps)
{
    if (prec == 0) {
        if (N == 2) return launch_b<double, double, double, 2>(b, grid, st, bps);
        if (N == 3) return launch_b<double, double, double, 3>(b, grid, st, bps);
    } else if (prec == 1) {
        // FP32 storage: FP32 per-population arithmetic, double-float per-site part
        if (N == 2) return launch_b<float, float, float, 2>(b, grid, st, bps);
        if (N == 3) return launch_b<float, float, float, 3>(b, grid, st, bps);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_batch_advance(const KernelArgs *probs, int n, int nsteps, cudaStream_t st)
{
    batch_advance_kernel<<<(n + 255) / 256, 256, 0, st>>>(probs, n, nsteps);
    return cudaGetLastError();
}

} // namespace rlbmk
