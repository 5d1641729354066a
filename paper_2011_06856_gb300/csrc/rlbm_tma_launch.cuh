// Template dispatch for the persistent TMA-staged step kernel; included once
// per storage type by the rlbm_t_*.cu units.
#pragma once
#include "rlbm_tma.cuh"

namespace rlbmk {

template <class St, class R, class LR, int N, int P>
static cudaError_t tma_np(bool two_d, bool full, int grid, dim3 block, size_t smem, cudaStream_t st,
                          const TmaArgs &a, int *blocks_per_sm)
{
    void (*k)(const TmaArgs) =
        full ? (two_d ? rlbm_step_tma<St, R, LR, N, P, true, true>
                      : rlbm_step_tma<St, R, LR, N, P, false, true>)
             : (two_d ? rlbm_step_tma<St, R, LR, N, P, true, false>
                      : rlbm_step_tma<St, R, LR, N, P, false, false>);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (blocks_per_sm) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k,
                                                          (int)(block.x * block.y), smem);
        if (e != cudaSuccess) return e;
        if (grid <= 0) return cudaSuccess; // occupancy query only
    }
    k<<<grid, block, smem, st>>>(a);
    return cudaGetLastError();
}

template <class St, class R, class LR, int N>
static cudaError_t tma_n(int P, bool two_d, bool full, int grid, dim3 block, size_t smem,
                         cudaStream_t st, const TmaArgs &a, int *bps)
{
    switch (P) {
    case 8: return tma_np<St, R, LR, N, 8>(two_d, full, grid, block, smem, st, a, bps);
    case 12: return tma_np<St, R, LR, N, 12>(two_d, full, grid, block, smem, st, a, bps);
    case 16: return tma_np<St, R, LR, N, 16>(two_d, full, grid, block, smem, st, a, bps);
    case 24: return tma_np<St, R, LR, N, 24>(two_d, full, grid, block, smem, st, a, bps);
    case 32: return tma_np<St, R, LR, N, 32>(two_d, full, grid, block, smem, st, a, bps);
    case 48: return tma_np<St, R, LR, N, 48>(two_d, full, grid, block, smem, st, a, bps);
    case 64: return tma_np<St, R, LR, N, 64>(two_d, full, grid, block, smem, st, a, bps);
    default: return cudaErrorInvalidValue;
    }
}

template <class St, class R, class LR>
static cudaError_t tma_t(int N, int P, bool two_d, bool full, int grid, dim3 block, size_t smem,
                         cudaStream_t st, const TmaArgs &a, int *bps)
{
    switch (N) {
    case 2: return tma_n<St, R, LR, 2>(P, two_d, full, grid, block, smem, st, a, bps);
    case 3: return tma_n<St, R, LR, 3>(P, two_d, full, grid, block, smem, st, a, bps);
    default: return cudaErrorInvalidValue;
    }
}

} // namespace rlbmk
