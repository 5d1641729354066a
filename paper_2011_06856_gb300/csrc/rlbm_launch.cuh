// Template dispatch from runtime (mode, N, P, two_d) to one kernel instance.
// Included once per storage type by the rlbm_k_*.cu units so that they
// compile in parallel.
#pragma once
#include "rlbm_device.cuh"

namespace rlbmk {

// QB: 0, or MODE_Q for the quantum statistics.
template <class St, class R, class LR, int N, int P, int QB = 0>
static cudaError_t launch_np(int mode, bool two_d, bool full, dim3 grid, dim3 block, size_t smem,
                            cudaStream_t st, const KernelArgs &a)
{
    void (*k)(const KernelArgs);
    if (mode == MODE_STEP) {
        if (full)
            k = two_d ? rlbm_kernel<St, R, LR, N, P, true, MODE_STEP | QB, true>
                      : rlbm_kernel<St, R, LR, N, P, false, MODE_STEP | QB, true>;
        else
            k = two_d ? rlbm_kernel<St, R, LR, N, P, true, MODE_STEP | QB, false>
                      : rlbm_kernel<St, R, LR, N, P, false, MODE_STEP | QB, false>;
    } else if (mode == MODE_INIT) {
        k = rlbm_kernel<St, R, LR, N, P, false, MODE_INIT | QB, false>;
    } else {
        k = rlbm_kernel<St, R, LR, N, P, false, MODE_MOMENTS | QB, false>;
    }
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    k<<<grid, block, smem, st>>>(a);
    return cudaGetLastError();
}

template <class St, class R, class LR, int N, int QB = 0>
static cudaError_t launch_n(int mode, int P, bool two_d, bool full, dim3 grid, dim3 block,
                           size_t smem, cudaStream_t st, const KernelArgs &a)
{
    switch (P) {
    case 8: return launch_np<St, R, LR, N, 8, QB>(mode, two_d, full, grid, block, smem, st, a);
    case 12: return launch_np<St, R, LR, N, 12, QB>(mode, two_d, full, grid, block, smem, st, a);
    case 16: return launch_np<St, R, LR, N, 16, QB>(mode, two_d, full, grid, block, smem, st, a);
    case 24: return launch_np<St, R, LR, N, 24, QB>(mode, two_d, full, grid, block, smem, st, a);
    case 32: return launch_np<St, R, LR, N, 32, QB>(mode, two_d, full, grid, block, smem, st, a);
    case 48: return launch_np<St, R, LR, N, 48, QB>(mode, two_d, full, grid, block, smem, st, a);
    case 64: return launch_np<St, R, LR, N, 64, QB>(mode, two_d, full, grid, block, smem, st, a);
    default: return cudaErrorInvalidValue;
    }
}

// N = 2, 3 here; N = 4, 5 (launch_t_hi) live in their own units (rlbm_k*_n45.cu).
template <class St, class R, class LR>
static cudaError_t launch_t(int mode, int N, int P, bool two_d, bool full, dim3 grid,
                           dim3 block, size_t smem, cudaStream_t st, const KernelArgs &a)
{
    switch (N) {
    case 2: return launch_n<St, R, LR, 2>(mode, P, two_d, full, grid, block, smem, st, a);
    case 3: return launch_n<St, R, LR, 3>(mode, P, two_d, full, grid, block, smem, st, a);
    default: return cudaErrorInvalidValue;
    }
}

template <class St, class R, class LR>
static cudaError_t launch_t_hi(int mode, int N, int P, bool two_d, bool full, dim3 grid,
                              dim3 block, size_t smem, cudaStream_t st, const KernelArgs &a)
{
    switch (N) {
    case 4: return launch_n<St, R, LR, 4>(mode, P, two_d, full, grid, block, smem, st, a);
    case 5: return launch_n<St, R, LR, 5>(mode, P, two_d, full, grid, block, smem, st, a);
    default: return cudaErrorInvalidValue;
    }
}

// The quantum statistics (N = 2, 3).
template <class St, class R, class LR>
static cudaError_t launch_tq(int mode, int N, int P, bool two_d, bool full, dim3 grid, dim3 block,
                             size_t smem, cudaStream_t st, const KernelArgs &a)
{
    switch (N) {
    case 2: return launch_n<St, R, LR, 2, MODE_Q>(mode, P, two_d, full, grid, block, smem, st, a);
    case 3: return launch_n<St, R, LR, 3, MODE_Q>(mode, P, two_d, full, grid, block, smem, st, a);
    default: return cudaErrorInvalidValue;
    }
}

// The on-lattice rule (Sec. 2.3): N = 3, 12 stencil vectors per shell, one warp
// of P = 12 populations per shell, perfect streaming.
template <class St, class R, class LR>
static cudaError_t launch_lattice_t(bool two_d, dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                    const KernelArgs &a)
{
    void (*k)(const KernelArgs) = two_d ? rlbm_kernel<St, R, LR, 3, 12, true, MODE_STEP_LATTICE, true>
                                        : rlbm_kernel<St, R, LR, 3, 12, false, MODE_STEP_LATTICE, true>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k<<<grid, block, smem, st>>>(a);
    return cudaGetLastError();
}

// FP32 storage, step kernels with the double-float per-site part (DDS in
// rlbm_kernel); the init and moments passes stay FP64.
template <int N, int P>
static cudaError_t launch_dd_np(bool two_d, bool full, dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                const KernelArgs &a)
{
    void (*k)(const KernelArgs);
    if (full)
        k = two_d ? rlbm_kernel<float, float, float, N, P, true, MODE_STEP, true>
                  : rlbm_kernel<float, float, float, N, P, false, MODE_STEP, true>;
    else
        k = two_d ? rlbm_kernel<float, float, float, N, P, true, MODE_STEP, false>
                  : rlbm_kernel<float, float, float, N, P, false, MODE_STEP, false>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k<<<grid, block, smem, st>>>(a);
    return cudaGetLastError();
}
template <int N>
static cudaError_t launch_dd_n(int P, bool two_d, bool full, dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                               const KernelArgs &a)
{
    switch (P) {
    case 8: return launch_dd_np<N, 8>(two_d, full, grid, block, smem, st, a);
    case 12: return launch_dd_np<N, 12>(two_d, full, grid, block, smem, st, a);
    case 16: return launch_dd_np<N, 16>(two_d, full, grid, block, smem, st, a);
    case 24: return launch_dd_np<N, 24>(two_d, full, grid, block, smem, st, a);
    case 32: return launch_dd_np<N, 32>(two_d, full, grid, block, smem, st, a);
    case 48: return launch_dd_np<N, 48>(two_d, full, grid, block, smem, st, a);
    case 64: return launch_dd_np<N, 64>(two_d, full, grid, block, smem, st, a);
    default: return cudaErrorInvalidValue;
    }
}

} // namespace rlbmk
