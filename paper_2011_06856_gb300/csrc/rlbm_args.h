// Launch arguments of the fused RLBM kernels and the per-storage-type
// launchers; shared by the host code and the kernel units.
#pragma once

#include <cuda_runtime.h>

namespace rlbmk {

enum Mode { MODE_STEP = 0, MODE_INIT = 1, MODE_MOMENTS = 2 };

constexpr int kMaxN = 5;
constexpr int kMaxWarps = 16;

// Everything a launch needs; passed by value (kernel parameter space).
struct KernelArgs {
    const void *fin;
    void *fout;
    int nx, ny;
    long long S;
    int K, Gs;      // angles per shell, warps per shell
    int P;          // populations per warp (the last warp of a shell may own fewer)
    int bcx, bcy;   // 0 periodic, 1 copy-out
    int collide;    // 0 for tau = +inf (free streaming)
    double inv_tau;
    double beta;    // stored-unit offset: f = alpha (s + beta)
    double off[8];  // moment contribution of the offset beta
    double smp_c[kMaxN + 1], smp_s[kMaxN + 1]; // equispaced sample directions
    const void *poptab;   // npop x tab_width(N), compute type
    const void *shelltab; // (N+1) x 2: alpha_r p_r, alpha_r p_r^2 (site type)
    const void *rtab;     // (N+1)^3 projection weights R'[r][m][k] (site type)
    const double *in_n, *in_T, *in_bx, *in_by; // MODE_INIT fields
    double *out[6];                            // MODE_MOMENTS fields
    int *status;
};

__host__ __device__ constexpr int tab_width(int N) { return ((2 * N + 5) + 3) / 4 * 4; }

// Host-side launcher for one storage type (defined in the per-type units).
cudaError_t launch_f64(int mode, int N, int P, bool two_d, dim3 grid, dim3 block, size_t smem,
                       cudaStream_t st, const KernelArgs &a);
cudaError_t launch_f32(int mode, int N, int P, bool two_d, bool site_fp64, dim3 grid, dim3 block,
                       size_t smem, cudaStream_t st, const KernelArgs &a);
cudaError_t launch_f16(int mode, int N, int P, bool two_d, dim3 grid, dim3 block, size_t smem,
                       cudaStream_t st, const KernelArgs &a);
cudaError_t launch_bf16(int mode, int N, int P, bool two_d, dim3 grid, dim3 block, size_t smem,
                        cudaStream_t st, const KernelArgs &a);

} // namespace rlbmk
