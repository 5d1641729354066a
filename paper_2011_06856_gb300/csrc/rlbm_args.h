// Launch arguments of the fused RLBM kernels and the per-storage-type
// launchers; shared by the host code and the kernel units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

namespace rlbmk {

// MODE_STEP_LATTICE: a step of the on-lattice rule (perfect streaming by the
// integer stencil vector of each population, no interpolation).
// MODE_Q (a bit added to STEP, INIT, MOMENTS): the quantum statistics.
enum Mode { MODE_STEP = 0, MODE_INIT = 1, MODE_MOMENTS = 2, MODE_STEP_LATTICE = 3, MODE_Q = 4 };

constexpr int kMaxN = 5;
// Suspend-time hint of the mbarrier waits (ns): a waiting thread sleeps until
// the phase completes or this time passes, instead of spinning through issue
// slots; the waits stay bounded by their clock deadline.
constexpr unsigned kWaitHintNs = 100000;
constexpr int kMaxWarps = 16;

// Everything a launch needs; passed by value (kernel parameter space).
struct KernelArgs {
    const void *fin;
    void *fout;
    int nx, ny;
    long long S;
    int K, Gs;      // angles per shell, warps per shell
    int P;          // populations per warp (the last warp of a shell may own fewer)
    int R;          // groups of P populations per warp (many angles); 0 or 1: one group
    int bcx, bcy;   // 0 periodic, 1 copy-out
    int collide;    // 0 for tau = +inf (free streaming)
    int stat;       // equilibrium statistic: 0 Maxwell-Juttner, +1 Fermi-Dirac, -1 Bose-Einstein
    double gdeg;    // normalisation g of f^eq = g / (z^-1 exp(U.p/T) + stat) (quantum statistics)
    double inv_tau;
    double beta;    // stored-unit offset: f = alpha (s + beta)
    double feq_off; // beta / (w_i / alpha_i): subtracted from the m = 0 coefficient
    double off[8];  // moment contribution of the offset beta
    double smp_c[kMaxN + 1], smp_s[kMaxN + 1]; // equispaced sample directions
    // FP32 copies of the scalars above, so FP32 kernels never touch the FP64 pipe
    float inv_tau_f, feq_off_f;
    float off_f[8];
    float smp_cf[kMaxN + 1], smp_sf[kMaxN + 1];
    // low parts of the double-float forms (value = FP32 copy + low part) of
    // the scalars above, for the double-float per-site part (rlbm_df64.cuh)
    float feq_off_l;
    float off_l[8];
    float smp_cl[kMaxN + 1], smp_sl[kMaxN + 1];
    const void *poptab;   // npop x tab_width(N), compute type
    const void *shelltab; // (N+1) x 2: alpha_r p_r, alpha_r p_r^2 (site type)
    const void *rtab;     // (N+1)^3 projection weights R'[r][m][k] (site type)
    const float2 *shell2; // the shell folds as double-floats (hi, lo): (N+1) x 2
    const float2 *rtab2;  // R'[r][m][k] as double-floats (hi, lo): (N+1)^3
    const double *in_n, *in_T, *in_bx, *in_by; // MODE_INIT fields
    double *out[6];                            // MODE_MOMENTS fields
    const unsigned long long *masks; // per warp: bit k = (v_x >= 0), (v_y >= 0) of its population k (k < 64)
    const void *pairtab; // npop x 3 float4: paired constants of the two-sites-per-lane kernel (FP32 arithmetic)
    const int2 *shifts;  // npop: integer stencil vectors of the on-lattice rule (else NULL)
    double *qeta;        // quantum statistics: per site, eta = ln z of the last solve (the next
                         // step's Newton start; NaN: none yet), else NULL
    long long wait_cycles; // bound of every mbarrier wait of the bulk-staged pair kernel (SM cycles)
    unsigned extra_tx;     // test hook: bytes expected on top of the copies (makes the waits run out)
    int *status;
    unsigned *ctr; // [0] completed step launches (seeds stochastic rounding), [1] CTAs done
};

__host__ __device__ constexpr int tab_width(int N) { return ((2 * N + 5) + 3) / 4 * 4; }

// Dynamic shared memory of the per-tile kernel (rlbm_kernel): the angular sums
// [5][G][32] in the per-site type (ls bytes), then either the per-site sums
// shared by the warps when the per-site part runs once per site in FP64
// [(N+1)^2 + 3][32] or, for the quantum statistics, T and the radial weights
// t_0..t_N [1 + N + 1][32] doubles.
__host__ __device__ constexpr size_t tile_smem_bytes(int N, int G, size_t ls, bool quantum)
{
    return ls * 5 * size_t(G) * 32 +
           (quantum ? size_t(N + 2) * 32 * sizeof(double)
                    : (ls == 8 ? size_t((N + 1) * (N + 1) + 3) * 32 * 8 : 0));
}
// The same for an FP32-storage step with the double-float per-site part split
// over the warps (site_split_dd): FP32 angular sums, then [2 (N+1)^2 + 3][32]
// floats (the sums as hi and lo rows, then U^a / tau), the frame
// [6 + 2 (N+1)][32] and the partial sums [N+1][2 (N+1)^2][32].
__host__ __device__ constexpr size_t tile_smem_bytes_dd(int N, int G)
{
    return 4 * 5 * size_t(G) * 32 +
           size_t(2 * (N + 1) * (N + 1) + 3 + 6 + 2 * (N + 1) + (N + 1) * 2 * (N + 1) * (N + 1)) * 32 * 4;
}

// Two-sites-per-lane step kernel: sites per CTA and dynamic shared memory:
// angular sums [5][G][64] and the per-site results [2 (N+1)^2 + 3][64] (FP32;
// the (N+1)^2 shell-independent equilibrium sums as double-floats, hi and lo
// rows, then U^a / tau); for the bulk-staged form then, per warp, kPairDepth
// mbarriers and kPairDepth slots of kPairChunk populations x rows x (64 sites
// + 16 bytes of halo on each side).
constexpr int kPairSites = 64;
constexpr int kPairChunk = 4;
constexpr int kPairDepth = 3;
__host__ __device__ constexpr int pair_site_rows(int N) { return 2 * (N + 1) * (N + 1) + 3; }
__host__ __device__ constexpr size_t pair_bars_offset(int N, int G)
{
    return ((size_t(5) * G + size_t(pair_site_rows(N))) * kPairSites * 4 + 15) / 16 * 16;
}
__host__ __device__ constexpr size_t pair_slots_offset(int N, int G)
{
    return pair_bars_offset(N, G) + (size_t(G) * kPairDepth * 8 + 15) / 16 * 16;
}
__host__ __device__ constexpr size_t pair_slot_bytes(int elem_bytes, bool two_d)
{
    return size_t(kPairChunk) * (two_d ? 2 : 1) * (kPairSites * elem_bytes + 32);
}
__host__ __device__ constexpr size_t pair_smem_bytes(int N, int G, bool bulk, int elem_bytes, bool two_d)
{
    return bulk ? pair_slots_offset(N, G) + size_t(G) * kPairDepth * pair_slot_bytes(elem_bytes, two_d)
                : pair_bars_offset(N, G);
}
// Rows of site_split_dd's frame [6 + 2 (N+1)] and partial sums [N+1][2 (N+1)^2].
__host__ __device__ constexpr int split_rows(int N) { return 6 + 2 * (N + 1) + (N + 1) * 2 * (N + 1) * (N + 1); }
// The two-sites-per-lane kernels with FP32 storage split their double-float
// per-site part over the warps when the CTA has a thread for every (sample
// direction, site) item; its frame and partial sums then follow the layout
// above ([split_rows(N)][64] floats).  With fewer warps two of them solve the
// sites whole (the split's extra shared memory would cost more occupancy than
// the shorter chain gains).
__host__ __device__ constexpr bool pair_split(int N, int G) { return G * 32 >= (N + 1) * kPairSites; }
__host__ __device__ constexpr size_t pair_smem_total(int N, int G, bool bulk, int elem_bytes, bool two_d)
{
    return pair_smem_bytes(N, G, bulk, elem_bytes, two_d) +
           (elem_bytes == 4 && pair_split(N, G) ? size_t(split_rows(N)) * kPairSites * 4 : 0);
}

// Arguments of the persistent TMA-staged step kernel.
struct alignas(128) TmaArgs {
    CUtensorMap tmap;      // 3D map over the input buffer: {nx, ny, npop}, box {BW, 1, BP}
    KernelArgs a;
    int BP;                // populations per box
    int nbox;              // boxes per row slot (npop <= nbox * BP)
    int ntiles_x, ntiles;  // tiles of 32 sites per row, total tiles
    long long stage_bytes; // bytes of one pipeline stage
    long long wait_cycles; // bound of every mbarrier wait
    unsigned extra_tx;     // test hook: extra expected bytes (0 in normal use)
};

__host__ __device__ constexpr size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Shared-memory layout of rlbm_step_tma: two stages, the per-warp table
// slice, two reduction buffers (tiles alternate), two mbarriers, a flag.
struct TmaSmem {
    size_t tab, red, bars, flag, total;
    __host__ __device__ TmaSmem(size_t stage_bytes, int G, int P, int N, size_t rs, size_t ls)
    {
        tab = 2 * stage_bytes;
        red = align_up(tab + size_t(G) * P * tab_width(N) * rs, 16);
        bars = align_up(red + 2 * 5 * size_t(G) * 32 * ls, 16);
        flag = bars + 16;
        total = flag + 16 + 1024; // + slack to align the base to 1 KB
    }
};

// Host-side launcher for one storage type (defined in the per-type units).
// Persistent TMA-staged step launchers; grid <= 0 with blocks_per_sm set only
// queries the occupancy.
#define RLBM_DECLARE_TMA(t)                                                                       \
    cudaError_t launch_tma_##t(int N, int P, bool two_d, bool full, bool site_fp64, int grid,      \
                               dim3 block, size_t smem, cudaStream_t st, const TmaArgs &a, int *bps);
RLBM_DECLARE_TMA(f64)
RLBM_DECLARE_TMA(f32)
RLBM_DECLARE_TMA(f16)
RLBM_DECLARE_TMA(bf16)
#undef RLBM_DECLARE_TMA
// full: K is a multiple of P (every warp owns exactly P populations)
cudaError_t launch_f64(int mode, int N, int P, bool two_d, bool full, dim3 grid, dim3 block,
                       size_t smem, cudaStream_t st, const KernelArgs &a);
cudaError_t launch_f32(int mode, int N, int P, bool two_d, bool full, bool site_fp64, dim3 grid,
                       dim3 block, size_t smem, cudaStream_t st, const KernelArgs &a);
// FP32 storage, a step (N = 2, 3) with the double-float per-site part once per
// site (needs the split tables shell2, rtab2 and the lo parts of KernelArgs;
// shared memory tile_smem_bytes_dd).
cudaError_t launch_f32_dd(int N, int P, bool two_d, bool full, dim3 grid, dim3 block, size_t smem,
                          cudaStream_t st, const KernelArgs &a);
cudaError_t launch_f32_dd_n2(int P, bool two_d, bool full, dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                             const KernelArgs &a);
cudaError_t launch_f32_dd_n3(int P, bool two_d, bool full, dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                             const KernelArgs &a);
cudaError_t launch_f16(int mode, int N, int P, bool two_d, bool full, dim3 grid, dim3 block,
                       size_t smem, cudaStream_t st, const KernelArgs &a);
cudaError_t launch_bf16(int mode, int N, int P, bool two_d, bool full, dim3 grid, dim3 block,
                        size_t smem, cudaStream_t st, const KernelArgs &a);
// A step of the on-lattice rule (per-tile kernel, N = 3, P = 12), FP64 and FP32 storage
// (FP32: the double-float per-site part, shared memory tile_smem_bytes_dd).
cudaError_t launch_lattice_f64(bool two_d, dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                               const KernelArgs &a);
cudaError_t launch_lattice_f32(bool two_d, dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                               const KernelArgs &a);
// The per-tile kernel with a quantum statistic (N = 2, 3; FP64 per-site arithmetic), FP64 and
// FP32 storage; mode is MODE_STEP, MODE_INIT or MODE_MOMENTS.
cudaError_t launch_quant_f64(int mode, int N, int P, bool two_d, bool full, dim3 grid, dim3 block,
                             size_t smem, cudaStream_t st, const KernelArgs &a);
cudaError_t launch_quant_f32(int mode, int N, int P, bool two_d, bool full, dim3 grid, dim3 block,
                             size_t smem, cudaStream_t st, const KernelArgs &a);
// The same per-tile kernel for N = 4, 5, with FP64 per-site arithmetic in every storage type.
cudaError_t launch_f64_n45(int mode, int N, int P, bool two_d, bool full, dim3 grid, dim3 block,
                           size_t smem, cudaStream_t st, const KernelArgs &a);
cudaError_t launch_f32_n45(int mode, int N, int P, bool two_d, bool full, dim3 grid, dim3 block,
                           size_t smem, cudaStream_t st, const KernelArgs &a);
cudaError_t launch_f16_n45(int mode, int N, int P, bool two_d, bool full, dim3 grid, dim3 block,
                           size_t smem, cudaStream_t st, const KernelArgs &a);
cudaError_t launch_bf16_n45(int mode, int N, int P, bool two_d, bool full, dim3 grid, dim3 block,
                            size_t smem, cudaStream_t st, const KernelArgs &a);
// Two-sites-per-lane step kernel (rlbm_pair.cuh): 64-site tiles, PP in {8, 12, 16, 24, 32};
// bulk: interior tiles staged through shared memory by cp.async.bulk.
// Two-sites-per-lane kernels: one compile unit per storage, order N and form
// (p plain, b bulk-staged first pass), compiled in parallel; the dispatchers
// below pick the unit.
#define RLBM_DECLARE_PAIR(name)                                                                          \
    cudaError_t launch_pair_##name##_n2p(int PP, bool two_d, dim3 grid, dim3 block, size_t smem,         \
                                         cudaStream_t st, const KernelArgs &a);                          \
    cudaError_t launch_pair_##name##_n2b(int PP, bool two_d, dim3 grid, dim3 block, size_t smem,         \
                                         cudaStream_t st, const KernelArgs &a);                          \
    cudaError_t launch_pair_##name##_n3p(int PP, bool two_d, dim3 grid, dim3 block, size_t smem,         \
                                         cudaStream_t st, const KernelArgs &a);                          \
    cudaError_t launch_pair_##name##_n3b(int PP, bool two_d, dim3 grid, dim3 block, size_t smem,         \
                                         cudaStream_t st, const KernelArgs &a);                          \
    inline cudaError_t launch_pair_##name(int N, int PP, bool two_d, bool bulk, dim3 grid, dim3 block,   \
                                          size_t smem, cudaStream_t st, const KernelArgs &a)             \
    {                                                                                                    \
        if (N == 2)                                                                                      \
            return bulk ? launch_pair_##name##_n2b(PP, two_d, grid, block, smem, st, a)                  \
                        : launch_pair_##name##_n2p(PP, two_d, grid, block, smem, st, a);                 \
        if (N == 3)                                                                                      \
            return bulk ? launch_pair_##name##_n3b(PP, two_d, grid, block, smem, st, a)                  \
                        : launch_pair_##name##_n3p(PP, two_d, grid, block, smem, st, a);                 \
        return cudaErrorInvalidValue;                                                                    \
    }
RLBM_DECLARE_PAIR(f32)
RLBM_DECLARE_PAIR(f16)
RLBM_DECLARE_PAIR(bf16)
#undef RLBM_DECLARE_PAIR
// several population groups per warp (FP32 storage)
cudaError_t launch_pair_groups_f32_n2(int PP, bool two_d, dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                      const KernelArgs &a);
cudaError_t launch_pair_groups_f32_n3(int PP, bool two_d, dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                      const KernelArgs &a);
inline cudaError_t launch_pair_groups_f32(int N, int PP, bool two_d, dim3 grid, dim3 block, size_t smem,
                                          cudaStream_t st, const KernelArgs &a)
{
    if (N == 2) return launch_pair_groups_f32_n2(PP, two_d, grid, block, smem, st, a);
    if (N == 3) return launch_pair_groups_f32_n3(PP, two_d, grid, block, smem, st, a);
    return cudaErrorInvalidValue;
}

// Arguments of the tile-staged two-sites-per-lane kernel (rlbm_pair_tma.cuh).
struct alignas(128) PairTmaArgs {
    CUtensorMap cmap; // 3D map over the input buffer {nx, ny, npop}, box {BW, 1, CB}: centre rows
    CUtensorMap pmap; // the same map with box {BW, 1, DB}: pull rows
    KernelArgs a;
    int CB, ncbox;    // populations per centre box, boxes per tile (CB ncbox = npop)
    int DB, npbox;    // populations per pull-row chunk, chunks per tile (DB npbox = npop)
    unsigned long long chunk_up[4]; // bit c: chunk c pulls from row y - 1 (its v_y >= 0), else y + 1
};

// Shared-memory layout of rlbm_pair_tma_kernel: the staged tile (centre rows,
// then pull rows in 2D: [rows][npop][BW] storage elements, BW = 64 sites +
// 16 bytes of halo on each side), the pair table [npop][3] float4, the
// angular sums [5][G][64], the per-site results [pair_site_rows(N)][64], the
// mbarrier; + 1 KB of slack to align the base for the TMA.
// The angular sums and the per-site results are needed only after pass 1, when
// the stage is dead: where the stage is large enough they alias it (alias = true;
// the kernel then separates the last stage read from the first write by a CTA
// barrier), which lets more CTAs share an SM.
struct PairTmaSmem {
    size_t stage, tab, red, sres, bar, total;
    bool alias;
    __host__ __device__ PairTmaSmem(int N, int G, int npop, int es, bool two_d)
    {
        const size_t BW = size_t(kPairSites) + 2 * size_t(16 / es);
        const size_t stage_bytes = size_t(two_d ? 2 : 1) * size_t(npop) * BW * size_t(es);
        const size_t red_bytes = size_t(5) * G * kPairSites * 4;
        const size_t sres_bytes = size_t(pair_site_rows(N)) * kPairSites * 4;
        stage = 0;
        tab = align_up(stage_bytes, 128);
        alias = stage_bytes >= red_bytes + sres_bytes;
        if (alias) {
            red = 0;
            sres = red_bytes;
            bar = align_up(tab + size_t(npop) * 3 * 16, 16);
        } else {
            red = align_up(tab + size_t(npop) * 3 * 16, 16);
            sres = red + red_bytes;
            bar = align_up(sres + sres_bytes, 16);
        }
        total = bar + 16 + 1024;
    }
};

#define RLBM_DECLARE_PAIR_TMA(name)                                                                      \
    cudaError_t launch_pair_tma_##name##_n2(int PP, bool two_d, dim3 block, size_t smem,       \
                                            cudaStream_t st, const PairTmaArgs &ta, int *bps);           \
    cudaError_t launch_pair_tma_##name##_n3(int PP, bool two_d, dim3 block, size_t smem,       \
                                            cudaStream_t st, const PairTmaArgs &ta, int *bps);           \
    inline cudaError_t launch_pair_tma_##name(int N, int PP, bool two_d, dim3 block,           \
                                              size_t smem, cudaStream_t st, const PairTmaArgs &ta,       \
                                              int *bps)                                                  \
    {                                                                                                    \
        if (N == 2) return launch_pair_tma_##name##_n2(PP, two_d, block, smem, st, ta, bps);       \
        if (N == 3) return launch_pair_tma_##name##_n3(PP, two_d, block, smem, st, ta, bps);       \
        return cudaErrorInvalidValue;                                                                    \
    }
RLBM_DECLARE_PAIR_TMA(f32)
RLBM_DECLARE_PAIR_TMA(f16)
RLBM_DECLARE_PAIR_TMA(bf16)
#undef RLBM_DECLARE_PAIR_TMA

// Batched persistent form (rlbm_batch.cuh).
constexpr int kBatchWarps = 6;

struct BatchUnit {
    int prob;  // problem index
    int tile0; // first tile (row-major: y * ntiles_x + xt)
};

struct BatchArgs {
    const KernelArgs *probs; // per problem: fin = buffer 0, fout = buffer 1
    const int *ntiles_x;     // per problem
    const int *ntiles;       // per problem
    const int *tiles_per_unit;
    const BatchUnit *units;
    int nunits;
    int nsteps;
    const int *parity0;      // per problem: buffer holding the current state (0 / 1)
    unsigned *sync;          // [0] arrivals, [1] generation, [2], [3] work counters (by step parity)
    int *status;             // bit 1: a barrier wait ran out
    long long wait_cycles;
    unsigned barrier_extra;  // test hook: arrivals the barrier waits for beyond the grid (0)
};

cudaError_t launch_batch(int prec, int N, const BatchArgs &b, int grid, cudaStream_t st,
                         int *blocks_per_sm);
// Advance every problem's launch counter by nsteps (after a batched launch).
cudaError_t launch_batch_advance(const KernelArgs *probs, int n, int nsteps, cudaStream_t st);

} // namespace rlbmk
