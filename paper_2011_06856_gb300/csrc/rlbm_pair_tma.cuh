// Tile-staged form of the two-sites-per-lane step (arXiv 2011.06856, Sec. 2.2).
//
// The arithmetic is that of rlbm_pair_kernel (two sites per lane as packed
// f32x2 pairs, the per-site part once per site in two warps); what changes is
// how the populations reach the registers.  A CTA owns one 64-site tile.  At
// its start the lanes of warp 0 issue the TMA loads of the whole tile into
// shared memory -- cp.async.bulk.tensor over the 3D map {nx, ny, npop}:
//   centre rows  row y of every population, x0 - HX .. x0 + 64 + HX
//                (HX = 16 bytes of halo on each side), CB populations per box;
//   pull rows    (2D) row y - sgn(v_y) of every population (the upwind row of
//                the bilinear pull, Eqs. streaming, interpolation), DB
//                populations per box; the host groups the populations in
//                chunks of DB that share sgn(v_y) (populations with v_y = 0
//                give the pull row the weight 0 and join either side), so one
//                box fetches the right row for a whole chunk;
// and one mbarrier counts the bytes.  While the copies fly, every thread
// copies the per-population pair table into shared memory.  After a bounded
// wait the first pass reads shared memory only, with compile-time offsets; on
// the domain edges the halo cells outside the grid (zero-filled by the TMA)
// are first rewritten with their periodic / copy-out source values.  Several
// CTAs per SM overlap one another's loads, per-site solve and stores.
//
// Stores round stochastically: 16-bit ones with the cvt.rs instruction, FP32
// ones from the FMA residual (relax_pair_sr); random bits from a per-thread
// LCG (the high halves of its draws, next_bits2).
//
// One tile per CTA, three CTAs per SM (64 registers, about 71 KB of shared
// memory with 144 populations in FP16) measured faster than persistent CTAs
// cycling their tiles through one or two stages: 1.44 ms against 1.61 ms (one
// stage, three CTAs) and 1.89 ms (two stages, two CTAs) per 2048^2 FP16 step.
//
// Every wait is bounded: on expiry the CTA sets bit 1 of the status word,
// waits (again bounded) for its copies and returns without storing.
#pragma once

#include "rlbm_pair.cuh"
#include "rlbm_tma.cuh"

namespace rlbmk {

template <class St> struct PairTmaGeom {
    static constexpr int HX = 16 / int(sizeof(St)); // halo columns on each side (16 bytes)
    static constexpr int BW = kPairSites + 2 * HX;  // box width in x (a multiple of 16 bytes)
};

// 16-bit pair stores with the stochastic-rounding conversion (the first
// source operand lands in the upper half: the site at the higher address)
template <class St> __device__ __forceinline__ void st2_rs(St *p, float2 v, unsigned rbits);
template <> __device__ __forceinline__ void st2_rs<__half>(__half *p, float2 v, unsigned rbits)
{
    unsigned d;
    asm("cvt.rs.satfinite.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(v.y), "f"(v.x), "r"(rbits));
    *reinterpret_cast<unsigned *>(p) = d;
}
template <> __device__ __forceinline__ void st2_rs<__nv_bfloat16>(__nv_bfloat16 *p, float2 v, unsigned rbits)
{
    unsigned d;
    asm("cvt.rs.satfinite.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(v.y), "f"(v.x), "r"(rbits));
    *reinterpret_cast<unsigned *>(p) = d;
}

template <class St, int N, int PP, bool TWO_D>
__device__ __forceinline__ void pair_tma_body(const PairTmaArgs &ta)
{
    constexpr int NC = 2 * N + 1;
    constexpr int PQ = 3; // float4 per population in the pair table
    constexpr int HX = PairTmaGeom<St>::HX, BW = PairTmaGeom<St>::BW;
    constexpr int RW = TWO_D ? 2 : 1;
    const KernelArgs &a = ta.a;
    extern __shared__ __align__(16) unsigned char smem_pt[];
    // TMA destinations: align the base to 1 KB (the host adds the slack)
    unsigned char *sm = smem_pt + ((1024u - (smem_u32(smem_pt) & 1023u)) & 1023u);
    const int lane = threadIdx.x, g = threadIdx.y, G = blockDim.y;
    const int tid = g * 32 + lane, nthr = G * 32;
    const int npop = a.K * (N + 1);
    const PairTmaSmem L(N, G, npop, int(sizeof(St)), TWO_D);
    St *stage = reinterpret_cast<St *>(sm + L.stage); // [RW][npop][BW]
    float4 *tab = reinterpret_cast<float4 *>(sm + L.tab);
    float *red = reinterpret_cast<float *>(sm + L.red);   // [5][G][64]
    float *sres = reinterpret_cast<float *>(sm + L.sres); // [pair_site_rows(N)][64]
    unsigned long long *bar = reinterpret_cast<unsigned long long *>(sm + L.bar);
    const int x0 = blockIdx.x * kPairSites, y = blockIdx.y;
    const int ym = TWO_D ? bc_index(y - 1, a.ny, a.bcy) : y;
    const int yp = TWO_D ? bc_index(y + 1, a.ny, a.bcy) : y;

    if (tid == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (g == 0) {
        if (lane == 0) mbar_expect_tx(bar, unsigned(RW * npop * BW * int(sizeof(St))) + a.extra_tx);
        __syncwarp();
        const int nops = ta.ncbox + (TWO_D ? ta.npbox : 0);
        for (int o = lane; o < nops; o += 32) {
            if (o < ta.ncbox) {
                const int p0 = o * ta.CB;
                tma_load_3d(stage + size_t(p0) * BW, &ta.cmap, x0 - HX, y, p0, bar);
            } else {
                const int c = o - ta.ncbox, p0 = c * ta.DB;
                const bool up = (ta.chunk_up[c >> 6] >> (c & 63)) & 1ull;
                tma_load_3d(stage + size_t(npop + p0) * BW, &ta.pmap, x0 - HX, up ? ym : yp, p0, bar);
            }
        }
    }
    // while the copies fly: the pair table into shared memory
    {
        const float4 *gt = reinterpret_cast<const float4 *>(a.pairtab);
        for (int e = tid; e < npop * PQ; e += nthr) tab[e] = __ldg(gt + e);
    }
    const bool arrived = mbar_wait_bounded(bar, 0, a.wait_cycles);
    if (__syncthreads_or(!arrived)) {
        if (tid == 0) {
            atomicOr(a.status, 2);
            mbar_wait_bounded(bar, 0, a.wait_cycles); // the copies still in flight (bounded)
        }
        return;
    }
    const St *fin = reinterpret_cast<const St *>(a.fin);
    const long long S = a.S;
    // halo cells beyond the grid edge (TMA filled zeros): their source values
    const bool left = x0 == 0, right = a.nx - x0 < kPairSites + HX;
    if (left || right) {
        const int xr = a.nx - x0 + HX; // local column of x = nx
        for (int e = tid; e < RW * npop * 2; e += nthr) {
            const int side = e & 1, rest = e >> 1;
            const int rr = rest / npop, p = rest % npop;
            if (side == 0 ? !left : !right) continue;
            int row = y;
            if (rr == 1) {
                const int c = p / ta.DB;
                row = ((ta.chunk_up[c >> 6] >> (c & 63)) & 1ull) ? ym : yp;
            }
            const int xs = bc_index(side == 0 ? -1 : a.nx, a.nx, a.bcx);
            stage[(size_t(rr) * npop + p) * BW + (side == 0 ? HX - 1 : xr)] =
                fin[(long long)p * S + (long long)row * a.nx + xs];
        }
        __syncthreads();
    }

    const int xl = x0 + 2 * lane;
    const bool act = xl < a.nx;
    const int r = g / a.Gs, q = g % a.Gs;
    const int i0 = r * a.K + q * PP;
    const St *cb = stage + size_t(i0) * BW + HX + 2 * lane;         // centre row, this lane's pair
    const St *pb = stage + size_t(npop + i0) * BW + HX + 2 * lane;  // pull row
    const float4 *tb = tab + size_t(i0) * PQ;
    const unsigned long long mx = __ldg(a.masks + 2 * g);

    // pass 1: bilinear pull from shared memory, five angular sums
    float2 fs[PP];
    float2 s0 = f2(0.f, 0.f), sc = f2(0.f, 0.f), ss = f2(0.f, 0.f), scc = f2(0.f, 0.f), scs = f2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < PP; ++k) {
        const bool px = (mx >> k) & 1ull; // v_x >= 0: pull from x - 1
        const St *ra = cb + k * BW;
        const float2 C = lds2<St>(ra);
        const float e = lds1<St>(ra + (px ? -1 : 2));
        const float4 t0 = tb[k * PQ], t1 = tb[k * PQ + 1]; // (c,c,s,s), (|c|,|c|,|s|,|s|)
        const float2 B = px ? f2(e, C.x) : f2(C.y, e);
        const float2 ac = f2(t1.x, t1.y);
        float2 v = __ffma2_rn(ac, f2sub(B, C), C);
        if (TWO_D) {
            const St *rb = pb + k * BW;
            const float2 C2 = lds2<St>(rb);
            const float e2 = lds1<St>(rb + (px ? -1 : 2));
            const float2 B2 = px ? f2(e2, C2.x) : f2(C2.y, e2);
            const float2 hi = __ffma2_rn(ac, f2sub(B2, C2), C2);
            v = __ffma2_rn(f2(t1.z, t1.w), f2sub(hi, v), v);
        }
        fs[k] = v;
        const float2 c = f2(t0.x, t0.y), sn = f2(t0.z, t0.w);
        const float2 cv = __fmul2_rn(c, v);
        s0 = __fadd2_rn(s0, v);
        sc = __fadd2_rn(sc, cv);
        ss = __ffma2_rn(sn, v, ss);
        scc = __ffma2_rn(c, cv, scc);
        scs = __ffma2_rn(sn, cv, scs);
    }
    if (L.alias) __syncthreads(); // red and sres alias the stage: every warp is done reading it
    float2 *red2 = reinterpret_cast<float2 *>(red);
    red2[(0 * G + g) * 32 + lane] = s0;
    red2[(1 * G + g) * 32 + lane] = sc;
    red2[(2 * G + g) * 32 + lane] = ss;
    red2[(3 * G + g) * 32 + lane] = scc;
    red2[(4 * G + g) * 32 + lane] = scs;
    __syncthreads();
    constexpr bool DD = sizeof(St) == 4; // FP32 storage: FP64-class per-site part
    if (g < 2) {
        const int s = g * 32 + lane;
        if constexpr (DD) pair_site_solve_dd<N>(a, red, G, s, x0 + s < a.nx, sres);
        else pair_site_solve<N>(a, red, G, s, x0 + s < a.nx, sres);
    }
    __syncthreads();

    // pass 2: this warp's shell coefficients, f^eq, relaxation (Eq. discrete-rbe), stores
    float2 cr[NC], o0, o1, o2;
    pair_shell_coefficients<N, DD>(a, r, sres, lane, cr, o0, o1, o2);
    const float2 no1 = f2(-o1.x, -o1.y), no2 = f2(-o2.x, -o2.y);
    unsigned rng = mix32(unsigned(y * a.nx + xl) * 64u + unsigned(g) ^ mix32(__ldcg(a.ctr) * 0x9E3779B9u + 1u));
    St *ob = reinterpret_cast<St *>(a.fout) + (long long)i0 * S + (long long)y * a.nx + (act ? xl : 0);
#pragma unroll
    for (int k = 0; k < PP; ++k) {
        const float4 t0 = tb[k * PQ];                                      // (c,c,s,s)
        const float2 wq = *reinterpret_cast<const float2 *>(tb + k * PQ + 2); // (w', w')
        const float2 c = f2(t0.x, t0.y), sn = f2(t0.z, t0.w);
        const float2 cc = __fmul2_rn(c, c), cs = __fmul2_rn(c, sn);
        float2 pe = __ffma2_rn(cr[1], c, cr[0]);
        pe = __ffma2_rn(cr[2], sn, pe);
        pe = __ffma2_rn(cr[3], cc, pe);
        pe = __ffma2_rn(cr[4], cs, pe);
        if (N == 3) {
            pe = __ffma2_rn(cr[NC - 2], __fmul2_rn(c, cc), pe);
            pe = __ffma2_rn(cr[NC - 1], __fmul2_rn(sn, cc), pe);
        }
        const float2 feq = __fmul2_rn(wq, pe);
        const float2 om = __ffma2_rn(no2, sn, __ffma2_rn(no1, c, o0));
        const unsigned rb = next_bits2(rng);
        if constexpr (sizeof(St) == 4) {
            const float2 out = relax_pair_sr(fs[k], om, feq, rb);
            if (act) *reinterpret_cast<float2 *>(ob + (long long)k * S) = out;
        } else {
            const float2 out = __ffma2_rn(om, f2sub(feq, fs[k]), fs[k]);
            if (act) st2_rs<St>(ob + (long long)k * S, out, rb);
        }
    }
    __syncthreads();
    if (tid == 0) advance_launch_counter(a.ctr, gridDim.x * gridDim.y);
}

// FP32 storage: the launch bounds of the other two-sites-per-lane kernels.
template <class St, int N, int PP, bool TWO_D>
__global__ void __launch_bounds__(kMaxWarps * 32, PP <= 16 ? 2 : 1)
    rlbm_pair_tma_kernel(const __grid_constant__ PairTmaArgs ta)
{
    pair_tma_body<St, N, PP, TWO_D>(ta);
}

// 16-bit storage: with PP <= 16, at most 56 registers, so that four CTAs of nine
// warps (the 2048^2 N = 2 K = 48 tiling, 54 KB of shared memory with the aliased
// sums) share an SM.
template <class St, int N, int PP, bool TWO_D>
__global__ void __maxnreg__(PP <= 16 ? 56 : 128) rlbm_pair_tma_kernel16(const __grid_constant__ PairTmaArgs ta)
{
    pair_tma_body<St, N, PP, TWO_D>(ta);
}

template <class St, int N, int PP>
static cudaError_t launch_pair_tma_np(bool two_d, dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                      const PairTmaArgs &ta, int *bps)
{
    void (*k)(const PairTmaArgs);
    if constexpr (sizeof(St) == 2)
        k = two_d ? rlbm_pair_tma_kernel16<St, N, PP, true> : rlbm_pair_tma_kernel16<St, N, PP, false>;
    else
        k = two_d ? rlbm_pair_tma_kernel<St, N, PP, true> : rlbm_pair_tma_kernel<St, N, PP, false>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (bps) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k, int(block.x * block.y), smem);
    k<<<grid, block, smem, st>>>(ta);
    return cudaGetLastError();
}

// The instances of storage St and order N (one compile unit each): one CTA per
// 64-site tile; with bps set, only the occupancy query (CTAs per SM).
template <class St, int N>
static cudaError_t launch_pair_tma_n(int PP, bool two_d, dim3 block, size_t smem, cudaStream_t st,
                                     const PairTmaArgs &ta, int *bps)
{
    const dim3 grid((ta.a.nx + kPairSites - 1) / kPairSites, ta.a.ny);
    switch (PP) {
    case 8: return launch_pair_tma_np<St, N, 8>(two_d, grid, block, smem, st, ta, bps);
    case 12: return launch_pair_tma_np<St, N, 12>(two_d, grid, block, smem, st, ta, bps);
    case 16: return launch_pair_tma_np<St, N, 16>(two_d, grid, block, smem, st, ta, bps);
    case 24: return launch_pair_tma_np<St, N, 24>(two_d, grid, block, smem, st, ta, bps);
    case 32: return launch_pair_tma_np<St, N, 32>(two_d, grid, block, smem, st, ta, bps);
    default: return cudaErrorInvalidValue;
    }
}

} // namespace rlbmk
