// Persistent, TMA-staged variant of the fused RLBM step (Sec. 2.2).
//
// Each CTA owns a stripe of tiles (tile = 32 consecutive sites of one row x
// all N_pop populations) and walks them with a two-stage pipeline:
//
//   TMA      one elected thread loads the tile's populations with their
//            halo (16 bytes on each side in x, rows y-1..y+1 in 2D) into a
//            shared-memory stage with cp.async.bulk.tensor (3D tensor map
//            over f[pop][y][x]); completion is an mbarrier transaction count;
//   patch    tiles on the domain boundary rewrite the halo cells that lie
//            outside the grid with their periodic / copy-out source values;
//   pass 1   warp g streams its P populations from shared memory (bilinear
//            pull, Eqs. streaming and interpolation), keeps f* in registers
//            and forms the five per-shell angular sums;
//   refill   once every warp is done with the stage, the elected thread
//            issues the TMA of the tile two steps ahead into it;
//   site     every warp: moments, Landau frame and its own shell's
//            equilibrium coefficients (see rlbm_device.cuh);
//   pass 2   every warp: f^eq, relaxation (Eq. discrete-rbe), coalesced
//            stores to global memory.
//
// Every mbarrier wait is bounded (a clock64 deadline): on expiry the kernel
// sets bit 1 of the status word, waits (again bounded) for its own copies
// still in flight and returns.
#pragma once

#include "rlbm_device.cuh"

namespace rlbmk {

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity), "r"(kWaitHintNs)
                 : "memory");
    return ok != 0;
}

// Bounded wait for the phase with the given parity; false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, unsigned parity,
                                                  long long max_cycles)
{
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > max_cycles) return false;
    }
    return true;
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z,
                                            unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

template <class St> struct StageGeom {
    static constexpr int HX = 16 / int(sizeof(St)); // halo columns on each side (16 bytes)
    static constexpr int BW = 32 + 2 * HX;          // box width in x
};

// Issue the TMA loads of one tile into a stage: one box {BW, 1, BP} per row
// slot and population block.  In 2D the slots hold rows bc(y-1), y, bc(y+1),
// so the y boundary condition is applied by the choice of source row.
template <class St>
__device__ __forceinline__ void issue_tile(const TmaArgs &ta, unsigned char *stage,
                                           unsigned long long *bar, int tile, int BR)
{
    constexpr int HX = StageGeom<St>::HX, BW = StageGeom<St>::BW;
    const KernelArgs &a = ta.a;
    const int y = tile / ta.ntiles_x;
    const int x0 = (tile % ta.ntiles_x) * 32;
    const unsigned box_bytes = unsigned(ta.BP) * BW * sizeof(St);
    mbar_expect_tx(bar, box_bytes * ta.nbox * BR + ta.extra_tx);
    for (int rr = 0; rr < BR; ++rr) {
        const int ys = (BR == 3) ? bc_index(y - 1 + rr, a.ny, a.bcy) : y;
        for (int b = 0; b < ta.nbox; ++b)
            tma_load_3d(stage + (size_t(rr) * ta.nbox + b) * box_bytes, &ta.tmap, x0 - HX, ys,
                        b * ta.BP, bar);
    }
}

template <class R>
__device__ __forceinline__ void lds4(const R *p, R &x, R &y, R &z, R &w)
{
    x = p[0]; y = p[1]; z = p[2]; w = p[3];
}
template <>
__device__ __forceinline__ void lds4<float>(const float *p, float &x, float &y, float &z, float &w)
{
    const float4 v = *reinterpret_cast<const float4 *>(p);
    x = v.x; y = v.y; z = v.z; w = v.w;
}

template <class St, class R, class LR, int N, int P, bool TWO_D, bool FULL>
__global__ void __launch_bounds__(kMaxWarps * 32) rlbm_step_tma(const __grid_constant__ TmaArgs ta)
{
    constexpr int NC = 2 * N + 1;
    constexpr int TW = tab_width(N);
    constexpr int HX = StageGeom<St>::HX, BW = StageGeom<St>::BW;
    constexpr int BR = TWO_D ? 3 : 1;
    const KernelArgs &a = ta.a;
    extern __shared__ __align__(16) unsigned char smem_tma[];
    // TMA destinations must be 128-byte aligned: align the base (the host adds 1 KB)
    unsigned char *smem_raw = smem_tma + ((1024u - (smem_u32(smem_tma) & 1023u)) & 1023u);
    const int lane = threadIdx.x, g = threadIdx.y, G = blockDim.y;
    const int tid = g * 32 + lane, nthr = G * 32;
    const int npop = a.K * (N + 1);
    const int r = g / a.Gs, q = g % a.Gs;
    const int i0 = r * a.K + q * a.P;
    const int pc = FULL ? P : min(a.P, a.K - q * a.P);
    const long long S = a.S;

    // shared memory carve-up (the host sizes it with the same TmaSmem)
    const size_t stage_bytes = size_t(ta.stage_bytes);
    const TmaSmem L(stage_bytes, G, P, N, sizeof(R), sizeof(LR));
    unsigned char *stages = smem_raw;
    R *tab = reinterpret_cast<R *>(smem_raw + L.tab);                    // [G][P][TW]
    LR *red2 = reinterpret_cast<LR *>(smem_raw + L.red);                 // [2][5][G][32]
    unsigned long long *bars = reinterpret_cast<unsigned long long *>(smem_raw + L.bars);

    // per-warp slice of the population table
    const R *gtab = reinterpret_cast<const R *>(a.poptab);
    for (int e = lane; e < P * TW; e += 32) {
        const int k = e / TW;
        tab[(g * P) * TW + e] = (k < pc) ? gtab[(size_t)(i0 + k) * TW + (e % TW)] : R(0);
    }
    const unsigned long long mx = __ldg(a.masks + 2 * g), my = __ldg(a.masks + 2 * g + 1);
    if (tid == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
        fence_proxy_async();
    }
    __syncthreads();

    const unsigned step_seed = (sizeof(St) <= 4) ? mix32(__ldcg(a.ctr) * 0x9E3779B9u + 1u) : 0u;
    const int first = blockIdx.x, stride = gridDim.x;
    if (tid == 0) {
        if (first < ta.ntiles) issue_tile<St>(ta, stages, &bars[0], first, BR);
        if (first + stride < ta.ntiles) issue_tile<St>(ta, stages + stage_bytes, &bars[1], first + stride, BR);
    }
    const R *mytab = tab + (g * P) * TW;
    const St *fin = reinterpret_cast<const St *>(a.fin);
    St *fout = reinterpret_cast<St *>(a.fout);
    const int nissued_max = ta.ntiles;
    int j = 0;
    int last_issued = (first + stride < ta.ntiles) ? 1 : 0; // local index of the last tile issued
    bool aborted = false;
    for (int t = first; t < ta.ntiles; t += stride, ++j) {
        const int st = j & 1;
        unsigned char *stage = stages + st * stage_bytes;
        const St *sf = reinterpret_cast<const St *>(stage);
        const bool timed_out = !mbar_wait_bounded(&bars[st], (j >> 1) & 1, ta.wait_cycles);
        const int y = t / ta.ntiles_x;
        const int x0 = (t % ta.ntiles_x) * 32;
        const int npad = ta.nbox * ta.BP; // populations per row slot in the stage
        if (x0 == 0 || x0 + 32 >= a.nx) {
            // the halo column beyond the grid edge: TMA filled zeros; write the
            // periodic / copy-out source value of the same row slot instead
            St *sw = reinterpret_cast<St *>(stage);
            const int right = a.nx - x0; // local index of x = nx (if within the tile)
            for (int e = tid; e < npop * BR * 2; e += nthr) {
                const int side = e & 1, rest = e >> 1;
                const int rr = rest % BR, p = rest / BR;
                int lx;
                if (side == 0) { if (x0 != 0) continue; lx = -1; }
                else { if (right > 32) continue; lx = right; }
                const int ys = (BR == 3) ? bc_index(y - 1 + rr, a.ny, a.bcy) : y;
                const int xs = bc_index(x0 + lx, a.nx, a.bcx);
                sw[((size_t)rr * npad + p) * BW + HX + lx] = fin[(size_t)p * S + (size_t)ys * a.nx + xs];
            }
        }
        if (__syncthreads_or(timed_out)) { aborted = true; break; }

        const bool act = x0 + lane < a.nx;
        const int x = act ? x0 + lane : a.nx - 1;
        // pass 1: stream from shared memory
        R fs[P];
        R s0[2] = {R(0), R(0)}, sc[2] = {R(0), R(0)}, ss[2] = {R(0), R(0)};
        R scc[2] = {R(0), R(0)}, scs[2] = {R(0), R(0)};
        {
            const int cx = HX + (x - x0); // column of site x in the stage (lanes past nx repeat the last site)
            const size_t rowstride = size_t(npad) * BW;
            const St *base = sf + (TWO_D ? rowstride : 0) + (size_t)i0 * BW;
#pragma unroll
            for (int k = 0; k < P; ++k) {
                if (k < pc) {
                    const St *pk = base + k * BW;
                    const int cxs = ((mx >> k) & 1ull) ? cx - 1 : cx + 1;
                    R c, s, cc2, cs2;
                    lds4<R>(mytab + k * TW, c, s, cc2, cs2);
                    const R f00 = Io<St, R>::lds(pk + cx), f01 = Io<St, R>::lds(pk + cxs);
                    R v = f00 + fabs(c) * (f01 - f00);
                    if (TWO_D) {
                        const St *pr = pk + (((my >> k) & 1ull) ? -(long)rowstride : (long)rowstride);
                        const R f10 = Io<St, R>::lds(pr + cx), f11 = Io<St, R>::lds(pr + cxs);
                        const R hi = f10 + fabs(c) * (f11 - f10);
                        v = v + fabs(s) * (hi - v);
                    }
                    fs[k] = v;
                    s0[k & 1] += v;
                    sc[k & 1] += c * v;
                    ss[k & 1] += s * v;
                    scc[k & 1] += cc2 * v;
                    scs[k & 1] += cs2 * v;
                }
            }
        }
        LR *red = red2 + (j & 1) * 5 * G * 32;
        if (a.collide) {
            red[(0 * G + g) * 32 + lane] = LR(s0[0] + s0[1]);
            red[(1 * G + g) * 32 + lane] = LR(sc[0] + sc[1]);
            red[(2 * G + g) * 32 + lane] = LR(ss[0] + ss[1]);
            red[(3 * G + g) * 32 + lane] = LR(scc[0] + scc[1]);
            red[(4 * G + g) * 32 + lane] = LR(scs[0] + scs[1]);
        }
        __syncthreads();
        // the stage is free: refill it with the tile two ahead
        if (tid == 0 && t + 2 * stride < nissued_max) {
            fence_proxy_async();
            issue_tile<St>(ta, stage, &bars[st], t + 2 * stride, BR);
            last_issued = j + 2;
        }
        const long long site = (long long)y * a.nx + x;
        St *obase = fout + (long long)i0 * S + site;
        if (!a.collide) {
            if (act) {
#pragma unroll
                for (int k = 0; k < P; ++k)
                    if (k < pc) Io<St, R>::st(obase + (long long)k * S, fs[k]);
            }
            continue;
        }
        // every warp: the Landau frame of the tile's 32 sites and its own shell's
        // equilibrium coefficients (no second barrier; red alternates between tiles)
        LR m[8];
        fold_moments<N, LR>(a, red, G, lane, m);
        LR n, eps, U0, Ux, Uy;
        const bool ok = site_landau<St, LR>(m, n, eps, U0, Ux, Uy);
        const LR T = eps / (LR(2) * n);
        if (!ok && act && g == 0) atomicOr(a.status, 1);
        R cr[NC];
        shell_coefficients<N, LR, R>(a, r, n, T, U0, Ux, Uy, cr);
        const LR itau = Par<LR>::inv_tau(a);
        const R o0 = R(U0 * itau), o1 = R(Ux * itau), o2 = R(Uy * itau);
        constexpr bool kSR = sizeof(St) <= 4; // FP32 and 16-bit stores round stochastically
        unsigned rng = 0;
        if (kSR) rng = mix32(unsigned(site) * 64u + unsigned(g) ^ step_seed);
#pragma unroll
        for (int k = 0; k < P; ++k) {
            if (k < pc) {
                const R *tk = mytab + k * TW;
                R c, s, e0, e1;
                lds4<R>(tk, c, s, e0, e1);
                R E[TW - 4];
#pragma unroll
                for (int u = 0; u < TW - 4; u += 4) lds4<R>(tk + 4 + u, E[u], E[u + 1], E[u + 2], E[u + 3]);
                R feq = cr[0] * E[0];
#pragma unroll
                for (int u = 1; u < NC; ++u) feq += cr[u] * E[u];
                const R om = o0 - o1 * c - o2 * s;
                if (act) relax_store<St, R>(obase + (long long)k * S, fs[k], om, feq, rng);
            }
        }
    }
    if (sizeof(St) <= 4) {
        __syncthreads();
        if (tid == 0) advance_launch_counter(a.ctr, gridDim.x);
    }
    if (aborted && tid == 0) {
        atomicOr(a.status, 2);
        // drain copies still in flight (bounded)
        for (int jj = j; jj <= last_issued; ++jj)
            mbar_wait_bounded(&bars[jj & 1], (jj >> 1) & 1, ta.wait_cycles);
    }
}

} // namespace rlbmk
