// Batched persistent form: many independent RLBM problems of uneven size,
// order N and angle count K, advanced nsteps time steps by ONE kernel launch.
//
// Work units: a unit is T tiles (T = 6 / G_p, G_p = warps per tile of problem
// p) of 32 consecutive sites of one row of one problem; the CTA (6 warps)
// processes them side by side, warp group t on tile t.  Units are taken from
// an atomic counter per step (dynamic load balance over uneven problems).
// Between time steps all CTAs meet at a grid barrier (arrive counter +
// generation word, every wait bounded by a clock deadline); the last CTA to
// arrive resets the next step's work counter and releases the others.  The
// launch is cooperative, so all CTAs are co-resident.
//
// Per tile the arithmetic is that of the per-tile kernel (rlbm_device.cuh):
// bilinear pull from global memory (L2-coherent loads, since the values were
// written by other CTAs earlier in the same launch), per-warp angular sums,
// the Landau frame and the equilibrium (Sec. 2.2) -- FP64 storage: every warp
// solves the frame and its own shell's equilibrium in FP64; FP32 storage: the
// group solves each site once in double-float, split over its warps by sample
// direction (site_split_dd), and every warp combines its shell's coefficients
// from the shared sums --
// and relaxation; FP32 stores round stochastically (relax_store).
#pragma once

#include "rlbm_device.cuh"

namespace rlbmk {

// One tile of one problem, computed by a group of G warps (gw = warp in group).
template <class St, class R, class LR, int N, bool TWO_D>
__device__ __forceinline__ void batch_tile(const KernelArgs &a, const St *fin, St *fout, int tile,
                                           int ntiles_x, bool valid, int gw, int G, int lane,
                                           LR *red, float *wdd, unsigned seed)
{
    // FP32 storage: the per-site part once per site in double-float, split over
    // the group's warps (site_split_dd); wdd holds the group's [2 (N+1)^2 + 3][32]
    // sums and U^a / tau, then the frame and the partial sums
    constexpr bool DDS = (sizeof(St) == 4) && (sizeof(LR) == 4);
    constexpr int W = (N + 1) * (N + 1);
    constexpr int P = 32;
    constexpr int NC = 2 * N + 1;
    constexpr int TW = tab_width(N);
    const int y = valid ? tile / ntiles_x : 0;
    const int x0 = valid ? (tile % ntiles_x) * 32 : 0;
    const bool act = valid && (x0 + lane < a.nx);
    const int x = min(x0 + lane, a.nx - 1);
    const int r = gw / a.Gs, q = gw % a.Gs;
    const int i0 = r * a.K + q * a.P;
    const int pc = min(a.P, a.K - q * a.P);
    const long long S = a.S;
    const R *tab = reinterpret_cast<const R *>(a.poptab) + (long long)i0 * TW;

    R fs[P];
    R s0 = R(0), sc = R(0), ss = R(0), scc = R(0), scs = R(0);
    const int xm = bc_index(x - 1, a.nx, a.bcx), xp = bc_index(x + 1, a.nx, a.bcx);
    const int ym = TWO_D ? bc_index(y - 1, a.ny, a.bcy) : y;
    const int yp = TWO_D ? bc_index(y + 1, a.ny, a.bcy) : y;
    const unsigned long long mx = __ldg(a.masks + 2 * gw), my = __ldg(a.masks + 2 * gw + 1);
    const St *base = fin + (long long)i0 * S + (long long)y * a.nx;
    const long long dym = (long long)(ym - y) * a.nx, dyp = (long long)(yp - y) * a.nx;
#pragma unroll
    for (int k = 0; k < P; ++k) {
        if (k < pc) {
            const St *pk = base + (long long)k * S;
            const int xs = ((mx >> k) & 1ull) ? xm : xp;
            R c, s, cc, cs;
            ld4<R>(tab + k * TW, c, s, cc, cs);
            // L2-coherent loads: other CTAs wrote these values in the previous step of
            // this same launch, and L1 is not coherent across CTAs
            const R f00 = Io<St, R>::ldcg(pk + x), f01 = Io<St, R>::ldcg(pk + xs);
            R v = f00 + fabs(c) * (f01 - f00);
            if (TWO_D) {
                const long long dy = ((my >> k) & 1ull) ? dym : dyp;
                const R f10 = Io<St, R>::ldcg(pk + dy + x), f11 = Io<St, R>::ldcg(pk + dy + xs);
                const R hi = f10 + fabs(c) * (f11 - f10);
                v = v + fabs(s) * (hi - v);
            }
            fs[k] = v;
            s0 += v;
            sc += c * v;
            ss += s * v;
            scc += cc * v;
            scs += cs * v;
        }
    }
    const long long site = (long long)y * a.nx + x;
    St *obase = fout + (long long)i0 * S + site;
    if (!a.collide) { // uniform across the CTA: the unit's tiles share one problem
        if (act) {
#pragma unroll
            for (int k = 0; k < P; ++k)
                if (k < pc) Io<St, R>::st(obase + (long long)k * S, fs[k]);
        }
        __syncthreads();
        return;
    }
    red[(0 * G + gw) * 32 + lane] = LR(s0);
    red[(1 * G + gw) * 32 + lane] = LR(sc);
    red[(2 * G + gw) * 32 + lane] = LR(ss);
    red[(3 * G + gw) * 32 + lane] = LR(scc);
    red[(4 * G + gw) * 32 + lane] = LR(scs);
    __syncthreads();
    R cr[NC];
    R o0, o1, o2;
    if constexpr (DDS) {
        site_split_dd<N, 32>(a, reinterpret_cast<const float *>(red), G, gw * 32 + lane, G * 32, act, wdd,
                             wdd + (2 * W + 3) * 32, wdd + (2 * W + 3 + kSplitFrameRows(N)) * 32);
        shell_from_sums_dd<N>(a, r, wdd + lane, 32, cr);
        o0 = wdd[(2 * W + 0) * 32 + lane];
        o1 = wdd[(2 * W + 1) * 32 + lane];
        o2 = wdd[(2 * W + 2) * 32 + lane];
    } else {
        LR m[8];
        fold_moments<N, LR>(a, red, G, lane, m);
        LR n, eps, U0, Ux, Uy;
        const bool ok = site_landau<St, LR>(m, n, eps, U0, Ux, Uy);
        const LR T = eps / (LR(2) * n);
        if (!ok && act && gw == 0) atomicOr(a.status, 1);
        shell_coefficients<N, LR, R>(a, r, n, T, U0, Ux, Uy, cr);
        const LR itau = Par<LR>::inv_tau(a);
        o0 = R(U0 * itau);
        o1 = R(Ux * itau);
        o2 = R(Uy * itau);
    }
    unsigned rng = mix32(unsigned(y * a.nx + x) * 64u + unsigned(gw) ^ seed);
#pragma unroll
    for (int k = 0; k < P; ++k) {
        if (k < pc) {
            const R *t = tab + k * TW;
            R c, s, e0, e1;
            ld4<R>(t, c, s, e0, e1);
            R E[TW - 4];
#pragma unroll
            for (int u = 0; u < TW - 4; u += 4) ld4<R>(t + 4 + u, E[u], E[u + 1], E[u + 2], E[u + 3]);
            R feq = cr[0] * E[0];
#pragma unroll
            for (int t2 = 1; t2 < NC; ++t2) feq += cr[t2] * E[t2];
            const R om = o0 - o1 * c - o2 * s;
            if (act) relax_store<St, R>(obase + (long long)k * S, fs[k], om, feq, rng);
        }
    }
    __syncthreads(); // red is reused by the next unit
}

// Grid barrier with a bounded wait.  Returns false (and sets status bit 1)
// when the wait ran out; the caller then stops.
__device__ __forceinline__ bool batch_grid_barrier(const BatchArgs &b, int next_step)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        volatile unsigned *gen = b.sync + 1;
        const unsigned g0 = *gen;
        __threadfence();
        const unsigned arrived = atomicAdd(&b.sync[0], 1u) + 1u;
        int ok = 1;
        if (arrived == gridDim.x + b.barrier_extra) {
            b.sync[0] = 0u;
            b.sync[2 + (next_step & 1)] = 0u; // work counter of the next step
            __threadfence();
            atomicAdd(&b.sync[1], 1u);
        } else {
            const long long t0 = clock64();
            while (*gen == g0) {
                if (clock64() - t0 > b.wait_cycles) {
                    ok = 0;
                    atomicOr(b.status, 2);
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// FP32 storage: at most 56 registers, six 6-warp CTAs per SM (FP64: no bound).  On the
// 256-problem set 4, 5, 6 and 8 CTAs per SM gave 62.9, 57.1, 52.5 and 59.6 ms per time
// step (more warps hide the per-site chain; at 8 the spills win).
template <class St, class R, class LR, int N>
__global__ void __launch_bounds__(kBatchWarps * 32, sizeof(St) == 4 ? 6 : 1) rlbm_batch_kernel(const BatchArgs b)
{
    __shared__ LR red_all[kBatchWarps * 5 * 32];
    // FP32 storage: the double-float per-site sums of each tile of a unit
    // (at most kBatchWarps / (N + 1) tiles per unit)
    constexpr bool DDS = (sizeof(St) == 4) && (sizeof(LR) == 4);
    constexpr int kRows = 2 * (N + 1) * (N + 1) + 3 + kSplitFrameRows(N) + (N + 1) * 2 * (N + 1) * (N + 1);
    __shared__ float wdd_all[DDS ? (kBatchWarps / (N + 1)) * kRows * 32 : 1];
    __shared__ int s_unit;
    const int lane = threadIdx.x, g = threadIdx.y;
    for (int step = 0; step < b.nsteps; ++step) {
        unsigned *work = b.sync + 2 + (step & 1);
        for (;;) {
            if (lane == 0 && g == 0) s_unit = int(atomicAdd(work, 1u));
            __syncthreads();
            const int u = s_unit;
            __syncthreads();
            if (u >= b.nunits) break;
            const BatchUnit bu = b.units[u];
            const KernelArgs &a = b.probs[bu.prob];
            const int tpu = b.tiles_per_unit[bu.prob];
            const int G = kBatchWarps / tpu;
            const int grp = g / G, gw = g % G;
            const int tile = bu.tile0 + grp;
            const bool valid = tile < b.ntiles[bu.prob];
            const int par = (b.parity0[bu.prob] + step) & 1;
            const St *fin = reinterpret_cast<const St *>(par ? a.fout : a.fin);
            St *fout = reinterpret_cast<St *>(par ? const_cast<void *>(a.fin) : a.fout);
            LR *red = red_all + grp * (G * 5 * 32);
            float *wdd = DDS ? wdd_all + grp * kRows * 32 : nullptr;
            // stochastic rounding of FP32 stores: seeded by the problem's launch
            // counter plus the step (the host advances the counters by nsteps after
            // the launch, batch_advance_kernel)
            const unsigned seed = mix32((__ldcg(a.ctr) + unsigned(step)) * 0x9E3779B9u + 1u);
            if (a.ny > 1)
                batch_tile<St, R, LR, N, true>(a, fin, fout, tile, b.ntiles_x[bu.prob], valid, gw, G, lane, red,
                                               wdd, seed);
            else
                batch_tile<St, R, LR, N, false>(a, fin, fout, tile, b.ntiles_x[bu.prob], valid, gw, G, lane, red,
                                                wdd, seed);
        }
        if (step + 1 < b.nsteps && !batch_grid_barrier(b, step + 1)) return;
    }
}

// After a launch of nsteps steps: every problem's launch counter (the seed of
// its stochastic rounding) advances by nsteps, as nsteps single launches would.
__global__ void batch_advance_kernel(const KernelArgs *probs, int n, int nsteps)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) probs[i].ctr[0] += unsigned(nsteps);
}

} // namespace rlbmk
