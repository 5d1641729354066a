// Two-sites-per-lane form of the fused RLBM step (arXiv 2011.06856, Sec. 2.2)
// for FP32 arithmetic (FP32, FP16 or BF16 storage).
//
// A CTA owns 64 consecutive sites of one grid row and all N_pop populations
// of them; lane l holds sites x0 + 2l and x0 + 2l + 1 as one packed pair, so
// that every per-population operation is one Blackwell f32x2 instruction
// (add / sub / mul / fma .f32x2) for two sites, every population-table load
// serves two sites, and the centre values of a pair are one 8-byte load.
// Warp g owns PP populations of energy shell r = g / Gs.
//
//   pass 1  bilinear pull (Eqs. streaming, interpolation): the pair pulled
//           from x - sgn(v_x) is (f[x0+2l-1], f[x0+2l]) or (f[x0+2l+1],
//           f[x0+2l+2]), i.e. one neighbour value plus one of the centre
//           pair; five per-shell angular sums S0, Sc, Ss, Scc, Scs of f*;
//   site    two warps (one site per lane) fold the sums of all warps into
//           N^a and T^ab (Eq. discrete_sum_moments), solve the Landau frame
//           (landau_fast), and form the shell-independent part of the
//           truncated-equilibrium coefficients (Eqs. mj-projection-coefficients,
//           mj-feq-expansion-truncated) once per site, into shared memory;
//           every warp then combines them into its own shell's coefficients;
//   pass 2  f^eq_i and the relaxation f <- f* + omega_i (f^eq - f*)
//           (Eq. discrete-rbe), one paired store per population.
//
// Per-population constants come from a pair table (each constant twice, so a
// 16-byte load gives two packed operands): (c,c,s,s), (|c|,|c|,|s|,|s|) and
// (w',w',0,0), w' = w_i / alpha_i in stored units.  The equilibrium of shell
// r at angle theta is a trigonometric polynomial of degree N; with
// cos 2t = 2 cc - 1, sin 2t = 2 cs, cos 3t = 4 c cc - 3 c, sin 3t = 4 s cc - s
// it becomes w' (b0 + b1 c + b2 s + b3 cc + b4 cs [+ b5 c cc + b6 s cc]),
// the b's formed once per site from the Fourier coefficients, so that the
// per-population basis is a few packed products of c and s.
//
// BULK form (row pitch a whole number of 16-byte chunks): on interior tiles
// pass 1 reads shared memory.  Each warp streams its own populations through
// kPairDepth slots, kPairChunk populations per slot, two slots ahead of the
// arithmetic: one lane per (population, row) issues one cp.async.bulk of the
// row segment [x0 - 16 bytes, x0 + 64 sites + 16 bytes) (the row y and, in
// 2D, the boundary-mapped row y - sgn(v_y)), and the slot's mbarrier counts
// the bytes.  Every wait is bounded (wait_cycles): on expiry the warp sets
// bit 1 of the status word, waits (bounded) for its copies in flight, skips
// its stores and still takes part in the CTA barriers.  Tiles touching the
// x boundary use plain loads.
#pragma once

#include "rlbm_device.cuh"

namespace rlbmk {

__device__ __forceinline__ float2 f2sub(float2 a, float2 b)
{
    unsigned long long ua, ub, ud;
    memcpy(&ua, &a, 8);
    memcpy(&ub, &b, 8);
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(ud) : "l"(ua), "l"(ub));
    float2 d;
    memcpy(&d, &ud, 8);
    return d;
}
__device__ __forceinline__ float2 f2(float x, float y) { return make_float2(x, y); }

__device__ __forceinline__ unsigned sptr(const void *p) { return static_cast<unsigned>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ bool pbar_try_wait(unsigned bar, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(bar), "r"(parity), "r"(kWaitHintNs)
                 : "memory");
    return ok != 0;
}

// bounded wait for the phase of the given parity; false when the bound ran out
__device__ __forceinline__ bool pbar_wait(unsigned bar, unsigned parity, long long max_cycles)
{
    const long long t0 = clock64();
    while (!pbar_try_wait(bar, parity))
        if (clock64() - t0 > max_cycles) return false;
    return true;
}

template <class St> __device__ __forceinline__ float2 lds2(const St *p);
template <> __device__ __forceinline__ float2 lds2<float>(const float *p) { return *reinterpret_cast<const float2 *>(p); }
template <> __device__ __forceinline__ float2 lds2<__half>(const __half *p)
{
    return __half22float2(*reinterpret_cast<const __half2 *>(p));
}
template <> __device__ __forceinline__ float2 lds2<__nv_bfloat16>(const __nv_bfloat16 *p)
{
    const unsigned u = *reinterpret_cast<const unsigned *>(p);
    return make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xFFFF0000u));
}
template <class St> __device__ __forceinline__ float lds1(const St *p);
template <> __device__ __forceinline__ float lds1<float>(const float *p) { return *p; }
template <> __device__ __forceinline__ float lds1<__half>(const __half *p) { return __half2float(*p); }
template <> __device__ __forceinline__ float lds1<__nv_bfloat16>(const __nv_bfloat16 *p)
{
    return __bfloat162float(*p);
}


// paired storage access: two consecutive sites (the first at an even index)
template <class St> struct PIo;
// Loads are volatile asm so that the compiler issues a chunk's loads in
// program order before the arithmetic that uses them (many in flight).
template <> struct PIo<float> {
    static __device__ __forceinline__ float2 ld2(const float *p)
    {
        float2 v;
        asm volatile("ld.global.nc.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p));
        return v;
    }
    static __device__ __forceinline__ float ld1(const float *p)
    {
        float v;
        asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(v) : "l"(p));
        return v;
    }
    static __device__ __forceinline__ void st2(float *p, float2 v, unsigned &) { *reinterpret_cast<float2 *>(p) = v; }
};
template <> struct PIo<__half> {
    static __device__ __forceinline__ float2 ld2(const __half *p)
    {
        unsigned u;
        asm volatile("ld.global.nc.b32 %0, [%1];" : "=r"(u) : "l"(p));
        __half2 h;
        memcpy(&h, &u, 4);
        return __half22float2(h);
    }
    static __device__ __forceinline__ float ld1(const __half *p)
    {
        unsigned short u;
        asm volatile("ld.global.nc.b16 %0, [%1];" : "=h"(u) : "l"(p));
        return __half2float(__ushort_as_half(u));
    }
    static __device__ __forceinline__ void st2(__half *p, float2 v, unsigned &rng)
    {
        // stochastic rounding of both values (13 dropped mantissa bits)
        const __half h0 = __float2half_rz(__uint_as_float(__float_as_uint(v.x) + (lcg_next(rng) >> 19)));
        const __half h1 = __float2half_rz(__uint_as_float(__float_as_uint(v.y) + (lcg_next(rng) >> 19)));
        const unsigned u = unsigned(__half_as_ushort(h0)) | (unsigned(__half_as_ushort(h1)) << 16);
        *reinterpret_cast<unsigned *>(p) = u;
    }
};
template <> struct PIo<__nv_bfloat16> {
    static __device__ __forceinline__ float2 ld2(const __nv_bfloat16 *p)
    {
        unsigned u;
        asm volatile("ld.global.nc.b32 %0, [%1];" : "=r"(u) : "l"(p));
        return make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xFFFF0000u));
    }
    static __device__ __forceinline__ float ld1(const __nv_bfloat16 *p)
    {
        unsigned short u;
        asm volatile("ld.global.nc.b16 %0, [%1];" : "=h"(u) : "l"(p));
        return __uint_as_float(unsigned(u) << 16);
    }
    static __device__ __forceinline__ void st2(__nv_bfloat16 *p, float2 v, unsigned &rng)
    {
        // stochastic rounding of both values (16 dropped mantissa bits)
        const unsigned b0 = __float_as_uint(v.x) + (lcg_next(rng) >> 16);
        const unsigned b1 = __float_as_uint(v.y) + (lcg_next(rng) >> 16);
        *reinterpret_cast<unsigned *>(p) = (b0 >> 16) | (b1 & 0xFFFF0000u);
    }
};

// The relaxation f* + om (f^eq - f*) of two sites (packed), rounded
// stochastically to FP32 (relax_sr in rlbm_device.cuh, for both sites at
// once): rb gives 16 random bits per site.
__device__ __forceinline__ float2 relax_pair_sr(float2 fs, float2 om, float2 feq, unsigned rb)
{
    const float2 d = f2sub(feq, fs);
    const float2 r = __ffma2_rn(om, d, fs);
    const float2 e = __ffma2_rn(om, d, f2sub(fs, r));
    const float2 ulp = __fmul2_rn(f2(__uint_as_float(__float_as_uint(r.x) & 0x7f800000u),
                                     __uint_as_float(__float_as_uint(r.y) & 0x7f800000u)),
                                  f2(1.1920928955078125e-7f, 1.1920928955078125e-7f));
    const float2 u = __fadd2_rn(f2(__uint_as_float(0x3f800000u | ((rb & 0xffffu) << 7)),
                                   __uint_as_float(0x3f800000u | ((rb >> 16) << 7))),
                                f2(-1.5f, -1.5f));
    return __fadd2_rn(r, __ffma2_rn(u, ulp, e));
}

// 32 random bits from the thread's LCG stream: the high halves of two draws
// (the low bits of a power-of-two LCG have short periods; each 16-bit half
// of the result feeds the rounding of one site)
__device__ __forceinline__ unsigned next_bits2(unsigned &rng)
{
    const unsigned a = lcg_next(rng), b = lcg_next(rng);
    return __byte_perm(a, b, 0x7632);
}

// The per-site part for site s of the tile with FP32 accumulation (16-bit
// storage): moments from the warps' angular sums, the Landau frame in FP32,
// refined in double-float where T^ab is near-degenerate
// (landau_f32_adaptive), and the shell-independent part of the
// equilibrium coefficients (the boosted-direction sums acc, weighted by
// n T^(k-1)), written to sres[row 64 + s]; then U^a / tau at rows
// (N+1)^2 + 0..2.  Every warp forms its own shell's coefficients from these.
template <int N>
__device__ __forceinline__ void pair_site_solve(const KernelArgs &a, const float *red, int G, int s, bool act,
                                                float *sres)
{
    constexpr int NC = 2 * N + 1;
    const float *sh = reinterpret_cast<const float *>(a.shelltab);
    float m[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) m[u] = a.off_f[u];
#pragma unroll
    for (int rr = 0; rr <= N; ++rr) {
        float p0 = 0.f, pc = 0.f, ps = 0.f, pcc = 0.f, pcs = 0.f;
        for (int qq = 0; qq < a.Gs; ++qq) {
            const int w = rr * a.Gs + qq;
            p0 += red[(0 * G + w) * kPairSites + s];
            pc += red[(1 * G + w) * kPairSites + s];
            ps += red[(2 * G + w) * kPairSites + s];
            pcc += red[(3 * G + w) * kPairSites + s];
            pcs += red[(4 * G + w) * kPairSites + s];
        }
        const float f1 = __ldg(sh + 2 * rr), f2v = __ldg(sh + 2 * rr + 1);
        m[0] += f1 * p0;
        m[1] += f1 * pc;
        m[2] += f1 * ps;
        m[3] += f2v * p0;
        m[4] += f2v * pc;
        m[5] += f2v * ps;
        m[6] += f2v * pcc;
        m[7] += f2v * pcs;
    }
    float n, eps, U0, Ux, Uy;
    const bool ok = landau_f32_adaptive(m, n, eps, U0, Ux, Uy);
    const float T = __fdividef(eps, 2.f * n);
    if (!ok && act) atomicOr(a.status, 1);
    // boosted rest-frame directions: acc_{m,k} = sum_j q0^(k-m) z^m (as in shell_coefficients)
    float accr[N + 1][N + 1], acci[N + 1][N + 1];
#pragma unroll
    for (int mm = 0; mm <= N; ++mm)
#pragma unroll
        for (int k = 0; k <= N; ++k) { accr[mm][k] = 0.f; acci[mm][k] = 0.f; }
    const float inv1g = __fdividef(1.f, 1.f + U0);
#pragma unroll
    for (int j = 0; j <= N; ++j) {
        const float cj = a.smp_cf[j], sj = a.smp_sf[j];
        const float un = Ux * cj + Uy * sj;
        const float q0 = U0 + un;
        const float h = 1.f + un * inv1g;
        const float zr = cj + Ux * h, zi = sj + Uy * h;
        float qp[N + 1], pr[N + 1], pi[N + 1];
        qp[0] = 1.f;
        pr[0] = 1.f;
        pi[0] = 0.f;
#pragma unroll
        for (int t = 1; t <= N; ++t) {
            qp[t] = qp[t - 1] * q0;
            pr[t] = pr[t - 1] * zr - pi[t - 1] * zi;
            pi[t] = pr[t - 1] * zi + pi[t - 1] * zr;
        }
#pragma unroll
        for (int mm = 0; mm <= N; ++mm)
#pragma unroll
            for (int k = mm; k <= N; ++k) {
                accr[mm][k] += qp[k - mm] * pr[mm];
                acci[mm][k] += qp[k - mm] * pi[mm];
            }
    }
    float tk[N + 1];
    tk[0] = __fdividef(n, T);
#pragma unroll
    for (int k = 1; k <= N; ++k) tk[k] = (k == 1) ? n : tk[k - 1] * T;
    // shell-independent part of the coefficients, T^(k-1)-weighted: w_{m,k} = tk[k] acc_{m,k}
    // (rows: Re for m = 0..N, k = m..N, then Im for m = 1..N; then U^a / tau)
    int row = 0;
#pragma unroll
    for (int mm = 0; mm <= N; ++mm)
#pragma unroll
        for (int k = mm; k <= N; ++k) sres[(row++) * kPairSites + s] = tk[k] * accr[mm][k];
#pragma unroll
    for (int mm = 1; mm <= N; ++mm)
#pragma unroll
        for (int k = mm; k <= N; ++k) sres[(row++) * kPairSites + s] = tk[k] * acci[mm][k];
    const float itau = a.inv_tau_f;
    sres[((N + 1) * (N + 1) + 0) * kPairSites + s] = U0 * itau;
    sres[((N + 1) * (N + 1) + 1) * kPairSites + s] = Ux * itau;
    sres[((N + 1) * (N + 1) + 2) * kPairSites + s] = Uy * itau;
}

// Shell r's equilibrium coefficients for the lane's two sites, in the basis
// (1, c, s, cc, cs [, c cc, s cc]) of the pair kernels' second pass, and the
// relaxation factors o = U^a / tau.  The Fourier coefficients are
// C_{r,m} = sum_k R'[r][m][k] w_{m,k} (Eq. mj-feq-expansion-truncated in the
// per-shell Fourier form); with cos 2t = 2 cc - 1, sin 2t = 2 cs,
// cos 3t = 4 c cc - 3 c and sin 3t = 4 s cc - s they become cr.  DD: the
// w_{m,k} are double-floats (pair_site_solve_dd) and the radial sums and the
// change of basis run in packed double-float, rounded to FP32 at the end;
// otherwise everything is packed FP32.
template <int N, bool DD>
__device__ __forceinline__ void pair_shell_coefficients(const KernelArgs &a, int r, const float *sres, int lane,
                                                        float2 *cr, float2 &o0, float2 &o1, float2 &o2)
{
    static_assert(N == 2 || N == 3, "the polynomial basis below is written for N = 2, 3");
    constexpr int NC = 2 * N + 1;
    constexpr int W = (N + 1) * (N + 1);
    const float2 *sres2 = reinterpret_cast<const float2 *>(sres);
    if constexpr (DD) {
        const float2 *rt = a.rtab2 + r * (N + 1) * (N + 1);
        df2 cf[NC];
        int row = 0;
#pragma unroll
        for (int mm = 0; mm <= N; ++mm) {
            df2 acc{f2(0.f, 0.f), f2(0.f, 0.f)};
#pragma unroll
            for (int k = mm; k <= N; ++k, ++row) {
                const float2 t = __ldg(rt + mm * (N + 1) + k);
                const df2 w{sres2[row * 32 + lane], sres2[(W + row) * 32 + lane]};
                acc = acc + w * dd(t.x, t.y);
            }
            if (mm == 0)
                cf[0] = acc - df2{f2(a.feq_off_f, a.feq_off_f), f2(a.feq_off_l, a.feq_off_l)};
            else
                cf[2 * mm - 1] = acc;
        }
#pragma unroll
        for (int mm = 1; mm <= N; ++mm) {
            df2 acc{f2(0.f, 0.f), f2(0.f, 0.f)};
#pragma unroll
            for (int k = mm; k <= N; ++k, ++row) {
                const float2 t = __ldg(rt + mm * (N + 1) + k);
                const df2 w{sres2[row * 32 + lane], sres2[(W + row) * 32 + lane]};
                acc = acc + w * dd(t.x, t.y);
            }
            cf[2 * mm] = acc;
        }
        df2 c1 = cf[1], c2 = cf[2];
        if (N == 3) {
            c1 = c1 - scale(cf[NC - 2], 3.f);
            c2 = c2 - cf[NC - 1];
            cr[NC - 2] = to_float2(scale(cf[NC - 2], 4.f));
            cr[NC - 1] = to_float2(scale(cf[NC - 1], 4.f));
        }
        cr[0] = to_float2(cf[0] - cf[3]);
        cr[1] = to_float2(c1);
        cr[2] = to_float2(c2);
        cr[3] = to_float2(scale(cf[3], 2.f));
        cr[4] = to_float2(scale(cf[4], 2.f));
    } else {
        const float *rt = reinterpret_cast<const float *>(a.rtab) + r * (N + 1) * (N + 1);
        float2 cf[NC];
        int row = 0;
#pragma unroll
        for (int mm = 0; mm <= N; ++mm) {
            float2 acc = f2(0.f, 0.f);
#pragma unroll
            for (int k = mm; k <= N; ++k) {
                const float w = __ldg(rt + mm * (N + 1) + k);
                acc = __ffma2_rn(f2(w, w), sres2[(row++) * 32 + lane], acc);
            }
            if (mm == 0) cf[0] = __fadd2_rn(acc, f2(-a.feq_off_f, -a.feq_off_f));
            else cf[2 * mm - 1] = acc;
        }
#pragma unroll
        for (int mm = 1; mm <= N; ++mm) {
            float2 acc = f2(0.f, 0.f);
#pragma unroll
            for (int k = mm; k <= N; ++k) {
                const float w = __ldg(rt + mm * (N + 1) + k);
                acc = __ffma2_rn(f2(w, w), sres2[(row++) * 32 + lane], acc);
            }
            cf[2 * mm] = acc;
        }
        cr[0] = f2sub(cf[0], cf[3]);
        cr[1] = cf[1];
        cr[2] = cf[2];
        cr[3] = __fmul2_rn(f2(2.f, 2.f), cf[3]);
        cr[4] = __fmul2_rn(f2(2.f, 2.f), cf[4]);
        if (N == 3) {
            cr[1] = __ffma2_rn(f2(-3.f, -3.f), cf[NC - 2], cr[1]);
            cr[2] = f2sub(cr[2], cf[NC - 1]);
            cr[NC - 2] = __fmul2_rn(f2(4.f, 4.f), cf[NC - 2]);
            cr[NC - 1] = __fmul2_rn(f2(4.f, 4.f), cf[NC - 1]);
        }
    }
    constexpr int OR = DD ? 2 * W : W; // row of U^0 / tau
    o0 = sres2[(OR + 0) * 32 + lane];
    o1 = sres2[(OR + 1) * 32 + lane];
    o2 = sres2[(OR + 2) * 32 + lane];
}

// St: storage type; N: quadrature order; PP: populations per warp (K is a
// multiple of PP); TWO_D: ny > 1; BULK: staged pass 1 on interior tiles (row
// pitch a multiple of 16 bytes, buffers 16-byte aligned).  Requires nx even
// (paired access) and a collision (tau finite).
template <class St, int N, int PP, bool TWO_D, bool BULK>
__global__ void __launch_bounds__(kMaxWarps * 32, PP <= 16 ? 2 : 1) rlbm_pair_kernel(const KernelArgs a)
{
    constexpr int NC = 2 * N + 1;
    constexpr int PQ = 3; // float4 per population in the pair table
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x, g = threadIdx.y, G = blockDim.y;
    const int x0 = blockIdx.x * kPairSites;
    const int xl = x0 + 2 * lane;
    const bool act = xl < a.nx;
    const int xa = act ? xl : a.nx - 2;
    const int y = blockIdx.y;
    const int r = g / a.Gs, q = g % a.Gs;
    const int i0 = r * a.K + q * PP;
    const long long S = a.S;
    const St *fin = reinterpret_cast<const St *>(a.fin);
    St *fout = reinterpret_cast<St *>(a.fout);
    float *red = reinterpret_cast<float *>(smem_raw); // [5][G][64]
    float *sres = red + 5 * G * kPairSites;           // [pair_site_rows(N)][64]
    const float4 *tb = reinterpret_cast<const float4 *>(a.pairtab) + size_t(i0) * PQ;

    const int xm = bc_index(xa - 1, a.nx, a.bcx), xp = bc_index(xa + 2, a.nx, a.bcx);
    const int ym = TWO_D ? bc_index(y - 1, a.ny, a.bcy) : y;
    const int yp = TWO_D ? bc_index(y + 1, a.ny, a.bcy) : y;
    const unsigned long long mx = __ldg(a.masks + 2 * g), my = __ldg(a.masks + 2 * g + 1);
    const St *base = fin + (long long)i0 * S + (long long)y * a.nx;
    const long long dym = (long long)(ym - y) * a.nx, dyp = (long long)(yp - y) * a.nx;

    float2 fs[PP];
    float2 s0 = f2(0.f, 0.f), sc = f2(0.f, 0.f), ss = f2(0.f, 0.f), scc = f2(0.f, 0.f), scs = f2(0.f, 0.f);
    // streamed pair of population k from its centre pair C, neighbour e (row y),
    // and, in 2D, C2, e2 of the pull row; accumulates the angular sums
    auto stream_pop = [&](int k, float2 C, float e, float2 C2, float e2) {
        const float4 t0 = __ldg(tb + k * PQ), t1 = __ldg(tb + k * PQ + 1); // (c,c,s,s), (|c|,|c|,|s|,|s|)
        const bool px = (mx >> k) & 1ull; // v_x >= 0: pull from x - 1
        const float2 B = px ? f2(e, C.x) : f2(C.y, e);
        const float2 ac = f2(t1.x, t1.y);
        float2 v = __ffma2_rn(ac, f2sub(B, C), C);
        if (TWO_D) {
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
    };

    constexpr int HX = 16 / int(sizeof(St));    // halo elements on each side (16 bytes)
    constexpr int BW = kPairSites + 2 * HX;      // staged row width (elements)
    constexpr int RW = TWO_D ? 2 : 1;            // staged rows per population
    constexpr int NCH = PP / kPairChunk;         // chunks per warp
    const bool staged = BULK && x0 >= HX && x0 + kPairSites + HX <= a.nx;
    bool good = true; // every bounded wait of this warp completed
    if (staged) {
        static_assert(PP % kPairChunk == 0, "chunking");
        constexpr unsigned SLOT = unsigned(pair_slot_bytes(int(sizeof(St)), TWO_D));
        unsigned char *slots = smem_raw + pair_slots_offset(N, G) + size_t(g) * kPairDepth * SLOT;
        const unsigned bar0 = sptr(smem_raw + pair_bars_offset(N, G) + size_t(g) * kPairDepth * 8);
        if (lane == 0) {
            for (int d = 0; d < kPairDepth; ++d)
                asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8 * d) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncwarp();
        // lane j < kPairChunk * RW copies row (j % RW) of population j / RW of a chunk
        const int jk = lane / RW, jr = lane % RW;
        auto issue = [&](int c) {
            const unsigned bar = bar0 + 8 * (c % kPairDepth);
            if (lane == 0)
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
                             "r"(unsigned(kPairChunk * RW * BW * int(sizeof(St))) + a.extra_tx)
                             : "memory");
            __syncwarp();
            if (lane < kPairChunk * RW) {
                const int k = c * kPairChunk + jk;
                const long long dy = jr == 0 ? 0 : (((my >> k) & 1ull) ? dym : dyp);
                const St *src = base + (long long)k * S + dy + (x0 - HX);
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                                 sptr(slots + (c % kPairDepth) * SLOT + lane * (BW * int(sizeof(St))))),
                             "l"(src), "r"(unsigned(BW * int(sizeof(St)))), "r"(bar)
                             : "memory");
            }
        };
        int issued = 0;
        for (; issued < kPairDepth - 1 && issued < NCH; ++issued) issue(issued);
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
            if (good && issued < NCH && issued == c + kPairDepth - 1) issue(issued++);
            if (good) good = __all_sync(0xffffffffu, pbar_wait(bar0 + 8 * (c % kPairDepth), (c / kPairDepth) & 1, a.wait_cycles));
            if (!good) break;
            const St *slot = reinterpret_cast<const St *>(slots + (c % kPairDepth) * SLOT);
#pragma unroll
            for (int kk = 0; kk < kPairChunk; ++kk) {
                const int k = c * kPairChunk + kk;
                const bool px = (mx >> k) & 1ull;
                const St *ra = slot + (kk * RW) * BW + HX + 2 * lane;
                const float2 C = lds2<St>(ra);
                const float e = lds1<St>(ra + (px ? -1 : 2));
                float2 C2 = f2(0.f, 0.f);
                float e2 = 0.f;
                if (TWO_D) {
                    C2 = lds2<St>(ra + BW);
                    e2 = lds1<St>(ra + BW + (px ? -1 : 2));
                }
                stream_pop(k, C, e, C2, e2);
            }
            __syncwarp(); // the slot is refilled by a later issue
        }
        if (!good) {
            if (lane == 0) atomicOr(a.status, 2);
            // drain this warp's copies still in flight (bounded) before the CTA can exit
            for (int c = 0; c < issued; ++c) pbar_wait(bar0 + 8 * (c % kPairDepth), (c / kPairDepth) & 1, a.wait_cycles);
        }
    } else {
        // populations whose loads are in flight together (registers: 6 per population in 2D)
        constexpr int CH = TWO_D ? (PP <= 8 ? PP : (PP == 12 ? 6 : 4)) : (PP <= 16 ? PP : 8);
        static_assert(PP % CH == 0, "chunking");
#pragma unroll
        for (int c0 = 0; c0 < PP; c0 += CH) {
            float2 ca[CH], cb[TWO_D ? CH : 1];
            float ea[CH], eb[TWO_D ? CH : 1];
#pragma unroll
            for (int kk = 0; kk < CH; ++kk) {
                const int k = c0 + kk;
                const St *pk = base + (long long)k * S;
                const int xs = ((mx >> k) & 1ull) ? xm : xp;
                ca[kk] = PIo<St>::ld2(pk + xa);
                ea[kk] = PIo<St>::ld1(pk + xs);
                if (TWO_D) {
                    const long long dy = ((my >> k) & 1ull) ? dym : dyp;
                    cb[kk] = PIo<St>::ld2(pk + dy + xa);
                    eb[kk] = PIo<St>::ld1(pk + dy + xs);
                }
            }
#pragma unroll
            for (int kk = 0; kk < CH; ++kk)
                stream_pop(c0 + kk, ca[kk], ea[kk], TWO_D ? cb[kk] : f2(0.f, 0.f), TWO_D ? eb[kk] : 0.f);
        }
    }
    float2 *red2 = reinterpret_cast<float2 *>(red);
    red2[(0 * G + g) * 32 + lane] = s0;
    red2[(1 * G + g) * 32 + lane] = sc;
    red2[(2 * G + g) * 32 + lane] = ss;
    red2[(3 * G + g) * 32 + lane] = scc;
    red2[(4 * G + g) * 32 + lane] = scs;
    __syncthreads();
    constexpr bool DD = sizeof(St) == 4; // FP32 storage: FP64-class per-site part
    if (DD && pair_split(N, G)) { // double-float, split over the warps by sample direction
        float *fr = reinterpret_cast<float *>(smem_raw + pair_smem_bytes(N, G, BULK, 4, TWO_D));
        const int tid = g * 32 + lane;
        site_split_dd<N, kPairSites>(a, red, G, tid, G * 32, x0 + tid < a.nx, sres, fr,
                                     fr + kSplitFrameRows(N) * kPairSites);
    } else {
        if (g < 2) {
            const int s = g * 32 + lane;
            if constexpr (DD) pair_site_solve_dd<N>(a, red, G, s, x0 + s < a.nx, sres);
            else pair_site_solve<N>(a, red, G, s, x0 + s < a.nx, sres);
        }
        __syncthreads();
    }

    // this warp's shell: its equilibrium coefficients for its two sites
    float2 cr[NC], o0, o1, o2;
    pair_shell_coefficients<N, DD>(a, r, sres, lane, cr, o0, o1, o2);
    const float2 no1 = f2(-o1.x, -o1.y), no2 = f2(-o2.x, -o2.y);
    constexpr bool kSR = sizeof(St) <= 4; // FP32 and 16-bit stores round stochastically
    unsigned rng = mix32(unsigned(y * a.nx + xa) * 64u + unsigned(g) ^ mix32(__ldcg(a.ctr) * 0x9E3779B9u + 1u));
    St *ob = fout + (long long)i0 * S + (long long)y * a.nx + xa;
#pragma unroll
    for (int k = 0; k < PP; ++k) {
        const float4 t0 = __ldg(tb + k * PQ);                                       // (c,c,s,s)
        const float2 wq = __ldg(reinterpret_cast<const float2 *>(tb + k * PQ + 2)); // (w', w')
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
        if constexpr (sizeof(St) == 4) {
            const float2 out = relax_pair_sr(fs[k], om, feq, next_bits2(rng));
            if (act && good) *reinterpret_cast<float2 *>(ob + (long long)k * S) = out;
        } else {
            const float2 out = __ffma2_rn(om, f2sub(feq, fs[k]), fs[k]);
            if (act && good) PIo<St>::st2(ob + (long long)k * S, out, rng);
        }
    }
    if (kSR) {
        __syncthreads();
        if (threadIdx.x == 0 && threadIdx.y == 0) advance_launch_counter(a.ctr, gridDim.x * gridDim.y);
    }
}

// Many angles (K beyond one group of PP populations per warp), FP32 storage:
// the arithmetic of rlbm_pair_kernel with plain loads, warp (r, q) owning
// groups rho = 0, 1, ... of PP populations, group rho being virtual warp
// v = rho Gs + q (populations r K + v PP + k; K is a multiple of PP, so a group
// is full or empty).  Pass 1 streams the groups one after another and parks
// the packed f* of all but the warp's last non-empty group in their own output
// slots; pass 2 handles the last group from registers and reads the others
// back (the same thread wrote them: no synchronisation).
template <int N, int PP, bool TWO_D>
__global__ void __launch_bounds__(kMaxWarps * 32, PP <= 16 ? 2 : 1) rlbm_pair_groups_kernel(const KernelArgs a)
{
    constexpr int NC = 2 * N + 1;
    constexpr int PQ = 3;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x, g = threadIdx.y, G = blockDim.y;
    const int x0 = blockIdx.x * kPairSites;
    const int xl = x0 + 2 * lane;
    const bool act = xl < a.nx;
    const int xa = act ? xl : a.nx - 2;
    const int y = blockIdx.y;
    const int r = g / a.Gs, q = g % a.Gs;
    const long long S = a.S;
    const float *fin = reinterpret_cast<const float *>(a.fin);
    float *fout = reinterpret_cast<float *>(a.fout);
    float *red = reinterpret_cast<float *>(smem_raw); // [5][G][64]
    float *sres = red + 5 * G * kPairSites;           // [pair_site_rows(N)][64]
    const float4 *ptab = reinterpret_cast<const float4 *>(a.pairtab);
    const int xm = bc_index(xa - 1, a.nx, a.bcx), xp = bc_index(xa + 2, a.nx, a.bcx);
    const int ym = TWO_D ? bc_index(y - 1, a.ny, a.bcy) : y;
    const int yp = TWO_D ? bc_index(y + 1, a.ny, a.bcy) : y;
    const long long row = (long long)y * a.nx;
    const long long dym = (long long)(ym - y) * a.nx, dyp = (long long)(yp - y) * a.nx;
    const int Gv = a.Gs * a.R;                                      // virtual warps per shell
    const int nrho = min(a.R, (a.K / PP - q + a.Gs - 1) / a.Gs); // non-empty groups of this warp

    float2 fs[PP];
    float2 s0 = f2(0.f, 0.f), sc = f2(0.f, 0.f), ss = f2(0.f, 0.f), scc = f2(0.f, 0.f), scs = f2(0.f, 0.f);
    constexpr int CH = TWO_D ? (PP <= 8 ? PP : (PP == 12 ? 6 : 4)) : (PP <= 16 ? PP : 8);
    static_assert(PP % CH == 0, "chunking");
#pragma unroll 1
    for (int rho = 0; rho < nrho; ++rho) {
        const int vw = rho * a.Gs + q;
        const int i0 = r * a.K + vw * PP;
        const float4 *tb = ptab + size_t(i0) * PQ;
        const unsigned long long mx = __ldg(a.masks + 2 * (r * Gv + vw));
        const unsigned long long my = __ldg(a.masks + 2 * (r * Gv + vw) + 1);
        const float *base = fin + (long long)i0 * S + row;
#pragma unroll
        for (int c0 = 0; c0 < PP; c0 += CH) {
            float2 ca[CH], cb[TWO_D ? CH : 1];
            float ea[CH], eb[TWO_D ? CH : 1];
#pragma unroll
            for (int kk = 0; kk < CH; ++kk) {
                const int k = c0 + kk;
                const float *pk = base + (long long)k * S;
                const int xs = ((mx >> k) & 1ull) ? xm : xp;
                ca[kk] = PIo<float>::ld2(pk + xa);
                ea[kk] = PIo<float>::ld1(pk + xs);
                if (TWO_D) {
                    const long long dy = ((my >> k) & 1ull) ? dym : dyp;
                    cb[kk] = PIo<float>::ld2(pk + dy + xa);
                    eb[kk] = PIo<float>::ld1(pk + dy + xs);
                }
            }
#pragma unroll
            for (int kk = 0; kk < CH; ++kk) {
                const int k = c0 + kk;
                const float4 t0 = __ldg(tb + k * PQ), t1 = __ldg(tb + k * PQ + 1); // (c,c,s,s), (|c|,|c|,|s|,|s|)
                const bool px = (mx >> k) & 1ull;                                    // v_x >= 0: pull from x - 1
                const float2 C = ca[kk];
                const float2 B = px ? f2(ea[kk], C.x) : f2(C.y, ea[kk]);
                const float2 ac = f2(t1.x, t1.y);
                float2 v = __ffma2_rn(ac, f2sub(B, C), C);
                if (TWO_D) {
                    const float2 C2 = cb[kk];
                    const float2 B2 = px ? f2(eb[kk], C2.x) : f2(C2.y, eb[kk]);
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
        }
        if (rho + 1 < nrho && act) { // park f* of every group but the last
            float *pb = fout + (long long)i0 * S + row + xa;
#pragma unroll
            for (int k = 0; k < PP; ++k) *reinterpret_cast<float2 *>(pb + (long long)k * S) = fs[k];
        }
    }
    float2 *red2 = reinterpret_cast<float2 *>(red);
    red2[(0 * G + g) * 32 + lane] = s0;
    red2[(1 * G + g) * 32 + lane] = sc;
    red2[(2 * G + g) * 32 + lane] = ss;
    red2[(3 * G + g) * 32 + lane] = scc;
    red2[(4 * G + g) * 32 + lane] = scs;
    __syncthreads();
    if (pair_split(N, G)) { // the per-site part in double-float, split over the warps by sample direction
        float *fr = reinterpret_cast<float *>(smem_raw + pair_bars_offset(N, G));
        const int tid = g * 32 + lane;
        site_split_dd<N, kPairSites>(a, red, G, tid, G * 32, x0 + tid < a.nx, sres, fr,
                                     fr + kSplitFrameRows(N) * kPairSites);
    } else {
        if (g < 2) {
            const int s = g * 32 + lane;
            pair_site_solve_dd<N>(a, red, G, s, x0 + s < a.nx, sres);
        }
        __syncthreads();
    }

    // this warp's shell coefficients for its two sites (as in rlbm_pair_kernel)
    float2 cr[NC], o0, o1, o2;
    pair_shell_coefficients<N, true>(a, r, sres, lane, cr, o0, o1, o2);
    const float2 no1 = f2(-o1.x, -o1.y), no2 = f2(-o2.x, -o2.y);
    unsigned rng = mix32(unsigned(y * a.nx + xa) * 64u + unsigned(g) ^ mix32(__ldcg(a.ctr) * 0x9E3779B9u + 1u));
#pragma unroll 1
    for (int rho = nrho - 1; rho >= 0; --rho) {
        const int vw = rho * a.Gs + q;
        const int i0 = r * a.K + vw * PP;
        const float4 *tb = ptab + size_t(i0) * PQ;
        float *ob = fout + (long long)i0 * S + row + xa;
        if (rho + 1 < nrho && act) { // a parked group: f* back from its output slots
#pragma unroll
            for (int k = 0; k < PP; ++k) fs[k] = *reinterpret_cast<const float2 *>(ob + (long long)k * S);
        }
#pragma unroll
        for (int k = 0; k < PP; ++k) {
            const float4 t0 = __ldg(tb + k * PQ);                                       // (c,c,s,s)
            const float2 wq = __ldg(reinterpret_cast<const float2 *>(tb + k * PQ + 2)); // (w', w')
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
            const float2 out = relax_pair_sr(fs[k], om, feq, next_bits2(rng));
            if (act) *reinterpret_cast<float2 *>(ob + (long long)k * S) = out;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) advance_launch_counter(a.ctr, gridDim.x * gridDim.y);
}

// Several population groups per warp (FP32 storage, plain loads): the
// instances of one order N (one compile unit per N).
template <int N, int PP>
static cudaError_t launch_pair_groups_np(bool two_d, dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                         const KernelArgs &a)
{
    void (*k)(const KernelArgs) = two_d ? rlbm_pair_groups_kernel<N, PP, true> : rlbm_pair_groups_kernel<N, PP, false>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k<<<grid, block, smem, st>>>(a);
    return cudaGetLastError();
}

template <int N>
static cudaError_t launch_pair_groups_n(int PP, bool two_d, dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                        const KernelArgs &a)
{
    switch (PP) {
    case 8: return launch_pair_groups_np<N, 8>(two_d, grid, block, smem, st, a);
    case 12: return launch_pair_groups_np<N, 12>(two_d, grid, block, smem, st, a);
    case 16: return launch_pair_groups_np<N, 16>(two_d, grid, block, smem, st, a);
    case 24: return launch_pair_groups_np<N, 24>(two_d, grid, block, smem, st, a);
    case 32: return launch_pair_groups_np<N, 32>(two_d, grid, block, smem, st, a);
    default: return cudaErrorInvalidValue;
    }
}

// The two-sites-per-lane kernel of storage St, order N, plain (BULK false) or
// bulk-staged first pass: the instances of one compile unit.
template <class St, int N, int PP, bool BULK>
static cudaError_t launch_pair_one(bool two_d, dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                   const KernelArgs &a)
{
    void (*k)(const KernelArgs) =
        two_d ? rlbm_pair_kernel<St, N, PP, true, BULK> : rlbm_pair_kernel<St, N, PP, false, BULK>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k<<<grid, block, smem, st>>>(a);
    return cudaGetLastError();
}

template <class St, int N, bool BULK>
static cudaError_t launch_pair_nb(int PP, bool two_d, dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                  const KernelArgs &a)
{
    switch (PP) {
    case 8: return launch_pair_one<St, N, 8, BULK>(two_d, grid, block, smem, st, a);
    case 12: return launch_pair_one<St, N, 12, BULK>(two_d, grid, block, smem, st, a);
    case 16: return launch_pair_one<St, N, 16, BULK>(two_d, grid, block, smem, st, a);
    case 24: return launch_pair_one<St, N, 24, BULK>(two_d, grid, block, smem, st, a);
    case 32: return launch_pair_one<St, N, 32, BULK>(two_d, grid, block, smem, st, a);
    default: return cudaErrorInvalidValue;
    }
}

} // namespace rlbmk
