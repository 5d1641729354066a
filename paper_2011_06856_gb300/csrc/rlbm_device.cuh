// Device side of the fused RLBM step (arXiv 2011.06856, Sec. 2.2): one CTA
// owns 32 consecutive sites of one grid row and all N_pop populations of
// them.  Warp g handles P populations of one energy shell r = g / Gs
// (Gs warps per shell), lane = site.  A step is:
//
//   pass 1  bilinear pull of the warp's P populations (Eqs. streaming,
//           interpolation), kept in registers, and five angular sums
//           S0, Sc, Ss, Scc, Scs of them, exchanged through shared memory;
//   site    every warp folds the G x 5 sums of its 32 sites with p_r, p_r^2
//           into N^a and T^ab (Eq. discrete_sum_moments; T^yy = T^tt - T^xx
//           on the light cone), solves the Landau frame eps U^a = T^ab U_b
//           (landau_fast), n = U_a N^a, T = eps / 2n, and builds the truncated
//           equilibrium of its own shell as a trigonometric polynomial of
//           degree N in theta (shell_coefficients).  The work is repeated per
//           warp so that no warp waits on another;
//   pass 2  f^eq_i from those coefficients, relaxation
//           f <- f* + omega_i (f^eq - f*), omega_i = (U^0 - U.v_i)/tau
//           (Eq. discrete-rbe), one store per population.
//
// Populations are read once and written once per step; halo values of the
// neighbouring tile come through L1/L2.  All per-population constants are
// warp-uniform loads of a small table (L1 resident).
//
// Many angles (K beyond what 16 warps of at most 64 populations hold): warp
// (r, q) then owns a.R groups of P populations of its shell, group rho being
// "virtual warp" v = rho Gs + q (populations r K + v P + k).  Pass 1 streams
// the groups one after another and parks the streamed values f* of all but
// the last group in their own output slots (same thread, same address: no
// synchronisation needed); pass 2 handles the last group from registers and
// reads the others back.  FP32 and FP64 storage only (f* is parked exactly).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "rlbm_args.h"
#include "rlbm_df64.cuh"
#include "rlbm_stat.cuh"

namespace rlbmk {

// ---- storage <-> compute conversions -------------------------------------
template <class St, class R> struct Io;
template <> struct Io<double, double> {
    static __device__ __forceinline__ double ld(const double *p) { return __ldg(p); }
    static __device__ __forceinline__ double lds(const double *p) { return *p; }
    static __device__ __forceinline__ double ldcg(const double *p) { return __ldcg(p); }
    static __device__ __forceinline__ void st(double *p, double v) { *p = v; }
};
template <> struct Io<float, float> {
    static __device__ __forceinline__ float ld(const float *p) { return __ldg(p); }
    static __device__ __forceinline__ float lds(const float *p) { return *p; }
    static __device__ __forceinline__ float ldcg(const float *p) { return __ldcg(p); }
    static __device__ __forceinline__ void st(float *p, float v) { *p = v; }
};
template <> struct Io<__half, float> {
    static __device__ __forceinline__ float ld(const __half *p)
    {
        return __half2float(__ushort_as_half(__ldg(reinterpret_cast<const unsigned short *>(p))));
    }
    static __device__ __forceinline__ float lds(const __half *p) { return __half2float(*p); }
    static __device__ __forceinline__ float ldcg(const __half *p)
    {
        return __half2float(__ushort_as_half(__ldcg(reinterpret_cast<const unsigned short *>(p))));
    }
    static __device__ __forceinline__ void st(__half *p, float v) { *p = __float2half_rn(v); }
};
template <> struct Io<__nv_bfloat16, float> {
    static __device__ __forceinline__ float ld(const __nv_bfloat16 *p)
    {
        return __bfloat162float(
            __ushort_as_bfloat16(__ldg(reinterpret_cast<const unsigned short *>(p))));
    }
    static __device__ __forceinline__ float lds(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
    static __device__ __forceinline__ float ldcg(const __nv_bfloat16 *p)
    {
        return __bfloat162float(
            __ushort_as_bfloat16(__ldcg(reinterpret_cast<const unsigned short *>(p))));
    }
    static __device__ __forceinline__ void st(__nv_bfloat16 *p, float v)
    {
        *p = __float2bfloat16_rn(v);
    }
};

__device__ __forceinline__ float r_acos(float v) { return acosf(v); }
__device__ __forceinline__ double r_acos(double v) { return acos(v); }
__device__ __forceinline__ float r_cos(float v) { return cosf(v); }
__device__ __forceinline__ double r_cos(double v) { return cos(v); }
__device__ __forceinline__ float r_sqrt(float v) { return sqrtf(v); }
__device__ __forceinline__ double r_sqrt(double v) { return sqrt(v); }
__device__ __forceinline__ float r_rsqrt(float v) { return rsqrtf(v); }
__device__ __forceinline__ double r_rsqrt(double v) { return rsqrt(v); }
// Division in the per-site arithmetic: FP32 uses the approximate quotient (2 ulp;
// the FP32 per-site part serves 16-bit storage, and where it is not accurate
// enough landau_f32_adaptive solves again in double-float), FP64 the exact one.
__device__ __forceinline__ float r_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double r_div(double a, double b) { return a / b; }

// Stochastic rounding of 16-bit stores.  Round-to-nearest repeats the same
// rounding error every step wherever the flow is steady, and the conserved
// moments drift linearly; with stochastic rounding the error has zero mean
// and only random-walks.  Random bits: one hash per thread and tile (of the
// site, the warp and the launch counter), then a 32-bit LCG step per store;
// the top bits are added below the kept mantissa and the value truncated.
__device__ __forceinline__ unsigned mix32(unsigned x)
{
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}
__device__ __forceinline__ unsigned lcg_next(unsigned &s)
{
    s = s * 1664525u + 1013904223u;
    return s;
}
template <class St> struct SR {
    static __device__ __forceinline__ void st(St *p, float v, unsigned &rng);
};
template <> struct SR<__half> {
    static __device__ __forceinline__ void st(__half *p, float v, unsigned &rng)
    {
        const unsigned b = __float_as_uint(v) + (lcg_next(rng) >> 19); // 13 dropped bits
        *p = __float2half_rz(__uint_as_float(b));
    }
};
template <> struct SR<__nv_bfloat16> {
    static __device__ __forceinline__ void st(__nv_bfloat16 *p, float v, unsigned &rng)
    {
        const unsigned b = __float_as_uint(v) + (lcg_next(rng) >> 16); // 16 dropped bits
        *reinterpret_cast<unsigned short *>(p) = (unsigned short)(b >> 16);
    }
};
template <> struct SR<float> {
    static __device__ __forceinline__ void st(float *p, float v, unsigned &) { *p = v; }
};
template <> struct SR<double> {
    static __device__ __forceinline__ void st(double *p, double v, unsigned &) { *p = v; }
};

// Stochastic rounding of the FP32 relaxation out = f* + om (f^eq - f*): the
// FMA's result r (round to nearest) and its exact residual e = f* + om d - r
// (d = f^eq - f*; f* - r is exact whenever the two are within a factor 2)
// give the exact value r + e; adding a uniform noise of +-ulp(r)/2 to e
// before the final rounding r + (e + noise) rounds it up or down with
// probabilities proportional to the distance -- stochastic rounding.  With
// round to nearest, FP32 stores repeat the same rounding error step after
// step wherever the flow changes slowly, and the conserved moments drift
// (1e-5 after ~3500 steps of the 8192 x 4 shock tube at tau = 82); with it
// the error only random-walks (3e-7).  u16: 16 random bits.
__device__ __forceinline__ float ulp_of(float r)
{
    return __uint_as_float(__float_as_uint(r) & 0x7f800000u) * 1.1920928955078125e-7f; // 2^-23
}
__device__ __forceinline__ float noise16(unsigned u16)
{
    return __uint_as_float(0x3f800000u | ((u16 & 0xffffu) << 7)) - 1.5f; // uniform in [-1/2, 1/2)
}
__device__ __forceinline__ float relax_sr(float fs, float om, float feq, unsigned u16)
{
    const float d = __fsub_rn(feq, fs);
    const float r = __fmaf_rn(om, d, fs);
    const float e = __fmaf_rn(om, d, __fsub_rn(fs, r));
    return __fadd_rn(r, __fmaf_rn(noise16(u16), ulp_of(r), e));
}

// The relaxation (Eq. discrete-rbe) and its store in storage St: FP64 rounds
// to nearest; FP32 and the 16-bit forms round stochastically (their random
// bits from the per-thread stream rng).
template <class St, class R>
__device__ __forceinline__ void relax_store(St *p, R fs, R om, R feq, unsigned &rng)
{
    if constexpr (sizeof(St) == 8) {
        *p = fs + om * (feq - fs);
    } else if constexpr (sizeof(St) == 4) {
        *p = relax_sr(fs, om, feq, lcg_next(rng) >> 16);
    } else {
        SR<St>::st(p, fs + om * (feq - fs), rng);
    }
}

// The last CTA of a step launch advances the launch counter that seeds the
// rounding of the next launch (graph replays keep their parameters fixed).
__device__ __forceinline__ void advance_launch_counter(unsigned *ctr, unsigned nblocks)
{
    __threadfence();
    if (atomicAdd(&ctr[1], 1u) == nblocks - 1) {
        ctr[1] = 0u;
        __threadfence();
        atomicAdd(&ctr[0], 1u);
    }
}

// Launch scalars in the per-site precision (FP32 kernels read the FP32 copies).
template <class LR> struct Par;
template <> struct Par<double> {
    static __device__ __forceinline__ double inv_tau(const KernelArgs &a) { return a.inv_tau; }
    static __device__ __forceinline__ double feq_off(const KernelArgs &a) { return a.feq_off; }
    static __device__ __forceinline__ double off(const KernelArgs &a, int u) { return a.off[u]; }
    static __device__ __forceinline__ double smp_c(const KernelArgs &a, int j) { return a.smp_c[j]; }
    static __device__ __forceinline__ double smp_s(const KernelArgs &a, int j) { return a.smp_s[j]; }
};
template <> struct Par<float> {
    static __device__ __forceinline__ float inv_tau(const KernelArgs &a) { return a.inv_tau_f; }
    static __device__ __forceinline__ float feq_off(const KernelArgs &a) { return a.feq_off_f; }
    static __device__ __forceinline__ float off(const KernelArgs &a, int u) { return a.off_f[u]; }
    static __device__ __forceinline__ float smp_c(const KernelArgs &a, int j) { return a.smp_cf[j]; }
    static __device__ __forceinline__ float smp_s(const KernelArgs &a, int j) { return a.smp_sf[j]; }
};

__device__ __forceinline__ int bc_index(int i, int L, int bc)
{
    if (bc == 0) return i < 0 ? i + L : (i >= L ? i - L : i);
    return i < 0 ? 0 : (i >= L ? L - 1 : i);
}

// The same for any offset (shifts of several cells, grids smaller than the shift).
__device__ __forceinline__ int bc_any(int i, int L, int bc)
{
    if (bc == 0) return ((i % L) + L) % L;
    return i < 0 ? 0 : (i >= L ? L - 1 : i);
}

template <class R>
__device__ __forceinline__ void ld4(const R *p, R &x, R &y, R &z, R &w);
template <>
__device__ __forceinline__ void ld4<float>(const float *p, float &x, float &y, float &z, float &w)
{
    const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
    x = v.x; y = v.y; z = v.z; w = v.w;
}
template <>
__device__ __forceinline__ void ld4<double>(const double *p, double &x, double &y, double &z,
                                            double &w)
{
    const double2 v0 = __ldg(reinterpret_cast<const double2 *>(p));
    const double2 v1 = __ldg(reinterpret_cast<const double2 *>(p) + 1);
    x = v0.x; y = v0.y; z = v1.x; w = v1.y;
}

// Sum the per-warp angular sums of one site (lane) and fold them with the
// shell factors alpha_r p_r, alpha_r p_r^2 into
// m = (N^t, N^x, N^y, T^tt, T^tx, T^ty, T^xx, T^xy)  (Eq. discrete_sum_moments).
template <int N, class LR>
__device__ __forceinline__ void fold_moments(const KernelArgs &a, const LR *red, int G, int lane,
                                             LR *m)
{
    const LR *sh = reinterpret_cast<const LR *>(a.shelltab);
#pragma unroll
    for (int u = 0; u < 8; ++u) m[u] = Par<LR>::off(a, u);
#pragma unroll
    for (int rr = 0; rr <= N; ++rr) {
        LR p0 = LR(0), pc = LR(0), ps = LR(0), pcc = LR(0), pcs = LR(0);
        for (int qq = 0; qq < a.Gs; ++qq) {
            const int w = rr * a.Gs + qq;
            p0 += red[(0 * G + w) * 32 + lane];
            pc += red[(1 * G + w) * 32 + lane];
            ps += red[(2 * G + w) * 32 + lane];
            pcc += red[(3 * G + w) * 32 + lane];
            pcs += red[(4 * G + w) * 32 + lane];
        }
        const LR f1 = __ldg(sh + 2 * rr), f2 = __ldg(sh + 2 * rr + 1);
        m[0] += f1 * p0;
        m[1] += f1 * pc;
        m[2] += f1 * ps;
        m[3] += f2 * p0;
        m[4] += f2 * pc;
        m[5] += f2 * ps;
        m[6] += f2 * pcc;
        m[7] += f2 * pcs;
    }
}

// Landau frame, eps U^a = T^ab U_b (Sec. 2.2), in a form cheap enough to run
// per site in every warp.  With E = T^tt and M = |T^ti|, an equilibrium has
// beta = (3E - sqrt(9E^2 - 8M^2)) / 2M and eps = E - beta M exactly; that is the
// starting point of Newton's method on the trace-free characteristic cubic
// lambda^3 + c1 lambda - c0.  If it lies below the root, T^tt (an upper bound
// of the rest-frame energy density) is used instead, so Newton approaches the
// largest root from above, monotonically.  The eigenvector is the cross
// product of the last two rows of A - eps I (A = T eta), whose spatial 2x2
// block T^ij + eps delta^ij is positive definite for a physical state.
template <class LR>
__device__ __forceinline__ bool landau_fast(const LR *m, LR &n, LR &eps, LR &U0, LR &Ux, LR &Uy)
{
    const LR Nt = m[0], Nx = m[1], Ny = m[2];
    const LR E = m[3], Ttx = m[4], Tty = m[5], Txx = m[6], Txy = m[7];
    const LR Tyy = E - Txx;
    const LR c1 = -E * E + Ttx * Ttx + Tty * Tty + Txx * Tyy - Txy * Txy;
    const LR c0 = E * (Txx * Tyy - Txy * Txy) - Ttx * Ttx * Tyy + LR(2) * Ttx * Tty * Txy -
                  Tty * Tty * Txx;
    const LR M = r_sqrt(Ttx * Ttx + Tty * Tty);
    const LR disc = LR(9) * E * E - LR(8) * M * M;
    const LR b0 = r_div(LR(4) * M, LR(3) * E + r_sqrt(disc > LR(0) ? disc : LR(0)));
    LR lam = E - b0 * M;
    if ((lam * lam + c1) * lam - c0 < LR(0)) lam = E;
    const LR tol = LR(sizeof(LR) == 8 ? 4e-16 : 2e-7);
#pragma unroll 1
    for (int it = 0; it < 24; ++it) {
        const LR P = (lam * lam + c1) * lam - c0;
        const LR dP = LR(3) * lam * lam + c1;
        if (!(dP > LR(0))) break;
        const LR d = r_div(P, dP);
        lam -= d;
        if (!(fabs(d) > tol * lam)) break;
    }
    eps = lam;
    const LR bx = Txx + lam, by = Tyy + lam;
    const LR v0 = bx * by - Txy * Txy;
    const LR v1 = Ttx * by - Txy * Tty;
    const LR v2 = bx * Tty - Ttx * Txy;
    const LR mink = v0 * v0 - v1 * v1 - v2 * v2;
    bool ok = (c1 < LR(0)) && (v0 > LR(0)) && (mink > LR(0));
    if (ok) {
        const LR s = r_rsqrt(mink);
        U0 = v0 * s;
        Ux = v1 * s;
        Uy = v2 * s;
    } else {
        U0 = LR(1);
        Ux = LR(0);
        Uy = LR(0);
    }
    n = U0 * Nt - Ux * Nx - Uy * Ny;
    if (!(n > LR(0)) || !(eps > LR(0))) {
        ok = false;
        n = Nt > LR(0) ? Nt : LR(1e-30);
        if (!(eps > LR(0))) eps = E > LR(0) ? E : LR(1e-30);
    }
    return ok;
}

// The Landau frame in double-float arithmetic (rlbm_df64.cuh), for moments m
// given as double-floats.  The FP32 root of landau_fast is polished by two
// Newton steps on the trace-free characteristic cubic whose coefficients c1,
// c0 are formed in double-float; then the eigenvector (the cross product of
// the last two rows of A - eps I), its Minkowski norm and n = U_a N^a.  Where
// T^ab is close to degenerate (a strongly boosted or strongly anisotropic
// state) the cross product and the norm cancel many digits: the FP32 frame
// loses them, the double-float one keeps about 48 bits.
__device__ __forceinline__ bool landau_dd(const df64 *m, df64 &n, df64 &eps, df64 &U0, df64 &Ux, df64 &Uy)
{
    float mf[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) mf[u] = to_float(m[u]);
    float nf, ef, u0f, uxf, uyf;
    landau_fast<float>(mf, nf, ef, u0f, uxf, uyf);
    const df64 Nt = m[0], Nx = m[1], Ny = m[2];
    const df64 E = m[3], Ttx = m[4], Tty = m[5], Txx = m[6], Txy = m[7];
    const df64 Tyy = E - Txx;
    const df64 tx2 = Ttx * Ttx, ty2 = Tty * Tty, xy2 = Txy * Txy, xxyy = Txx * Tyy;
    const df64 c1 = tx2 + ty2 + xxyy - xy2 - E * E;
    const df64 c0 = E * (xxyy - xy2) - tx2 * Tyy + (Ttx * Tty * Txy) * 2.f - ty2 * Txx;
    df64 lam = dd(ef);
#pragma unroll
    for (int it = 0; it < 2; ++it) {
        const df64 P = (lam * lam + c1) * lam - c0;
        const float dP = __fmaf_rn(3.f * lam.hi, lam.hi, c1.hi);
        if (!(dP > 0.f)) break;
        lam = lam - __fdividef(P.hi, dP);
    }
    eps = lam;
    const df64 bx = Txx + lam, by = Tyy + lam;
    const df64 v0 = bx * by - xy2;
    const df64 v1 = Ttx * by - Txy * Tty;
    const df64 v2 = bx * Tty - Ttx * Txy;
    const df64 mink = v0 * v0 - v1 * v1 - v2 * v2;
    bool ok = (c1.hi < 0.f) && (v0.hi > 0.f) && (mink.hi > 0.f);
    if (ok) {
        const df64 s = dd_rsqrt(mink);
        U0 = v0 * s;
        Ux = v1 * s;
        Uy = v2 * s;
    } else {
        U0 = dd(1.f);
        Ux = dd(0.f);
        Uy = dd(0.f);
    }
    n = U0 * Nt - Ux * Nx - Uy * Ny;
    if (!(n.hi > 0.f) || !(eps.hi > 0.f)) {
        ok = false;
        n = Nt.hi > 0.f ? Nt : dd(1e-30f);
        if (!(eps.hi > 0.f)) eps = E.hi > 0.f ? E : dd(1e-30f);
    }
    return ok;
}

// FP32 moments in, FP32 frame out, the frame solved in double-float: the form
// of the kernels that store 16-bit populations and accumulate in FP32.
__device__ __forceinline__ bool landau_f32dd(const float *m, float &n, float &eps, float &U0, float &Ux, float &Uy)
{
    df64 md[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) md[u] = dd(m[u]);
    df64 nd, ed, u0, ux, uy;
    const bool ok = landau_dd(md, nd, ed, u0, ux, uy);
    n = to_float(nd);
    eps = to_float(ed);
    U0 = to_float(u0);
    Ux = to_float(ux);
    Uy = to_float(uy);
    return ok;
}

// The Landau frame for FP32 per-site arithmetic, refined in double-float where
// T^ab is close to degenerate.  The FP32 root of the characteristic cubic
// carries a relative error of about u_32 (E / eps)^3 / (P'(eps) / eps^2) (E =
// T^tt; P' = 3 eps^2 + c1 is (eps + P)^2 = 2.25 eps^2 for a fluid at rest): it
// grows like gamma^6 with the boost and blows up near a double root.  Where
// E > 3 eps (gamma^2 above ~2.3), P'(eps) < eps^2 / 2, or the FP32 solve failed,
// the frame is solved again in double-float (landau_f32dd); elsewhere the FP32
// frame is accurate to a few 1e-7, far below the rounding of 16-bit storage.
__device__ __forceinline__ bool landau_f32_adaptive(const float *m, float &n, float &eps, float &U0, float &Ux,
                                                    float &Uy)
{
    bool ok = landau_fast<float>(m, n, eps, U0, Ux, Uy);
    const float E = m[3], Ttx = m[4], Tty = m[5], Txx = m[6], Txy = m[7];
    const float c1 = -E * E + Ttx * Ttx + Tty * Tty + Txx * (E - Txx) - Txy * Txy;
    const bool refine = !ok || E > 3.f * eps || 3.f * eps * eps + c1 < 0.5f * eps * eps;
    if (refine) ok = landau_f32dd(m, n, eps, U0, Ux, Uy);
    return ok;
}

// The Landau solve of a kernel with storage St and per-site type LR: 16-bit
// storage with FP32 per-site arithmetic refines the FP32 frame in
// double-float where T^ab is near-degenerate (landau_f32_adaptive); every other
// combination solves it in LR itself (FP64 for FP32 and FP64 storage).
template <class St, class LR>
__device__ __forceinline__ bool site_landau(const LR *m, LR &n, LR &eps, LR &U0, LR &Ux, LR &Uy)
{
    if constexpr (sizeof(St) == 2 && sizeof(LR) == 4) return landau_f32_adaptive(m, n, eps, U0, Ux, Uy);
    else return landau_fast<LR>(m, n, eps, U0, Ux, Uy);
}

// Truncated equilibrium (Eqs. mj-feq-expansion, mj-projection-coefficients,
// mj-feq-expansion-truncated) as per-shell Fourier coefficients.  On the light
// cone the polynomials of degree <= N split by angular mode m: mode m uses the
// radial powers p^k, m <= k <= N, orthogonal across modes under
// omega = exp(-p).  The projection coefficients are the MJ moments
//   b_{m,k} = int f^MJ p^k e^{i m theta} d^2p/p^0
//           = n k! T^(k-1) / (2 pi) int (q^0)^(k-m) (q^x + i q^y)^m dphi,
// q = Lambda(U) (1, cos phi, sin phi) the boosted rest-frame direction; the
// integrand is a trigonometric polynomial of degree k <= N in phi, so N+1
// equispaced directions integrate it exactly.  The radial Gram inverse,
// k!/(N+1), the angular norms and p_r^l are folded into rtab = R'[r][m][k]:
//   C_{r,m} = sum_k R'[r][m][k] n T^(k-1) acc_{m,k},  acc = sum_j q0^(k-m) z^m.
// This returns the coefficients of one energy shell r in stored units:
// cr[0] = Re C_{r,0} - feq_off, cr[2m-1], cr[2m] = Re, Im C_{r,m}.
// shell_coefficients_tk takes the radial weights tk[k] as given (n T^(k-1) for
// Maxwell-Juttner, 2 pi g T^(k+1) phi_{k+1}(z) for the quantum statistics,
// rlbm_stat.cuh); shell_coefficients forms the Maxwell-Juttner ones.
template <int N, class LR, class R>
__device__ __forceinline__ void shell_coefficients_tk(const KernelArgs &a, int r, const LR *tk, LR U0,
                                                      LR Ux, LR Uy, R *cr)
{
    LR accr[N + 1][N + 1], acci[N + 1][N + 1];
#pragma unroll
    for (int m = 0; m <= N; ++m)
#pragma unroll
        for (int k = 0; k <= N; ++k) { accr[m][k] = LR(0); acci[m][k] = LR(0); }
    const LR inv1g = LR(1) / (LR(1) + U0);
#pragma unroll
    for (int j = 0; j <= N; ++j) {
        const LR cj = Par<LR>::smp_c(a, j), sj = Par<LR>::smp_s(a, j);
        const LR un = Ux * cj + Uy * sj;
        const LR q0 = U0 + un;
        const LR h = LR(1) + un * inv1g;
        const LR zr = cj + Ux * h, zi = sj + Uy * h;
        LR qp[N + 1], pr[N + 1], pi[N + 1];
        qp[0] = LR(1);
        pr[0] = LR(1);
        pi[0] = LR(0);
#pragma unroll
        for (int t = 1; t <= N; ++t) {
            qp[t] = qp[t - 1] * q0;
            pr[t] = pr[t - 1] * zr - pi[t - 1] * zi;
            pi[t] = pr[t - 1] * zi + pi[t - 1] * zr;
        }
#pragma unroll
        for (int m = 0; m <= N; ++m)
#pragma unroll
            for (int k = m; k <= N; ++k) {
                accr[m][k] += qp[k - m] * pr[m];
                acci[m][k] += qp[k - m] * pi[m];
            }
    }
    const LR *rt = reinterpret_cast<const LR *>(a.rtab) + r * (N + 1) * (N + 1);
#pragma unroll
    for (int m = 0; m <= N; ++m) {
        LR cre = LR(0), cim = LR(0);
#pragma unroll
        for (int k = m; k <= N; ++k) {
            const LR wgt = __ldg(rt + m * (N + 1) + k) * tk[k];
            cre += wgt * accr[m][k];
            cim += wgt * acci[m][k];
        }
        if (m == 0) {
            cr[0] = R(cre - Par<LR>::feq_off(a));
        } else {
            cr[2 * m - 1] = R(cre);
            cr[2 * m] = R(cim);
        }
    }
}

// The same in two halves, for kernels that solve each site once and share the
// result: site_sums forms the shell-independent sums w_{m,k} = tk[k] acc_{m,k}
// ((N+1)^2 rows: Re for m = 0..N, k = m..N, then Im for m = 1..N, k = m..N),
// shell_from_sums combines them into shell r's coefficients (w[row * ws]).
template <int N, class LR>
__device__ __forceinline__ void site_sums(const KernelArgs &a, const LR *tk, LR U0, LR Ux, LR Uy, LR *w, int ws)
{
    LR accr[N + 1][N + 1], acci[N + 1][N + 1];
#pragma unroll
    for (int m = 0; m <= N; ++m)
#pragma unroll
        for (int k = 0; k <= N; ++k) { accr[m][k] = LR(0); acci[m][k] = LR(0); }
    const LR inv1g = LR(1) / (LR(1) + U0);
#pragma unroll
    for (int j = 0; j <= N; ++j) {
        const LR cj = Par<LR>::smp_c(a, j), sj = Par<LR>::smp_s(a, j);
        const LR un = Ux * cj + Uy * sj;
        const LR q0 = U0 + un;
        const LR h = LR(1) + un * inv1g;
        const LR zr = cj + Ux * h, zi = sj + Uy * h;
        LR qp[N + 1], pr[N + 1], pi[N + 1];
        qp[0] = LR(1);
        pr[0] = LR(1);
        pi[0] = LR(0);
#pragma unroll
        for (int t = 1; t <= N; ++t) {
            qp[t] = qp[t - 1] * q0;
            pr[t] = pr[t - 1] * zr - pi[t - 1] * zi;
            pi[t] = pr[t - 1] * zi + pi[t - 1] * zr;
        }
#pragma unroll
        for (int m = 0; m <= N; ++m)
#pragma unroll
            for (int k = m; k <= N; ++k) {
                accr[m][k] += qp[k - m] * pr[m];
                acci[m][k] += qp[k - m] * pi[m];
            }
    }
    int row = 0;
#pragma unroll
    for (int m = 0; m <= N; ++m)
#pragma unroll
        for (int k = m; k <= N; ++k) w[(row++) * ws] = tk[k] * accr[m][k];
#pragma unroll
    for (int m = 1; m <= N; ++m)
#pragma unroll
        for (int k = m; k <= N; ++k) w[(row++) * ws] = tk[k] * acci[m][k];
}

template <int N, class LR, class R>
__device__ __forceinline__ void shell_from_sums(const KernelArgs &a, int r, const LR *w, int ws, R *cr)
{
    const LR *rt = reinterpret_cast<const LR *>(a.rtab) + r * (N + 1) * (N + 1);
    int row = 0;
#pragma unroll
    for (int m = 0; m <= N; ++m) {
        LR cre = LR(0);
#pragma unroll
        for (int k = m; k <= N; ++k) cre += __ldg(rt + m * (N + 1) + k) * w[(row++) * ws];
        if (m == 0) cr[0] = R(cre - Par<LR>::feq_off(a));
        else cr[2 * m - 1] = R(cre);
    }
#pragma unroll
    for (int m = 1; m <= N; ++m) {
        LR cim = LR(0);
#pragma unroll
        for (int k = m; k <= N; ++k) cim += __ldg(rt + m * (N + 1) + k) * w[(row++) * ws];
        cr[2 * m] = R(cim);
    }
}

template <int N, class LR, class R>
__device__ __forceinline__ void shell_coefficients(const KernelArgs &a, int r, LR n, LR T, LR U0,
                                                   LR Ux, LR Uy, R *cr)
{
    LR tk[N + 1];
    tk[0] = n / T;
#pragma unroll
    for (int k = 1; k <= N; ++k) tk[k] = (k == 1) ? n : tk[k - 1] * T;
    shell_coefficients_tk<N, LR, R>(a, r, tk, U0, Ux, Uy, cr);
}

// The per-site part for site s with FP64-class accuracy (FP32 storage), in
// double-float arithmetic (rlbm_df64.cuh): the warps' FP32 angular sums are
// folded into N^a and T^ab (Eq. discrete_sum_moments) in double-float, the
// Landau frame is solved in double-float (landau_dd), and the shell-independent
// equilibrium sums w_{m,k} = n T^(k-1) acc_{m,k} are formed in double-float
// and written as hi rows 0 .. (N+1)^2 - 1 and lo rows (N+1)^2 .. 2 (N+1)^2 - 1
// of sres; U^a / tau follow at rows 2 (N+1)^2 + 0..2 (FP32: the relaxation
// rate enters the conserved moments only at second order).  An FP32 per-site
// part carries the conserved moments to a relative bias of about 4e-7 per
// step (rounding of the moment fold, the frame and the radial projection,
// which cancels about one digit); the collision feeds omega of that into the
// state every step and it grows linearly; in double-float it is below 1e-12.
// ST: sites per tile (the stride of red and sres): 64 in the two-sites-per-lane
// kernels, 32 in the per-tile kernel.
template <int N, int ST = 64>
__device__ __forceinline__ void pair_site_solve_dd(const KernelArgs &a, const float *red, int G, int s, bool act,
                                                   float *sres)
{
    constexpr int W = (N + 1) * (N + 1);
    df64 m[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) m[u] = dd(a.off_f[u], a.off_l[u]);
#pragma unroll
    for (int rr = 0; rr <= N; ++rr) {
        float p0 = 0.f, pc = 0.f, ps = 0.f, pcc = 0.f, pcs = 0.f; // the warps' FP32 sums, in FP32
        for (int qq = 0; qq < a.Gs; ++qq) {
            const int w = rr * a.Gs + qq;
            p0 += red[(0 * G + w) * ST + s];
            pc += red[(1 * G + w) * ST + s];
            ps += red[(2 * G + w) * ST + s];
            pcc += red[(3 * G + w) * ST + s];
            pcs += red[(4 * G + w) * ST + s];
        }
        const float2 t1 = __ldg(a.shell2 + 2 * rr), t2 = __ldg(a.shell2 + 2 * rr + 1);
        const df64 f1 = dd(t1.x, t1.y), f2v = dd(t2.x, t2.y);
        m[0] = m[0] + f1 * p0;
        m[1] = m[1] + f1 * pc;
        m[2] = m[2] + f1 * ps;
        m[3] = m[3] + f2v * p0;
        m[4] = m[4] + f2v * pc;
        m[5] = m[5] + f2v * ps;
        m[6] = m[6] + f2v * pcc;
        m[7] = m[7] + f2v * pcs;
    }
    df64 n, eps, U0, Ux, Uy;
    const bool ok = landau_dd(m, n, eps, U0, Ux, Uy);
    if (!ok && act) atomicOr(a.status, 1);
    const df64 T = eps / (n * 2.f);
    const df64 inv1g = dd(1.f) / (U0 + 1.f);
    // boosted rest-frame directions: acc_{m,k} = sum_j q0^(k-m) z^m (as in shell_coefficients)
    df64 accr[N + 1][N + 1], acci[N + 1][N + 1];
#pragma unroll
    for (int mm = 0; mm <= N; ++mm)
#pragma unroll
        for (int k = 0; k <= N; ++k) { accr[mm][k] = dd(0.f); acci[mm][k] = dd(0.f); }
#pragma unroll
    for (int j = 0; j <= N; ++j) {
        const df64 cj = dd(a.smp_cf[j], a.smp_cl[j]), sj = dd(a.smp_sf[j], a.smp_sl[j]);
        const df64 un = Ux * cj + Uy * sj;
        const df64 h = un * inv1g + 1.f;
        df64 qp[N + 1], pr[N + 1], pi[N + 1];
        qp[1] = U0 + un;
        pr[1] = cj + Ux * h;
        pi[1] = sj + Uy * h;
#pragma unroll
        for (int t = 2; t <= N; ++t) {
            qp[t] = qp[t - 1] * qp[1];
            pr[t] = pr[t - 1] * pr[1] - pi[t - 1] * pi[1];
            pi[t] = pr[t - 1] * pi[1] + pi[t - 1] * pr[1];
        }
#pragma unroll
        for (int k = 1; k <= N; ++k) accr[0][k] = accr[0][k] + qp[k];
#pragma unroll
        for (int mm = 1; mm <= N; ++mm) {
            accr[mm][mm] = accr[mm][mm] + pr[mm];
            acci[mm][mm] = acci[mm][mm] + pi[mm];
#pragma unroll
            for (int k = mm + 1; k <= N; ++k) {
                accr[mm][k] = accr[mm][k] + qp[k - mm] * pr[mm];
                acci[mm][k] = acci[mm][k] + qp[k - mm] * pi[mm];
            }
        }
    }
    accr[0][0] = dd(float(N + 1));
    df64 tk[N + 1];
    tk[0] = n / T;
    tk[1] = n;
#pragma unroll
    for (int k = 2; k <= N; ++k) tk[k] = tk[k - 1] * T;
    int row = 0;
#pragma unroll
    for (int mm = 0; mm <= N; ++mm)
#pragma unroll
        for (int k = mm; k <= N; ++k, ++row) {
            const df64 w = tk[k] * accr[mm][k];
            sres[row * ST + s] = w.hi;
            sres[(W + row) * ST + s] = w.lo;
        }
#pragma unroll
    for (int mm = 1; mm <= N; ++mm)
#pragma unroll
        for (int k = mm; k <= N; ++k, ++row) {
            const df64 w = tk[k] * acci[mm][k];
            sres[row * ST + s] = w.hi;
            sres[(W + row) * ST + s] = w.lo;
        }
    const float itau = a.inv_tau_f;
    sres[(2 * W + 0) * ST + s] = to_float(U0) * itau;
    sres[(2 * W + 1) * ST + s] = to_float(Ux) * itau;
    sres[(2 * W + 2) * ST + s] = to_float(Uy) * itau;
}

// Shell r's equilibrium coefficients in the per-shell Fourier form of the
// per-tile kernel (cr[0] = Re C_{r,0} - feq_off, cr[2m-1], cr[2m] = Re, Im C_{r,m})
// from the double-float sums of pair_site_solve_dd (hi rows, then lo rows, of
// stride ws), in double-float, rounded to FP32 at the end.
template <int N>
__device__ __forceinline__ void shell_from_sums_dd(const KernelArgs &a, int r, const float *w, int ws, float *cr)
{
    constexpr int W = (N + 1) * (N + 1);
    const float2 *rt = a.rtab2 + r * (N + 1) * (N + 1);
    int row = 0;
#pragma unroll
    for (int m = 0; m <= N; ++m) {
        df64 acc = dd(0.f);
#pragma unroll
        for (int k = m; k <= N; ++k, ++row) {
            const float2 t = __ldg(rt + m * (N + 1) + k);
            acc = acc + dd(w[row * ws], w[(W + row) * ws]) * dd(t.x, t.y);
        }
        if (m == 0) cr[0] = to_float(acc - dd(a.feq_off_f, a.feq_off_l));
        else cr[2 * m - 1] = to_float(acc);
    }
#pragma unroll
    for (int m = 1; m <= N; ++m) {
        df64 acc = dd(0.f);
#pragma unroll
        for (int k = m; k <= N; ++k, ++row) {
            const float2 t = __ldg(rt + m * (N + 1) + k);
            acc = acc + dd(w[row * ws], w[(W + row) * ws]) * dd(t.x, t.y);
        }
        cr[2 * m] = to_float(acc);
    }
}

// The double-float per-site part of pair_site_solve_dd split over the threads
// of a CTA, for kernels with more threads than sites.  Three phases, each ended
// by a CTA barrier (every thread of the CTA calls site_split_dd):
//  1. threads tid < ST: moment fold and Landau frame of site tid; U^a and
//     t_k = n T^(k-1) (double-floats) into fr, U^a / tau into sres rows 2 W + 0..2;
//  2. item (j, s), j = 0..N: the boosted sample direction j's terms of the sums,
//     acc_{m,k}(j) = q0^(k-m) z^m (double-floats), into part[j];
//  3. item (row, s): w_{m,k} = t_k sum_j part[j], into sres (hi rows, then lo rows).
// The serial chain per site falls from the whole solve to the frame plus one
// direction; the partial sums cost (N + 1) 2 W ST floats of shared memory.
// Layouts (row stride ST): fr [kSplitFrameRows(N)][ST]: U0, Ux, Uy as hi, lo
// pairs, then t_0..t_N as hi, lo pairs; part [N + 1][2 W][ST].
__host__ __device__ constexpr int kSplitFrameRows(int N) { return 6 + 2 * (N + 1); }

template <int N, int ST>
__device__ __forceinline__ void site_frame_dd(const KernelArgs &a, const float *red, int G, int s, bool act,
                                              float *fr, float *sres)
{
    constexpr int W = (N + 1) * (N + 1);
    // The warps' FP32 angular sums of one shell are added in FP32 (one more
    // rounding of the kind the per-warp accumulation already carries); the shell
    // factors and the fold across shells are double-float.
    df64 m[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) m[u] = dd(a.off_f[u], a.off_l[u]);
#pragma unroll
    for (int rr = 0; rr <= N; ++rr) {
        float p0 = 0.f, pc = 0.f, ps = 0.f, pcc = 0.f, pcs = 0.f;
        for (int qq = 0; qq < a.Gs; ++qq) {
            const int w = rr * a.Gs + qq;
            p0 += red[(0 * G + w) * ST + s];
            pc += red[(1 * G + w) * ST + s];
            ps += red[(2 * G + w) * ST + s];
            pcc += red[(3 * G + w) * ST + s];
            pcs += red[(4 * G + w) * ST + s];
        }
        const float2 t1 = __ldg(a.shell2 + 2 * rr), t2 = __ldg(a.shell2 + 2 * rr + 1);
        const df64 f1 = dd(t1.x, t1.y), f2v = dd(t2.x, t2.y);
        m[0] = m[0] + f1 * p0;
        m[1] = m[1] + f1 * pc;
        m[2] = m[2] + f1 * ps;
        m[3] = m[3] + f2v * p0;
        m[4] = m[4] + f2v * pc;
        m[5] = m[5] + f2v * ps;
        m[6] = m[6] + f2v * pcc;
        m[7] = m[7] + f2v * pcs;
    }
    df64 n, eps, U0, Ux, Uy;
    const bool ok = landau_dd(m, n, eps, U0, Ux, Uy);
    if (!ok && act) atomicOr(a.status, 1);
    const df64 T = eps / (n * 2.f);
    fr[0 * ST + s] = U0.hi;
    fr[1 * ST + s] = U0.lo;
    fr[2 * ST + s] = Ux.hi;
    fr[3 * ST + s] = Ux.lo;
    fr[4 * ST + s] = Uy.hi;
    fr[5 * ST + s] = Uy.lo;
    df64 tk = n / T;
#pragma unroll
    for (int k = 0; k <= N; ++k) {
        if (k == 1) tk = n;
        else if (k > 1) tk = tk * T;
        fr[(6 + 2 * k) * ST + s] = tk.hi;
        fr[(7 + 2 * k) * ST + s] = tk.lo;
    }
    const float itau = a.inv_tau_f;
    sres[(2 * W + 0) * ST + s] = to_float(U0) * itau;
    sres[(2 * W + 1) * ST + s] = to_float(Ux) * itau;
    sres[(2 * W + 2) * ST + s] = to_float(Uy) * itau;
}

template <int N, int ST>
__device__ __forceinline__ void site_direction_dd(const KernelArgs &a, const float *fr, int j, int s, float *part)
{
    constexpr int W = (N + 1) * (N + 1);
    const df64 U0 = dd(fr[0 * ST + s], fr[1 * ST + s]);
    const df64 Ux = dd(fr[2 * ST + s], fr[3 * ST + s]);
    const df64 Uy = dd(fr[4 * ST + s], fr[5 * ST + s]);
    const df64 inv1g = dd(1.f) / (U0 + 1.f);
    const df64 cj = dd(a.smp_cf[j], a.smp_cl[j]), sj = dd(a.smp_sf[j], a.smp_sl[j]);
    const df64 un = Ux * cj + Uy * sj;
    const df64 h = un * inv1g + 1.f;
    df64 qp[N + 1], pr[N + 1], pi[N + 1];
    qp[1] = U0 + un;
    pr[1] = cj + Ux * h;
    pi[1] = sj + Uy * h;
#pragma unroll
    for (int t = 2; t <= N; ++t) {
        qp[t] = qp[t - 1] * qp[1];
        pr[t] = pr[t - 1] * pr[1] - pi[t - 1] * pi[1];
        pi[t] = pr[t - 1] * pi[1] + pi[t - 1] * pr[1];
    }
    float *pj = part + j * (2 * W) * ST + s;
    int row = 0;
    // Re rows: m = 0 (q0^k; the k = 0 row is 1 and is not stored), then
    // m = 1..N (q0^(k-m) Re z^m); the reduction multiplies by t_k
#pragma unroll
    for (int mm = 0; mm <= N; ++mm)
#pragma unroll
        for (int k = mm; k <= N; ++k, ++row) {
            if (mm == 0 && k == 0) continue;
            const df64 v = (mm == 0) ? qp[k] : ((k == mm) ? pr[mm] : qp[k - mm] * pr[mm]);
            pj[row * ST] = v.hi;
            pj[(W + row) * ST] = v.lo;
        }
#pragma unroll
    for (int mm = 1; mm <= N; ++mm)
#pragma unroll
        for (int k = mm; k <= N; ++k, ++row) {
            const df64 v = (k == mm) ? pi[mm] : qp[k - mm] * pi[mm];
            pj[row * ST] = v.hi;
            pj[(W + row) * ST] = v.lo;
        }
}

// The power k of T in row `row` of the sums (Re rows m = 0..N, k = m..N, then
// Im rows m = 1..N, k = m..N).
template <int N>
__device__ __forceinline__ int sums_row_k(int row)
{
    int k = 0;
    bool found = false;
#pragma unroll
    for (int mm = 0; mm <= N; ++mm) {
        const int len = N + 1 - mm;
        if (!found && row < len) { k = mm + row; found = true; }
        if (!found) row -= len;
    }
#pragma unroll
    for (int mm = 1; mm <= N; ++mm) {
        const int len = N + 1 - mm;
        if (!found && row < len) { k = mm + row; found = true; }
        if (!found) row -= len;
    }
    return k;
}

template <int N, int ST>
__device__ __forceinline__ void site_split_dd(const KernelArgs &a, const float *red, int G, int tid, int nthr,
                                              bool act, float *sres, float *fr, float *part)
{
    constexpr int W = (N + 1) * (N + 1);
    if (tid < ST) site_frame_dd<N, ST>(a, red, G, tid, act, fr, sres);
    __syncthreads();
    for (int e = tid; e < (N + 1) * ST; e += nthr) site_direction_dd<N, ST>(a, fr, e / ST, e % ST, part);
    __syncthreads();
    for (int e = tid; e < W * ST; e += nthr) {
        const int row = e / ST, s = e - row * ST;
        const int k = sums_row_k<N>(row);
        df64 acc;
        if (row == 0) {
            acc = dd(float(N + 1)); // sum over the N + 1 directions of q0^0
        } else {
            acc = dd(part[e], part[W * ST + e]);
#pragma unroll
            for (int j = 1; j <= N; ++j) acc = acc + dd(part[j * 2 * W * ST + e], part[(j * 2 * W + W) * ST + e]);
        }
        acc = acc * dd(fr[(6 + 2 * k) * ST + s], fr[(7 + 2 * k) * ST + s]);
        sres[e] = acc.hi;
        sres[W * ST + e] = acc.lo;
    }
    __syncthreads();
}

// St: storage type; R: per-population arithmetic; LR: per-site arithmetic
// (moment sums, Landau frame, equilibrium coefficients); N: quadrature order;
// P: populations per thread (compile-time upper bound); TWO_D: ny > 1;
// FULL: every warp owns exactly P populations (no per-population guard).
// MODEQ: a Mode, with the bit MODE_Q for the quantum statistics (Fermi-Dirac or
// Bose-Einstein per a.stat; FP64 per-site arithmetic only).
template <class St, class R, class LR, int N, int P, bool TWO_D, int MODEQ, bool FULL>
__global__ void __launch_bounds__(kMaxWarps * 32) rlbm_kernel(const KernelArgs a)
{
    constexpr int MODE = MODEQ & ~MODE_Q;
    constexpr bool QUANT = (MODEQ & MODE_Q) != 0;
    static_assert(!QUANT || sizeof(LR) == 8, "quantum statistics: FP64 per-site arithmetic");
    constexpr int NC = 2 * N + 1;
    constexpr int TW = tab_width(N);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x, g = threadIdx.y, G = blockDim.y;
    const int xr = blockIdx.x * 32 + lane;
    const bool act = xr < a.nx;
    const int x = act ? xr : a.nx - 1;
    const int y = blockIdx.y;
    const int r = g / a.Gs, q = g % a.Gs;
    const int NR = a.R > 1 ? a.R : 1; // groups of P populations per warp
    const int Gv = a.Gs * NR;         // virtual warps per shell
    const long long S = a.S;
    const long long site = (long long)y * a.nx + x;
    const St *fin = reinterpret_cast<const St *>(a.fin);
    St *fout = reinterpret_cast<St *>(a.fout);
    LR *red = reinterpret_cast<LR *>(smem_raw); // [5][G][32]

    R fs[P];
    constexpr bool LATTICE = (MODE == MODE_STEP_LATTICE); // on-lattice rule: exact shifts
    constexpr bool STEP = (MODE == MODE_STEP) || LATTICE;
    const bool stream = (MODE == MODE_STEP); // bilinear pull
    const bool need_site = !STEP || a.collide;

    if (MODE != MODE_INIT) {
        // two partial sums per moment (even / odd populations) halve the add chains
        R s0[2] = {R(0), R(0)}, sc[2] = {R(0), R(0)}, ss[2] = {R(0), R(0)};
        R scc[2] = {R(0), R(0)}, scs[2] = {R(0), R(0)};
        const int xm = bc_index(x - 1, a.nx, a.bcx), xp = bc_index(x + 1, a.nx, a.bcx);
        const int ym = TWO_D ? bc_index(y - 1, a.ny, a.bcy) : y;
        const int yp = TWO_D ? bc_index(y + 1, a.ny, a.bcy) : y;
        const long long dym = (long long)(ym - y) * a.nx, dyp = (long long)(yp - y) * a.nx;
#pragma unroll 1
        for (int rho = 0; rho < NR; ++rho) {
        const int vw = rho * a.Gs + q;
        const int i0 = r * a.K + vw * a.P;
        // populations of this group (FULL: every group owns exactly P)
        const int pc = FULL ? P : min(a.P, a.K - vw * a.P);
        const R *tab = reinterpret_cast<const R *>(a.poptab) + (long long)i0 * TW;
        const unsigned long long mx = stream ? __ldg(a.masks + 2 * (r * Gv + vw)) : 0ull;
        const unsigned long long my = stream ? __ldg(a.masks + 2 * (r * Gv + vw) + 1) : 0ull;
        const St *base = fin + (long long)i0 * S + (long long)y * a.nx;
        // Loads first (a chunk of populations at a time, all independent), then
        // arithmetic: the pull direction of population k comes from the warp's
        // sign masks, so no load waits for the table.
        constexpr int CH = TWO_D ? (P > 16 ? 8 : P) : (P > 32 ? 16 : P);
#pragma unroll
        for (int c0 = 0; c0 < P; c0 += CH) {
            R fa[CH], fb[CH], fc[TWO_D ? CH : 1], fd[TWO_D ? CH : 1];
#pragma unroll
            for (int kk = 0; kk < CH; ++kk) {
                const int k = c0 + kk;
                const St *pk = base + (long long)k * S;
                if (k < pc && LATTICE) { // perfect streaming: f_i(x - n_i), Sec. 2.3
                    const int2 sh = __ldg(a.shifts + i0 + k);
                    const int xs = bc_any(x - sh.x, a.nx, a.bcx), ys = bc_any(y - sh.y, a.ny, a.bcy);
                    fa[kk] = Io<St, R>::ld(fin + (long long)(i0 + k) * S + (long long)ys * a.nx + xs);
                } else if (k < pc) {
                    fa[kk] = Io<St, R>::ld(pk + x);
                    if (stream) {
                        const int xs = ((mx >> k) & 1ull) ? xm : xp; // pull from x - sgn(v_x)
                        fb[kk] = Io<St, R>::ld(pk + xs);
                        if (TWO_D) {
                            const long long dy = ((my >> k) & 1ull) ? dym : dyp;
                            fc[kk] = Io<St, R>::ld(pk + dy + x);
                            fd[kk] = Io<St, R>::ld(pk + dy + xs);
                        }
                    }
                }
            }
#pragma unroll
            for (int kk = 0; kk < CH; ++kk) {
                const int k = c0 + kk;
                if (k < pc) {
                    R c, s, cc, cs;
                    ld4<R>(tab + k * TW, c, s, cc, cs);
                    R v = fa[kk];
                    if (stream) {
                        v = v + fabs(c) * (fb[kk] - v);
                        if (TWO_D) {
                            const R hi = fc[kk] + fabs(c) * (fd[kk] - fc[kk]);
                            v = v + fabs(s) * (hi - v);
                        }
                    }
                    fs[k] = v;
                    s0[k & 1] += v;
                    sc[k & 1] += c * v;
                    ss[k & 1] += s * v;
                    scc[k & 1] += cc * v;
                    scs[k & 1] += cs * v;
                }
            }
        }
        // free streaming stores every group now; a collision parks all groups but the last
        if (STEP && (!need_site || rho + 1 < NR) && act) {
            St *ob = fout + (long long)i0 * S + site;
#pragma unroll
            for (int k = 0; k < P; ++k)
                if (k < pc) Io<St, R>::st(ob + (long long)k * S, fs[k]);
        }
        } // groups
        if (need_site) {
            red[(0 * G + g) * 32 + lane] = LR(s0[0] + s0[1]);
            red[(1 * G + g) * 32 + lane] = LR(sc[0] + sc[1]);
            red[(2 * G + g) * 32 + lane] = LR(ss[0] + ss[1]);
            red[(3 * G + g) * 32 + lane] = LR(scc[0] + scc[1]);
            red[(4 * G + g) * 32 + lane] = LR(scs[0] + scs[1]);
        }
    }

    if (!need_site) return; // free streaming: f <- f*, stored above
    if (MODE != MODE_INIT) __syncthreads();
    if (MODE == MODE_MOMENTS && g != 0) return;

    // the Landau frame of the tile's 32 sites and every warp's own shell coefficients:
    // with an FP64 per-site part once per site (ONCE), with a double-float one
    // once per site (DDS: FP32 storage, FP32 LR), else in every warp
    constexpr bool ONCE = (sizeof(LR) == 8) && STEP && !QUANT;
    constexpr bool DDS = (sizeof(St) == 4) && (sizeof(LR) == 4) && STEP && !QUANT;
    constexpr int W = (N + 1) * (N + 1);
    // ONCE: [W + 3][32] LR; DDS: [2 W + 3][32] floats (the sums as hi, lo rows, then
    // U^a / tau), then site_split_dd's frame and partial sums
    LR *wsh = reinterpret_cast<LR *>(smem_raw + size_t(5) * G * 32 * sizeof(LR));
    (void)wsh;
    LR n = LR(0), eps = LR(0), U0 = LR(0), Ux = LR(0), Uy = LR(0), T = LR(0);
    if constexpr (DDS) {
        // FP32 storage: the moment fold, the Landau frame and the shell-independent
        // sums in double-float (FP64-class accuracy on the FP32 pipes), split over
        // the CTA's warps by sample direction; U^a / tau follow in rows 2 W + 0..2
        float *sres = reinterpret_cast<float *>(wsh);
        float *fr = sres + (2 * W + 3) * 32;
        site_split_dd<N, 32>(a, reinterpret_cast<const float *>(red), G, g * 32 + lane, G * 32, act, sres, fr,
                             fr + kSplitFrameRows(N) * 32);
    } else if (MODE == MODE_INIT) {
        const double bx = a.in_bx[site], by = a.in_by[site];
        const double gam = 1.0 / sqrt(1.0 - bx * bx - by * by);
        n = LR(a.in_n[site]);
        T = LR(a.in_T[site]);
        U0 = LR(gam);
        Ux = LR(gam * bx);
        Uy = LR(gam * by);
        eps = LR(2) * n * T;
    } else if constexpr (ONCE) {
        // FP64 per-site part of a step: warp 0 solves the Landau frame of the
        // tile's 32 sites and forms the shell-independent sums w_{m,k} once; the
        // other warps read them (and U^a) from shared memory after the moments
        if (g == 0) {
            LR m[8];
            fold_moments<N, LR>(a, red, G, lane, m);
            const bool ok = site_landau<St, LR>(m, n, eps, U0, Ux, Uy);
            T = eps / (LR(2) * n);
            if (!ok && act) atomicOr(a.status, 1);
            LR tk[N + 1];
            tk[0] = n / T;
#pragma unroll
            for (int k = 1; k <= N; ++k) tk[k] = (k == 1) ? n : tk[k - 1] * T;
            site_sums<N, LR>(a, tk, U0, Ux, Uy, wsh + lane, 32);
            wsh[(W + 0) * 32 + lane] = U0;
            wsh[(W + 1) * 32 + lane] = Ux;
            wsh[(W + 2) * 32 + lane] = Uy;
        }
        __syncthreads();
        U0 = wsh[(W + 0) * 32 + lane];
        Ux = wsh[(W + 1) * 32 + lane];
        Uy = wsh[(W + 2) * 32 + lane];
    } else {
        LR m[8];
        fold_moments<N, LR>(a, red, G, lane, m);
        const bool ok = site_landau<St, LR>(m, n, eps, U0, Ux, Uy);
        T = eps / (LR(2) * n);
        if (!ok && act && g == 0) atomicOr(a.status, 1);
    }
    // quantum statistics: (T, z) of the equilibrium with these (n, eps), or z of (n, T) at init.
    // Warp 0 solves for its 32 sites and passes (eta, T) on through shared memory
    // (after the angular sums: qsh = [2][32] doubles); in the moments pass only warp 0 runs.
    LR tkq[N + 1];
    if constexpr (QUANT) {
        // warp 0 solves each site and forms its radial weights once; the other
        // warps read T and t_k from shared memory (qsh = [1 + N + 1][32] doubles)
        double qeta = 0.0, qT = T;
        double *qsh = reinterpret_cast<double *>(smem_raw + size_t(5) * G * 32 * sizeof(LR));
        if (g == 0) {
            // warm start from the site's eta of the previous solve, kept in a.qeta
            const double x0 = a.qeta ? a.qeta[site] : __longlong_as_double(0x7ff8000000000000ll);
            double phr[N + 1]; // phi_1..phi_{N+1} at the solved eta (steps)
            const bool ok = (MODE == MODE_INIT) ? stat_fugacity(n, T, a.gdeg, a.stat, qeta)
                                                : stat_solve(n, eps, a.gdeg, a.stat, qeta, qT, x0,
                                                             MODE == MODE_MOMENTS ? nullptr : phr,
                                                             MODE == MODE_MOMENTS ? 0 : N + 1,
                                                             sizeof(St) == 8 ? 1e-10 : 1e-5);
            if (!ok && act) atomicOr(a.status, 1);
            if (a.qeta && act && MODE != MODE_MOMENTS) a.qeta[site] = qeta;
            if (MODE != MODE_MOMENTS) {
                if (MODE == MODE_INIT) stat_radial<N>(qT, qeta, a.gdeg, a.stat, tkq);
                else stat_radial_from_phi<N>(qT, a.gdeg, phr, tkq);
                qsh[lane] = qT;
#pragma unroll
                for (int k = 0; k <= N; ++k) qsh[(1 + k) * 32 + lane] = tkq[k];
            }
        }
        if (MODE != MODE_MOMENTS) {
            __syncthreads();
            qT = qsh[lane];
#pragma unroll
            for (int k = 0; k <= N; ++k) tkq[k] = qsh[(1 + k) * 32 + lane];
        }
        T = qT;
    }
    if (MODE == MODE_MOMENTS) {
        if (act) {
            a.out[0][site] = double(n);
            a.out[1][site] = double(eps);
            a.out[2][site] = double(T);
            a.out[3][site] = double(U0);
            a.out[4][site] = double(Ux);
            a.out[5][site] = double(Uy);
        }
        return;
    }
    R cr[NC];
    if constexpr (QUANT)
        shell_coefficients_tk<N, LR, R>(a, r, tkq, U0, Ux, Uy, cr);
    else if constexpr (DDS)
        shell_from_sums_dd<N>(a, r, reinterpret_cast<const float *>(wsh) + lane, 32, cr);
    else if constexpr (ONCE)
        shell_from_sums<N, LR, R>(a, r, wsh + lane, 32, cr);
    else
        shell_coefficients<N, LR, R>(a, r, n, T, U0, Ux, Uy, cr);
    const LR itau = Par<LR>::inv_tau(a);
    R o0 = R(U0 * itau), o1 = R(Ux * itau), o2 = R(Uy * itau);
    if constexpr (DDS) {
        o0 = wsh[(2 * W + 0) * 32 + lane];
        o1 = wsh[(2 * W + 1) * 32 + lane];
        o2 = wsh[(2 * W + 2) * 32 + lane];
    }
    constexpr bool kSR = (sizeof(St) <= 4) && STEP; // FP32 and 16-bit stores round stochastically
    unsigned rng = 0;
    if (kSR) rng = mix32(unsigned(site) * 64u + unsigned(g) ^ mix32(__ldcg(a.ctr) * 0x9E3779B9u + 1u));
#pragma unroll 1
    for (int rho = NR - 1; rho >= 0; --rho) {
    const int vw = rho * a.Gs + q;
    const int i0 = r * a.K + vw * a.P;
    const int pc = FULL ? P : min(a.P, a.K - vw * a.P);
    const R *tab = reinterpret_cast<const R *>(a.poptab) + (long long)i0 * TW;
    St *obase = fout + (long long)i0 * S + site;
    if (STEP && rho + 1 < NR && act) { // parked group: f* back from its output slot
#pragma unroll
        for (int k = 0; k < P; ++k)
            if (k < pc) fs[k] = Io<St, R>::lds(obase + (long long)k * S);
    }
#pragma unroll
    for (int k = 0; k < P; ++k) {
        if (k < pc) {
            const R *t = tab + k * TW;
            R c, s, e0, e1;
            ld4<R>(t, c, s, e0, e1); // e0 = cc, e1 = cs (unused here)
            R E[TW - 4];
#pragma unroll
            for (int u = 0; u < TW - 4; u += 4) ld4<R>(t + 4 + u, E[u], E[u + 1], E[u + 2], E[u + 3]);
            R feq = cr[0] * E[0];
#pragma unroll
            for (int t2 = 1; t2 < NC; ++t2) feq += cr[t2] * E[t2];
            if (MODE == MODE_INIT) {
                if (act) Io<St, R>::st(obase + (long long)k * S, feq);
            } else {
                const R om = o0 - o1 * c - o2 * s;
                if (act) relax_store<St, R>(obase + (long long)k * S, fs[k], om, feq, rng);
            }
        }
    }
    } // groups
    if (kSR) {
        __syncthreads();
        if (threadIdx.x == 0 && threadIdx.y == 0) advance_launch_counter(a.ctr, gridDim.x * gridDim.y);
    }
}

} // namespace rlbmk
