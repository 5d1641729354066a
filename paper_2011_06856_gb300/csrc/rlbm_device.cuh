// Device side of the fused RLBM step (arXiv 2011.06856, Sec. 2.2): one CTA
// owns 32 consecutive sites of one grid row and all N_pop populations of
// them.  Warp g handles P populations of one energy shell r = g / Gs
// (Gs warps per shell), lane = site.  A step is:
//
//   pass 1  (every warp)   bilinear pull of its P populations (Eqs.
//           streaming, interpolation), kept in registers, and five
//           per-shell angular sums S0, Sc, Ss, Scc, Scs of them;
//   site    (warp 0)       the 5 x G partial sums folded with p_r, p_r^2 into
//           N^a and T^ab (Eq. discrete_sum_moments; T^yy = T^tt - T^xx on the
//           light cone), the Landau frame eps U^a = T^ab U_b (trace-free
//           cubic, Viete root + one Newton step, eigenvector by cross
//           products), n = U_a N^a, T = eps / 2n, and the truncated
//           equilibrium as one trigonometric polynomial of degree N in theta
//           per shell (see feq_coefficients);
//   pass 2  (every warp)   f^eq_i from those coefficients, relaxation
//           f <- f* + omega_i (f^eq - f*), omega_i = (U^0 - U.v_i)/tau
//           (Eq. discrete-rbe), one store per population.
//
// Populations are read once and written once per step; halo values of the
// neighbouring tile come through L1/L2.  All per-population constants are
// warp-uniform loads of a small table (L1 resident).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "rlbm_args.h"

namespace rlbmk {

// ---- storage <-> compute conversions -------------------------------------
template <class St, class R> struct Io;
template <> struct Io<double, double> {
    static __device__ __forceinline__ double ld(const double *p) { return __ldg(p); }
    static __device__ __forceinline__ void st(double *p, double v) { *p = v; }
};
template <> struct Io<float, float> {
    static __device__ __forceinline__ float ld(const float *p) { return __ldg(p); }
    static __device__ __forceinline__ void st(float *p, float v) { *p = v; }
};
template <> struct Io<__half, float> {
    static __device__ __forceinline__ float ld(const __half *p)
    {
        return __half2float(__ushort_as_half(__ldg(reinterpret_cast<const unsigned short *>(p))));
    }
    static __device__ __forceinline__ void st(__half *p, float v) { *p = __float2half_rn(v); }
};
template <> struct Io<__nv_bfloat16, float> {
    static __device__ __forceinline__ float ld(const __nv_bfloat16 *p)
    {
        return __bfloat162float(
            __ushort_as_bfloat16(__ldg(reinterpret_cast<const unsigned short *>(p))));
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

__device__ __forceinline__ int bc_index(int i, int L, int bc)
{
    if (bc == 0) return i < 0 ? i + L : (i >= L ? i - L : i);
    return i < 0 ? 0 : (i >= L ? L - 1 : i);
}

// Landau frame of the moments m = (N^t, N^x, N^y, T^tt, T^tx, T^ty, T^xx, T^xy)
// with T^yy = T^tt - T^xx (massless: T^a_a = 0).  A = T eta has zero trace, so
// its characteristic polynomial is lambda^3 + c1 lambda - c0; the largest
// real root is the energy density.  Returns false for a non-physical state
// (then a rest frame with n = N^t is returned so the caller stays finite).
template <class LR>
__device__ __forceinline__ bool landau_frame(const LR *m, LR &n, LR &eps, LR &U0, LR &Ux, LR &Uy)
{
    const LR Nt = m[0], Nx = m[1], Ny = m[2];
    const LR Ttt = m[3], Ttx = m[4], Tty = m[5], Txx = m[6], Txy = m[7];
    const LR Tyy = Ttt - Txx;
    const LR c1 = -Ttt * Ttt + Ttx * Ttx + Tty * Tty + Txx * Tyy - Txy * Txy;
    const LR c0 = Ttt * (Txx * Tyy - Txy * Txy) - Ttx * Ttx * Tyy + LR(2) * Ttx * Tty * Txy -
                  Tty * Tty * Txx;
    bool ok = c1 < LR(0);
    LR lam;
    {
        const LR r = r_sqrt(ok ? -c1 / LR(3) : LR(0));
        const LR r3 = r * r * r;
        LR arg = r3 > LR(0) ? c0 / (LR(2) * r3) : LR(1);
        arg = arg > LR(1) ? LR(1) : (arg < LR(-1) ? LR(-1) : arg);
        lam = LR(2) * r * r_cos(r_acos(arg) / LR(3));
        const LR P = (lam * lam + c1) * lam - c0;
        const LR dP = LR(3) * lam * lam + c1;
        if (dP != LR(0)) lam -= P / dP;
    }
    eps = lam;
    // eigenvector: orthogonal to the rows of A - eps I
    const LR a00 = Ttt - lam, a01 = -Ttx, a02 = -Tty;
    const LR a10 = Ttx, a11 = -Txx - lam, a12 = -Txy;
    const LR a20 = Tty, a21 = -Txy, a22 = -Tyy - lam;
    LR v0 = a01 * a12 - a02 * a11, v1 = a02 * a10 - a00 * a12, v2 = a00 * a11 - a01 * a10;
    LR nn = v0 * v0 + v1 * v1 + v2 * v2;
    {
        const LR w0 = a11 * a22 - a12 * a21, w1 = a12 * a20 - a10 * a22, w2 = a10 * a21 - a11 * a20;
        const LR wn = w0 * w0 + w1 * w1 + w2 * w2;
        if (wn > nn) { v0 = w0; v1 = w1; v2 = w2; nn = wn; }
        const LR z0 = a21 * a02 - a22 * a01, z1 = a22 * a00 - a20 * a02, z2 = a20 * a01 - a21 * a00;
        const LR zn = z0 * z0 + z1 * z1 + z2 * z2;
        if (zn > nn) { v0 = z0; v1 = z1; v2 = z2; nn = zn; }
    }
    const LR mink = v0 * v0 - v1 * v1 - v2 * v2;
    if (mink > LR(0)) {
        LR s = r_rsqrt(mink);
        if (v0 < LR(0)) s = -s;
        U0 = v0 * s;
        Ux = v1 * s;
        Uy = v2 * s;
    } else {
        ok = false;
        U0 = LR(1);
        Ux = LR(0);
        Uy = LR(0);
    }
    n = U0 * Nt - Ux * Nx - Uy * Ny;
    if (!(n > LR(0)) || !(eps > LR(0))) {
        ok = false;
        n = Nt > LR(0) ? Nt : LR(1e-30);
        if (!(eps > LR(0))) eps = Ttt > LR(0) ? Ttt : LR(1e-30);
    }
    return ok;
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
// Output coef[r][0] = Re C_{r,0} - beta; coef[r][2m-1], coef[r][2m] = Re, Im C_{r,m}.
template <int N, class LR>
__device__ __forceinline__ void feq_coefficients(const KernelArgs &a, const LR *rtab, LR n, LR T,
                                                 LR U0, LR Ux, LR Uy, LR *coef /* (N+1)(2N+1) */)
{
    LR accr[N + 1][N + 1], acci[N + 1][N + 1]; // [m][k]
#pragma unroll
    for (int m = 0; m <= N; ++m)
#pragma unroll
        for (int k = 0; k <= N; ++k) { accr[m][k] = LR(0); acci[m][k] = LR(0); }
    const LR inv1g = LR(1) / (LR(1) + U0);
#pragma unroll
    for (int j = 0; j <= N; ++j) {
        const LR cj = LR(a.smp_c[j]), sj = LR(a.smp_s[j]);
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
    LR tk[N + 1];
    tk[0] = n / T;
#pragma unroll
    for (int k = 1; k <= N; ++k) tk[k] = (k == 1) ? n : tk[k - 1] * T;
#pragma unroll
    for (int r = 0; r <= N; ++r) {
#pragma unroll
        for (int m = 0; m <= N; ++m) {
            LR cr = LR(0), ci = LR(0);
#pragma unroll
            for (int k = m; k <= N; ++k) {
                const LR wgt = rtab[(r * (N + 1) + m) * (N + 1) + k] * tk[k];
                cr += wgt * accr[m][k];
                ci += wgt * acci[m][k];
            }
            if (m == 0) {
                coef[r * (2 * N + 1)] = cr - LR(a.beta);
            } else {
                coef[r * (2 * N + 1) + 2 * m - 1] = cr;
                coef[r * (2 * N + 1) + 2 * m] = ci;
            }
        }
    }
}

template <class R> struct Vec4;
template <> struct Vec4<float> {
    using T = float4;
};
template <> struct Vec4<double> {
    using T = double4;
};

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

// St: storage type; R: per-population arithmetic; LR: per-site arithmetic
// (moment sums, Landau frame, equilibrium coefficients); N: quadrature order;
// P: populations per thread (compile-time upper bound); TWO_D: ny > 1.
template <class St, class R, class LR, int N, int P, bool TWO_D, int MODE>
__global__ void __launch_bounds__(kMaxWarps * 32) rlbm_kernel(const KernelArgs a)
{
    constexpr int NC = 2 * N + 1;
    constexpr int TW = tab_width(N);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x, g = threadIdx.y, G = blockDim.y;
    const int xr = blockIdx.x * 32 + lane;
    const bool act = xr < a.nx;
    const int x = act ? xr : a.nx - 1;
    const int y = blockIdx.y;
    const int r = g / a.Gs, q = g % a.Gs;
    const int i0 = r * a.K + q * a.P;
    const int pc = min(a.P, a.K - q * a.P); // populations of this warp
    const long long S = a.S;
    const long long site = (long long)y * a.nx + x;
    const R *tab = reinterpret_cast<const R *>(a.poptab) + (long long)i0 * TW;
    const St *fin = reinterpret_cast<const St *>(a.fin);
    St *fout = reinterpret_cast<St *>(a.fout);

    LR *red = reinterpret_cast<LR *>(smem_raw);                  // [5][G][32]
    LR *coefs = red + 5 * G * 32;                                  // [(N+1)*NC][32]
    LR *oms = coefs + (N + 1) * NC * 32;                           // [3][32]

    R fs[P];
    const bool stream = (MODE == MODE_STEP);
    const bool need_site = (MODE != MODE_STEP) || a.collide;

    if (MODE != MODE_INIT) {
        R s0 = R(0), sc = R(0), ss = R(0), scc = R(0), scs = R(0);
        const int xm = bc_index(x - 1, a.nx, a.bcx), xp = bc_index(x + 1, a.nx, a.bcx);
        const int ym = TWO_D ? bc_index(y - 1, a.ny, a.bcy) : y;
        const int yp = TWO_D ? bc_index(y + 1, a.ny, a.bcy) : y;
        const St *base = fin + (long long)i0 * S + (long long)y * a.nx;
#pragma unroll
        for (int k = 0; k < P; ++k) {
            if (k < pc) {
                R c, s, cc, cs;
                ld4<R>(tab + k * TW, c, s, cc, cs);
                R v;
                if (stream) {
                    const R ax = fabs(c);
                    const int xs = c >= R(0) ? xm : xp; // pull from x - sgn(v_x)
                    const R f00 = Io<St, R>::ld(base + x);
                    const R f01 = Io<St, R>::ld(base + xs);
                    R lo = f00 + ax * (f01 - f00);
                    if (TWO_D) {
                        const R ay = fabs(s);
                        const long long dy = (long long)((s >= R(0) ? ym : yp) - y) * a.nx;
                        const R f10 = Io<St, R>::ld(base + dy + x);
                        const R f11 = Io<St, R>::ld(base + dy + xs);
                        const R hi = f10 + ax * (f11 - f10);
                        lo = lo + ay * (hi - lo);
                    }
                    v = lo;
                } else {
                    v = Io<St, R>::ld(base + x);
                }
                fs[k] = v;
                s0 += v;
                sc += c * v;
                ss += s * v;
                scc += cc * v;
                scs += cs * v;
            }
            base += S;
        }
        if (need_site) {
            red[(0 * G + g) * 32 + lane] = LR(s0);
            red[(1 * G + g) * 32 + lane] = LR(sc);
            red[(2 * G + g) * 32 + lane] = LR(ss);
            red[(3 * G + g) * 32 + lane] = LR(scc);
            red[(4 * G + g) * 32 + lane] = LR(scs);
        }
    }

    if (need_site) {
        __syncthreads();
        if (g == 0) {
            LR n, eps, U0, Ux, Uy, T;
            bool ok = true;
            if (MODE == MODE_INIT) {
                const double bx = a.in_bx[site], by = a.in_by[site];
                const double gam = 1.0 / sqrt(1.0 - bx * bx - by * by);
                n = LR(a.in_n[site]);
                T = LR(a.in_T[site]);
                U0 = LR(gam);
                Ux = LR(gam * bx);
                Uy = LR(gam * by);
                eps = LR(2) * n * T;
            } else {
                const LR *sh = reinterpret_cast<const LR *>(a.shelltab);
                LR m[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) m[t] = LR(a.off[t]);
                for (int rr = 0; rr <= N; ++rr) {
                    LR p0 = LR(0), pc_ = LR(0), ps = LR(0), pcc = LR(0), pcs = LR(0);
                    for (int qq = 0; qq < a.Gs; ++qq) {
                        const int w = rr * a.Gs + qq;
                        p0 += red[(0 * G + w) * 32 + lane];
                        pc_ += red[(1 * G + w) * 32 + lane];
                        ps += red[(2 * G + w) * 32 + lane];
                        pcc += red[(3 * G + w) * 32 + lane];
                        pcs += red[(4 * G + w) * 32 + lane];
                    }
                    const LR f1 = sh[2 * rr], f2 = sh[2 * rr + 1];
                    m[0] += f1 * p0;
                    m[1] += f1 * pc_;
                    m[2] += f1 * ps;
                    m[3] += f2 * p0;
                    m[4] += f2 * pc_;
                    m[5] += f2 * ps;
                    m[6] += f2 * pcc;
                    m[7] += f2 * pcs;
                }
                ok = landau_frame<LR>(m, n, eps, U0, Ux, Uy);
                T = eps / (LR(2) * n);
                if (!ok && act) atomicOr(a.status, 1);
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
            } else {
                LR cf[(N + 1) * NC];
                feq_coefficients<N, LR>(a, reinterpret_cast<const LR *>(a.rtab), n, T, U0, Ux, Uy,
                                        cf);
#pragma unroll
                for (int t = 0; t < (N + 1) * NC; ++t) coefs[t * 32 + lane] = cf[t];
                const LR it = LR(a.inv_tau);
                oms[0 * 32 + lane] = U0 * it;
                oms[1 * 32 + lane] = Ux * it;
                oms[2 * 32 + lane] = Uy * it;
            }
        }
        __syncthreads();
    }
    if (MODE == MODE_MOMENTS) return;

    St *obase = fout + (long long)i0 * S + site;
    if (!need_site) { // free streaming: f <- f*
        if (act) {
#pragma unroll
            for (int k = 0; k < P; ++k)
                if (k < pc) Io<St, R>::st(obase + (long long)k * S, fs[k]);
        }
        return;
    }
    R cr[NC];
#pragma unroll
    for (int t = 0; t < NC; ++t) cr[t] = R(coefs[(r * NC + t) * 32 + lane]);
    const R o0 = R(oms[lane]), o1 = R(oms[32 + lane]), o2 = R(oms[64 + lane]);
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
            R out;
            if (MODE == MODE_INIT) {
                out = feq;
            } else {
                const R om = o0 - o1 * c - o2 * s;
                out = fs[k] + om * (feq - fs[k]);
            }
            if (act) Io<St, R>::st(obase + (long long)k * S, out);
        }
    }
}

} // namespace rlbmk
