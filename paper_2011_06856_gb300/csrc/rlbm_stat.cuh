// Fermi-Dirac and Bose-Einstein equilibria (Eq. feq_dist with eps = +1, -1),
// FP64, for the per-site part of the per-tile kernel and for host checks.
//
// f^eq = g / (z^-1 exp(U.p / T) + eps).  Its rest-frame radial integrals are
//   int_0^inf f p^k dp = g T^(k+1) k! phi_{k+1}(z),
//   phi_s = -Li_s(-z) (Fermi-Dirac),  Li_s(z) (Bose-Einstein, z < 1),
// so n = 2 pi g T^2 phi_2, e = 4 pi g T^3 phi_3 (massless, 2+1 dimensions) and
// the projection weights of the truncated equilibrium take
// 2 pi g T^(k+1) phi_{k+1}(z) where Maxwell-Juttner has n T^(k-1).
// Everything is a function of eta = ln z; d phi_s / d eta = phi_{s-1}.
#pragma once

#include <math.h>

// RLBM_HD: small helpers, inlined; RLBM_HDX: the solvers, called (one copy per
// translation unit instead of one per kernel instance).
#ifdef __CUDACC__
#define RLBM_HD __host__ __device__ __forceinline__
#define RLBM_HDX static __host__ __device__ __noinline__
#else
#define RLBM_HD inline
#define RLBM_HDX static inline
#endif

namespace rlbmk {


RLBM_HD double stat_ipow(double x, int e)
{
    double r = 1.0;
    for (int i = 0; i < e; ++i) r *= x;
    return r;
}

// sum_{j>=1} (-1)^(j+1) x^j / j^s for 0 < x <= 1 (= -Li_s(-x)), by the
// convergence acceleration of Cohen, Rodriguez Villegas and Zagier (Exp. Math.
// 9 (2000), Algorithm 1): the terms x^(k+1)/(k+1)^s form a totally monotone
// sequence, and n = 24 terms leave an error below 2 (3 + sqrt 8)^-24 ~ 1e-18 of
// the first.  The algorithm's weights c_k / d do not depend on x or s: they are
// formed once, at compile time, with the reciprocals 1 / (k + 1), so a term
// costs multiplications only.  d = ((3 + sqrt 8)^n + (3 + sqrt 8)^-n) / 2 is the
// Chebyshev value T_n(3), from T_{k+1} = 6 T_k - T_{k-1}, T_0 = 1, T_1 = 3.
constexpr int kStatTerms = 24;
// 16 terms (error below 2 (3 + sqrt 8)^-16 ~ 1e-12 of the first): the
// FP32-storage solve, whose accepted FP64 step needs no more.
constexpr int kStatTermsShort = 16;
struct StatSeriesTab {
    double w[kStatTerms];   // c_k / d
    double inv[kStatTerms]; // 1 / (k + 1)
};
constexpr StatSeriesTab stat_series_tab(int n)
{
    StatSeriesTab t{};
    double tm = 1.0, tc = 3.0;
    for (int k = 1; k < n; ++k) {
        const double tn = 6.0 * tc - tm;
        tm = tc;
        tc = tn;
    }
    const double d = tc;
    double b = -1.0, c = -d;
    for (int k = 0; k < n; ++k) {
        c = b - c;
        t.w[k] = c / d;
        t.inv[k] = 1.0 / (k + 1.0);
        b = (double(k) + n) * (double(k) - n) * b / ((k + 0.5) * (k + 1.0));
    }
    return t;
}
#ifdef __CUDACC__
static __constant__ StatSeriesTab kStatSeriesDev = stat_series_tab(kStatTerms);
static __constant__ StatSeriesTab kStatSeriesShortDev = stat_series_tab(kStatTermsShort);
#endif
static constexpr StatSeriesTab kStatSeriesHost = stat_series_tab(kStatTerms);
static constexpr StatSeriesTab kStatSeriesShortHost = stat_series_tab(kStatTermsShort);

RLBM_HD const StatSeriesTab &stat_series(bool short_series = false)
{
#ifdef __CUDA_ARCH__
    return short_series ? kStatSeriesShortDev : kStatSeriesDev;
#else
    return short_series ? kStatSeriesShortHost : kStatSeriesHost;
#endif
}

RLBM_HDX double stat_alt_series(int s, double x)
{
    const StatSeriesTab &tab = stat_series();
    double sum = 0.0, xk = x;
    for (int k = 0; k < kStatTerms; ++k) {
        double t = tab.w[k] * xk;
        const double r = tab.inv[k];
        for (int q = 0; q < s; ++q) t *= r;
        sum += t;
        xk *= x;
    }
    return sum;
}

// The same series for every s = 1..smax at once (smax <= 6): the weights of the
// acceleration do not depend on s, so one pass over the 24 terms serves all
// orders, out[s-1] = sum_j (-1)^(j+1) x^j / j^s.
RLBM_HDX void stat_alt_series_upto(int smax, double x, double *out, bool short_series = false)
{
    const StatSeriesTab &tab = stat_series(short_series);
    const int nt = short_series ? kStatTermsShort : kStatTerms;
    double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    double xk = x;
    for (int k = 0; k < nt; ++k) {
        double t = tab.w[k] * xk;
        const double r = tab.inv[k];
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            t *= r;
            if (q < smax) acc[q] += t;
        }
        xk *= x;
    }
#pragma unroll
    for (int q = 0; q < 6; ++q)
        if (q < smax) out[q] = acc[q];
}

// Fermi-Dirac F_s(eta) = -Li_s(-e^eta), s >= 1.  eta <= 0: the alternating series
// at x = e^eta; eta > 0: the inversion identity for integer s,
//   F_s(eta) = (-1)^(s+1) F_s(-eta) + 2 sum_{j=0}^{s/2} eta_D(2j) eta^(s-2j) / (s-2j)!,
// with the Dirichlet eta values eta_D(0) = 1/2, eta_D(2) = pi^2/12,
// eta_D(4) = 7 pi^4/720, eta_D(6) = 31 pi^6/30240.
RLBM_HDX double stat_fd(int s, double eta)
{
    if (s == 0) return 1.0 / (1.0 + exp(-eta)); // d F_1 / d eta
    if (eta <= 0.0) return stat_alt_series(s, exp(eta));
    const double pi2 = 9.8696044010893586188; // pi^2
    const double etaD[4] = {0.5, pi2 / 12.0, 7.0 * pi2 * pi2 / 720.0, 31.0 * pi2 * pi2 * pi2 / 30240.0};
    double poly = 0.0;
    for (int j = 0; 2 * j <= s; ++j) {
        const int m = s - 2 * j;
        double fact = 1.0;
        for (int i = 2; i <= m; ++i) fact *= i;
        poly += etaD[j] * stat_ipow(eta, m) / fact;
    }
    const double mirror = stat_alt_series(s, exp(-eta));
    return ((s & 1) ? mirror : -mirror) + 2.0 * poly;
}

// Bose-Einstein Li_s(e^eta), eta < 0, s >= 1.  z <= 1/2: the defining series;
// above, the duplication formula Li_s(z) = 2^(1-s) Li_s(z^2) + F_s(ln z) (from
// Li_s(z) + Li_s(-z) = 2^(1-s) Li_s(z^2)), applied until z^(2^m) <= 1/2.
RLBM_HDX double stat_be(int s, double eta)
{
    if (s == 0) return 1.0 / (exp(-eta) - 1.0); // d Li_1 / d eta
    if (s == 1) return -log1p(-exp(eta));
    double scale = 1.0, acc = 0.0, e = eta;
    const double half = -0.69314718055994530942; // ln 1/2
    int guard = 0;
    while (e > half && guard < 64) {
        acc += scale * stat_fd(s, e);
        scale *= stat_ipow(0.5, s - 1);
        e *= 2.0;
        ++guard;
    }
    const double z = exp(e);
    double term = z, sum = 0.0;
    for (int k = 1; k <= 64; ++k) {
        sum += term / stat_ipow(double(k), s);
        term *= z;
    }
    return acc + scale * sum;
}

// phi_1 .. phi_smax at once (smax <= 6): Fermi-Dirac from one pass of the
// accelerated series (and the inversion identity for eta > 0), Bose-Einstein
// order by order.
RLBM_HDX void stat_phi_upto(int smax, double eta, int stat, double *phi, bool short_series = false)
{
    if (stat < 0) {
        for (int q = 1; q <= smax; ++q) phi[q - 1] = stat_be(q, eta);
        return;
    }
    if (eta <= 0.0) {
        stat_alt_series_upto(smax, exp(eta), phi, short_series);
        return;
    }
    const double pi2 = 9.8696044010893586188; // pi^2
    const double etaD[4] = {0.5, pi2 / 12.0, 7.0 * pi2 * pi2 / 720.0, 31.0 * pi2 * pi2 * pi2 / 30240.0};
    double mirror[6];
    stat_alt_series_upto(smax, exp(-eta), mirror, short_series);
    for (int q = 1; q <= smax; ++q) {
        double poly = 0.0;
        for (int j = 0; 2 * j <= q; ++j) {
            const int m = q - 2 * j;
            double fact = 1.0;
            for (int i = 2; i <= m; ++i) fact *= i;
            poly += etaD[j] * stat_ipow(eta, m) / fact;
        }
        phi[q - 1] = ((q & 1) ? mirror[q - 1] : -mirror[q - 1]) + 2.0 * poly;
    }
}

// phi_s(eta) of the statistic (+1 Fermi-Dirac, -1 Bose-Einstein), s = 0..6.
RLBM_HD double stat_phi(int s, double eta, int stat) { return stat > 0 ? stat_fd(s, eta) : stat_be(s, eta); }

// Fermi-Dirac phi_1..phi_3 in FP32 (the same series and inversion identity),
// for the FP32 Newton steps that start stat_solve.
RLBM_HD void stat_fd3_f(float eta, float *phi)
{
    const StatSeriesTab &tab = stat_series();
    const float x = expf(-fabsf(eta));
    float a1 = 0.f, a2 = 0.f, a3 = 0.f, xk = x;
    for (int k = 0; k < kStatTerms; ++k) {
        const float r = float(tab.inv[k]);
        float t = float(tab.w[k]) * xk * r;
        a1 += t;
        t *= r;
        a2 += t;
        t *= r;
        a3 += t;
        xk *= x;
    }
    if (eta <= 0.f) {
        phi[0] = a1;
        phi[1] = a2;
        phi[2] = a3;
        return;
    }
    const float pi2 = 9.8696044f;
    // F_s(eta) = (-1)^(s+1) F_s(-eta) + 2 sum_j eta_D(2j) eta^(s-2j) / (s-2j)!
    phi[0] = a1 + 2.f * (0.5f * eta);
    phi[1] = -a2 + 2.f * (0.5f * eta * eta * 0.5f + pi2 / 12.f);
    phi[2] = a3 + 2.f * (0.5f * eta * eta * eta / 6.f + (pi2 / 12.f) * eta);
}

// FP32 Newton steps on the equation of stat_solve (Fermi-Dirac), from x: the
// start of its FP64 steps, accurate to about 1e-7.  Returns x unchanged where a
// step leaves the bracket (lo, hi) or the FP32 values are not positive.
RLBM_HD double stat_presolve_fd(double L, double x, double lo, double hi)
{
    float xf = float(x);
    const float Lf = float(L);
    for (int it = 0; it < 12; ++it) {
        float ph[3];
        stat_fd3_f(xf, ph);
        if (!(ph[0] > 0.f && ph[1] > 0.f && ph[2] > 0.f)) return x;
        const float H = logf(ph[2]) - 1.5f * logf(ph[1]) - Lf;
        const float dH = ph[1] / ph[2] - 1.5f * ph[0] / ph[1];
        const float xn = xf - H / dH;
        if (!(double(xn) > lo && double(xn) < hi)) return x;
        const bool done = fabsf(xn - xf) <= 1e-5f * (1.f + fabsf(xf));
        xf = xn;
        if (done) break;
    }
    return double(xf);
}

// (eta, T) of the equilibrium with density n and energy density e:
// ln phi_3 - 3/2 ln phi_2 = ln(e sqrt(2 pi g) / (2 n^1.5)) =: L is decreasing in eta
// (Maxwell-Boltzmann limit: -eta/2).  Start: x0 (the previous step's eta of the
// site; NaN or out of range: the Maxwell-Boltzmann value), refined by FP32 Newton
// steps for Fermi-Dirac; then FP64 Newton steps kept inside a bisection bracket
// (at most 100), until a Newton step is below tol (1 + |eta|).  With quadratic
// convergence the accepted iterate's error is about the square of that step:
// tol = 1e-10 leaves eta exact to rounding (FP64 storage); tol = 1e-5 accepts the
// first FP64 step after the FP32 ones, whose error stays below 1e-12 (FP32
// storage, whose own rounding is 1e-7).  phi_root (may be
// NULL): phi_1..phi_nphi at the returned eta (nphi <= 6), from the last
// evaluation by d phi_s / d eta = phi_{s-1} (the step is below 1e-10).  Returns
// false for a Bose-Einstein state beyond condensation (no z < 1), or bad
// input; eta then sits at the bracket end.
RLBM_HDX bool stat_solve(double n, double e, double g, int stat, double &eta, double &T, double x0,
                         double *phi_root = nullptr, int nphi = 0, double tol = 1e-10)
{
    const double twopi = 6.283185307179586477;
    if (!(n > 0.0) || !(e > 0.0)) { eta = -30.0; T = 1.0; return false; }
    const double L = log(e * sqrt(twopi * g) / (2.0 * n * sqrt(n)));
    double lo = -60.0, hi = stat > 0 ? 700.0 : -1e-13;
    double x = (x0 > lo && x0 < hi) ? x0 : -2.0 * L;
    if (x <= lo) x = lo + 1.0;
    if (x >= hi) x = stat > 0 ? hi - 1.0 : -1e-3;
    if (stat > 0) x = stat_presolve_fd(L, x, lo, hi);
    const int nq = nphi > 6 ? 6 : (nphi > 3 ? nphi : 3);
    const bool short_series = tol >= 1e-6; // the FP32-storage rule: 16 terms suffice
    bool ok = false;
    double xl = x, phl[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0}; // the last evaluation point and phi there
    for (int it = 0; it < 100; ++it) {
        stat_phi_upto(nq, x, stat, phl, short_series);
        xl = x;
        const double p1 = phl[0], p2 = phl[1], p3 = phl[2];
        const double H = log(p3) - 1.5 * log(p2) - L;
        if (H > 0.0) lo = x; else hi = x;
        const double dH = p2 / p3 - 1.5 * p1 / p2;
        double xn = x - H / dH;
        const bool newton = xn > lo && xn < hi;
        if (!newton) xn = 0.5 * (lo + hi);
        if (newton && fabs(xn - x) <= tol * (1.0 + fabs(x))) { x = xn; ok = true; break; }
        x = xn;
        if (hi - lo < 1e-15 * (1.0 + fabs(x))) { ok = true; break; }
    }
    if (stat < 0 && !(x < -1e-12)) ok = false; // condensation: no Bose-Einstein equilibrium
    eta = x;
    double phr[6];
    const double dx = x - xl;
    if (fabs(dx) <= 1e-4 * (1.0 + fabs(x)) && phl[1] > 0.0) {
        // phi_s(x) = phi_s(xl) + phi_{s-1}(xl) dx + O(dx^2); phi_0 = d phi_1 / d eta
        // (dx <= tol: the second-order term is below 1e-10 relative for FP32 storage)
        const double phi0 = stat > 0 ? 1.0 / (1.0 + double(expf(float(-xl)))) : 1.0 / (exp(-xl) - 1.0);
        phr[0] = phl[0] + phi0 * dx;
        for (int q = 1; q < nq; ++q) phr[q] = phl[q] + phl[q - 1] * dx;
    } else {
        stat_phi_upto(nq, x, stat, phr, short_series);
    }
    T = sqrt(n / (twopi * g * phr[1]));
    if (phi_root)
        for (int q = 0; q < nphi && q < 6; ++q) phi_root[q] = phr[q];
    return ok;
}

// eta of the equilibrium with density n at temperature T: phi_2(eta) = n / (2 pi g T^2).
RLBM_HDX bool stat_fugacity(double n, double T, double g, int stat, double &eta)
{
    const double twopi = 6.283185307179586477;
    const double target = log(n / (twopi * g * T * T));
    double lo = -60.0, hi = stat > 0 ? 700.0 : -1e-13;
    double x = target; // Maxwell-Boltzmann start (phi_2 = z)
    if (x <= lo) x = lo + 1.0;
    if (x >= hi) x = stat > 0 ? hi - 1.0 : -1e-3;
    bool ok = false;
    for (int it = 0; it < 100; ++it) {
        double ph[2];
        stat_phi_upto(2, x, stat, ph);
        const double p1 = ph[0], p2 = ph[1];
        const double H = log(p2) - target; // increasing in eta
        if (H < 0.0) lo = x; else hi = x;
        double xn = x - H * p2 / p1;
        if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
        if (fabs(xn - x) <= 1e-15 * (1.0 + fabs(x))) { x = xn; ok = true; break; }
        x = xn;
        if (hi - lo < 1e-15 * (1.0 + fabs(x))) { ok = true; break; }
    }
    if (stat < 0 && !(x < -1e-12)) ok = false;
    eta = x;
    return ok;
}

// Radial weights tk[k] = 2 pi g T^(k+1) phi_{k+1}, k = 0..N, from phi_1..phi_{N+1}.
template <int N>
RLBM_HD void stat_radial_from_phi(double T, double g, const double *ph, double *tk)
{
    const double twopi = 6.283185307179586477;
    double Tp = T;
    for (int k = 0; k <= N; ++k) {
        tk[k] = twopi * g * Tp * ph[k];
        Tp *= T;
    }
}

// Radial weights tk[k] = 2 pi g T^(k+1) phi_{k+1}(eta), k = 0..N.
template <int N>
RLBM_HD void stat_radial(double T, double eta, double g, int stat, double *tk)
{
    const double twopi = 6.283185307179586477;
    double ph[N + 1];
    stat_phi_upto(N + 1, eta, stat, ph);
    double Tp = T;
    for (int k = 0; k <= N; ++k) {
        tk[k] = twopi * g * Tp * ph[k];
        Tp *= T;
    }
}

} // namespace rlbmk
