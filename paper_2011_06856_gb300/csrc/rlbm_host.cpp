// Host side of librlbm.so: quadrature and projection tables (Sec. 2.3,
// Sec. 2.2), handle management and the C ABI of include/rlbm.h.
//
// The quadrature is computed here independently of any other component:
// Gauss-Laguerre nodes are the eigenvalues of the Laguerre Jacobi matrix
// (Golub-Welsch), found by Sturm-sequence bisection and polished by Newton
// steps on L_{N+1}; weights use the closed form printed in Sec. 2.3.
#include "rlbm.h"
#include "rlbm_args.h"
#include "rlbm_stat.cuh"

#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

namespace {

constexpr double kPi = 3.14159265358979323846264338327950288;

thread_local std::string g_create_error;

// ---------------------------------------------------------------- quadrature

// L_n(x) and L_{n-1}(x) by the three-term recurrence.
void laguerre_pair(int n, double x, double &ln, double &lnm1)
{
    double a = 1.0, b = 1.0 - x; // L_0, L_1
    if (n == 0) { ln = 1.0; lnm1 = 0.0; return; }
    for (int k = 1; k < n; ++k) {
        const double c = ((2.0 * k + 1.0 - x) * b - k * a) / (k + 1.0);
        a = b;
        b = c;
    }
    ln = b;
    lnm1 = a;
}

// Number of eigenvalues below x of the symmetric tridiagonal Jacobi matrix of
// the Laguerre weight (diagonal 2k+1, off-diagonal k), by Sturm sequence.
int sturm_count(int n, double x)
{
    int cnt = 0;
    double d = 1.0;
    for (int k = 0; k < n; ++k) {
        const double off2 = (k == 0) ? 0.0 : double(k) * double(k);
        d = (2.0 * k + 1.0 - x) - (k == 0 ? 0.0 : off2 / d);
        if (d == 0.0) d = -1e-300;
        if (d < 0.0) ++cnt;
    }
    return cnt;
}

// Gauss-Laguerre nodes (roots of L_n) in increasing order.
std::vector<double> laguerre_nodes(int n)
{
    std::vector<double> x(n);
    const double hi0 = 4.0 * n + 2.0; // Gershgorin bound: (2n-1) + 2(n-1) < 4n
    for (int k = 0; k < n; ++k) {
        double lo = 0.0, hi = hi0;
        // k-th eigenvalue: smallest x with sturm_count(x) >= k+1
        for (int it = 0; it < 2000; ++it) {
            const double mid = 0.5 * (lo + hi);
            if (mid <= lo || mid >= hi) break;
            if (sturm_count(n, mid) >= k + 1) hi = mid; else lo = mid;
        }
        double r = 0.5 * (lo + hi);
        for (int it = 0; it < 3; ++it) { // Newton: x L_n' = n (L_n - L_{n-1})
            double ln, lnm1;
            laguerre_pair(n, r, ln, lnm1);
            const double d = n * (ln - lnm1) / r;
            if (d == 0.0) break;
            const double step = ln / d;
            if (!std::isfinite(step)) break;
            r -= step;
        }
        x[k] = r;
    }
    return x;
}

// Cholesky inverse of a small SPD matrix (row-major); false if not SPD.
bool spd_inverse(int n, const std::vector<double> &A, std::vector<double> &inv)
{
    std::vector<double> L(n * n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j <= i; ++j) {
            double s = A[i * n + j];
            for (int k = 0; k < j; ++k) s -= L[i * n + k] * L[j * n + k];
            if (i == j) {
                if (s <= 0.0) return false;
                L[i * n + i] = std::sqrt(s);
            } else {
                L[i * n + j] = s / L[j * n + j];
            }
        }
    inv.assign(n * n, 0.0);
    for (int c = 0; c < n; ++c) { // solve L L^T x = e_c
        std::vector<double> z(n, 0.0);
        for (int i = 0; i < n; ++i) {
            double s = (i == c) ? 1.0 : 0.0;
            for (int k = 0; k < i; ++k) s -= L[i * n + k] * z[k];
            z[i] = s / L[i * n + i];
        }
        for (int i = n - 1; i >= 0; --i) {
            double s = z[i];
            for (int k = i + 1; k < n; ++k) s -= L[k * n + i] * inv[k * n + c];
            inv[i * n + c] = s / L[i * n + i];
        }
    }
    return true;
}

double factorial(int k)
{
    double r = 1.0;
    for (int i = 2; i <= k; ++i) r *= i;
    return r;
}

struct Quad {
    int N = 0, K = 0, npop = 0;
    std::vector<double> pr, wr;            // radial nodes / weights (N+1)
    std::vector<double> p0, vx, vy, w;     // per population
    bool onlat = false;                    // on-lattice rule: perfect streaming by (sx, sy)
    std::vector<int> sx, sy;               // per population integer stencil vector (on-lattice)
};

bool make_quadrature(int N, int K, Quad &q)
{
    if (N < 0 || N > 12 || K < 2 * N + 1) return false;
    q.N = N;
    q.K = K;
    q.npop = K * (N + 1);
    q.pr = laguerre_nodes(N + 1);
    q.wr.resize(N + 1);
    for (int r = 0; r <= N; ++r) { // w^(p)_r = p_r / ((N+2)^2 L_{N+2}(p_r)^2)
        double l, lm1;
        laguerre_pair(N + 2, q.pr[r], l, lm1);
        q.wr[r] = q.pr[r] / ((N + 2.0) * (N + 2.0) * l * l);
    }
    q.p0.resize(q.npop);
    q.vx.resize(q.npop);
    q.vy.resize(q.npop);
    q.w.resize(q.npop);
    for (int r = 0; r <= N; ++r)
        for (int j = 0; j < K; ++j) {
            const int i = r * K + j;
            const double th = (j + r / double(N + 1)) * (2.0 * kPi / K);
            double c = std::cos(th), s = std::sin(th);
            if (std::fabs(c) < 1e-15) c = 0.0; // exact axis directions
            if (std::fabs(s) < 1e-15) s = 0.0;
            q.p0[i] = q.pr[r];
            q.vx[i] = c;
            q.vy[i] = s;
            q.w[i] = q.wr[r] * (2.0 * kPi / K);
        }
    return true;
}

// On-lattice rule of Sec. 2.3 (Fig. 1, left), order N = 3: the 12 integer
// vectors of length 5 on each of the 4 Gauss-Laguerre shells,
// p = p_r (1, n / 5).  A product rule satisfies the orthonormal conditions
// (Eq. mj-orthogonal-conditions) when its radial part integrates p^k exactly
// for k <= 2N (the Gauss-Laguerre rule does to 2N+1) and its angular part
// integrates trigonometric polynomials of degree <= 2N = 6.  The stencil is
// invariant under rotations by 90 degrees, so every harmonic m not divisible by
// 4 sums to zero over it; with one weight v_a on the 4 axis vectors and one v_o
// on the 8 others, what remains is sum v = 2 pi (m = 0) and
// sum v cos 4 theta = 0 (m = 4):  4 v_a + 8 v_o = 2 pi,  4 v_a + S v_o = 0 with
// S = sum over the off-axis vectors of cos 4 theta (= 8 cos 4 atan(4/3)).
// Populations shell-major, i = 12 r + j, the vectors ordered by angle from 0.
bool make_onlattice_quadrature(Quad &q)
{
    const int N = 3, K = 12;
    if (!make_quadrature(N, K, q)) return false; // radial nodes and weights
    std::vector<std::pair<double, std::pair<int, int>>> vec;
    for (int a = -5; a <= 5; ++a)
        for (int b = -5; b <= 5; ++b)
            if (a * a + b * b == 25) {
                double th = std::atan2(double(b), double(a));
                if (th < 0.0) th += 2.0 * kPi;
                vec.push_back({th, {a, b}});
            }
    if (int(vec.size()) != K) return false;
    std::sort(vec.begin(), vec.end());
    double S = 0.0;
    for (auto &v : vec)
        if (v.second.first != 0 && v.second.second != 0) S += std::cos(4.0 * v.first);
    const double vo = 2.0 * kPi / (8.0 - S), va = -S * vo / 4.0;
    if (!(vo > 0.0) || !(va > 0.0)) return false;
    q.onlat = true;
    q.sx.assign(q.npop, 0);
    q.sy.assign(q.npop, 0);
    for (int r = 0; r <= N; ++r)
        for (int j = 0; j < K; ++j) {
            const int i = r * K + j;
            const int a = vec[j].second.first, b = vec[j].second.second;
            q.vx[i] = a / 5.0;
            q.vy[i] = b / 5.0;
            q.w[i] = q.wr[r] * ((a == 0 || b == 0) ? va : vo);
            q.sx[i] = a;
            q.sy[i] = b;
        }
    return true;
}

// ---------------------------------------------------------------- handle

// FP64 per-site tables (moment folds, projection weights) for the kernels of
// non-FP64 storage whose per-site part runs in FP64: the init and moments
// passes, the TMA-staged per-tile kernel, N >= 4 and the quantum statistics.
// (FP32-storage steps with N <= 3 in the per-tile, batched and
// two-sites-per-lane kernels run it in double-float from the split tables.)
//  - FP32 storage: an FP32 per-site part carries the conserved moments to a
//    relative bias of about 4e-7 per step, which the collision accumulates
//    linearly (1e-5 after a few hundred steps at tau ~ 4);
//  - N >= 4: the radial projection weights (inverse of a factorial Gram
//    matrix) cancel too many digits for FP32;
//  - the quantum statistics: the (T, z) solve.
// 16-bit storage accumulates in FP32 and solves the Landau frame in
// double-float (site_landau): its error is set by the storage rounding.
bool site_fp64_for(int prec, int N, int stat)
{
    return prec != RLBM_FP64 && (prec == RLBM_FP32 || N >= 4 || stat != 0);
}

size_t storage_size(int prec)
{
    switch (prec) {
    case RLBM_FP64: return 8;
    case RLBM_FP32: return 4;
    case RLBM_FP16_DEV:
    case RLBM_BF16_DEV:
    case RLBM_FP16_NORM:
    case RLBM_BF16_NORM: return 2;
    default: return 0;
    }
}

} // namespace

struct rlbm {
    rlbm_grid grid{};
    int N = 0, K = 0, npop = 0, prec = 0;
    double tau = 0.0;
    Quad q;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    void *buf = nullptr; // 2 population buffers
    bool own_buf = false;
    size_t pop_bytes = 0;
    int cur = 0; // index of the buffer holding the current state
    long long steps = 0;
    long long launches = 0;
    void *d_tabs = nullptr; // poptab | shelltab | rtab
    int *d_status = nullptr;
    rlbmk::KernelArgs base{};
    int P = 0, Gs = 0, G = 0;
    int R = 1; // groups of P populations per warp (K beyond one group per warp)
    int stat = 0;       // equilibrium statistic: 0 Maxwell-Juttner, +1 Fermi-Dirac, -1 Bose-Einstein
    double *d_qeta = nullptr; // quantum statistics: per-site eta of the last solve (Newton warm start)
    double gdeg = 1.0;  // normalisation g of the quantum statistics
    bool site_fp64 = false;
    // CUDA graphs of kGraphSteps steps starting from buffer 0 / buffer 1
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    // persistent TMA-staged step kernel (when the grid allows it)
    bool use_tma = false;
    rlbmk::TmaArgs *tma = nullptr; // [2]: input buffer 0 / 1
    int tma_grid = 0;
    size_t tma_smem = 0;
    int sm_count = 0;
    bool stall_next = false; // test hook: next launch waits for bytes that never arrive
    bool no_tma = false;     // tiling choice: per-tile kernel even where TMA is possible
    bool use_pair = false;   // two-sites-per-lane step kernel (rlbm_pair.cuh)
    bool pair_bulk = false;  // ... with its first pass staged by cp.async.bulk on interior tiles
    bool use_pair_tma = false;          // ... with the whole tile staged by TMA (rlbm_pair_tma.cuh)
    rlbmk::PairTmaArgs *ptma = nullptr; // [2]: input buffer 0 / 1
    size_t ptma_smem = 0;
    long long wait_cycles = 4000000000LL; // bound of the device waits (about 2 s at the maximum clock)
    std::string err;
};

namespace {

constexpr int kGraphSteps = 32;

rlbm_status fail(rlbm_t *h, rlbm_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (h) h->err = buf; else g_create_error = buf;
    return st;
}

rlbm_status cuda_fail(rlbm_t *h, cudaError_t e, const char *what)
{
    return fail(h, e == cudaErrorMemoryAllocation ? RLBM_ERR_OOM : RLBM_ERR_CUDA, "%s: %s (%s)",
                what, cudaGetErrorString(e), cudaGetErrorName(e));
}

#define RLBM_CUDA(h, call)                                                                       \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, #call);                                   \
    } while (0)

// Pick P (populations per warp, one of the compiled sizes) and Gs (warps per
// energy shell, G = Gs (N+1) warps per CTA): fewest idle population slots,
// then the larger P (fewer warps sharing the per-site work).
// Warps per shell and groups per warp of a tiling with P populations per
// warp: one group while ceil(K / P) warps per shell fit the CTA, otherwise
// as many warps as fit and several groups, but only when K exceeds what one
// group per warp can hold at all (K > 64 floor(16 / (N+1))).
int single_group_capacity(int N) { return 64 * (rlbmk::kMaxWarps / (N + 1)); }
bool group_tiling(int N, int K, int P, int &Gs, int &R)
{
    const int gs = (K + P - 1) / P;
    if (gs * (N + 1) <= rlbmk::kMaxWarps && (gs - 1) * P < K) {
        Gs = gs;
        R = 1;
        return true;
    }
    if (K <= single_group_capacity(N)) return false;
    Gs = rlbmk::kMaxWarps / (N + 1);
    R = (K + Gs * P - 1) / (Gs * P); // trailing groups may be empty (the kernel skips them)
    return true;
}

bool choose_tiling(int N, int K, int &P, int &Gs, int &R)
{
    static const int sizes[] = {8, 12, 16, 24, 32, 48, 64};
    R = 1;
    if (K > single_group_capacity(N)) { // fewest groups, then least padding
        int best = 1 << 30;
        for (int p : sizes) {
            int gs = 0, r = 0;
            if (!group_tiling(N, K, p, gs, r)) continue;
            const int score = r * 4096 + (r * gs * p - K);
            if (score < best) { best = score; P = p; Gs = gs; R = r; }
        }
        return best < (1 << 30);
    }
    int best_waste = 1 << 30;
    bool found = false;
    for (int gs = 1; gs * (N + 1) <= rlbmk::kMaxWarps; ++gs) {
        const int need = (K + gs - 1) / gs;
        if (need > 64 || (gs - 1) * need >= K) continue;
        int p = 0;
        for (int s : sizes)
            if (s >= need) { p = s; break; }
        const int waste = gs * p - K;
        if (waste < best_waste || (waste == best_waste && p > P)) {
            best_waste = waste;
            P = p;
            Gs = gs;
            found = true;
        }
    }
    return found;
}

template <class T>
void put(std::vector<unsigned char> &blob, size_t off, const std::vector<double> &v)
{
    for (size_t i = 0; i < v.size(); ++i) {
        T t = T(v[i]);
        std::memcpy(blob.data() + off + i * sizeof(T), &t, sizeof(T));
    }
}

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

rlbm_status build_tables(rlbm_t *h)
{
    const int N = h->N, K = h->K, npop = h->npop;
    const Quad &q = h->q;
    // 16-bit storage keeps f_i relative to the rest equilibrium at n = 1, T = 1,
    // f^rest_i = w_i / (2 pi):  f_i = alpha_i (s_i + beta), alpha_i = f^rest_i,
    // beta = 1 for the deviation form, 0 for the normalised form.
    const bool scaled = storage_size(h->prec) == 2;
    const bool dev = (h->prec == RLBM_FP16_DEV || h->prec == RLBM_BF16_DEV);
    const double beta = dev ? 1.0 : 0.0;
    const int TW = rlbmk::tab_width(N);

    // per-population table in stored units
    std::vector<double> pop(size_t(npop) * TW, 0.0);
    for (int i = 0; i < npop; ++i) {
        const double c = q.vx[i], s = q.vy[i];
        const double alpha = scaled ? q.w[i] / (2.0 * kPi) : 1.0;
        const double th = std::atan2(s, c);
        double *t = &pop[size_t(i) * TW];
        t[0] = c;
        t[1] = s;
        t[2] = c * c;
        t[3] = c * s;
        t[4] = q.w[i] / alpha;
        for (int m = 1; m <= N; ++m) {
            t[4 + 2 * m - 1] = q.w[i] / alpha * std::cos(m * th);
            t[4 + 2 * m] = q.w[i] / alpha * std::sin(m * th);
        }
    }
    // per-shell folds alpha_r p_r, alpha_r p_r^2
    std::vector<double> shell(size_t(N + 1) * 2);
    for (int r = 0; r <= N; ++r) {
        const double alpha = scaled ? q.w[r * K] / (2.0 * kPi) : 1.0;
        shell[2 * r] = alpha * q.pr[r];
        shell[2 * r + 1] = alpha * q.pr[r] * q.pr[r];
    }
    // projection weights R'[r][m][k] = sum_l p_r^l (G_m^-1)_{lk} / norm_m * k! / (N+1)
    std::vector<double> rt(size_t(N + 1) * (N + 1) * (N + 1), 0.0);
    for (int m = 0; m <= N; ++m) {
        const int d = N - m + 1;
        std::vector<double> Gm(d * d), Gi;
        for (int l = 0; l < d; ++l)
            for (int k = 0; k < d; ++k) Gm[l * d + k] = factorial(2 * m + l + k);
        if (!spd_inverse(d, Gm, Gi)) return fail(h, RLBM_ERR_ARG, "projection Gram matrix not SPD");
        const double norm = (m == 0) ? 2.0 * kPi : kPi;
        for (int r = 0; r <= N; ++r)
            for (int k = m; k <= N; ++k) {
                double s = 0.0;
                for (int l = m; l <= N; ++l) s += std::pow(q.pr[r], l) * Gi[(l - m) * d + (k - m)];
                rt[(size_t(r) * (N + 1) + m) * (N + 1) + k] = s / norm * factorial(k) / (N + 1);
            }
    }
    // moment contribution of the offset beta: beta * sum_i alpha_i p^a (p^b)
    double off[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (dev) {
        for (int i = 0; i < npop; ++i) {
            const double a = q.w[i] / (2.0 * kPi) * beta, p = q.p0[i], c = q.vx[i], s = q.vy[i];
            off[0] += a * p;
            off[1] += a * p * c;
            off[2] += a * p * s;
            off[3] += a * p * p;
            off[4] += a * p * p * c;
            off[5] += a * p * p * s;
            off[6] += a * p * p * c * c;
            off[7] += a * p * p * c * s;
        }
    }

    // per-warp sign masks of the populations it owns
    static_assert(sizeof(unsigned long long) == 8, "64-bit masks");
    if (h->P > 64) return fail(h, RLBM_ERR_UNSUPPORTED, "at most 64 populations per warp");
    // (one pair per group of populations: virtual warp v of shell r at r Gs R + v)
    const int Gv = h->Gs * h->R;
    std::vector<unsigned long long> masks(size_t(N + 1) * Gv * 2, 0ull);
    for (int g = 0; g < (N + 1) * Gv; ++g) {
        const int r = g / Gv, vv = g % Gv;
        for (int k = 0; k < h->P; ++k) {
            const int j = vv * h->P + k;
            if (j >= K) break;
            const int i = r * K + j;
            if (q.vx[i] >= 0.0) masks[2 * g] |= 1ull << k;
            if (q.vy[i] >= 0.0) masks[2 * g + 1] |= 1ull << k;
        }
    }

    const bool r64 = (h->prec == RLBM_FP64);
    const bool l64 = r64 || h->site_fp64;
    const size_t rs = r64 ? 8 : 4, ls = l64 ? 8 : 4;
    const size_t o_pop = 0;
    const size_t o_shell = align256(pop.size() * rs);
    const size_t o_rt = o_shell + align256(shell.size() * ls);
    const size_t o_mask = o_rt + align256(rt.size() * ls);
    // pair table of the two-sites-per-lane kernel (FP32 arithmetic only):
    // (c,c,s,s), (|c|,|c|,|s|,|s|), (w/alpha, w/alpha, 0, 0) per population
    const int PQ = 3;
    std::vector<double> ptab;
    if (!r64) {
        ptab.assign(size_t(npop) * PQ * 4, 0.0);
        for (int i = 0; i < npop; ++i) {
            const double *t = &pop[size_t(i) * TW];
            double *o = &ptab[size_t(i) * PQ * 4];
            const double v[12] = {t[0], t[0], t[1], t[1], std::fabs(t[0]), std::fabs(t[0]),
                                  std::fabs(t[1]), std::fabs(t[1]), t[4], t[4], 0.0, 0.0};
            for (int u = 0; u < 12; ++u) o[u] = v[u];
        }
    }
    const size_t o_pair0 = o_mask + align256(masks.size() * sizeof(unsigned long long));
    // double-float (hi, lo) copies of the shell folds and projection weights
    // for the double-float per-site part of the two-sites-per-lane kernels
    auto split = [](const std::vector<double> &v) {
        std::vector<float> o(2 * v.size());
        for (size_t i = 0; i < v.size(); ++i) {
            o[2 * i] = float(v[i]);
            o[2 * i + 1] = float(v[i] - double(o[2 * i]));
        }
        return o;
    };
    const std::vector<float> shell2 = split(shell), rt2 = split(rt);
    const size_t o_shell2 = o_pair0;
    const size_t o_rt2 = o_shell2 + align256(shell2.size() * 4);
    const size_t o_pair = o_rt2 + align256(rt2.size() * 4);
    // on-lattice rule: per population integer stencil vector (sx, sy)
    std::vector<int> shifts;
    if (q.onlat)
        for (int i = 0; i < npop; ++i) { shifts.push_back(q.sx[i]); shifts.push_back(q.sy[i]); }
    const size_t o_shift = o_pair + align256(ptab.size() * 4);
    const size_t total = o_shift + align256(shifts.size() * sizeof(int));
    std::vector<unsigned char> blob(total, 0);
    if (r64) put<double>(blob, o_pop, pop); else put<float>(blob, o_pop, pop);
    if (l64) { put<double>(blob, o_shell, shell); put<double>(blob, o_rt, rt); }
    else { put<float>(blob, o_shell, shell); put<float>(blob, o_rt, rt); }
    std::memcpy(blob.data() + o_mask, masks.data(), masks.size() * sizeof(unsigned long long));
    put<float>(blob, o_pair, ptab);
    std::memcpy(blob.data() + o_shell2, shell2.data(), shell2.size() * 4);
    std::memcpy(blob.data() + o_rt2, rt2.data(), rt2.size() * 4);
    if (!shifts.empty()) std::memcpy(blob.data() + o_shift, shifts.data(), shifts.size() * sizeof(int));

    if (h->d_tabs) { // re-tiling: replace the tables
        RLBM_CUDA(h, cudaStreamSynchronize(h->stream));
        cudaFree(h->d_tabs);
        h->d_tabs = nullptr;
    }
    RLBM_CUDA(h, cudaMalloc(&h->d_tabs, total));
    if (!h->d_status) {
        RLBM_CUDA(h, cudaMalloc(&h->d_status, 4 * sizeof(int))); // status, launch counter, CTAs done
        RLBM_CUDA(h, cudaMemsetAsync(h->d_status, 0, 4 * sizeof(int), h->stream));
    }
    RLBM_CUDA(h, cudaMemcpyAsync(h->d_tabs, blob.data(), total, cudaMemcpyHostToDevice, h->stream));
    RLBM_CUDA(h, cudaStreamSynchronize(h->stream));

    rlbmk::KernelArgs &a = h->base;
    std::memset(&a, 0, sizeof(a));
    a.nx = h->grid.nx;
    a.ny = h->grid.ny;
    a.S = (long long)h->grid.nx * h->grid.ny;
    a.K = K;
    a.Gs = h->Gs;
    a.P = h->P;
    a.R = h->R;
    a.bcx = h->grid.bc_x;
    a.bcy = h->grid.bc_y;
    a.collide = std::isinf(h->tau) ? 0 : 1;
    a.stat = h->stat;
    a.gdeg = h->gdeg;
    a.inv_tau = std::isinf(h->tau) ? 0.0 : 1.0 / h->tau;
    a.beta = beta;
    a.inv_tau_f = float(a.inv_tau);
    a.feq_off = scaled ? beta / (2.0 * kPi) : 0.0;
    a.feq_off_f = float(a.feq_off);
    a.feq_off_l = float(a.feq_off - double(a.feq_off_f));
    for (int t = 0; t < 8; ++t) {
        a.off[t] = off[t];
        a.off_f[t] = float(off[t]);
        a.off_l[t] = float(off[t] - double(a.off_f[t]));
    }
    for (int j = 0; j <= N; ++j) {
        const double ph = 2.0 * kPi * j / (N + 1);
        a.smp_c[j] = std::cos(ph);
        a.smp_s[j] = std::sin(ph);
        a.smp_cf[j] = float(a.smp_c[j]);
        a.smp_sf[j] = float(a.smp_s[j]);
        a.smp_cl[j] = float(a.smp_c[j] - double(a.smp_cf[j]));
        a.smp_sl[j] = float(a.smp_s[j] - double(a.smp_sf[j]));
    }
    a.poptab = (const unsigned char *)h->d_tabs + o_pop;
    a.shelltab = (const unsigned char *)h->d_tabs + o_shell;
    a.rtab = (const unsigned char *)h->d_tabs + o_rt;
    a.shell2 = reinterpret_cast<const float2 *>((const unsigned char *)h->d_tabs + o_shell2);
    a.rtab2 = reinterpret_cast<const float2 *>((const unsigned char *)h->d_tabs + o_rt2);
    a.masks = reinterpret_cast<const unsigned long long *>((const unsigned char *)h->d_tabs + o_mask);
    a.pairtab = ptab.empty() ? nullptr : (const unsigned char *)h->d_tabs + o_pair;
    a.shifts = shifts.empty() ? nullptr : reinterpret_cast<const int2 *>((const unsigned char *)h->d_tabs + o_shift);
    a.status = h->d_status;
    a.ctr = reinterpret_cast<unsigned *>(h->d_status + 1);
    a.qeta = h->d_qeta;
    a.wait_cycles = h->wait_cycles;
    a.extra_tx = 0;
    return RLBM_OK;
}

void *buffer(rlbm_t *h, int which) { return (unsigned char *)h->buf + size_t(which) * h->pop_bytes; }

size_t smem_bytes(const rlbm_t *h)
{
    const size_t ls = (h->prec == RLBM_FP64 || h->site_fp64) ? 8 : 4;
    return rlbmk::tile_smem_bytes(h->N, h->G, ls, h->stat != 0);
}

cudaError_t launch(rlbm_t *h, int mode, const rlbmk::KernelArgs &a)
{
    const dim3 grid((h->grid.nx + 31) / 32, h->grid.ny);
    const dim3 block(32, h->G);
    const size_t smem = smem_bytes(h);
    const bool two_d = h->grid.ny > 1;
    const bool full = h->K == h->R * h->Gs * h->P;
    cudaError_t e;
    if (h->stat) { // quantum statistics (FP64 per-site part; rlbm_set_statistics checks the rest)
        e = h->prec == RLBM_FP64
                ? rlbmk::launch_quant_f64(mode, h->N, h->P, two_d, full, grid, block, smem, h->stream, a)
                : rlbmk::launch_quant_f32(mode, h->N, h->P, two_d, full, grid, block, smem, h->stream, a);
        if (e == cudaSuccess) ++h->launches;
        return e;
    }
    // an FP32-storage step carries its per-site part in double-float (N = 2, 3)
    const bool dd_step = mode == rlbmk::MODE_STEP && h->prec == RLBM_FP32 && h->N <= 3;
    const size_t smem_dd = rlbmk::tile_smem_bytes_dd(h->N, h->G);
    if (mode == rlbmk::MODE_STEP && h->q.onlat) { // perfect streaming (FP32/FP64, P = 12: create, set_tiling)
        e = h->prec == RLBM_FP64 ? rlbmk::launch_lattice_f64(two_d, grid, block, smem, h->stream, a)
                                 : rlbmk::launch_lattice_f32(two_d, grid, block, smem_dd, h->stream, a);
        if (e == cudaSuccess) ++h->launches;
        return e;
    }
    if (dd_step) {
        e = rlbmk::launch_f32_dd(h->N, h->P, two_d, full, grid, block, smem_dd, h->stream, a);
        if (e == cudaSuccess) ++h->launches;
        return e;
    }
    switch (h->prec) {
    case RLBM_FP64: e = rlbmk::launch_f64(mode, h->N, h->P, two_d, full, grid, block, smem, h->stream, a); break;
    case RLBM_FP32:
        e = rlbmk::launch_f32(mode, h->N, h->P, two_d, full, h->site_fp64, grid, block, smem, h->stream, a);
        break;
    case RLBM_FP16_DEV:
    case RLBM_FP16_NORM: e = rlbmk::launch_f16(mode, h->N, h->P, two_d, full, grid, block, smem, h->stream, a); break;
    default: e = rlbmk::launch_bf16(mode, h->N, h->P, two_d, full, grid, block, smem, h->stream, a); break;
    }
    if (e == cudaSuccess) ++h->launches;
    return e;
}

// The two-sites-per-lane step kernel applies to FP32 per-population arithmetic
// (FP32 storage with a double-float per-site part, 16-bit storage with FP32
// accumulation and a double-float Landau solve) with a collision, N <= 3, an
// even row length, K a multiple of P and P in {8, 12, 16, 24, 32}; with
// several population groups per warp (many angles) to FP32 storage only.
bool pair_possible(const rlbm_t *h, int P)
{
    if (h->prec == RLBM_FP64 || std::isinf(h->tau) || h->N > 3 || h->q.onlat || h->stat) return false;
    if (h->grid.nx < 2 || h->grid.nx % 2 != 0) return false;
    if (!(P == 8 || P == 12 || P == 16 || P == 24 || P == 32) || h->K % P != 0) return false;
    int gs = 0, ng = 0;
    if (!group_tiling(h->N, h->K, P, gs, ng)) return false;
    return ng == 1 || h->prec == RLBM_FP32;
}

// The bulk-staged form copies row segments of whole 16-byte chunks from
// 16-byte aligned buffers.
bool pair_bulk_possible(const rlbm_t *h)
{
    return (size_t(h->grid.nx) * storage_size(h->prec)) % 16 == 0 && reinterpret_cast<uintptr_t>(h->buf) % 16 == 0;
}

cudaError_t launch_pair(rlbm_t *h, const rlbmk::KernelArgs &a)
{
    const dim3 grid((h->grid.nx + rlbmk::kPairSites - 1) / rlbmk::kPairSites, h->grid.ny);
    const dim3 block(32, h->G);
    // the population-groups kernel has no bulk staging
    const bool two_d = h->grid.ny > 1, bulk = h->pair_bulk && h->R == 1;
    const size_t smem = rlbmk::pair_smem_total(h->N, h->G, bulk, int(storage_size(h->prec)), two_d);
    cudaError_t e;
    if (h->R > 1) { // several population groups per warp (FP32 storage: pair_possible)
        e = rlbmk::launch_pair_groups_f32(h->N, h->P, two_d, grid, block, smem, h->stream, a);
        if (e == cudaSuccess) ++h->launches;
        return e;
    }
    switch (h->prec) {
    case RLBM_FP32: e = rlbmk::launch_pair_f32(h->N, h->P, two_d, bulk, grid, block, smem, h->stream, a); break;
    case RLBM_FP16_DEV:
    case RLBM_FP16_NORM:
        e = rlbmk::launch_pair_f16(h->N, h->P, two_d, bulk, grid, block, smem, h->stream, a);
        break;
    default: e = rlbmk::launch_pair_bf16(h->N, h->P, two_d, bulk, grid, block, smem, h->stream, a); break;
    }
    if (e == cudaSuccess) ++h->launches;
    return e;
}

// with bps set: only the occupancy query (CTAs per SM)
cudaError_t launch_pair_tma_raw(rlbm_t *h, const rlbmk::PairTmaArgs &ta, int *bps)
{
    const dim3 block(32, h->G);
    const bool two_d = h->grid.ny > 1;
    switch (h->prec) {
    case RLBM_FP32: return rlbmk::launch_pair_tma_f32(h->N, h->P, two_d, block, h->ptma_smem, h->stream, ta, bps);
    case RLBM_FP16_DEV:
    case RLBM_FP16_NORM:
        return rlbmk::launch_pair_tma_f16(h->N, h->P, two_d, block, h->ptma_smem, h->stream, ta, bps);
    default: return rlbmk::launch_pair_tma_bf16(h->N, h->P, two_d, block, h->ptma_smem, h->stream, ta, bps);
    }
}

cudaError_t launch_pair_tma(rlbm_t *h, const rlbmk::PairTmaArgs &ta)
{
    cudaError_t e = launch_pair_tma_raw(h, ta, nullptr);
    if (e == cudaSuccess) ++h->launches;
    return e;
}

cudaError_t launch_tma(rlbm_t *h, const rlbmk::TmaArgs &ta, int grid, int *bps)
{
    const dim3 block(32, h->G);
    const bool two_d = h->grid.ny > 1;
    const bool full = (h->K % h->P) == 0;
    switch (h->prec) {
    case RLBM_FP64: return rlbmk::launch_tma_f64(h->N, h->P, two_d, full, false, grid, block, h->tma_smem, h->stream, ta, bps);
    case RLBM_FP32: return rlbmk::launch_tma_f32(h->N, h->P, two_d, full, h->site_fp64, grid, block, h->tma_smem, h->stream, ta, bps);
    case RLBM_FP16_DEV:
    case RLBM_FP16_NORM: return rlbmk::launch_tma_f16(h->N, h->P, two_d, full, false, grid, block, h->tma_smem, h->stream, ta, bps);
    default: return rlbmk::launch_tma_bf16(h->N, h->P, two_d, full, false, grid, block, h->tma_smem, h->stream, ta, bps);
    }
}

cudaError_t launch_step(rlbm_t *h, int from)
{
    if (h->use_tma) {
        rlbmk::TmaArgs &ta = h->tma[from];
        ta.a.fin = buffer(h, from);
        ta.a.fout = buffer(h, 1 - from);
        ta.extra_tx = h->stall_next ? 16u : 0u;
        h->stall_next = false;
        cudaError_t e = launch_tma(h, ta, h->tma_grid, nullptr);
        ta.extra_tx = 0;
        if (e == cudaSuccess) ++h->launches;
        return e;
    }
    if (h->use_pair_tma) {
        rlbmk::PairTmaArgs &ta = h->ptma[from];
        ta.a.fin = buffer(h, from);
        ta.a.fout = buffer(h, 1 - from);
        ta.a.extra_tx = h->stall_next ? 16u : 0u;
        h->stall_next = false;
        cudaError_t e = launch_pair_tma(h, ta);
        ta.a.extra_tx = 0;
        return e;
    }
    rlbmk::KernelArgs a = h->base;
    a.fin = buffer(h, from);
    a.fout = buffer(h, 1 - from);
    if (h->use_pair) {
        if (h->pair_bulk && h->stall_next) a.extra_tx = 16u;
        h->stall_next = false;
        return launch_pair(h, a);
    }
    return launch(h, rlbmk::MODE_STEP, a);
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// Set up the persistent TMA-staged step kernel if the grid satisfies the
// tensor-map rules (16-byte row pitch, at least one box wide); otherwise the
// per-tile kernel is used.
rlbm_status setup_tma(rlbm_t *h)
{
    h->use_tma = false;
    delete[] h->tma;
    h->tma = nullptr;
    const char *off = std::getenv("RLBM_NO_TMA");
    if ((off && off[0] == '1') || h->no_tma || h->N > 3 || h->R > 1 || h->q.onlat || h->stat) return RLBM_OK;
    const size_t es = storage_size(h->prec);
    const int HX = int(16 / es), BW = 32 + 2 * HX;
    const int nx = h->grid.nx, ny = h->grid.ny, npop = h->npop;
    if ((size_t(nx) * es) % 16 != 0 || nx < BW) return RLBM_OK;
    int nbox = (npop + 255) / 256;
    int BP = (npop + nbox - 1) / nbox;
    BP = (BP + 3) / 4 * 4;
    if (BP > 256 || (npop <= 256 && BP != npop)) return RLBM_OK; // keep every box inside the tensor
    const int BR = ny > 1 ? 3 : 1;
    const size_t box_bytes = size_t(BP) * BW * es;
    const size_t stage = rlbmk::align_up(size_t(BR) * nbox * box_bytes, 1024);
    const size_t ls = (h->prec == RLBM_FP64 || h->site_fp64) ? 8 : 4;
    const size_t rs = (h->prec == RLBM_FP64) ? 8 : 4;
    const rlbmk::TmaSmem L(stage, h->G, h->P, h->N, rs, ls);
    int dev = 0, max_smem = 0;
    RLBM_CUDA(h, cudaGetDevice(&dev));
    RLBM_CUDA(h, cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    RLBM_CUDA(h, cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, dev));
    if (L.total > size_t(max_smem)) return RLBM_OK;

    void *fn = nullptr;
    cudaDriverEntryPointQueryResult qres;
    RLBM_CUDA(h, cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                   cudaEnableDefault, &qres));
    if (!fn || qres != cudaDriverEntryPointSuccess)
        return fail(h, RLBM_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    EncodeTiledFn encode = reinterpret_cast<EncodeTiledFn>(fn);
    CUtensorMapDataType dt;
    switch (h->prec) {
    case RLBM_FP64: dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT64; break;
    case RLBM_FP32: dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT32; break;
    case RLBM_FP16_DEV:
    case RLBM_FP16_NORM: dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT16; break;
    default: dt = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16; break;
    }
    h->tma = new (std::nothrow) rlbmk::TmaArgs[2];
    if (!h->tma) return fail(h, RLBM_ERR_OOM, "host allocation failed");
    const cuuint64_t dims[3] = {cuuint64_t(nx), cuuint64_t(ny), cuuint64_t(npop)};
    const cuuint64_t strides[2] = {cuuint64_t(nx) * es, cuuint64_t(nx) * ny * es};
    const cuuint32_t box[3] = {cuuint32_t(BW), 1u, cuuint32_t(BP)};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    const int ntiles_x = (nx + 31) / 32;
    for (int b = 0; b < 2; ++b) {
        rlbmk::TmaArgs &ta = h->tma[b];
        std::memset(&ta, 0, sizeof(ta));
        CUresult r = encode(&ta.tmap, dt, 3, buffer(h, b), dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(h, RLBM_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", int(r));
        ta.a = h->base;
        ta.BP = BP;
        ta.nbox = nbox;
        ta.ntiles_x = ntiles_x;
        ta.ntiles = ntiles_x * ny;
        ta.stage_bytes = (long long)stage;
        ta.wait_cycles = 4000000000LL; // about 2 s at the maximum SM clock
        ta.extra_tx = 0;
    }
    h->tma_smem = L.total;
    int bps = 0;
    cudaError_t e = launch_tma(h, h->tma[0], 0, &bps);
    if (e != cudaSuccess) return cuda_fail(h, e, "occupancy query of the TMA step kernel");
    if (bps < 1) return RLBM_OK;
    const long long ntiles = (long long)ntiles_x * ny;
    h->tma_grid = int(std::min<long long>(ntiles, (long long)bps * h->sm_count));
    h->use_tma = true;
    return RLBM_OK;
}

// Pull-row chunks of the tile-staged pair kernel: the largest DB in {8, 4}
// dividing npop for which every chunk of DB consecutive populations shares
// sgn(v_y) (a population with v_y = 0 gives its pull row the weight 0 and
// joins either side); bit c of up: chunk c pulls from row y - 1.  0 if none.
int pull_chunking(const Quad &q, int npop, unsigned long long *up)
{
    for (int db : {8, 4}) {
        if (npop % db || npop / db > 256) continue;
        unsigned long long m[4] = {0, 0, 0, 0};
        bool ok = true;
        for (int c = 0; c < npop / db && ok; ++c) {
            int sgn = 0;
            for (int i = c * db; i < (c + 1) * db; ++i) {
                const int si = q.vy[i] > 0.0 ? 1 : (q.vy[i] < 0.0 ? -1 : 0);
                if (si == 0) continue;
                if (sgn == 0) sgn = si;
                else if (si != sgn) { ok = false; break; }
            }
            if (sgn >= 0) m[c >> 6] |= 1ull << (c & 63);
        }
        if (ok) {
            std::memcpy(up, m, sizeof(m));
            return db;
        }
    }
    return 0;
}

// Set up the tile-staged two-sites-per-lane kernel for the current tiling, if
// the pair kernel applies with one population group, the rows are whole
// 16-byte chunks (the TMA's pitch rule), nx covers one box, the pull rows
// chunk by sgn(v_y) and the shared memory fits.  Otherwise use_pair_tma stays
// false.
rlbm_status setup_pair_tma(rlbm_t *h)
{
    h->use_pair_tma = false;
    delete[] h->ptma;
    h->ptma = nullptr;
    const size_t es = storage_size(h->prec);
    const int BW = rlbmk::kPairSites + 2 * int(16 / es);
    const int nx = h->grid.nx, ny = h->grid.ny, npop = h->npop;
    if (!pair_possible(h, h->P) || h->R != 1) return RLBM_OK;
    if ((size_t(nx) * es) % 16 != 0 || nx < BW || reinterpret_cast<uintptr_t>(h->buf) % 16 != 0) return RLBM_OK;
    unsigned long long up[4];
    const int DB = pull_chunking(h->q, npop, up);
    if (!DB) return RLBM_OK;
    const int ncbox = (npop + 255) / 256;
    const int CB = npop / ncbox;
    if (CB * ncbox != npop || CB % 4 != 0) return RLBM_OK; // whole boxes, 128-byte aligned destinations
    const bool two_d = ny > 1;
    int dev = 0, max_smem = 0;
    RLBM_CUDA(h, cudaGetDevice(&dev));
    RLBM_CUDA(h, cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    RLBM_CUDA(h, cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, dev));
    const size_t need = rlbmk::PairTmaSmem(h->N, h->G, npop, int(es), two_d).total;
    if (need > size_t(max_smem)) return RLBM_OK;
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult qres;
    RLBM_CUDA(h, cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &qres));
    if (!fn || qres != cudaDriverEntryPointSuccess) return fail(h, RLBM_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    EncodeTiledFn encode = reinterpret_cast<EncodeTiledFn>(fn);
    CUtensorMapDataType dt;
    switch (h->prec) {
    case RLBM_FP32: dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT32; break;
    case RLBM_FP16_DEV:
    case RLBM_FP16_NORM: dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT16; break;
    default: dt = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16; break;
    }
    h->ptma = new (std::nothrow) rlbmk::PairTmaArgs[2];
    if (!h->ptma) return fail(h, RLBM_ERR_OOM, "host allocation failed");
    const cuuint64_t dims[3] = {cuuint64_t(nx), cuuint64_t(ny), cuuint64_t(npop)};
    const cuuint64_t strides[2] = {cuuint64_t(nx) * es, cuuint64_t(nx) * ny * es};
    const cuuint32_t cbox[3] = {cuuint32_t(BW), 1u, cuuint32_t(CB)};
    const cuuint32_t pbox[3] = {cuuint32_t(BW), 1u, cuuint32_t(DB)};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    for (int b = 0; b < 2; ++b) {
        rlbmk::PairTmaArgs &ta = h->ptma[b];
        std::memset(&ta, 0, sizeof(ta));
        for (int m = 0; m < 2; ++m) {
            CUresult r = encode(m == 0 ? &ta.cmap : &ta.pmap, dt, 3, buffer(h, b), dims, strides, m == 0 ? cbox : pbox,
                                estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) {
                delete[] h->ptma;
                h->ptma = nullptr;
                return fail(h, RLBM_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", int(r));
            }
        }
        ta.a = h->base;
        ta.CB = CB;
        ta.ncbox = ncbox;
        ta.DB = DB;
        ta.npbox = npop / DB;
        std::memcpy(ta.chunk_up, up, sizeof(up));
    }
    h->ptma_smem = need;
    int bps = 0;
    cudaError_t e = launch_pair_tma_raw(h, h->ptma[0], &bps);
    if (e != cudaSuccess) return cuda_fail(h, e, "occupancy query of the tile-staged step kernel");
    if (bps < 1) {
        delete[] h->ptma;
        h->ptma = nullptr;
        return RLBM_OK;
    }
    h->use_pair_tma = true;
    return RLBM_OK;
}

rlbm_status check_status(rlbm_t *h)
{
    int st = 0;
    RLBM_CUDA(h, cudaMemcpyAsync(&st, h->d_status, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    RLBM_CUDA(h, cudaStreamSynchronize(h->stream));
    if (st) {
        RLBM_CUDA(h, cudaMemsetAsync(h->d_status, 0, sizeof(int), h->stream));
        RLBM_CUDA(h, cudaStreamSynchronize(h->stream));
        if (st & 2)
            return fail(h, RLBM_ERR_TIMEOUT,
                        "a bounded wait in the step kernel ran out (its copies did not complete in time)");
        return fail(h, RLBM_ERR_UNPHYSICAL,
                    "a cell had no physical Landau frame (non-positive n or eps, or no timelike eigenvector)");
    }
    return RLBM_OK;
}

rlbm_status ensure_graph(rlbm_t *h, int from)
{
    if (h->graph[from]) return RLBM_OK;
    cudaGraph_t g = nullptr;
    const long long l0 = h->launches;
    RLBM_CUDA(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaSuccess;
    int cur = from;
    for (int s = 0; s < kGraphSteps && e == cudaSuccess; ++s) {
        e = launch_step(h, cur);
        cur = 1 - cur;
    }
    cudaError_t e2 = cudaStreamEndCapture(h->stream, &g);
    h->launches = l0; // captured launches are counted at replay
    if (e != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_fail(h, e, "kernel launch during graph capture"); }
    if (e2 != cudaSuccess) return cuda_fail(h, e2, "cudaStreamEndCapture");
    cudaError_t e3 = cudaGraphInstantiate(&h->graph[from], g, 0);
    cudaGraphDestroy(g);
    if (e3 != cudaSuccess) { h->graph[from] = nullptr; return cuda_fail(h, e3, "cudaGraphInstantiate"); }
    return RLBM_OK;
}

rlbm_status validate_fields_ptrs(rlbm_t *h, const void *a, const void *b, const void *c, const void *d)
{
    if (!a || !b || !c || !d) return fail(h, RLBM_ERR_ARG, "NULL field pointer");
    return RLBM_OK;
}

// Switch the handle to another tiling: P populations per warp and the step
// kernel kind (0 per-tile, 1 persistent TMA-staged where possible, 2 two
// sites per lane where possible; otherwise the per-tile kernel).
rlbm_status retile(rlbm_t *h, int P, int kind)
{
    RLBM_CUDA(h, cudaStreamSynchronize(h->stream));
    for (auto &g : h->graph)
        if (g) { cudaGraphExecDestroy(g); g = nullptr; }
    h->P = P;
    if (!group_tiling(h->N, h->K, P, h->Gs, h->R)) {
        h->Gs = (h->K + P - 1) / P;
        h->R = 1;
    }
    h->G = h->Gs * (h->N + 1);
    h->no_tma = kind != 1;
    h->use_pair = (kind == 2 || kind == 3 || kind == 4) && pair_possible(h, P);
    h->pair_bulk = h->use_pair && kind == 3 && pair_bulk_possible(h) && h->R == 1;
    rlbm_status st = build_tables(h);
    if (st) return st;
    st = setup_tma(h);
    if (st) return st;
    h->use_pair_tma = false;
    if (h->use_pair && kind == 4) {
        st = setup_pair_tma(h);
        if (st) return st;
        if (!h->use_pair_tma) h->use_pair = false; // not possible here: the per-tile kernel
    }
    return RLBM_OK;
}

int kernel_kind(const rlbm_t *h)
{
    if (h->use_pair_tma) return 4;
    if (h->use_pair) return h->pair_bulk ? 3 : 2;
    return h->use_tma ? 1 : 0;
}

struct TuneKey {
    int nx, ny, N, K, prec, bcx, bcy, site64;
    bool operator<(const TuneKey &o) const
    {
        return std::memcmp(this, &o, sizeof(TuneKey)) < 0;
    }
};
struct TuneChoice { int P; int kind; float ms; };

std::map<TuneKey, TuneChoice> &tune_cache()
{
    static std::map<TuneKey, TuneChoice> m;
    return m;
}
std::mutex g_tune_mutex;

} // namespace

extern "C" {

rlbm_status rlbm_quadrature(int order_N, int angles_K, double *p0, double *vx, double *vy, double *w)
{
    Quad q;
    if (!make_quadrature(order_N, angles_K, q))
        return fail(nullptr, RLBM_ERR_ARG, "need 0 <= N <= 12 and K >= 2N+1 (N=%d, K=%d)", order_N,
                    angles_K);
    const size_t nb = sizeof(double) * q.npop;
    if (p0) std::memcpy(p0, q.p0.data(), nb);
    if (vx) std::memcpy(vx, q.vx.data(), nb);
    if (vy) std::memcpy(vy, q.vy.data(), nb);
    if (w) std::memcpy(w, q.w.data(), nb);
    return RLBM_OK;
}

size_t rlbm_population_bytes(rlbm_grid grid, int order_N, int angles_K, int precision)
{
    if (grid.nx < 1 || grid.ny < 1 || order_N < 0 || angles_K < 1) return 0;
    return storage_size(precision) * size_t(angles_K) * size_t(order_N + 1) * size_t(grid.nx) *
           size_t(grid.ny);
}

static rlbm_status create_impl(rlbm_t **out, rlbm_grid grid, int order_N, int angles_K, double tau,
                               int precision, void *cuda_stream, void *dev_buffers, size_t dev_buffer_bytes,
                               bool onlat)
{
    if (!out) return fail(nullptr, RLBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (grid.nx < 1 || grid.ny < 1)
        return fail(nullptr, RLBM_ERR_ARG, "grid must be at least 1x1 (got %dx%d)", grid.nx, grid.ny);
    if ((long long)grid.ny > 65535)
        return fail(nullptr, RLBM_ERR_ARG, "ny must be <= 65535 (got %d)", grid.ny);
    if (grid.bc_x < 0 || grid.bc_x > 1 || grid.bc_y < 0 || grid.bc_y > 1)
        return fail(nullptr, RLBM_ERR_ARG, "boundary conditions must be 0 (periodic) or 1 (copy-out)");
    if (order_N < 2)
        return fail(nullptr, RLBM_ERR_ARG,
                    "order N must be >= 2 (the collision conserves N^0 and T^0nu only from N = 2)");
    if (angles_K < 2 * order_N + 1)
        return fail(nullptr, RLBM_ERR_ARG, "K must be >= 2N+1 (N=%d, K=%d)", order_N, angles_K);
    if (!(tau > 0.0)) return fail(nullptr, RLBM_ERR_ARG, "tau must be > 0 or +inf (got %g)", tau);
    if (storage_size(precision) == 0)
        return fail(nullptr, RLBM_ERR_ARG, "unknown precision %d", precision);
    if (order_N > rlbmk::kMaxN)
        return fail(nullptr, RLBM_ERR_UNSUPPORTED, "kernels are built for N = 2..%d (got N=%d)", rlbmk::kMaxN,
                    order_N);
    if (onlat && precision != RLBM_FP32 && precision != RLBM_FP64)
        return fail(nullptr, RLBM_ERR_UNSUPPORTED,
                    "the on-lattice rule is built for FP32 and FP64 storage (its weights differ within a shell)");

    rlbm_t *h = new (std::nothrow) rlbm();
    if (!h) return fail(nullptr, RLBM_ERR_OOM, "host allocation failed");
    h->grid = grid;
    h->N = order_N;
    h->K = angles_K;
    h->npop = angles_K * (order_N + 1);
    h->prec = precision;
    h->tau = tau;
    h->site_fp64 = site_fp64_for(precision, order_N, 0);
    if (!(onlat ? make_onlattice_quadrature(h->q) : make_quadrature(order_N, angles_K, h->q))) {
        delete h;
        return fail(nullptr, RLBM_ERR_ARG, "quadrature construction failed");
    }
    if (!choose_tiling(order_N, angles_K, h->P, h->Gs, h->R)) {
        delete h;
        return fail(nullptr, RLBM_ERR_UNSUPPORTED, "no compiled tiling for K=%d", angles_K);
    }
    if (h->R > 1 && storage_size(precision) == 2) {
        delete h;
        return fail(nullptr, RLBM_ERR_UNSUPPORTED,
                    "K=%d needs several population groups per warp, built for FP32 and FP64 storage only "
                    "(at most %d angles with N=%d in 16-bit storage)",
                    angles_K, single_group_capacity(order_N), order_N);
    }
    if (const char *ep = onlat ? nullptr : std::getenv("RLBM_TILE_P")) { // experiment hook: force P if it fits
        const int P = std::atoi(ep);
        const int gs = (angles_K + P - 1) / P;
        if ((P == 8 || P == 12 || P == 16 || P == 24 || P == 32 || P == 48 || P == 64) &&
            gs * (order_N + 1) <= rlbmk::kMaxWarps &&
            (gs - 1) * P < angles_K) {
            h->P = P;
            h->Gs = gs;
        }
    }
    h->G = h->Gs * (order_N + 1);
    h->pop_bytes = rlbm_population_bytes(grid, order_N, angles_K, precision);

    rlbm_status st = RLBM_OK;
    if (cuda_stream) {
        h->stream = (cudaStream_t)cuda_stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) { st = cuda_fail(h, e, "cudaStreamCreate"); }
        h->own_stream = (e == cudaSuccess);
    }
    if (st == RLBM_OK) {
        if (dev_buffers) {
            if (dev_buffer_bytes < 2 * h->pop_bytes)
                st = fail(h, RLBM_ERR_ARG, "dev_buffers holds %zu bytes, need %zu", dev_buffer_bytes,
                          2 * h->pop_bytes);
            else if (((uintptr_t)dev_buffers) % 256)
                st = fail(h, RLBM_ERR_ARG, "dev_buffers must be 256-byte aligned");
            else
                h->buf = dev_buffers;
        } else {
            cudaError_t e = cudaMalloc(&h->buf, 2 * h->pop_bytes);
            if (e != cudaSuccess) st = cuda_fail(h, e, "cudaMalloc(populations)");
            else h->own_buf = true;
        }
    }
    if (st == RLBM_OK) st = build_tables(h);
    if (st == RLBM_OK) st = setup_tma(h);
    if (st != RLBM_OK) {
        g_create_error = h->err;
        rlbm_destroy(h);
        return st;
    }
    *out = h;
    return RLBM_OK;
}

rlbm_status rlbm_create(rlbm_t **out, rlbm_grid grid, int order_N, int angles_K, double tau,
                        int precision, void *cuda_stream, void *dev_buffers, size_t dev_buffer_bytes)
{
    return create_impl(out, grid, order_N, angles_K, tau, precision, cuda_stream, dev_buffers,
                       dev_buffer_bytes, false);
}

rlbm_status rlbm_create_onlattice(rlbm_t **out, rlbm_grid grid, double tau, int precision, void *cuda_stream,
                                  void *dev_buffers, size_t dev_buffer_bytes)
{
    return create_impl(out, grid, 3, 12, tau, precision, cuda_stream, dev_buffers, dev_buffer_bytes, true);
}

int rlbm_is_onlattice(const rlbm_t *h) { return h ? (h->q.onlat ? 1 : 0) : -1; }

rlbm_status rlbm_set_statistics(rlbm_t *h, int statistics, double g)
{
    if (!h) return fail(nullptr, RLBM_ERR_ARG, "NULL handle");
    if (statistics < -1 || statistics > 1) return fail(h, RLBM_ERR_ARG, "statistics must be 0, 1 or -1");
    if (statistics != 0 && !(g > 0.0 && std::isfinite(g))) return fail(h, RLBM_ERR_ARG, "g must be > 0");
    if (statistics != 0) {
        if (h->prec != RLBM_FP64 && h->prec != RLBM_FP32)
            return fail(h, RLBM_ERR_UNSUPPORTED, "quantum statistics are built for FP64 and FP32 storage");
        if (h->N > 3) return fail(h, RLBM_ERR_UNSUPPORTED, "quantum statistics are built for N = 2, 3");
        if (h->q.onlat) return fail(h, RLBM_ERR_UNSUPPORTED, "quantum statistics use the off-lattice rule");
    }
    h->stat = statistics;
    h->gdeg = statistics != 0 ? g : 1.0;
    // the per-site eta of the last solve, the Newton start of the next one (NaN: none yet)
    if (statistics != 0 && !h->d_qeta) {
        const size_t bytes = sizeof(double) * size_t(h->grid.nx) * size_t(h->grid.ny);
        RLBM_CUDA(h, cudaMalloc(&h->d_qeta, bytes));
        RLBM_CUDA(h, cudaMemsetAsync(h->d_qeta, 0xff, bytes, h->stream));
    }
    // the quantum per-site part runs in FP64 (FP32 storage: FP64 site tables)
    h->site_fp64 = site_fp64_for(h->prec, h->N, statistics);
    return retile(h, h->P, 0);
}

int rlbm_statistics(const rlbm_t *h) { return h ? h->stat : -2; }

double rlbm_quantum_phi(int s, double eta, int statistics)
{
    if (s < 0 || s > 6 || (statistics != 1 && statistics != -1) || (statistics < 0 && !(eta < 0.0)))
        return std::nan("");
    if (s == 0) return rlbmk::stat_phi(0, eta, statistics);
    double ph[6]; // the fused evaluation the kernels use (phi_1 .. phi_s in one pass)
    rlbmk::stat_phi_upto(s, eta, statistics, ph);
    return ph[s - 1];
}

int rlbm_quantum_solve(double n, double e, double g, int statistics, double eta0, int fp32_storage,
                       double *eta, double *T)
{
    if (!eta || !T) return 0;
    *eta = std::nan("");
    *T = std::nan("");
    if ((statistics != 1 && statistics != -1) || !(g > 0.0)) return 0;
    return rlbmk::stat_solve(n, e, g, statistics, *eta, *T, eta0, nullptr, 0, fp32_storage ? 1e-5 : 1e-10) ? 1 : 0;
}

void rlbm_destroy(rlbm_t *h)
{
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (auto &g : h->graph)
        if (g) cudaGraphExecDestroy(g);
    if (h->own_buf && h->buf) cudaFree(h->buf);
    if (h->d_tabs) cudaFree(h->d_tabs);
    if (h->d_status) cudaFree(h->d_status);
    if (h->d_qeta) cudaFree(h->d_qeta);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete[] h->tma;
    delete[] h->ptma;
    delete h;
}

const char *rlbm_last_error(const rlbm_t *h)
{
    return h ? h->err.c_str() : g_create_error.c_str();
}

rlbm_status rlbm_init_device(rlbm_t *h, const double *d_n, const double *d_T, const double *d_bx,
                             const double *d_by)
{
    if (!h) return fail(nullptr, RLBM_ERR_ARG, "NULL handle");
    rlbm_status st = validate_fields_ptrs(h, d_n, d_T, d_bx, d_by);
    if (st) return st;
    rlbmk::KernelArgs a = h->base;
    a.fin = nullptr;
    a.fout = buffer(h, 0);
    a.in_n = d_n;
    a.in_T = d_T;
    a.in_bx = d_bx;
    a.in_by = d_by;
    // the launch counter seeds the stochastic rounding of 16-bit storage: restart it
    RLBM_CUDA(h, cudaMemsetAsync(h->d_status + 1, 0, 2 * sizeof(int), h->stream));
    cudaError_t e = launch(h, rlbmk::MODE_INIT, a);
    if (e != cudaSuccess) return cuda_fail(h, e, "init kernel");
    h->cur = 0;
    h->steps = 0;
    return RLBM_OK;
}

rlbm_status rlbm_init(rlbm_t *h, const double *n, const double *T, const double *bx, const double *by)
{
    if (!h) return fail(nullptr, RLBM_ERR_ARG, "NULL handle");
    rlbm_status st = validate_fields_ptrs(h, n, T, bx, by);
    if (st) return st;
    const size_t S = size_t(h->grid.nx) * h->grid.ny;
    for (size_t s = 0; s < S; ++s) {
        if (!(n[s] > 0.0) || !(T[s] > 0.0) || !(bx[s] * bx[s] + by[s] * by[s] < 1.0))
            return fail(h, RLBM_ERR_ARG, "non-physical initial state at site %zu (need n > 0, T > 0, |beta| < 1)", s);
    }
    double *d = nullptr;
    RLBM_CUDA(h, cudaMallocAsync((void **)&d, 4 * S * sizeof(double), h->stream));
    const double *src[4] = {n, T, bx, by};
    for (int k = 0; k < 4; ++k)
        RLBM_CUDA(h, cudaMemcpyAsync(d + k * S, src[k], S * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    st = rlbm_init_device(h, d, d + S, d + 2 * S, d + 3 * S);
    cudaFreeAsync(d, h->stream);
    if (st) return st;
    RLBM_CUDA(h, cudaStreamSynchronize(h->stream));
    return RLBM_OK;
}

rlbm_status rlbm_step(rlbm_t *h, int nsteps)
{
    if (!h) return fail(nullptr, RLBM_ERR_ARG, "NULL handle");
    if (nsteps < 0) return fail(h, RLBM_ERR_ARG, "nsteps must be >= 0");
    int left = nsteps;
    while (left >= kGraphSteps) {
        rlbm_status st = ensure_graph(h, h->cur);
        if (st) return st;
        RLBM_CUDA(h, cudaGraphLaunch(h->graph[h->cur], h->stream));
        h->launches += kGraphSteps;
        // an even number of steps returns to the same buffer
        if (kGraphSteps & 1) h->cur = 1 - h->cur;
        h->steps += kGraphSteps;
        left -= kGraphSteps;
    }
    for (; left > 0; --left) {
        cudaError_t e = launch_step(h, h->cur);
        if (e != cudaSuccess) return cuda_fail(h, e, "step kernel");
        h->cur = 1 - h->cur;
        ++h->steps;
    }
    return RLBM_OK;
}

rlbm_status rlbm_moments_device(rlbm_t *h, double *d_n, double *d_eps, double *d_T, double *d_U0,
                                double *d_Ux, double *d_Uy)
{
    if (!h) return fail(nullptr, RLBM_ERR_ARG, "NULL handle");
    if (!d_n || !d_eps || !d_T || !d_U0 || !d_Ux || !d_Uy) return fail(h, RLBM_ERR_ARG, "NULL output pointer");
    rlbmk::KernelArgs a = h->base;
    a.fin = buffer(h, h->cur);
    a.fout = nullptr;
    a.out[0] = d_n;
    a.out[1] = d_eps;
    a.out[2] = d_T;
    a.out[3] = d_U0;
    a.out[4] = d_Ux;
    a.out[5] = d_Uy;
    cudaError_t e = launch(h, rlbmk::MODE_MOMENTS, a);
    if (e != cudaSuccess) return cuda_fail(h, e, "moments kernel");
    return RLBM_OK;
}

rlbm_status rlbm_moments(rlbm_t *h, double *n, double *eps, double *T, double *U0, double *Ux, double *Uy)
{
    if (!h) return fail(nullptr, RLBM_ERR_ARG, "NULL handle");
    double *outs[6] = {n, eps, T, U0, Ux, Uy};
    for (double *p : outs)
        if (!p) return fail(h, RLBM_ERR_ARG, "NULL output pointer");
    const size_t S = size_t(h->grid.nx) * h->grid.ny;
    double *d = nullptr;
    RLBM_CUDA(h, cudaMallocAsync((void **)&d, 6 * S * sizeof(double), h->stream));
    rlbm_status st = rlbm_moments_device(h, d, d + S, d + 2 * S, d + 3 * S, d + 4 * S, d + 5 * S);
    if (st == RLBM_OK) {
        for (int k = 0; k < 6; ++k) {
            cudaError_t e = cudaMemcpyAsync(outs[k], d + k * S, S * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
            if (e != cudaSuccess) { st = cuda_fail(h, e, "cudaMemcpyAsync(moments)"); break; }
        }
    }
    cudaFreeAsync(d, h->stream);
    if (st) return st;
    return check_status(h);
}

rlbm_status rlbm_get_populations(rlbm_t *h, void *host, size_t bytes)
{
    if (!h) return fail(nullptr, RLBM_ERR_ARG, "NULL handle");
    if (!host || bytes != h->pop_bytes)
        return fail(h, RLBM_ERR_ARG, "need a host buffer of exactly %zu bytes", h->pop_bytes);
    RLBM_CUDA(h, cudaMemcpyAsync(host, buffer(h, h->cur), bytes, cudaMemcpyDeviceToHost, h->stream));
    RLBM_CUDA(h, cudaStreamSynchronize(h->stream));
    return RLBM_OK;
}

rlbm_status rlbm_set_populations(rlbm_t *h, const void *host, size_t bytes, long long step)
{
    if (!h) return fail(nullptr, RLBM_ERR_ARG, "NULL handle");
    if (!host || bytes != h->pop_bytes)
        return fail(h, RLBM_ERR_ARG, "need a host buffer of exactly %zu bytes", h->pop_bytes);
    RLBM_CUDA(h, cudaMemcpyAsync(buffer(h, 0), host, bytes, cudaMemcpyHostToDevice, h->stream));
    const unsigned ctr[2] = {unsigned(step), 0u};
    RLBM_CUDA(h, cudaMemcpyAsync(h->d_status + 1, ctr, sizeof(ctr), cudaMemcpyHostToDevice, h->stream));
    if (h->d_qeta) // a new state: no previous eta to start from
        RLBM_CUDA(h, cudaMemsetAsync(h->d_qeta, 0xff, sizeof(double) * size_t(h->grid.nx) * h->grid.ny, h->stream));
    RLBM_CUDA(h, cudaStreamSynchronize(h->stream));
    h->cur = 0;
    h->steps = step;
    return RLBM_OK;
}

void *rlbm_current_buffer(rlbm_t *h) { return h ? buffer(h, h->cur) : nullptr; }

long long rlbm_steps_done(const rlbm_t *h) { return h ? h->steps : -1; }

rlbm_status rlbm_sync(rlbm_t *h)
{
    if (!h) return fail(nullptr, RLBM_ERR_ARG, "NULL handle");
    return check_status(h);
}

long long rlbm_kernel_launches(const rlbm_t *h) { return h ? h->launches : -1; }

int rlbm_step_kernel_variant(const rlbm_t *h) { return h ? kernel_kind(h) : -1; }

rlbm_status rlbm_set_tiling(rlbm_t *h, int P, int kind)
{
    if (!h) return fail(nullptr, RLBM_ERR_ARG, "NULL handle");
    if (kind < 0 || kind > 4) return fail(h, RLBM_ERR_ARG, "kernel kind must be 0..4 (got %d)", kind);
    static const int sizes[] = {8, 12, 16, 24, 32, 48, 64};
    bool ok = false;
    for (int v : sizes) ok = ok || v == P;
    int gs = 0, ng = 0;
    if (!ok || !group_tiling(h->N, h->K, P, gs, ng))
        return fail(h, RLBM_ERR_UNSUPPORTED, "no compiled tiling with P=%d for N=%d, K=%d", P, h->N, h->K);
    if (h->q.onlat && (P != 12 || kind != 0))
        return fail(h, RLBM_ERR_UNSUPPORTED, "the on-lattice rule runs the per-tile kernel with P=12 only");
    if (ng > 1 && kind != 0 && kind != 2)
        return fail(h, RLBM_ERR_UNSUPPORTED,
                    "K=%d needs several population groups per warp: per-tile or two-sites-per-lane kernel only",
                    h->K);
    if ((kind == 2 || kind == 3 || kind == 4) && !pair_possible(h, P)) {
        rlbm_status st0 = retile(h, P, 0);
        if (st0) return st0;
        return fail(h, RLBM_ERR_UNSUPPORTED,
                    "two-sites-per-lane kernel needs FP32 arithmetic, tau finite, N <= 3, nx even, P in "
                    "{8,12,16,24,32} dividing K, and FP32 storage when K needs several population groups");
    }
    rlbm_status st = retile(h, P, kind);
    if (st) return st;
    if (kernel_kind(h) != kind) {
        st = retile(h, P, 0);
        if (st) return st;
        return fail(h, RLBM_ERR_UNSUPPORTED,
                    kind == 1   ? "TMA-staged kernel not possible for this grid and tiling"
                    : kind == 4 ? "tile-staged pair kernel not possible here (rows of whole 16-byte chunks, "
                                  "nx >= one box, pull rows in chunks of 4 or 8 populations sharing sgn(v_y), "
                                  "one population group)"
                                : "bulk staging needs rows of whole 16-byte chunks");
    }
    return RLBM_OK;
}

int rlbm_tile_populations(const rlbm_t *h) { return h ? h->P : -1; }

int rlbm_population_groups(const rlbm_t *h) { return h ? h->R : -1; }

rlbm_status rlbm_autotune(rlbm_t *h, int launches_per_trial, float *best_ms)
{
    if (!h) return fail(nullptr, RLBM_ERR_ARG, "NULL handle");
    if (launches_per_trial < 1) return fail(h, RLBM_ERR_ARG, "launches_per_trial must be >= 1");
    const TuneKey key{h->grid.nx, h->grid.ny, h->N, h->K, h->prec, h->grid.bc_x, h->grid.bc_y,
                      (h->site_fp64 ? 1 : 0) | (h->q.onlat ? 2 : 0) | (h->stat ? (h->stat > 0 ? 4 : 8) : 0)};
    {
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        auto it = tune_cache().find(key);
        if (it != tune_cache().end()) {
            if (best_ms) *best_ms = it->second.ms;
            if (it->second.P == h->P && it->second.kind == kernel_kind(h)) return RLBM_OK;
            return retile(h, it->second.P, it->second.kind);
        }
    }
    static const int sizes[] = {8, 12, 16, 24, 32, 48, 64};
    cudaEvent_t e0, e1;
    RLBM_CUDA(h, cudaEventCreate(&e0));
    RLBM_CUDA(h, cudaEventCreate(&e1));
    TuneChoice best{h->P, kernel_kind(h), 1e30f};
    const long long launches0 = h->launches;
    rlbm_status st = RLBM_OK;
    for (int P : sizes) {
        int gs = 0, ng = 0;
        if (!group_tiling(h->N, h->K, P, gs, ng)) continue;
        if (h->q.onlat && P != 12) continue; // the on-lattice kernel is built for P = 12
        if (P > 2 * h->K) continue;
        for (int kind = 4; kind >= 0 && st == RLBM_OK; --kind) {
            st = retile(h, P, kind);
            if (st) break;
            if (kernel_kind(h) != kind) continue; // kernel kind not possible for this tiling
            // time cur -> other launches (the state in buffer cur is not modified)
            cudaError_t e = launch_step(h, h->cur);
            if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
            for (int k = 0; k < launches_per_trial && e == cudaSuccess; ++k) e = launch_step(h, h->cur);
            if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) { st = cuda_fail(h, e, "autotune trial"); break; }
            ms /= launches_per_trial;
            if (ms < best.ms) best = TuneChoice{P, kind, ms};
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->launches = launches0; // trial launches are not steps
    if (st) return st;
    st = retile(h, best.P, best.kind);
    if (st) return st;
    {
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        tune_cache()[key] = best;
    }
    if (best_ms) *best_ms = best.ms;
    // trial launches may flag cells of a state that was never stepped: clear
    RLBM_CUDA(h, cudaMemsetAsync(h->d_status, 0, sizeof(int), h->stream));
    RLBM_CUDA(h, cudaStreamSynchronize(h->stream));
    return RLBM_OK;
}

rlbm_status rlbm_set_wait_limit(rlbm_t *h, long long cycles)
{
    if (!h) return fail(nullptr, RLBM_ERR_ARG, "NULL handle");
    if (cycles < 1000) return fail(h, RLBM_ERR_ARG, "wait limit must be >= 1000 cycles");
    if (h->tma)
        for (int b = 0; b < 2; ++b) h->tma[b].wait_cycles = cycles;
    if (h->ptma)
        for (int b = 0; b < 2; ++b) h->ptma[b].a.wait_cycles = cycles;
    h->wait_cycles = cycles;
    h->base.wait_cycles = cycles;
    for (auto &g : h->graph)
        if (g) { cudaGraphExecDestroy(g); g = nullptr; }
    return RLBM_OK;
}

rlbm_status rlbm_test_stall_next_step(rlbm_t *h)
{
    if (!h) return fail(nullptr, RLBM_ERR_ARG, "NULL handle");
    if (!h->use_tma && !h->pair_bulk && !h->use_pair_tma)
        return fail(h, RLBM_ERR_UNSUPPORTED, "this step kernel has no device waits");
    h->stall_next = true;
    return RLBM_OK;
}

} // extern "C"

// ============================================================== batched form

struct rlbm_batch {
    std::vector<rlbm_t *> probs;
    int N = 0, prec = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    void *arena = nullptr;
    bool own_arena = false;
    std::vector<size_t> offs;
    std::vector<int> tpu;       // tiles per unit (per problem)
    std::vector<int> ntiles_x, ntiles;
    int nunits = 0, grid = 0;
    // device arrays
    rlbmk::KernelArgs *d_args = nullptr;
    int *d_ints = nullptr;                // ntiles_x | ntiles | tpu | parity
    rlbmk::BatchUnit *d_units = nullptr;
    unsigned *d_sync = nullptr;           // 4 words
    int *d_status = nullptr;
    long long wait_cycles = 4000000000LL;
    bool stall_next = false;
    std::map<int, cudaGraphExec_t> graphs; // by nsteps
    long long launches = 0, steps = 0;
    // execution mode: 0 = one persistent cooperative launch per call (tilings
    // batch_P); 1 = every problem runs its own step kernel (tilings solo_P /
    // solo_kind), all its steps back to back, on one of a pool of streams
    int mode = 0;
    std::vector<int> batch_P, solo_P, solo_kind, lane_of;
    std::vector<cudaStream_t> pool;
    std::vector<cudaEvent_t> pool_ev;
    cudaEvent_t fork_ev = nullptr;
    std::string err;
};

namespace {

rlbm_status bfail(rlbm_batch *b, rlbm_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (b) b->err = buf; else g_create_error = buf;
    return st;
}

#define BATCH_CUDA(b, call)                                                                      \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return bfail(b, e_ == cudaErrorMemoryAllocation ? RLBM_ERR_OOM : RLBM_ERR_CUDA,        \
                         "%s: %s", #call, cudaGetErrorString(e_));                               \
    } while (0)

// Tiling of one problem in a 6-warp CTA: G = gs (N+1) warps per tile must divide 6.
bool batch_tiling(int N, int K, int gs, int &P)
{
    static const int sizes[] = {8, 12, 16, 24, 32};
    if (rlbmk::kBatchWarps % (gs * (N + 1)) != 0) return false;
    const int need = (K + gs - 1) / gs;
    for (int s : sizes)
        if (s >= need) {
            if ((gs - 1) * s >= K) return false;
            P = s;
            return true;
        }
    return false;
}

rlbm_status batch_build_units(rlbm_batch *b)
{
    const int n = int(b->probs.size());
    b->tpu.assign(n, 1);
    b->ntiles_x.assign(n, 0);
    b->ntiles.assign(n, 0);
    std::vector<rlbmk::KernelArgs> args(n);
    std::vector<std::pair<double, int>> order;
    for (int i = 0; i < n; ++i) {
        rlbm_t *h = b->probs[i];
        b->tpu[i] = rlbmk::kBatchWarps / h->G;
        b->ntiles_x[i] = (h->grid.nx + 31) / 32;
        b->ntiles[i] = b->ntiles_x[i] * h->grid.ny;
        args[i] = h->base;
        args[i].fin = buffer(h, 0);
        args[i].fout = buffer(h, 1);
        order.push_back({-double(h->npop) * h->grid.nx * h->grid.ny, i}); // largest first
    }
    std::sort(order.begin(), order.end());
    std::vector<rlbmk::BatchUnit> units;
    for (auto &o : order) {
        const int i = o.second;
        for (int t = 0; t < b->ntiles[i]; t += b->tpu[i]) units.push_back({i, t});
    }
    b->nunits = int(units.size());
    if (b->d_units) { cudaFree(b->d_units); b->d_units = nullptr; }
    BATCH_CUDA(b, cudaMalloc(&b->d_units, sizeof(rlbmk::BatchUnit) * std::max<size_t>(1, units.size())));
    BATCH_CUDA(b, cudaMemcpyAsync(b->d_units, units.data(), sizeof(rlbmk::BatchUnit) * units.size(),
                                  cudaMemcpyHostToDevice, b->stream));
    BATCH_CUDA(b, cudaMemcpyAsync(b->d_args, args.data(), sizeof(rlbmk::KernelArgs) * n,
                                  cudaMemcpyHostToDevice, b->stream));
    std::vector<int> ints(4 * size_t(n));
    for (int i = 0; i < n; ++i) {
        ints[i] = b->ntiles_x[i];
        ints[n + i] = b->ntiles[i];
        ints[2 * n + i] = b->tpu[i];
        ints[3 * n + i] = b->probs[i]->cur;
    }
    BATCH_CUDA(b, cudaMemcpyAsync(b->d_ints, ints.data(), sizeof(int) * ints.size(),
                                  cudaMemcpyHostToDevice, b->stream));
    BATCH_CUDA(b, cudaStreamSynchronize(b->stream));
    for (auto &g : b->graphs) cudaGraphExecDestroy(g.second);
    b->graphs.clear();
    return RLBM_OK;
}

rlbmk::BatchArgs batch_args(rlbm_batch *b, int nsteps)
{
    const int n = int(b->probs.size());
    rlbmk::BatchArgs a{};
    a.probs = b->d_args;
    a.ntiles_x = b->d_ints;
    a.ntiles = b->d_ints + n;
    a.tiles_per_unit = b->d_ints + 2 * n;
    a.parity0 = b->d_ints + 3 * n;
    a.units = b->d_units;
    a.nunits = b->nunits;
    a.nsteps = nsteps;
    a.sync = b->d_sync;
    a.status = b->d_status;
    a.wait_cycles = b->wait_cycles;
    a.barrier_extra = 0;
    return a;
}

rlbm_status batch_launch(rlbm_batch *b, int nsteps, bool use_graph)
{
    const bool stall = b->stall_next;
    b->stall_next = false;
    if (use_graph && !stall) {
        auto it = b->graphs.find(nsteps);
        if (it == b->graphs.end()) {
            cudaGraph_t g = nullptr;
            BATCH_CUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = cudaMemsetAsync(b->d_sync, 0, 4 * sizeof(unsigned), b->stream);
            if (e == cudaSuccess)
                e = rlbmk::launch_batch(b->prec, b->N, batch_args(b, nsteps), b->grid, b->stream, nullptr);
            if (e == cudaSuccess)
                e = rlbmk::launch_batch_advance(b->d_args, int(b->probs.size()), nsteps, b->stream);
            cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
            if (e != cudaSuccess) { if (g) cudaGraphDestroy(g); BATCH_CUDA(b, e); }
            BATCH_CUDA(b, e2);
            cudaGraphExec_t ge = nullptr;
            cudaError_t e3 = cudaGraphInstantiate(&ge, g, 0);
            cudaGraphDestroy(g);
            BATCH_CUDA(b, e3);
            it = b->graphs.emplace(nsteps, ge).first;
        }
        BATCH_CUDA(b, cudaGraphLaunch(it->second, b->stream));
    } else {
        BATCH_CUDA(b, cudaMemsetAsync(b->d_sync, 0, 4 * sizeof(unsigned), b->stream));
        rlbmk::BatchArgs a = batch_args(b, nsteps);
        if (stall) a.barrier_extra = 1;
        BATCH_CUDA(b, rlbmk::launch_batch(b->prec, b->N, a, b->grid, b->stream, nullptr));
        BATCH_CUDA(b, rlbmk::launch_batch_advance(b->d_args, int(b->probs.size()), nsteps, b->stream));
    }
    b->launches += 2; // the batched kernel and the counter advance
    return RLBM_OK;
}

rlbm_status batch_check(rlbm_batch *b)
{
    int st = 0;
    BATCH_CUDA(b, cudaMemcpyAsync(&st, b->d_status, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    BATCH_CUDA(b, cudaStreamSynchronize(b->stream));
    if (st) {
        BATCH_CUDA(b, cudaMemsetAsync(b->d_status, 0, sizeof(int), b->stream));
        BATCH_CUDA(b, cudaStreamSynchronize(b->stream));
        return bfail(b, RLBM_ERR_TIMEOUT, "a grid-barrier wait in the batched kernel ran out");
    }
    for (size_t i = 0; i < b->probs.size(); ++i) {
        rlbm_status s2 = check_status(b->probs[i]);
        if (s2) return bfail(b, s2, "problem %zu: %s", i, b->probs[i]->err.c_str());
    }
    return RLBM_OK;
}

constexpr int kBatchStreams = 16;

// Smallest two-sites-per-lane tiling of a problem (more, lighter warps per
// SM), else the per-tile kernel with the default tiling.
void solo_default(const rlbm_t *h, int &P, int &kind)
{
    static const int sizes[] = {8, 12, 16, 24, 32};
    for (int v : sizes)
        if (pair_possible(h, v)) { P = v; kind = pair_bulk_possible(h) ? 3 : 2; return; }
    int gs = 0, ng = 0;
    choose_tiling(h->N, h->K, P, gs, ng);
    kind = 0;
}

rlbm_status batch_sync_all(rlbm_batch *b)
{
    for (cudaStream_t s : b->pool) BATCH_CUDA(b, cudaStreamSynchronize(s));
    BATCH_CUDA(b, cudaStreamSynchronize(b->stream));
    return RLBM_OK;
}

// Switch the execution mode, re-tiling every problem accordingly.
rlbm_status batch_set_mode(rlbm_batch *b, int mode)
{
    const int n = int(b->probs.size());
    rlbm_status st = batch_sync_all(b);
    if (st) return st;
    if (mode == 1) {
        if (b->pool.empty()) {
            b->pool.resize(kBatchStreams);
            b->pool_ev.resize(kBatchStreams);
            for (int s = 0; s < kBatchStreams; ++s) {
                BATCH_CUDA(b, cudaStreamCreateWithFlags(&b->pool[s], cudaStreamNonBlocking));
                BATCH_CUDA(b, cudaEventCreateWithFlags(&b->pool_ev[s], cudaEventDisableTiming));
            }
            BATCH_CUDA(b, cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming));
            // longest-processing-time assignment of problems to streams
            std::vector<std::pair<double, int>> order;
            for (int i = 0; i < n; ++i)
                order.push_back({-double(b->probs[i]->npop) * b->probs[i]->grid.nx * b->probs[i]->grid.ny, i});
            std::sort(order.begin(), order.end());
            std::vector<double> load(kBatchStreams, 0.0);
            b->lane_of.assign(n, 0);
            for (auto &o : order) {
                const int s = int(std::min_element(load.begin(), load.end()) - load.begin());
                b->lane_of[o.second] = s;
                load[s] -= o.first;
            }
        }
        if (b->solo_P.empty()) {
            b->solo_P.resize(n);
            b->solo_kind.resize(n);
            for (int i = 0; i < n; ++i) solo_default(b->probs[i], b->solo_P[i], b->solo_kind[i]);
        }
        for (int i = 0; i < n; ++i) {
            st = retile(b->probs[i], b->solo_P[i], b->solo_kind[i]);
            if (st) return bfail(b, st, "problem %d: %s", i, b->probs[i]->err.c_str());
        }
    } else {
        for (int i = 0; i < n; ++i) {
            b->probs[i]->no_tma = true;
            st = retile(b->probs[i], b->batch_P[i], 0);
            if (st) return bfail(b, st, "problem %d: %s", i, b->probs[i]->err.c_str());
        }
        st = batch_build_units(b);
        if (st) return st;
    }
    b->mode = mode;
    return RLBM_OK;
}

// Mode 1: fork the pool from the batch stream, run every problem's nsteps
// steps on its stream, join back.
rlbm_status batch_streams_step(rlbm_batch *b, int nsteps)
{
    BATCH_CUDA(b, cudaEventRecord(b->fork_ev, b->stream));
    for (cudaStream_t s : b->pool) BATCH_CUDA(b, cudaStreamWaitEvent(s, b->fork_ev, 0));
    for (size_t i = 0; i < b->probs.size(); ++i) {
        rlbm_t *h = b->probs[i];
        cudaStream_t saved = h->stream;
        h->stream = b->pool[b->lane_of[i]];
        const long long l0 = h->launches;
        rlbm_status st = rlbm_step(h, nsteps);
        h->stream = saved;
        if (st) return bfail(b, st, "problem %zu: %s", i, h->err.c_str());
        b->launches += h->launches - l0;
    }
    for (size_t s = 0; s < b->pool.size(); ++s) {
        BATCH_CUDA(b, cudaEventRecord(b->pool_ev[s], b->pool[s]));
        BATCH_CUDA(b, cudaStreamWaitEvent(b->stream, b->pool_ev[s], 0));
    }
    b->steps += nsteps;
    return RLBM_OK;
}

} // namespace

extern "C" {

size_t rlbm_batch_arena_bytes(const rlbm_problem *p, int count, int order_N, int precision)
{
    if (!p || count < 1) return 0;
    size_t tot = 0;
    for (int i = 0; i < count; ++i) {
        const rlbm_grid g{p[i].nx, p[i].ny, p[i].bc_x, p[i].bc_y};
        tot += align256(2 * rlbm_population_bytes(g, order_N, p[i].angles_K, precision));
    }
    return tot;
}

rlbm_status rlbm_batch_create(rlbm_batch_t **out, const rlbm_problem *p, int count, int order_N,
                              int precision, void *cuda_stream, void *dev_arena, size_t arena_bytes)
{
    if (!out) return bfail(nullptr, RLBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!p || count < 1) return bfail(nullptr, RLBM_ERR_ARG, "need at least one problem");
    if (precision != RLBM_FP64 && precision != RLBM_FP32)
        return bfail(nullptr, RLBM_ERR_UNSUPPORTED, "the batched kernel is built for FP64 and FP32 storage");
    if (order_N != 2 && order_N != 3)
        return bfail(nullptr, RLBM_ERR_UNSUPPORTED, "the batched kernel is built for N = 2, 3");
    for (int i = 0; i < count; ++i) {
        int P;
        if (!batch_tiling(order_N, p[i].angles_K, 1, P) && !batch_tiling(order_N, p[i].angles_K, 2, P))
            return bfail(nullptr, RLBM_ERR_UNSUPPORTED,
                         "problem %d: K=%d has no batched tiling (6 warps per CTA; N=2: K <= 64, N=3: none)",
                         i, p[i].angles_K);
        if (p[i].nx < 1 || p[i].ny < 1 || !(p[i].tau > 0.0) || p[i].angles_K < 2 * order_N + 1 ||
            p[i].bc_x < 0 || p[i].bc_x > 1 || p[i].bc_y < 0 || p[i].bc_y > 1)
            return bfail(nullptr, RLBM_ERR_ARG, "problem %d: invalid grid, K, tau or boundary condition", i);
    }
    const size_t need = rlbm_batch_arena_bytes(p, count, order_N, precision);
    if (dev_arena && (arena_bytes < need || ((uintptr_t)dev_arena) % 256))
        return bfail(nullptr, RLBM_ERR_ARG, "dev_arena must be 256-byte aligned and hold %zu bytes", need);
    rlbm_batch *b = new (std::nothrow) rlbm_batch();
    if (!b) return bfail(nullptr, RLBM_ERR_OOM, "host allocation failed");
    b->N = order_N;
    b->prec = precision;
    rlbm_status st = RLBM_OK;
    auto bail = [&](rlbm_status s) {
        g_create_error = b->err;
        rlbm_batch_destroy(b);
        return s;
    };
    if (cuda_stream) {
        b->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess)
            return bail(bfail(b, RLBM_ERR_CUDA, "cudaStreamCreate failed"));
        b->own_stream = true;
    }
    if (dev_arena) {
        b->arena = dev_arena;
    } else {
        if (cudaMalloc(&b->arena, need) != cudaSuccess)
            return bail(bfail(b, RLBM_ERR_OOM, "cudaMalloc of a %zu-byte arena failed", need));
        b->own_arena = true;
    }
    size_t off = 0;
    for (int i = 0; i < count; ++i) {
        const rlbm_grid g{p[i].nx, p[i].ny, p[i].bc_x, p[i].bc_y};
        const size_t bytes = 2 * rlbm_population_bytes(g, order_N, p[i].angles_K, precision);
        rlbm_t *h = nullptr;
        st = rlbm_create(&h, g, order_N, p[i].angles_K, p[i].tau, precision, b->stream,
                         (unsigned char *)b->arena + off, bytes);
        if (st) return bail(bfail(b, st, "problem %d: %s", i, g_create_error.c_str()));
        b->probs.push_back(h);
        b->offs.push_back(off);
        int P = 0;
        const int gs = batch_tiling(order_N, p[i].angles_K, 1, P) ? 1 : 2;
        batch_tiling(order_N, p[i].angles_K, gs, P);
        h->no_tma = true;
        st = retile(h, P, 0);
        if (st) return bail(bfail(b, st, "problem %d: %s", i, h->err.c_str()));
        b->batch_P.push_back(P);
        off += align256(bytes);
    }
    const int n = count;
    if (cudaMalloc(&b->d_args, sizeof(rlbmk::KernelArgs) * n) != cudaSuccess ||
        cudaMalloc(&b->d_ints, sizeof(int) * 4 * n) != cudaSuccess ||
        cudaMalloc(&b->d_sync, 4 * sizeof(unsigned)) != cudaSuccess ||
        cudaMalloc(&b->d_status, sizeof(int)) != cudaSuccess)
        return bail(bfail(b, RLBM_ERR_OOM, "device allocation of batch tables failed"));
    if (cudaMemsetAsync(b->d_status, 0, sizeof(int), b->stream) != cudaSuccess)
        return bail(bfail(b, RLBM_ERR_CUDA, "cudaMemsetAsync failed"));
    st = batch_build_units(b);
    if (st) return bail(st);
    int bps = 0, dev = 0, sms = 0;
    if (rlbmk::launch_batch(precision, order_N, batch_args(b, 0), 0, b->stream, &bps) != cudaSuccess ||
        cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || bps < 1)
        return bail(bfail(b, RLBM_ERR_CUDA, "occupancy query of the batched kernel failed"));
    b->grid = bps * sms;
    *out = b;
    return RLBM_OK;
}

void rlbm_batch_destroy(rlbm_batch_t *b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    for (cudaStream_t s : b->pool) { cudaStreamSynchronize(s); cudaStreamDestroy(s); }
    for (cudaEvent_t e : b->pool_ev) cudaEventDestroy(e);
    if (b->fork_ev) cudaEventDestroy(b->fork_ev);
    for (auto &g : b->graphs) cudaGraphExecDestroy(g.second);
    for (rlbm_t *h : b->probs) rlbm_destroy(h);
    if (b->d_args) cudaFree(b->d_args);
    if (b->d_ints) cudaFree(b->d_ints);
    if (b->d_units) cudaFree(b->d_units);
    if (b->d_sync) cudaFree(b->d_sync);
    if (b->d_status) cudaFree(b->d_status);
    if (b->own_arena && b->arena) cudaFree(b->arena);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

const char *rlbm_batch_last_error(const rlbm_batch_t *b) { return b ? b->err.c_str() : g_create_error.c_str(); }

int rlbm_batch_count(const rlbm_batch_t *b) { return b ? int(b->probs.size()) : -1; }

rlbm_t *rlbm_batch_problem(rlbm_batch_t *b, int i)
{
    if (!b || i < 0 || i >= int(b->probs.size())) return nullptr;
    return b->probs[i];
}

rlbm_status rlbm_batch_step(rlbm_batch_t *b, int nsteps)
{
    if (!b) return bfail(nullptr, RLBM_ERR_ARG, "NULL batch");
    if (nsteps < 0) return bfail(b, RLBM_ERR_ARG, "nsteps must be >= 0");
    if (nsteps == 0) return RLBM_OK;
    if (b->mode == 1) return batch_streams_step(b, nsteps);
    // current buffer parity of every problem (problems can be re-initialised one by one)
    const int n = int(b->probs.size());
    std::vector<int> par(n);
    for (int i = 0; i < n; ++i) par[i] = b->probs[i]->cur;
    BATCH_CUDA(b, cudaMemcpyAsync(b->d_ints + 3 * n, par.data(), sizeof(int) * n,
                                  cudaMemcpyHostToDevice, b->stream));
    BATCH_CUDA(b, cudaStreamSynchronize(b->stream)); // par is a stack buffer
    rlbm_status st = batch_launch(b, nsteps, true);
    if (st) return st;
    for (rlbm_t *h : b->probs) {
        h->cur = (h->cur + nsteps) & 1;
        h->steps += nsteps;
    }
    b->steps += nsteps;
    return RLBM_OK;
}

rlbm_status rlbm_batch_sync(rlbm_batch_t *b)
{
    if (!b) return bfail(nullptr, RLBM_ERR_ARG, "NULL batch");
    return batch_check(b);
}

long long rlbm_batch_kernel_launches(const rlbm_batch_t *b) { return b ? b->launches : -1; }

rlbm_status rlbm_batch_set_wait_limit(rlbm_batch_t *b, long long cycles)
{
    if (!b) return bfail(nullptr, RLBM_ERR_ARG, "NULL batch");
    if (cycles < 1000) return bfail(b, RLBM_ERR_ARG, "wait limit must be >= 1000 cycles");
    b->wait_cycles = cycles;
    for (auto &g : b->graphs) cudaGraphExecDestroy(g.second);
    b->graphs.clear();
    return RLBM_OK;
}

rlbm_status rlbm_batch_test_stall_next_step(rlbm_batch_t *b)
{
    if (!b) return bfail(nullptr, RLBM_ERR_ARG, "NULL batch");
    if (b->mode != 0) return bfail(b, RLBM_ERR_UNSUPPORTED, "the stream-pool mode has no grid barrier");
    b->stall_next = true;
    return RLBM_OK;
}

rlbm_status rlbm_batch_set_mode(rlbm_batch_t *b, int mode)
{
    if (!b) return bfail(nullptr, RLBM_ERR_ARG, "NULL batch");
    if (mode != 0 && mode != 1) return bfail(b, RLBM_ERR_ARG, "mode must be 0 or 1 (got %d)", mode);
    if (mode == b->mode) return RLBM_OK;
    return batch_set_mode(b, mode);
}

int rlbm_batch_mode(const rlbm_batch_t *b) { return b ? b->mode : -1; }

rlbm_status rlbm_batch_autotune(rlbm_batch_t *b, int steps_per_trial, float *best_ms)
{
    if (!b) return bfail(nullptr, RLBM_ERR_ARG, "NULL batch");
    if (steps_per_trial < 1) return bfail(b, RLBM_ERR_ARG, "steps_per_trial must be >= 1");
    const int n = int(b->probs.size());
    if (b->mode != 0) {
        rlbm_status st0 = batch_set_mode(b, 0);
        if (st0) return st0;
    }
    // a uniform rest state (n = 1, T = 1) in every problem: realistic timing, no NaNs
    for (int i = 0; i < n; ++i) {
        rlbm_t *h = b->probs[i];
        const size_t S = size_t(h->grid.nx) * h->grid.ny;
        std::vector<double> one(S, 1.0), zero(S, 0.0);
        rlbm_status st = rlbm_init(h, one.data(), one.data(), zero.data(), zero.data());
        if (st) return bfail(b, st, "problem %d: %s", i, h->err.c_str());
    }
    cudaEvent_t e0, e1;
    BATCH_CUDA(b, cudaEventCreate(&e0));
    BATCH_CUDA(b, cudaEventCreate(&e1));
    auto trial = [&](float &ms) -> rlbm_status {
        rlbm_status st = batch_build_units(b);
        if (st) return st;
        BATCH_CUDA(b, cudaEventRecord(e0, b->stream));
        st = batch_launch(b, steps_per_trial, false);
        if (st) return st;
        BATCH_CUDA(b, cudaEventRecord(e1, b->stream));
        BATCH_CUDA(b, cudaEventSynchronize(e1));
        BATCH_CUDA(b, cudaEventElapsedTime(&ms, e0, e1));
        return RLBM_OK;
    };
    // greedy over classes of K: warps per tile gs (N+1) in {N+1, 2 (N+1)}
    std::map<int, std::vector<int>> classes;
    for (int i = 0; i < n; ++i) classes[b->probs[i]->K].push_back(i);
    float best = 0.f;
    rlbm_status st = trial(best);
    for (auto &c : classes) {
        if (st) break;
        const int K = c.first;
        const int cur_gs = b->probs[c.second[0]]->Gs;
        int best_gs = cur_gs;
        for (int gs = 1; gs <= 2 && !st; ++gs) {
            int P;
            if (gs == cur_gs || !batch_tiling(b->N, K, gs, P)) continue;
            for (int i : c.second) {
                st = retile(b->probs[i], P, 0);
                if (st) break;
            }
            float ms = 0.f;
            if (!st) st = trial(ms);
            if (!st && ms < best) { best = ms; best_gs = gs; }
        }
        if (!st && best_gs != b->probs[c.second[0]]->Gs) {
            int P;
            batch_tiling(b->N, K, best_gs, P);
            for (int i : c.second)
                if (!st) st = retile(b->probs[i], P, 0);
        }
    }
    if (!st) st = batch_build_units(b);
    for (int i = 0; i < n && !st; ++i) b->batch_P[i] = b->probs[i]->P;
    // stream-pool mode: per class of K, the two-sites-per-lane tilings
    float best1 = 0.f;
    auto trial1 = [&](float &ms) -> rlbm_status {
        BATCH_CUDA(b, cudaEventRecord(e0, b->stream));
        rlbm_status s1 = batch_streams_step(b, steps_per_trial);
        if (s1) return s1;
        BATCH_CUDA(b, cudaEventRecord(e1, b->stream));
        BATCH_CUDA(b, cudaEventSynchronize(e1));
        BATCH_CUDA(b, cudaEventElapsedTime(&ms, e0, e1));
        return RLBM_OK;
    };
    if (!st) st = batch_set_mode(b, 1);
    if (!st) st = trial1(best1); // graphs captured on the first call: time the second
    if (!st) st = trial1(best1);
    static const int psizes[] = {8, 12, 16, 24, 32};
    for (auto &c : classes) {
        if (st) break;
        for (int P : psizes) {
            std::vector<int> members;
            for (int i : c.second)
                if (pair_possible(b->probs[i], P) && !(b->solo_kind[i] >= 2 && b->solo_P[i] == P)) members.push_back(i);
            if (members.empty()) continue;
            std::vector<int> oldP, oldK;
            if (!st) st = batch_sync_all(b);
            for (int i : members) {
                oldP.push_back(b->solo_P[i]);
                oldK.push_back(b->solo_kind[i]);
                b->solo_P[i] = P;
                b->solo_kind[i] = pair_bulk_possible(b->probs[i]) ? 3 : 2;
                if (!st) st = retile(b->probs[i], P, b->solo_kind[i]);
            }
            float ms = 0.f;
            if (!st) st = trial1(ms);
            if (!st) st = trial1(ms);
            if (st) break;
            if (ms < best1) {
                best1 = ms;
            } else {
                st = batch_sync_all(b);
                for (size_t m = 0; m < members.size() && !st; ++m) {
                    b->solo_P[members[m]] = oldP[m];
                    b->solo_kind[members[m]] = oldK[m];
                    st = retile(b->probs[members[m]], oldP[m], oldK[m]);
                }
            }
        }
    }
    if (!st && best < best1) st = batch_set_mode(b, 0);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) return st;
    b->launches = 0;
    if (best_ms) *best_ms = std::min(best, best1) / steps_per_trial;
    BATCH_CUDA(b, cudaMemsetAsync(b->d_status, 0, sizeof(int), b->stream));
    for (rlbm_t *h : b->probs) {
        BATCH_CUDA(b, cudaMemsetAsync(h->d_status, 0, sizeof(int), b->stream));
        h->steps = 0;
    }
    b->steps = 0;
    BATCH_CUDA(b, cudaStreamSynchronize(b->stream));
    return RLBM_OK;
}

} // extern "C"
