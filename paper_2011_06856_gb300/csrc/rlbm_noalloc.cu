// rlbm_step_noalloc: one fused step from a caller's input buffer to a caller's
// output buffer with no device allocation at all.
//
// Every other entry point of the library keeps its constant tables and its
// status word in device memory it allocates itself (cudaMalloc).  Some callers
// cannot let a library do that: their device memory is owned by their own
// pool or framework allocator, or they run under a fixed memory budget in
// which a side allocation may fail at the worst moment.  For them this entry
// point keeps its scratch -- the per-population tables, the projection weights,
// the sign masks and the status word -- in one file-scope __device__ array of
// kScratchBytes bytes that every GPU loading the library holds until the
// process exits.  The caller passes the populations in and out.
//
// The array is shared by every call: each call rewrites the tables and
// clears the status word before its kernel runs, so calls that overlap on the
// GPU (different streams, different host threads) race with each other and
// must be serialised by the caller.
#include "rlbm.h"
#include "rlbm_args.h"

#include <cmath>
#include <cstring>
#include <mutex>

namespace {

constexpr size_t kScratchBytes = 32768;
constexpr int kMaxDevices = 64;
constexpr int kMaxNpop = 256;
constexpr double kPi = 3.14159265358979323846264338327950288;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mutex;
void *g_scratch_ptr[kMaxDevices] = {};
thread_local char g_err[256];
thread_local unsigned char g_blob[kScratchBytes]; // host staging, static storage

rlbm_status fail(rlbm_status st, const char *msg)
{
    std::strncpy(g_err, msg, sizeof(g_err) - 1);
    g_err[sizeof(g_err) - 1] = 0;
    return st;
}

// Device address of the scratch array, looked up once per device with that
// device current (in host code the symbol is only a host-side stand-in).
rlbm_status scratch_address(void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return fail(RLBM_ERR_CUDA, "cudaGetDevice failed");
    std::lock_guard<std::mutex> lk(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) return fail(RLBM_ERR_CUDA, cudaGetErrorString(e));
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return RLBM_OK;
}

void laguerre2(int n, double x, double &ln, double &lnm1)
{
    double a = 1.0, b = 1.0 - x;
    if (n == 0) { ln = 1.0; lnm1 = 0.0; return; }
    for (int k = 1; k < n; ++k) {
        const double c = ((2.0 * k + 1.0 - x) * b - k * a) / (k + 1.0);
        a = b;
        b = c;
    }
    ln = b;
    lnm1 = a;
}

// Roots of L_n (n <= 4): Sturm bisection on the Jacobi matrix, Newton polish.
void nodes(int n, double *x)
{
    for (int k = 0; k < n; ++k) {
        double lo = 0.0, hi = 4.0 * n + 2.0;
        for (int it = 0; it < 2000; ++it) {
            const double mid = 0.5 * (lo + hi);
            if (mid <= lo || mid >= hi) break;
            int cnt = 0;
            double d = 1.0;
            for (int j = 0; j < n; ++j) {
                d = (2.0 * j + 1.0 - mid) - (j == 0 ? 0.0 : double(j) * j / d);
                if (d == 0.0) d = -1e-300;
                if (d < 0.0) ++cnt;
            }
            if (cnt >= k + 1) hi = mid; else lo = mid;
        }
        double r = 0.5 * (lo + hi);
        for (int it = 0; it < 3; ++it) {
            double l, lm;
            laguerre2(n, r, l, lm);
            const double dl = n * (l - lm) / r;
            if (dl != 0.0) r -= l / dl;
        }
        x[k] = r;
    }
}

// Inverse of the (small) Hankel matrix (l+k+2m)! by Gauss-Jordan, fixed arrays.
bool hankel_inverse(int d, int m, double inv[4][4])
{
    double A[4][8];
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < 2 * d; ++j) {
            if (j < d) {
                double f = 1.0;
                for (int t = 2; t <= 2 * m + i + j; ++t) f *= t;
                A[i][j] = f;
            } else {
                A[i][j] = (j - d == i) ? 1.0 : 0.0;
            }
        }
    for (int c = 0; c < d; ++c) {
        int p = c;
        for (int i = c + 1; i < d; ++i)
            if (std::fabs(A[i][c]) > std::fabs(A[p][c])) p = i;
        if (A[p][c] == 0.0) return false;
        for (int j = 0; j < 2 * d; ++j) { const double t = A[c][j]; A[c][j] = A[p][j]; A[p][j] = t; }
        const double piv = A[c][c];
        for (int j = 0; j < 2 * d; ++j) A[c][j] /= piv;
        for (int i = 0; i < d; ++i) {
            if (i == c) continue;
            const double f = A[i][c];
            for (int j = 0; j < 2 * d; ++j) A[i][j] -= f * A[c][j];
        }
    }
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) inv[i][j] = A[i][d + j];
    return true;
}

template <class T> void put(unsigned char *dst, double v)
{
    const T t = T(v);
    std::memcpy(dst, &t, sizeof(T));
}

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

} // namespace

extern "C" rlbm_status rlbm_step_noalloc(rlbm_grid grid, int order_N, int angles_K, double tau,
                                         int precision, const void *d_fin, void *d_fout,
                                         void *cuda_stream)
{
    const int N = order_N, K = angles_K, npop = K * (N + 1);
    if (grid.nx < 1 || grid.ny < 1 || grid.ny > 65535 || grid.bc_x < 0 || grid.bc_x > 1 ||
        grid.bc_y < 0 || grid.bc_y > 1)
        return fail(RLBM_ERR_ARG, "invalid grid or boundary condition");
    if (N < 2 || K < 2 * N + 1 || !(tau > 0.0)) return fail(RLBM_ERR_ARG, "need N >= 2, K >= 2N+1, tau > 0");
    if (!d_fin || !d_fout) return fail(RLBM_ERR_ARG, "need input and output buffers");
    if (precision != RLBM_FP64 && precision != RLBM_FP32)
        return fail(RLBM_ERR_UNSUPPORTED, "rlbm_step_noalloc supports FP64 and FP32 storage");
    if (N > 3 || npop > kMaxNpop)
        return fail(RLBM_ERR_ARG, "rlbm_step_noalloc is limited to N <= 3 and K (N+1) <= 256 populations "
                                  "(its scratch array holds 32 KB)");
    const bool r64 = precision == RLBM_FP64;
    const size_t es = r64 ? 8 : 4;
    if (((uintptr_t)d_fin % es) || ((uintptr_t)d_fout % es))
        return fail(RLBM_ERR_ARG, "buffers must be aligned to the element size");
    // the step streams from d_fin into d_fout: the two byte ranges must not overlap
    const size_t len = size_t(npop) * size_t(grid.nx) * size_t(grid.ny) * es;
    const uintptr_t pi = (uintptr_t)d_fin, po = (uintptr_t)d_fout;
    if (pi < po + len && po < pi + len)
        return fail(RLBM_ERR_ARG, "input and output buffers overlap");

    // tiling: fewest idle population slots, then the larger P (as rlbm_create)
    static const int sizes[] = {8, 12, 16, 24, 32, 48, 64};
    int P = 0, Gs = 0, best = 1 << 30;
    for (int gs = 1; gs * (N + 1) <= rlbmk::kMaxWarps; ++gs) {
        const int need = (K + gs - 1) / gs;
        if (need > 64 || (gs - 1) * need >= K) continue;
        int p = 0;
        for (int s : sizes)
            if (s >= need) { p = s; break; }
        const int waste = gs * p - K;
        if (waste < best || (waste == best && p > P)) { best = waste; P = p; Gs = gs; }
    }
    if (!P) return fail(RLBM_ERR_UNSUPPORTED, "no compiled tiling for this K");
    const int G = Gs * (N + 1);

    // tables (the same quantities rlbm_create builds), in the host staging buffer
    const int TW = rlbmk::tab_width(N);
    double pr[4], wr[4];
    nodes(N + 1, pr);
    for (int r = 0; r <= N; ++r) {
        double l, lm;
        laguerre2(N + 2, pr[r], l, lm);
        wr[r] = pr[r] / ((N + 2.0) * (N + 2.0) * l * l);
    }
    // per-population table in the storage's arithmetic type; the per-site part
    // (moment folds, Landau frame, projection weights) runs in FP64 for FP32
    // storage as well, as it does in the handle's per-tile kernel
    const size_t ls = 8;
    const size_t o_status = 0;
    const size_t o_pop = 256;
    const size_t o_shell = o_pop + align256(size_t(npop) * TW * es);
    const size_t o_rt = o_shell + align256(size_t(N + 1) * 2 * ls);
    const size_t o_mask = o_rt + align256(size_t(N + 1) * (N + 1) * (N + 1) * ls);
    const size_t total = o_mask + align256(size_t(G) * 2 * 8);
    if (total > kScratchBytes) return fail(RLBM_ERR_ARG, "tables exceed the 32 KB scratch array");
    std::memset(g_blob, 0, total);
    unsigned long long masks[2 * rlbmk::kMaxWarps] = {};
    for (int r = 0; r <= N; ++r)
        for (int j = 0; j < K; ++j) {
            const int i = r * K + j;
            const double th = (j + r / double(N + 1)) * (2.0 * kPi / K);
            double c = std::cos(th), s = std::sin(th);
            if (std::fabs(c) < 1e-15) c = 0.0;
            if (std::fabs(s) < 1e-15) s = 0.0;
            const double w = wr[r] * (2.0 * kPi / K);
            const double tha = std::atan2(s, c);
            double t[16] = {};
            t[0] = c; t[1] = s; t[2] = c * c; t[3] = c * s; t[4] = w;
            for (int m = 1; m <= N; ++m) {
                t[4 + 2 * m - 1] = w * std::cos(m * tha);
                t[4 + 2 * m] = w * std::sin(m * tha);
            }
            for (int u = 0; u < TW; ++u) {
                unsigned char *dst = g_blob + o_pop + (size_t(i) * TW + u) * es;
                if (r64) put<double>(dst, t[u]); else put<float>(dst, t[u]);
            }
            const int q = j / P, k = j % P, g = r * Gs + q;
            if (c >= 0.0) masks[2 * g] |= 1ull << k;
            if (s >= 0.0) masks[2 * g + 1] |= 1ull << k;
        }
    for (int r = 0; r <= N; ++r) {
        unsigned char *d = g_blob + o_shell + size_t(2 * r) * ls;
        put<double>(d, pr[r]);
        put<double>(d + ls, pr[r] * pr[r]);
    }
    for (int m = 0; m <= N; ++m) {
        const int d = N - m + 1;
        double Gi[4][4];
        if (!hankel_inverse(d, m, Gi)) return fail(RLBM_ERR_ARG, "projection matrix is singular");
        const double norm = (m == 0) ? 2.0 * kPi : kPi;
        for (int r = 0; r <= N; ++r)
            for (int k = m; k <= N; ++k) {
                double s = 0.0;
                for (int l = m; l <= N; ++l) s += std::pow(pr[r], l) * Gi[l - m][k - m];
                double kf = 1.0;
                for (int t = 2; t <= k; ++t) kf *= t;
                unsigned char *dst = g_blob + o_rt + (size_t(r * (N + 1) + m) * (N + 1) + k) * ls;
                put<double>(dst, s / norm * kf / (N + 1));
            }
    }
    std::memcpy(g_blob + o_mask, masks, size_t(G) * 2 * 8);

    void *scratch = nullptr;
    rlbm_status st = scratch_address(&scratch);
    if (st) return st;
    cudaStream_t stream = (cudaStream_t)cuda_stream;
    // tables and a cleared status word into the shared scratch array
    if (cudaMemcpyAsync(scratch, g_blob, total, cudaMemcpyHostToDevice, stream) != cudaSuccess)
        return fail(RLBM_ERR_CUDA, "copy of the tables into the scratch array failed");

    rlbmk::KernelArgs a;
    std::memset(&a, 0, sizeof(a));
    unsigned char *base = static_cast<unsigned char *>(scratch);
    a.fin = d_fin;
    a.fout = d_fout;
    a.nx = grid.nx;
    a.ny = grid.ny;
    a.S = (long long)grid.nx * grid.ny;
    a.K = K;
    a.Gs = Gs;
    a.P = P;
    a.bcx = grid.bc_x;
    a.bcy = grid.bc_y;
    a.collide = std::isinf(tau) ? 0 : 1;
    a.inv_tau = std::isinf(tau) ? 0.0 : 1.0 / tau;
    a.inv_tau_f = float(a.inv_tau);
    for (int j = 0; j <= N; ++j) {
        const double ph = 2.0 * kPi * j / (N + 1);
        a.smp_c[j] = std::cos(ph);
        a.smp_s[j] = std::sin(ph);
        a.smp_cf[j] = float(a.smp_c[j]);
        a.smp_sf[j] = float(a.smp_s[j]);
    }
    a.poptab = base + o_pop;
    a.shelltab = base + o_shell;
    a.rtab = base + o_rt;
    a.masks = reinterpret_cast<const unsigned long long *>(base + o_mask);
    a.status = reinterpret_cast<int *>(base + o_status);
    a.ctr = reinterpret_cast<unsigned *>(base + o_status + 4);

    const dim3 gridd((grid.nx + 31) / 32, grid.ny), block(32, G);
    const size_t smem = rlbmk::tile_smem_bytes(N, G, ls, false);
    const bool full = (K % P) == 0;
    const cudaError_t e = r64 ? rlbmk::launch_f64(rlbmk::MODE_STEP, N, P, grid.ny > 1, full, gridd,
                                                  block, smem, stream, a)
                              : rlbmk::launch_f32(rlbmk::MODE_STEP, N, P, grid.ny > 1, full, true,
                                                  gridd, block, smem, stream, a);
    if (e != cudaSuccess) return fail(RLBM_ERR_CUDA, cudaGetErrorString(e));
    int status = 0;
    if (cudaMemcpyAsync(&status, base + o_status, sizeof(int), cudaMemcpyDeviceToHost, stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
        return fail(RLBM_ERR_CUDA, "reading the status word failed");
    if (status & 1) return fail(RLBM_ERR_UNPHYSICAL, "a cell had no physical Landau frame");
    return RLBM_OK;
}

extern "C" const char *rlbm_noalloc_last_error(void) { return g_err; }
