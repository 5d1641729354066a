// Learned angular closure: a small MLP that corrects a coarse-angle run
// toward the fine-angle solution (not part of the paper; the build adds it).
//
//   features  x = (N^a, T^ab) / N^0 (9), Kn, f_i / (w_i N^0) (N_pop)      F = 10 + N_pop
//   network   y = W3 GELU(W2 GELU(W1 x + b1) + b2) + b3, hidden width 64, O = N_pop
//   apply     d_i = y_i w_i N^0, minus its weighted least-squares component
//             along p^0, p^0 p^0, p^0 p^x, p^0 p^y (so N^0, T^00, T^0x, T^0y of
//             the site are unchanged), added to the post-collision populations
//   training  target = (R f_fine(t+1) - Step_coarse(R f_fine(t))) / (w_i N^0),
//             R the per-shell spectral angular restriction (Fourier modes below
//             the coarse Nyquist mode; exact for equilibria, keeps N^a, T^0a);
//             mean-squared error, backprop, Adam on FP32 master weights.
//
// Weights are kept in BF16 for the forward passes, products accumulate in
// FP32.  Activations are feature-major ([feature][site]) so that a thread
// (one site) reads its inputs with coalesced loads across the warp.
#include "rlbm.h"
#include "rlbm_args.h"

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <random>
#include <string>
#include <vector>

namespace {

constexpr int H = 64;        // hidden width
constexpr int MAXO = 128;    // max populations handled (outputs)
constexpr int MAXF = 10 + MAXO;
constexpr int TS = 64;       // sites per training tile
constexpr float kPiF = 3.14159265358979f;

__device__ __forceinline__ float gelu(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float x)
{
    return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * expf(-0.5f * x * x) * 0.39894228040143268f;
}

struct Net {
    int F, O;
    const __nv_bfloat16 *W1, *W2, *W3; // [F][H], [H][H], [H][O]  (input-major)
    const float *b1, *b2, *b3;
};

// ---------------------------------------------------------------- forward
// One thread per site; weights in shared memory (BF16).  Writes y[O][ld], and
// for training the pre-activations z1, z2 [H][ld] and dY = 2 (y - t) / count.
template <bool TRAIN>
__global__ void __launch_bounds__(128) mlp_forward_kernel(Net net, const float *__restrict__ X, long long ld,
                                                          long long off, int count, float *__restrict__ Y,
                                                          float *__restrict__ Z1, float *__restrict__ Z2,
                                                          const float *__restrict__ T, float *__restrict__ dY,
                                                          float inv_count, float *__restrict__ loss)
{
    extern __shared__ __align__(16) unsigned char sm[];
    const int F = net.F, O = net.O;
    __nv_bfloat16 *w1 = reinterpret_cast<__nv_bfloat16 *>(sm);
    __nv_bfloat16 *w2 = w1 + F * H;
    __nv_bfloat16 *w3 = w2 + H * H;
    float *hbuf = reinterpret_cast<float *>(w3 + ((H * O + 7) / 8) * 8); // [H][128]
    for (int i = threadIdx.x; i < F * H; i += blockDim.x) w1[i] = net.W1[i];
    for (int i = threadIdx.x; i < H * H; i += blockDim.x) w2[i] = net.W2[i];
    for (int i = threadIdx.x; i < H * O; i += blockDim.x) w3[i] = net.W3[i];
    __syncthreads();
    float lsum = 0.f;
    for (long long base = (long long)blockIdx.x * blockDim.x; base < count; base += (long long)gridDim.x * blockDim.x) {
        const long long s = base + threadIdx.x;
        const bool act = s < count;
        const long long col = off + (act ? s : 0);
        float acc[H];
#pragma unroll
        for (int j = 0; j < H; ++j) acc[j] = net.b1[j];
        for (int i = 0; i < F; ++i) {
            const float xi = X[(long long)i * ld + col];
#pragma unroll
            for (int j = 0; j < H; ++j) acc[j] += xi * __bfloat162float(w1[i * H + j]);
        }
#pragma unroll
        for (int j = 0; j < H; ++j) {
            if (TRAIN && act) Z1[(long long)j * ld + col] = acc[j];
            hbuf[j * 128 + threadIdx.x] = gelu(acc[j]);
        }
#pragma unroll
        for (int j = 0; j < H; ++j) acc[j] = net.b2[j];
        for (int i = 0; i < H; ++i) {
            const float hi = hbuf[i * 128 + threadIdx.x];
#pragma unroll
            for (int j = 0; j < H; ++j) acc[j] += hi * __bfloat162float(w2[i * H + j]);
        }
#pragma unroll
        for (int j = 0; j < H; ++j) {
            if (TRAIN && act) Z2[(long long)j * ld + col] = acc[j];
            hbuf[j * 128 + threadIdx.x] = gelu(acc[j]);
        }
        // output layer in chunks of 32 outputs (registers)
        for (int o0 = 0; o0 < O; o0 += 32) {
            float out[32];
#pragma unroll
            for (int k = 0; k < 32; ++k) out[k] = (o0 + k < O) ? net.b3[o0 + k] : 0.f;
            for (int i = 0; i < H; ++i) {
                const float hi = hbuf[i * 128 + threadIdx.x];
#pragma unroll
                for (int k = 0; k < 32; ++k)
                    if (o0 + k < O) out[k] += hi * __bfloat162float(w3[i * O + o0 + k]);
            }
#pragma unroll
            for (int k = 0; k < 32; ++k) {
                if (o0 + k >= O || !act) continue;
                const long long a = (long long)(o0 + k) * ld + col;
                if (TRAIN) {
                    const float d = out[k] - T[a];
                    dY[a] = 2.0f * d * inv_count;
                    lsum += d * d;
                } else {
                    Y[a] = out[k];
                }
            }
        }
    }
    if (TRAIN) {
        for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(loss, lsum);
    }
}

// ---------------------------------------------------------------- backward
// Tiles of TS sites.  Weight gradients are tile-local GEMMs over sites
// (G = A^T B), accumulated in FP32 and added to the global gradient once per
// tile; the back-propagated deltas are per-site matrix-vector products.
__device__ __forceinline__ void tile_outer(const float *A, int na, const float *B, int nb, int nsite,
                                           float *grad, int ldg)
{
    // grad[a][b] += sum_s A[a][s] B[b][s]   (A, B in shared memory, [dim][TS])
    for (int e = threadIdx.x; e < na * nb; e += blockDim.x) {
        const int a = e / nb, b = e % nb;
        float s = 0.f;
        for (int t = 0; t < nsite; ++t) s += A[a * TS + t] * B[b * TS + t];
        atomicAdd(&grad[a * ldg + b], s);
    }
}

__global__ void __launch_bounds__(128) mlp_backward_kernel(Net net, const float *__restrict__ X, long long ld,
                                                           long long off, int count,
                                                           const float *__restrict__ Z1,
                                                           const float *__restrict__ Z2,
                                                           const float *__restrict__ dY, float *__restrict__ g)
{
    extern __shared__ __align__(16) float fsm[];
    const int F = net.F, O = net.O;
    float *sdy = fsm;               // [O][TS]
    float *sa = sdy + MAXO * TS;    // [H][TS]  h2, then dz2
    float *sb = sa + H * TS;        // [H][TS]  h1, then dz1
    float *sx = sb + H * TS;        // [F][TS]
    float *gW1 = g, *gb1 = g + F * H, *gW2 = gb1 + H, *gb2 = gW2 + H * H, *gW3 = gb2 + H, *gb3 = gW3 + H * O;
    const int ntiles = (count + TS - 1) / TS;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long long s0 = (long long)tile * TS;
        const int ns = (int)min((long long)TS, count - s0);
        __syncthreads();
        for (int e = threadIdx.x; e < O * TS; e += blockDim.x) {
            const int o = e / TS, t = e % TS;
            sdy[e] = t < ns ? dY[(long long)o * ld + off + s0 + t] : 0.f;
        }
        for (int e = threadIdx.x; e < H * TS; e += blockDim.x) {
            const int j = e / TS, t = e % TS;
            sa[e] = t < ns ? gelu(Z2[(long long)j * ld + off + s0 + t]) : 0.f;
            sb[e] = t < ns ? gelu(Z1[(long long)j * ld + off + s0 + t]) : 0.f;
        }
        for (int e = threadIdx.x; e < F * TS; e += blockDim.x) {
            const int i = e / TS, t = e % TS;
            sx[e] = t < ns ? X[(long long)i * ld + off + s0 + t] : 0.f;
        }
        __syncthreads();
        tile_outer(sa, H, sdy, O, ns, gW3, O); // dW3 = h2^T dY
        for (int o = threadIdx.x; o < O; o += blockDim.x) {
            float s = 0.f;
            for (int t = 0; t < ns; ++t) s += sdy[o * TS + t];
            atomicAdd(&gb3[o], s);
        }
        __syncthreads();
        // dz2 = (dY W3^T) * gelu'(z2)  (overwrites h2)
        for (int e = threadIdx.x; e < H * TS; e += blockDim.x) {
            const int j = e / TS, t = e % TS;
            float s = 0.f;
            for (int o = 0; o < O; ++o) s += sdy[o * TS + t] * __bfloat162float(net.W3[j * O + o]);
            sa[e] = t < ns ? s * gelu_grad(Z2[(long long)j * ld + off + s0 + t]) : 0.f;
        }
        __syncthreads();
        tile_outer(sb, H, sa, H, ns, gW2, H); // dW2 = h1^T dz2
        for (int j = threadIdx.x; j < H; j += blockDim.x) {
            float s = 0.f;
            for (int t = 0; t < ns; ++t) s += sa[j * TS + t];
            atomicAdd(&gb2[j], s);
        }
        __syncthreads();
        // dz1 = (dz2 W2^T) * gelu'(z1)  (overwrites h1)
        for (int e = threadIdx.x; e < H * TS; e += blockDim.x) {
            const int j = e / TS, t = e % TS;
            float s = 0.f;
            for (int k = 0; k < H; ++k) s += sa[k * TS + t] * __bfloat162float(net.W2[j * H + k]);
            sb[e] = t < ns ? s * gelu_grad(Z1[(long long)j * ld + off + s0 + t]) : 0.f;
        }
        __syncthreads();
        tile_outer(sx, F, sb, H, ns, gW1, H); // dW1 = x^T dz1
        for (int j = threadIdx.x; j < H; j += blockDim.x) {
            float s = 0.f;
            for (int t = 0; t < ns; ++t) s += sb[j * TS + t];
            atomicAdd(&gb1[j], s);
        }
    }
}

// ---------------------------------------------------------------- Adam
__global__ void adam_kernel(float *p, const float *g, float *m, float *v, int n, float lr, float b1,
                            float b2, float eps, float c1, float c2)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    }
}

__global__ void to_bf16_kernel(const float *p, __nv_bfloat16 *w, const int *map, int nw)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nw; i += gridDim.x * blockDim.x)
        w[i] = __float2bfloat16_rn(p[map[i]]);
}

// ---------------------------------------------------------------- LB-side kernels
struct CoarseTab {
    int npop, N, K;
    const float *p0, *c, *s, *w; // per population
    const float *Ainv;          // 4x4 inverse of C W C^T
};

// moments (9) of one site's populations, FP32
__device__ __forceinline__ void site_moments(const CoarseTab &q, const float *f, long long S, long long site,
                                             float *m)
{
    for (int k = 0; k < 9; ++k) m[k] = 0.f;
    for (int i = 0; i < q.npop; ++i) {
        const float v = f[(long long)i * S + site];
        const float p = q.p0[i], px = p * q.c[i], py = p * q.s[i];
        m[0] += p * v; m[1] += px * v; m[2] += py * v;
        m[3] += p * p * v; m[4] += p * px * v; m[5] += p * py * v;
        m[6] += px * px * v; m[7] += px * py * v; m[8] += py * py * v;
    }
}

__global__ void features_kernel(CoarseTab q, const float *__restrict__ f, long long S, float kn,
                                float *__restrict__ X, long long ld, long long off)
{
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < S; s += (long long)gridDim.x * blockDim.x) {
        float m[9];
        site_moments(q, f, S, s, m);
        const float inv = 1.f / m[0];
        for (int k = 0; k < 9; ++k) X[(long long)k * ld + off + s] = m[k] * inv;
        X[9 * ld + off + s] = kn;
        for (int i = 0; i < q.npop; ++i)
            X[(long long)(10 + i) * ld + off + s] = f[(long long)i * S + s] * inv / q.w[i];
    }
}

__global__ void target_kernel(CoarseTab q, const float *__restrict__ fr, const float *__restrict__ fc, long long S,
                              float *__restrict__ T, long long ld, long long off)
{
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < S; s += (long long)gridDim.x * blockDim.x) {
        float n0 = 0.f;
        for (int i = 0; i < q.npop; ++i) n0 += q.p0[i] * fc[(long long)i * S + s];
        const float inv = 1.f / n0;
        for (int i = 0; i < q.npop; ++i) {
            const long long a = (long long)i * S + s;
            T[(long long)i * ld + off + s] = (fr[a] - fc[a]) * inv / q.w[i];
        }
    }
}

// sparse restriction: for coarse population k, entries [beg[k], beg[k+1]) of (j, weight)
__global__ void restrict_kernel(const float *__restrict__ ff, long long S, int npc, const int *beg,
                                const int *idx, const float *wt, float *__restrict__ fc)
{
    for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < S; s += (long long)gridDim.x * blockDim.x) {
        for (int k = 0; k < npc; ++k) {
            float acc = 0.f;
            for (int e = beg[k]; e < beg[k + 1]; ++e) acc += wt[e] * ff[(long long)idx[e] * S + s];
            fc[(long long)k * S + s] = acc;
        }
    }
}

// features + network + conservative projection + update, one thread per site
__global__ void __launch_bounds__(128) apply_kernel(Net net, CoarseTab q, float *__restrict__ f, long long S,
                                                    float kn)
{
    extern __shared__ __align__(16) unsigned char sm[];
    const int F = net.F, O = net.O;
    __nv_bfloat16 *w1 = reinterpret_cast<__nv_bfloat16 *>(sm);
    __nv_bfloat16 *w2 = w1 + F * H;
    __nv_bfloat16 *w3 = w2 + H * H;
    float *hbuf = reinterpret_cast<float *>(w3 + ((H * O + 7) / 8) * 8); // [H][128]
    float *xbuf = hbuf + H * 128;                                        // [F][128]
    for (int i = threadIdx.x; i < F * H; i += blockDim.x) w1[i] = net.W1[i];
    for (int i = threadIdx.x; i < H * H; i += blockDim.x) w2[i] = net.W2[i];
    for (int i = threadIdx.x; i < H * O; i += blockDim.x) w3[i] = net.W3[i];
    __syncthreads();
    for (long long base = (long long)blockIdx.x * blockDim.x; base < S; base += (long long)gridDim.x * blockDim.x) {
        const long long s = base + threadIdx.x;
        const bool act = s < S;
        const long long site = act ? s : 0;
        float m[9];
        site_moments(q, f, S, site, m);
        const float n0 = m[0], inv = 1.f / n0;
        for (int k = 0; k < 9; ++k) xbuf[k * 128 + threadIdx.x] = m[k] * inv;
        xbuf[9 * 128 + threadIdx.x] = kn;
        for (int i = 0; i < q.npop; ++i)
            xbuf[(10 + i) * 128 + threadIdx.x] = f[(long long)i * S + site] * inv / q.w[i];
        float acc[H];
#pragma unroll
        for (int j = 0; j < H; ++j) acc[j] = net.b1[j];
        for (int i = 0; i < F; ++i) {
            const float xi = xbuf[i * 128 + threadIdx.x];
#pragma unroll
            for (int j = 0; j < H; ++j) acc[j] += xi * __bfloat162float(w1[i * H + j]);
        }
#pragma unroll
        for (int j = 0; j < H; ++j) hbuf[j * 128 + threadIdx.x] = gelu(acc[j]);
#pragma unroll
        for (int j = 0; j < H; ++j) acc[j] = net.b2[j];
        for (int i = 0; i < H; ++i) {
            const float hi = hbuf[i * 128 + threadIdx.x];
#pragma unroll
            for (int j = 0; j < H; ++j) acc[j] += hi * __bfloat162float(w2[i * H + j]);
        }
#pragma unroll
        for (int j = 0; j < H; ++j) hbuf[j * 128 + threadIdx.x] = gelu(acc[j]);
        // output, denormalised into xbuf rows 10.. (reused), conserved sums on the fly
        float cs[4] = {0.f, 0.f, 0.f, 0.f};
        for (int o0 = 0; o0 < O; o0 += 32) {
            float out[32];
#pragma unroll
            for (int k = 0; k < 32; ++k) out[k] = (o0 + k < O) ? net.b3[o0 + k] : 0.f;
            for (int i = 0; i < H; ++i) {
                const float hi = hbuf[i * 128 + threadIdx.x];
#pragma unroll
                for (int k = 0; k < 32; ++k)
                    if (o0 + k < O) out[k] += hi * __bfloat162float(w3[i * O + o0 + k]);
            }
#pragma unroll
            for (int k = 0; k < 32; ++k) {
                const int i = o0 + k;
                if (i >= O) continue;
                const float d = out[k] * q.w[i] * n0;
                xbuf[(10 + i) * 128 + threadIdx.x] = d;
                const float p = q.p0[i];
                cs[0] += p * d;
                cs[1] += p * p * d;
                cs[2] += p * p * q.c[i] * d;
                cs[3] += p * p * q.s[i] * d;
            }
        }
        float lam[4];
        for (int a = 0; a < 4; ++a)
            lam[a] = q.Ainv[a * 4 + 0] * cs[0] + q.Ainv[a * 4 + 1] * cs[1] + q.Ainv[a * 4 + 2] * cs[2] +
                     q.Ainv[a * 4 + 3] * cs[3];
        if (act) {
            for (int i = 0; i < O; ++i) {
                const float p = q.p0[i];
                const float corr = q.w[i] * (lam[0] * p + lam[1] * p * p + lam[2] * p * p * q.c[i] +
                                             lam[3] * p * p * q.s[i]);
                f[(long long)i * S + s] += xbuf[(10 + i) * 128 + threadIdx.x] - corr;
            }
        }
    }
}

} // namespace

// ==================================================================== host side

struct rlbm_closure {
    int N = 0, K = 0, npop = 0, F = 0, O = 0;
    cudaStream_t stream = nullptr;
    size_t nparam = 0;
    float *d_p = nullptr, *d_g = nullptr, *d_m = nullptr, *d_v = nullptr; // FP32 master, grad, Adam moments
    __nv_bfloat16 *d_w = nullptr;   // W1 | W2 | W3 in BF16
    int *d_wmap = nullptr;          // BF16 weight -> master index
    float *d_tab = nullptr;         // p0 | c | s | w | Ainv
    float *d_loss = nullptr;
    int adam_t = 0;
    std::string err;
    size_t off_W1, off_b1, off_W2, off_b2, off_W3, off_b3;
};

namespace {

thread_local std::string g_cerr;

rlbm_status cfail(rlbm_closure *c, rlbm_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c) c->err = buf; else g_cerr = buf;
    return st;
}

#define CL_CUDA(c, call)                                                                         \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess) return cfail(c, RLBM_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

Net net_of(const rlbm_closure *c)
{
    Net n;
    n.F = c->F;
    n.O = c->O;
    n.W1 = c->d_w;
    n.W2 = c->d_w + size_t(c->F) * H;
    n.W3 = n.W2 + size_t(H) * H;
    n.b1 = c->d_p + c->off_b1;
    n.b2 = c->d_p + c->off_b2;
    n.b3 = c->d_p + c->off_b3;
    return n;
}

CoarseTab tab_of(const rlbm_closure *c)
{
    CoarseTab q;
    q.npop = c->npop;
    q.N = c->N;
    q.K = c->K;
    q.p0 = c->d_tab;
    q.c = c->d_tab + c->npop;
    q.s = c->d_tab + 2 * c->npop;
    q.w = c->d_tab + 3 * c->npop;
    q.Ainv = c->d_tab + 4 * c->npop;
    return q;
}

size_t fwd_smem(const rlbm_closure *c, bool with_x)
{
    size_t b = (size_t(c->F) * H + size_t(H) * H + ((size_t(H) * c->O + 7) / 8) * 8) * 2 + size_t(H) * 128 * 4;
    if (with_x) b += size_t(c->F) * 128 * 4;
    return b;
}

size_t bwd_smem(const rlbm_closure *c) { return (size_t(MAXO) + 2 * H + c->F) * TS * 4; }

rlbm_status refresh_bf16(rlbm_closure *c)
{
    const int nw = c->F * H + H * H + H * c->O;
    to_bf16_kernel<<<(nw + 255) / 256, 256, 0, c->stream>>>(c->d_p, c->d_w, c->d_wmap, nw);
    CL_CUDA(c, cudaGetLastError());
    return RLBM_OK;
}

bool invert4(const double *A, double *inv)
{
    double M[4][8];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 8; ++j) M[i][j] = j < 4 ? A[i * 4 + j] : (j - 4 == i ? 1.0 : 0.0);
    for (int c = 0; c < 4; ++c) {
        int p = c;
        for (int i = c + 1; i < 4; ++i)
            if (std::fabs(M[i][c]) > std::fabs(M[p][c])) p = i;
        if (M[p][c] == 0.0) return false;
        for (int j = 0; j < 8; ++j) std::swap(M[c][j], M[p][j]);
        const double d = M[c][c];
        for (int j = 0; j < 8; ++j) M[c][j] /= d;
        for (int i = 0; i < 4; ++i) {
            if (i == c) continue;
            const double f = M[i][c];
            for (int j = 0; j < 8; ++j) M[i][j] -= f * M[c][j];
        }
    }
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) inv[i * 4 + j] = M[i][4 + j];
    return true;
}

} // namespace

extern "C" {

const char *rlbm_closure_last_error(const rlbm_closure_t *c) { return c ? c->err.c_str() : g_cerr.c_str(); }

size_t rlbm_closure_param_count(const rlbm_closure_t *c) { return c ? c->nparam : 0; }

rlbm_status rlbm_closure_create(rlbm_closure_t **out, int order_N, int angles_K, unsigned long long seed,
                                void *cuda_stream)
{
    if (!out) return cfail(nullptr, RLBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    const int npop = angles_K * (order_N + 1);
    if (order_N < 2 || angles_K < 2 * order_N + 1 || npop > MAXO)
        return cfail(nullptr, RLBM_ERR_ARG, "closure needs N >= 2, K >= 2N+1 and K (N+1) <= %d", MAXO);
    rlbm_closure *c = new (std::nothrow) rlbm_closure();
    if (!c) return cfail(nullptr, RLBM_ERR_OOM, "host allocation failed");
    c->N = order_N;
    c->K = angles_K;
    c->npop = npop;
    c->F = 10 + npop;
    c->O = npop;
    c->stream = (cudaStream_t)cuda_stream;
    c->off_W1 = 0;
    c->off_b1 = c->off_W1 + size_t(c->F) * H;
    c->off_W2 = c->off_b1 + H;
    c->off_b2 = c->off_W2 + size_t(H) * H;
    c->off_W3 = c->off_b2 + H;
    c->off_b3 = c->off_W3 + size_t(H) * c->O;
    c->nparam = c->off_b3 + c->O;
    auto bail = [&](rlbm_status s) { g_cerr = c->err; rlbm_closure_destroy(c); return s; };
    // initial weights: uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)), biases 0; output layer scaled down
    std::vector<float> p(c->nparam, 0.f);
    std::mt19937_64 rng(seed);
    auto fill = [&](size_t off, int fan_in, int n, float scale) {
        std::uniform_real_distribution<float> U(-scale / std::sqrt(float(fan_in)), scale / std::sqrt(float(fan_in)));
        for (int i = 0; i < n; ++i) p[off + i] = U(rng);
    };
    fill(c->off_W1, c->F, c->F * H, 1.f);
    fill(c->off_W2, H, H * H, 1.f);
    fill(c->off_W3, H, H * c->O, 0.1f);
    // quadrature tables of the coarse rule and the 4x4 projection inverse
    std::vector<double> qp0(npop), qvx(npop), qvy(npop), qw(npop);
    rlbm_status st = rlbm_quadrature(order_N, angles_K, qp0.data(), qvx.data(), qvy.data(), qw.data());
    if (st) return bail(cfail(c, st, "quadrature failed"));
    double A[16] = {0};
    for (int i = 0; i < npop; ++i) {
        const double cvec[4] = {qp0[i], qp0[i] * qp0[i], qp0[i] * qp0[i] * qvx[i], qp0[i] * qp0[i] * qvy[i]};
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) A[a * 4 + b] += qw[i] * cvec[a] * cvec[b];
    }
    double Ai[16];
    if (!invert4(A, Ai)) return bail(cfail(c, RLBM_ERR_ARG, "singular projection matrix"));
    std::vector<float> tab(4 * size_t(npop) + 16);
    for (int i = 0; i < npop; ++i) {
        tab[i] = float(qp0[i]);
        tab[npop + i] = float(qvx[i]);
        tab[2 * npop + i] = float(qvy[i]);
        tab[3 * npop + i] = float(qw[i]);
    }
    for (int k = 0; k < 16; ++k) tab[4 * npop + k] = float(Ai[k]);
    const int nw = c->F * H + H * H + H * c->O;
    std::vector<int> wmap(nw);
    {
        int k = 0;
        for (int i = 0; i < c->F * H; ++i) wmap[k++] = int(c->off_W1) + i;
        for (int i = 0; i < H * H; ++i) wmap[k++] = int(c->off_W2) + i;
        for (int i = 0; i < H * c->O; ++i) wmap[k++] = int(c->off_W3) + i;
    }
    if (cudaMalloc(&c->d_p, c->nparam * 4) != cudaSuccess || cudaMalloc(&c->d_g, c->nparam * 4) != cudaSuccess ||
        cudaMalloc(&c->d_m, c->nparam * 4) != cudaSuccess || cudaMalloc(&c->d_v, c->nparam * 4) != cudaSuccess ||
        cudaMalloc(&c->d_w, size_t(nw) * 2) != cudaSuccess || cudaMalloc(&c->d_wmap, size_t(nw) * 4) != cudaSuccess ||
        cudaMalloc(&c->d_tab, tab.size() * 4) != cudaSuccess || cudaMalloc(&c->d_loss, 4) != cudaSuccess)
        return bail(cfail(c, RLBM_ERR_OOM, "device allocation failed"));
    if (cudaMemcpyAsync(c->d_p, p.data(), c->nparam * 4, cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->d_m, 0, c->nparam * 4, c->stream) != cudaSuccess ||
        cudaMemsetAsync(c->d_v, 0, c->nparam * 4, c->stream) != cudaSuccess ||
        cudaMemcpyAsync(c->d_wmap, wmap.data(), size_t(nw) * 4, cudaMemcpyHostToDevice, c->stream) != cudaSuccess ||
        cudaMemcpyAsync(c->d_tab, tab.data(), tab.size() * 4, cudaMemcpyHostToDevice, c->stream) != cudaSuccess)
        return bail(cfail(c, RLBM_ERR_CUDA, "upload failed"));
    st = refresh_bf16(c);
    if (st) return bail(st);
    if (cudaFuncSetAttribute(mlp_forward_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_smem(c, false)) != cudaSuccess ||
        cudaFuncSetAttribute(mlp_forward_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_smem(c, false)) != cudaSuccess ||
        cudaFuncSetAttribute(apply_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fwd_smem(c, true)) != cudaSuccess ||
        cudaFuncSetAttribute(mlp_backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bwd_smem(c)) != cudaSuccess)
        return bail(cfail(c, RLBM_ERR_CUDA, "shared-memory attribute failed"));
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return bail(cfail(c, RLBM_ERR_CUDA, "sync failed"));
    *out = c;
    return RLBM_OK;
}

void rlbm_closure_destroy(rlbm_closure_t *c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    cudaFree(c->d_p); cudaFree(c->d_g); cudaFree(c->d_m); cudaFree(c->d_v);
    cudaFree(c->d_w); cudaFree(c->d_wmap); cudaFree(c->d_tab); cudaFree(c->d_loss);
    delete c;
}

rlbm_status rlbm_closure_get_params(rlbm_closure_t *c, float *host, size_t n)
{
    if (!c || !host || n != c->nparam) return cfail(c, RLBM_ERR_ARG, "need %zu floats", c ? c->nparam : 0);
    CL_CUDA(c, cudaMemcpyAsync(host, c->d_p, n * 4, cudaMemcpyDeviceToHost, c->stream));
    CL_CUDA(c, cudaStreamSynchronize(c->stream));
    return RLBM_OK;
}

rlbm_status rlbm_closure_set_params(rlbm_closure_t *c, const float *host, size_t n)
{
    if (!c || !host || n != c->nparam) return cfail(c, RLBM_ERR_ARG, "need %zu floats", c ? c->nparam : 0);
    CL_CUDA(c, cudaMemcpyAsync(c->d_p, host, n * 4, cudaMemcpyHostToDevice, c->stream));
    rlbm_status st = refresh_bf16(c);
    if (st) return st;
    CL_CUDA(c, cudaStreamSynchronize(c->stream));
    c->adam_t = 0;
    CL_CUDA(c, cudaMemsetAsync(c->d_m, 0, c->nparam * 4, c->stream));
    CL_CUDA(c, cudaMemsetAsync(c->d_v, 0, c->nparam * 4, c->stream));
    return RLBM_OK;
}

rlbm_status rlbm_closure_features(rlbm_closure_t *c, const float *d_f, long long sites, double kn, float *d_x,
                                  long long ld, long long off)
{
    if (!c || !d_f || !d_x || sites < 1) return cfail(c, RLBM_ERR_ARG, "bad arguments");
    features_kernel<<<1024, 128, 0, c->stream>>>(tab_of(c), d_f, sites, float(kn), d_x, ld, off);
    CL_CUDA(c, cudaGetLastError());
    return RLBM_OK;
}

rlbm_status rlbm_closure_target(rlbm_closure_t *c, const float *d_fr, const float *d_fc, long long sites,
                                float *d_t, long long ld, long long off)
{
    if (!c || !d_fr || !d_fc || !d_t || sites < 1) return cfail(c, RLBM_ERR_ARG, "bad arguments");
    target_kernel<<<1024, 128, 0, c->stream>>>(tab_of(c), d_fr, d_fc, sites, d_t, ld, off);
    CL_CUDA(c, cudaGetLastError());
    return RLBM_OK;
}

rlbm_status rlbm_closure_restrict(rlbm_closure_t *c, int fine_K, const float *d_ff, long long sites, float *d_fc)
{
    if (!c || !d_ff || !d_fc || sites < 1 || fine_K < c->K) return cfail(c, RLBM_ERR_ARG, "bad arguments");
    // per shell spectral restriction: the fine angular function g = f / w truncated to its
    // Fourier modes |m| <= (Kc - 1) / 2 and evaluated at the coarse angles (exact for
    // equilibria; keeps the m = 0, 1 modes and so N^0, N^i, T^00, T^0i)
    const int N = c->N, Kc = c->K, Kf = fine_K;
    const int M = (Kc - 1) / 2;
    const double two_pi = 2.0 * 3.14159265358979323846;
    std::vector<std::vector<std::pair<int, float>>> rows(size_t(N + 1) * Kc);
    for (int r = 0; r <= N; ++r) {
        const double off = double(r) / (N + 1);
        for (int k = 0; k < Kc; ++k) {
            const double tc = (k + off) * two_pi / Kc;
            for (int j = 0; j < Kf; ++j) {
                const double d = tc - (j + off) * two_pi / Kf;
                double ker = 1.0;
                for (int m = 1; m <= M; ++m) ker += 2.0 * std::cos(m * d);
                rows[size_t(r) * Kc + k].push_back({r * Kf + j, float(ker / Kc)});
            }
        }
    }
    std::vector<int> beg(rows.size() + 1, 0), idx;
    std::vector<float> wt;
    for (size_t k = 0; k < rows.size(); ++k) {
        for (auto &e : rows[k]) { idx.push_back(e.first); wt.push_back(e.second); }
        beg[k + 1] = int(idx.size());
    }
    int *d_beg = nullptr, *d_idx = nullptr;
    float *d_wt = nullptr;
    CL_CUDA(c, cudaMallocAsync(&d_beg, beg.size() * 4, c->stream));
    CL_CUDA(c, cudaMallocAsync(&d_idx, idx.size() * 4, c->stream));
    CL_CUDA(c, cudaMallocAsync(&d_wt, wt.size() * 4, c->stream));
    CL_CUDA(c, cudaMemcpyAsync(d_beg, beg.data(), beg.size() * 4, cudaMemcpyHostToDevice, c->stream));
    CL_CUDA(c, cudaMemcpyAsync(d_idx, idx.data(), idx.size() * 4, cudaMemcpyHostToDevice, c->stream));
    CL_CUDA(c, cudaMemcpyAsync(d_wt, wt.data(), wt.size() * 4, cudaMemcpyHostToDevice, c->stream));
    restrict_kernel<<<1024, 128, 0, c->stream>>>(d_ff, sites, c->npop, d_beg, d_idx, d_wt, d_fc);
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(d_beg, c->stream);
    cudaFreeAsync(d_idx, c->stream);
    cudaFreeAsync(d_wt, c->stream);
    CL_CUDA(c, e);
    CL_CUDA(c, cudaStreamSynchronize(c->stream)); // host tables go out of scope
    return RLBM_OK;
}

rlbm_status rlbm_closure_forward(rlbm_closure_t *c, const float *d_x, long long ld, long long off, int count,
                                 float *d_y)
{
    if (!c || !d_x || !d_y || count < 1) return cfail(c, RLBM_ERR_ARG, "bad arguments");
    const int grid = std::min(2048, (count + 127) / 128);
    mlp_forward_kernel<false><<<grid, 128, fwd_smem(c, false), c->stream>>>(
        net_of(c), d_x, ld, off, count, d_y, nullptr, nullptr, nullptr, nullptr, 0.f, nullptr);
    CL_CUDA(c, cudaGetLastError());
    return RLBM_OK;
}

// gradient of the mean-squared error over columns [off, off + count) into d_g; loss to host
static rlbm_status closure_grad(rlbm_closure_t *c, const float *d_x, const float *d_t, long long ld, long long off,
                                int count, float *d_z1, float *d_z2, float *d_dy, float *loss)
{
    CL_CUDA(c, cudaMemsetAsync(c->d_g, 0, c->nparam * 4, c->stream));
    CL_CUDA(c, cudaMemsetAsync(c->d_loss, 0, 4, c->stream));
    const int grid = std::min(2048, (count + 127) / 128);
    const float inv = 1.0f / (float(count) * float(c->O));
    // activations are stored with leading dimension `count`, columns relative to off
    mlp_forward_kernel<true><<<grid, 128, fwd_smem(c, false), c->stream>>>(
        net_of(c), d_x + off, ld, 0, count, nullptr, d_z1, d_z2, d_t + off, d_dy, inv, c->d_loss);
    CL_CUDA(c, cudaGetLastError());
    const int tiles = (count + TS - 1) / TS;
    mlp_backward_kernel<<<std::min(tiles, 1024), 128, bwd_smem(c), c->stream>>>(net_of(c), d_x + off, ld, 0, count,
                                                                            d_z1, d_z2, d_dy, c->d_g);
    CL_CUDA(c, cudaGetLastError());
    if (loss) {
        float l = 0.f;
        CL_CUDA(c, cudaMemcpyAsync(&l, c->d_loss, 4, cudaMemcpyDeviceToHost, c->stream));
        CL_CUDA(c, cudaStreamSynchronize(c->stream));
        *loss = l / (float(count) * float(c->O));
    }
    return RLBM_OK;
}

rlbm_status rlbm_closure_gradient(rlbm_closure_t *c, const float *d_x, const float *d_t, long long ld, long long off,
                                  int count, float *d_work, float *host_grad, float *loss)
{
    if (!c || !d_x || !d_t || !d_work || count < 1) return cfail(c, RLBM_ERR_ARG, "bad arguments");
    rlbm_status st = closure_grad(c, d_x, d_t, ld, off, count, d_work, d_work + size_t(H) * ld,
                                  d_work + size_t(2 * H) * ld, loss);
    if (st) return st;
    if (host_grad) {
        CL_CUDA(c, cudaMemcpyAsync(host_grad, c->d_g, c->nparam * 4, cudaMemcpyDeviceToHost, c->stream));
        CL_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    return RLBM_OK;
}

size_t rlbm_closure_work_floats(const rlbm_closure_t *c, long long ld)
{
    return c ? size_t(2 * H + c->O) * size_t(ld) : 0;
}

rlbm_status rlbm_closure_train_step(rlbm_closure_t *c, const float *d_x, const float *d_t, long long ld,
                                    long long off, int count, float lr, float *d_work, float *loss)
{
    if (!c || !d_x || !d_t || !d_work || count < 1 || !(lr > 0.f)) return cfail(c, RLBM_ERR_ARG, "bad arguments");
    rlbm_status st = closure_grad(c, d_x, d_t, ld, off, count, d_work, d_work + size_t(H) * ld,
                                  d_work + size_t(2 * H) * ld, loss);
    if (st) return st;
    ++c->adam_t;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f / (1.f - std::pow(b1, float(c->adam_t)));
    const float c2 = 1.f / (1.f - std::pow(b2, float(c->adam_t)));
    adam_kernel<<<64, 256, 0, c->stream>>>(c->d_p, c->d_g, c->d_m, c->d_v, int(c->nparam), lr, b1, b2, 1e-8f, c1,
                                          c2);
    CL_CUDA(c, cudaGetLastError());
    return refresh_bf16(c);
}

rlbm_status rlbm_closure_apply_buffer(rlbm_closure_t *c, float *d_f, long long sites, double kn)
{
    if (!c || !d_f || sites < 1) return cfail(c, RLBM_ERR_ARG, "bad arguments");
    const int grid = int(std::min<long long>(4096, (sites + 127) / 128));
    apply_kernel<<<grid, 128, fwd_smem(c, true), c->stream>>>(net_of(c), tab_of(c), d_f, sites, float(kn));
    CL_CUDA(c, cudaGetLastError());
    return RLBM_OK;
}

} // extern "C"
