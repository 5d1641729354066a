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

// ---------------------------------------------------------------- tensor-core apply
// The fused correction with the three layers on BF16 tensor cores
// (mma.sync.m16n8k16, FP32 accumulation), specialised for the coarse rule
// (N, K).  A CTA of TC_WARPS warps works on tiles of 16 TC_WARPS sites; the
// populations of the next tile stream into shared memory (cp.async, double
// buffered) while the current one is processed.
//
// * Conservation folded into the last layer.  With d = n0 W y (W = diag w) the
//   projection d - W C^T A^-1 C d equals n0 W Q y, Q = I - C^T A^-1 C W, a
//   constant matrix (C rows p^0, p^0 p^0, p^0 p^x, p^0 p^y; A = C W C^T).  So
//   y' = Q y = h2 (W3 Q^T) + Q b3: each CTA forms W3' = W3 - (W3 V^T) U^T with
//   V = C W and U = C^T A^-1 (FP32) and keeps it as a BF16 pair hi + lo
//   (relative error 2^-17), so that C W y' vanishes to FP32 rounding.  The
//   update is then f += n0 w_i y'_i.
// * Features.  Warp w owns sites 16w..16w+15 of the tile; lane (site, half)
//   sums half of every shell's angles (per-shell angular sums S0, Sc, Ss,
//   Scc, Scs, Sss folded with p_r, p_r^2), the halves are joined by a shuffle,
//   and the lane writes its populations / (w_i n0) as BF16 pairs into the
//   warp's input row.
// * Layers: [16 x K] x [K x N] products, fragments by ldmatrix from
//   transposed, padded BF16 weights; GELU between them (gelu_as below).
constexpr int TC_WARPS = 12;
constexpr int TC_SITES = 16 * TC_WARPS; // sites per CTA tile
constexpr int LDF = TC_SITES + 4;       // population-row stride of the tile (bank spread)
constexpr int SH = 72;                  // row stride of hidden tiles and of W2^T, W3'^T

__device__ __forceinline__ void mma_bf16(float *d, unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                         unsigned b0, unsigned b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
                 "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ unsigned smem_addr(const void *p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void ldsm_x4(const void *p, unsigned &r0, unsigned &r1, unsigned &r2, unsigned &r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(smem_addr(p)));
}

__device__ __forceinline__ void ldsm_x2(const void *p, unsigned &r0, unsigned &r1)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];"
                 : "=r"(r0), "=r"(r1)
                 : "r"(smem_addr(p)));
}

__device__ __forceinline__ unsigned pack_bf16(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const unsigned *>(&v);
}

// GELU(x) = x Phi(x) = x (1 + erf(x / sqrt 2)) / 2 with erf from Abramowitz &
// Stegun 7.1.26 (Hastings' rational approximation, |error| <= 1.5e-7):
// erf(z) = 1 - t (a1 + t (a2 + t (a3 + t (a4 + t a5)))) exp(-z^2), t = 1 / (1 + p z),
// z >= 0, extended to z < 0 by symmetry.  The layers' inputs are BF16, so
// this accuracy is far below their rounding.
__device__ __forceinline__ float gelu_as(float x)
{
    const float z = fabsf(x) * 0.70710678118654752f;
    float t;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(t) : "f"(fmaf(0.3275911f, z, 1.0f)));
    float q = fmaf(1.061405429f, t, -1.453152027f);
    q = fmaf(q, t, 1.421413741f);
    q = fmaf(q, t, -0.284496736f);
    q = fmaf(q, t, 0.254829592f);
    q *= t;
    float e; // exp(-z^2)
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e) : "f"(-1.4426950408889634f * z * z));
    const float h = 0.5f * q * e;                          // (1 - erf(z)) / 2
    return x * (x >= 0.f ? 1.f - h : h);
}

// GELU of two values with packed f32x2 arithmetic (same formula as gelu_as)
__device__ __forceinline__ float2 gelu2(float2 x)
{
    const float2 z = make_float2(fabsf(x.x) * 0.70710678118654752f, fabsf(x.y) * 0.70710678118654752f);
    const float2 den = __ffma2_rn(make_float2(0.3275911f, 0.3275911f), z, make_float2(1.f, 1.f));
    float2 t;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(t.x) : "f"(den.x));
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(t.y) : "f"(den.y));
    float2 q = __ffma2_rn(make_float2(1.061405429f, 1.061405429f), t, make_float2(-1.453152027f, -1.453152027f));
    q = __ffma2_rn(q, t, make_float2(1.421413741f, 1.421413741f));
    q = __ffma2_rn(q, t, make_float2(-0.284496736f, -0.284496736f));
    q = __ffma2_rn(q, t, make_float2(0.254829592f, 0.254829592f));
    q = __fmul2_rn(q, t);
    const float2 a = __fmul2_rn(__fmul2_rn(z, z), make_float2(-1.4426950408889634f, -1.4426950408889634f));
    float2 e;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e.x) : "f"(a.x));
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(e.y) : "f"(a.y));
    const float2 xh = __fmul2_rn(x, __fmul2_rn(__fmul2_rn(q, e), make_float2(0.5f, 0.5f))); // x (1 - erf(z)) / 2
    return make_float2(x.x >= 0.f ? x.x - xh.x : xh.x, x.y >= 0.f ? x.y - xh.y : xh.y);
}

// acc[nt][4] += A[16 x 16 KS] (row stride sa) x Bt[8 NT x 16 KS]^T (row stride sb)
template <int KS, int NT>
__device__ __forceinline__ void warp_gemm(const __nv_bfloat16 *A, int sa, const __nv_bfloat16 *Bt, int sb,
                                          float (*acc)[4], int lane)
{
    const int mi = lane >> 3, r8 = lane & 7;
#pragma unroll
    for (int ks = 0; ks < KS; ++ks) {
        unsigned a0, a1, a2, a3;
        // matrices: rows 0-7 | rows 8-15 at k0, then the same at k0 + 8
        ldsm_x4(A + ((mi & 1) * 8 + r8) * sa + ks * 16 + (mi >> 1) * 8, a0, a1, a2, a3);
#pragma unroll
        for (int np = 0; np < NT / 2; ++np) {
            unsigned b0, b1, b2, b3;
            // matrices: n-tile 2np at k0 | k0 + 8, n-tile 2np+1 at k0 | k0 + 8
            ldsm_x4(Bt + (np * 16 + (mi >> 1) * 8 + r8) * sb + ks * 16 + (mi & 1) * 8, b0, b1, b2, b3);
            mma_bf16(acc[2 * np], a0, a1, a2, a3, b0, b1);
            mma_bf16(acc[2 * np + 1], a0, a1, a2, a3, b2, b3);
        }
        if (NT & 1) {
            unsigned b0, b1;
            ldsm_x2(Bt + ((NT - 1) * 8 + r8) * sb + ks * 16 + (mi & 1) * 8, b0, b1);
            mma_bf16(acc[NT - 1], a0, a1, a2, a3, b0, b1);
        }
    }
}

__device__ __forceinline__ void bias_init(float (*acc)[4], const float *b, int nts, int lane)
{
    const int t = lane & 3;
    for (int nt = 0; nt < nts; ++nt) {
        const float2 v = *reinterpret_cast<const float2 *>(b + nt * 8 + 2 * t);
        acc[nt][0] = v.x; acc[nt][1] = v.y; acc[nt][2] = v.x; acc[nt][3] = v.y;
    }
}

__device__ __forceinline__ void gelu_rows(float (*acc)[4], __nv_bfloat16 *h, int lane)
{
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const int c = nt * 8 + t * 2;
        const float2 a = gelu2(make_float2(acc[nt][0], acc[nt][1]));
        const float2 b = gelu2(make_float2(acc[nt][2], acc[nt][3]));
        *reinterpret_cast<unsigned *>(h + g * SH + c) = pack_bf16(a.x, a.y);
        *reinterpret_cast<unsigned *>(h + (g + 8) * SH + c) = pack_bf16(b.x, b.y);
    }
}

// Populations of the tile at site0 into the shared tile (rows of LDF floats);
// sites >= S read as zero.  VEC = 4: 16-byte copies (S % 4 == 0, f 16-byte
// aligned); VEC = 1: 4-byte copies.
template <int VEC>
__device__ __forceinline__ void load_tile(float *tile, const float *f, long long S, long long site0, int npop)
{
    constexpr int CH = TC_SITES / VEC;
    for (int e = threadIdx.x; e < npop * CH; e += blockDim.x) {
        const int i = e / CH, c = e % CH;
        const long long site = site0 + c * VEC;
        const bool ok = site < S;
        const float *src = ok ? f + (long long)i * S + site : f;
        const unsigned dst = smem_addr(tile + i * LDF + c * VEC);
        if (VEC == 4)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(ok ? 16 : 0)
                         : "memory");
        else
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(dst), "l"(src), "r"(ok ? 4 : 0)
                         : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

template <int VEC>
__device__ __forceinline__ void store_tile(const float *tile, float *f, long long S, long long site0, int npop)
{
    constexpr int CH = TC_SITES / VEC;
    for (int e = threadIdx.x; e < npop * CH; e += blockDim.x) {
        const int i = e / CH, c = e % CH;
        const long long site = site0 + c * VEC;
        if (site >= S) continue;
        if (VEC == 4)
            *reinterpret_cast<float4 *>(f + (long long)i * S + site) =
                *reinterpret_cast<const float4 *>(tile + i * LDF + c * 4);
        else
            f[(long long)i * S + site] = tile[i * LDF + c];
    }
}

template <int N, int K>
struct TcGeom {
    static constexpr int NPOP = (N + 1) * K;
    static constexpr int F = 10 + NPOP;
    static constexpr int KS1 = (F + 15) / 16; // k-steps of layer 1
    static constexpr int SX = 16 * KS1 + 8;   // input row stride: odd number of 16-byte units
    static constexpr int NT3 = NPOP / 8;      // n-tiles of layer 3
    // shared memory carve-up, bytes
    static constexpr size_t W1 = 0, W2 = W1 + size_t(64) * SX * 2, W3H = W2 + size_t(64) * SH * 2,
                            W3L = W3H + size_t(NPOP) * SH * 2, BIAS = W3L + size_t(NPOP) * SH * 2,
                            TAB = BIAS + size_t(128 + NPOP) * 4,
                            WV = TAB + size_t(4 * NPOP + 8) * 4, // cs (2 NPOP), invw, wq, p_r (<= 8)
                            FT = (WV + 64 * 4 * 4 + 8 * 4 + 15) / 16 * 16,
                            WARP = FT + size_t(2) * NPOP * LDF * 4, TOTAL = WARP + size_t(TC_WARPS) * 16 * SX * 2;
};

template <int N, int K, int VEC>
__global__ void __launch_bounds__(TC_WARPS * 32, 1) apply_tc_kernel(Net net, CoarseTab q, float *__restrict__ f,
                                                                    long long S, float kn)
{
    using Gm = TcGeom<N, K>;
    constexpr int NPOP = Gm::NPOP, F = Gm::F, SX = Gm::SX, KH = K / 2;
    static_assert(K % 4 == 0 && NPOP % 8 == 0 && NPOP <= 2 * 64, "tile geometry");
    extern __shared__ __align__(16) unsigned char sm[];
    __nv_bfloat16 *w1t = reinterpret_cast<__nv_bfloat16 *>(sm + Gm::W1);  // [64][SX]
    __nv_bfloat16 *w2t = reinterpret_cast<__nv_bfloat16 *>(sm + Gm::W2);  // [64][SH]
    __nv_bfloat16 *w3h = reinterpret_cast<__nv_bfloat16 *>(sm + Gm::W3H); // [NPOP][SH]
    __nv_bfloat16 *w3l = reinterpret_cast<__nv_bfloat16 *>(sm + Gm::W3L); // [NPOP][SH]
    float *bias = reinterpret_cast<float *>(sm + Gm::BIAS);               // b1[64] b2[64] b3'[NPOP]
    float *cvec = reinterpret_cast<float *>(sm + Gm::TAB);                // v_x per population
    float *svec = cvec + NPOP;                                            // v_y per population
    float *invw = svec + NPOP;
    float *wq = invw + NPOP;
    float *pr = wq + NPOP;                                                // p_r per shell
    float *wv = reinterpret_cast<float *>(sm + Gm::WV);                   // (W3 V^T)[64][4], V b3 [4]
    float *ftile = reinterpret_cast<float *>(sm + Gm::FT);                // [2][NPOP][LDF]
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    __nv_bfloat16 *xa = reinterpret_cast<__nv_bfloat16 *>(sm + Gm::WARP) + size_t(wid) * 16 * SX;
    const long long ntile = (S + TC_SITES - 1) / TC_SITES;
    long long tile = blockIdx.x;
    if (tile < ntile) load_tile<VEC>(ftile, f, S, tile * TC_SITES, NPOP);

    // ---- per-CTA setup: weights, tables, the folded last layer
    for (int e = tid; e < 64 * SX; e += blockDim.x) {
        const int n = e / SX, k = e % SX;
        w1t[e] = (k < F) ? net.W1[k * H + n] : __float2bfloat16_rn(0.f);
    }
    for (int e = tid; e < 64 * SH; e += blockDim.x) {
        const int n = e / SH, k = e % SH;
        w2t[e] = (k < H) ? net.W2[k * H + n] : __float2bfloat16_rn(0.f);
    }
    for (int e = tid; e < 64; e += blockDim.x) { bias[e] = net.b1[e]; bias[64 + e] = net.b2[e]; }
    for (int e = tid; e < NPOP; e += blockDim.x) {
        cvec[e] = q.c[e];
        svec[e] = q.s[e];
        invw[e] = 1.f / q.w[e];
        wq[e] = q.w[e];
    }
    for (int e = tid; e <= N; e += blockDim.x) pr[e] = q.p0[e * K];
    // C[a][j] for a = 0..3: p, p^2, p^2 c, p^2 s
    auto Cm = [&](int a0, int j) {
        const float p = q.p0[j];
        return a0 == 0 ? p : a0 == 1 ? p * p : a0 == 2 ? p * p * q.c[j] : p * p * q.s[j];
    };
    // (W3 V^T)[k][a] = sum_j W3[k][j] C[a][j] w_j, and (V b3)[a]
    for (int e = tid; e < 64 * 4 + 4; e += blockDim.x) {
        float acc = 0.f;
        if (e < 256) {
            const int k = e >> 2, a0 = e & 3;
            for (int j = 0; j < NPOP; ++j) acc += __bfloat162float(net.W3[k * NPOP + j]) * Cm(a0, j) * q.w[j];
        } else {
            const int a0 = e - 256;
            for (int j = 0; j < NPOP; ++j) acc += net.b3[j] * Cm(a0, j) * q.w[j];
        }
        wv[e] = acc;
    }
    __syncthreads();
    // W3'[k][i] = W3[k][i] - sum_a (W3 V^T)[k][a] U[i][a], U = C^T A^-1; b3' likewise
    for (int e = tid; e < NPOP * SH; e += blockDim.x) {
        const int i = e / SH, k = e % SH;
        float u[4];
#pragma unroll
        for (int a0 = 0; a0 < 4; ++a0)
            u[a0] = Cm(0, i) * q.Ainv[0 * 4 + a0] + Cm(1, i) * q.Ainv[1 * 4 + a0] + Cm(2, i) * q.Ainv[2 * 4 + a0] +
                    Cm(3, i) * q.Ainv[3 * 4 + a0];
        if (k < H) {
            const float v = __bfloat162float(net.W3[k * NPOP + i]) -
                            (wv[k * 4] * u[0] + wv[k * 4 + 1] * u[1] + wv[k * 4 + 2] * u[2] + wv[k * 4 + 3] * u[3]);
            const __nv_bfloat16 hi = __float2bfloat16_rn(v);
            w3h[e] = hi;
            w3l[e] = __float2bfloat16_rn(v - __bfloat162float(hi));
        } else {
            w3h[e] = __float2bfloat16_rn(0.f);
            w3l[e] = __float2bfloat16_rn(0.f);
        }
        if (k == 0)
            bias[128 + i] = net.b3[i] - (wv[256] * u[0] + wv[257] * u[1] + wv[258] * u[2] + wv[259] * u[3]);
    }
    for (int e = lane; e < 16 * SX; e += 32) xa[e] = __float2bfloat16_rn(0.f);
    __syncthreads();

    const int g = lane >> 2, t = lane & 3;
    const int ls = lane & 15, half = lane >> 4;
    for (int k = 0; tile < ntile; ++k, tile += gridDim.x) {
        float *cur = ftile + (k & 1) * NPOP * LDF;
        const long long site0 = tile * TC_SITES;
        if (tile + gridDim.x < ntile)
            load_tile<VEC>(ftile + ((k + 1) & 1) * NPOP * LDF, f, S, (tile + gridDim.x) * TC_SITES, NPOP);
        else
            asm volatile("cp.async.commit_group;" ::: "memory");
        asm volatile("cp.async.wait_group 1;" ::: "memory");
        __syncthreads();
        // ---- features of the warp's 16 sites: this lane takes angles [half K/2, (half+1) K/2) of every shell
        const int col = wid * 16 + ls;
        const bool valid = site0 + col < S;
        // populations in pairs (i, i+1): the angular sums run on packed f32x2 operands
        float2 v[N + 1][KH / 2];
        float m[9];
#pragma unroll
        for (int a0 = 0; a0 < 9; ++a0) m[a0] = 0.f;
#pragma unroll
        for (int r = 0; r <= N; ++r) {
            float2 S0 = make_float2(0.f, 0.f), Sc = S0, Ss = S0, Scc = S0, Scs = S0, Sss = S0;
#pragma unroll
            for (int jj = 0; jj < KH; jj += 2) {
                const int i = r * K + half * KH + jj;
                const float2 x = make_float2(cur[i * LDF + col], cur[(i + 1) * LDF + col]);
                const float2 cp = *reinterpret_cast<const float2 *>(cvec + i);
                const float2 sp = *reinterpret_cast<const float2 *>(svec + i);
                v[r][jj / 2] = x;
                const float2 cx = __fmul2_rn(cp, x), sx = __fmul2_rn(sp, x);
                S0 = __fadd2_rn(S0, x); Sc = __fadd2_rn(Sc, cx); Ss = __fadd2_rn(Ss, sx);
                Scc = __ffma2_rn(cp, cx, Scc); Scs = __ffma2_rn(cp, sx, Scs); Sss = __ffma2_rn(sp, sx, Sss);
            }
            const float s0 = S0.x + S0.y, sc = Sc.x + Sc.y, ss = Ss.x + Ss.y;
            const float scc = Scc.x + Scc.y, scs = Scs.x + Scs.y, sss = Sss.x + Sss.y;
            const float p = pr[r], p2 = p * p;
            m[0] = fmaf(p, s0, m[0]); m[1] = fmaf(p, sc, m[1]); m[2] = fmaf(p, ss, m[2]);
            m[3] = fmaf(p2, s0, m[3]); m[4] = fmaf(p2, sc, m[4]); m[5] = fmaf(p2, ss, m[5]);
            m[6] = fmaf(p2, scc, m[6]); m[7] = fmaf(p2, scs, m[7]); m[8] = fmaf(p2, sss, m[8]);
        }
#pragma unroll
        for (int a0 = 0; a0 < 9; ++a0) m[a0] += __shfl_xor_sync(0xffffffffu, m[a0], 16);
        const float n0 = m[0], inv = valid ? __frcp_rn(n0) : 0.f;
        __nv_bfloat16 *xr = xa + ls * SX;
        if (half == 0) {
#pragma unroll
            for (int a0 = 0; a0 < 8; a0 += 2)
                *reinterpret_cast<unsigned *>(xr + a0) = pack_bf16(m[a0] * inv, m[a0 + 1] * inv);
            *reinterpret_cast<unsigned *>(xr + 8) = pack_bf16(m[8] * inv, kn);
        }
#pragma unroll
        for (int r = 0; r <= N; ++r)
#pragma unroll
            for (int jj = 0; jj < KH; jj += 2) {
                const int i = r * K + half * KH + jj;
                const float2 iw = *reinterpret_cast<const float2 *>(invw + i);
                const float2 sc2 = __fmul2_rn(__fmul2_rn(v[r][jj / 2], iw), make_float2(inv, inv));
                *reinterpret_cast<unsigned *>(xr + 10 + i) = pack_bf16(sc2.x, sc2.y);
            }
        // zero padding of layer 1's k range (the hidden tile of the previous tile overlaps it)
        constexpr int PADP = (16 * Gm::KS1 - F) / 2;
        for (int e = lane; e < 16 * PADP; e += 32)
            *reinterpret_cast<unsigned *>(xa + (e / PADP) * SX + F + 2 * (e % PADP)) = 0u;
        __syncwarp();
        // ---- layer 1: [16 x 16 KS1] x [16 KS1 x 64]; the hidden tile reuses the input rows
        float acc[Gm::NT3 > 8 ? Gm::NT3 : 8][4];
        bias_init(acc, bias, 8, lane);
        warp_gemm<Gm::KS1, 8>(xa, SX, w1t, SX, acc, lane);
        __syncwarp();
        gelu_rows(acc, xa, lane);
        __syncwarp();
        // ---- layer 2
        bias_init(acc, bias + 64, 8, lane);
        warp_gemm<4, 8>(xa, SH, w2t, SH, acc, lane);
        __syncwarp();
        gelu_rows(acc, xa, lane);
        __syncwarp();
        // ---- layer 3 with the folded projection (hi + lo)
        bias_init(acc, bias + 128, Gm::NT3, lane);
        warp_gemm<4, Gm::NT3>(xa, SH, w3h, SH, acc, lane);
        warp_gemm<4, Gm::NT3>(xa, SH, w3l, SH, acc, lane);
        // ---- update: f_i += n0 w_i y'_i; rows g (u = 0, 1) and g + 8 (u = 2, 3)
        const float na = __shfl_sync(0xffffffffu, n0, g), nb = __shfl_sync(0xffffffffu, n0, g + 8);
        float *fa = cur + wid * 16 + g;
#pragma unroll
        for (int nt = 0; nt < Gm::NT3; ++nt) {
            const int c = nt * 8 + 2 * t;
            const float2 w2 = *reinterpret_cast<const float2 *>(wq + c);
            fa[c * LDF] = fmaf(na * w2.x, acc[nt][0], fa[c * LDF]);
            fa[(c + 1) * LDF] = fmaf(na * w2.y, acc[nt][1], fa[(c + 1) * LDF]);
            fa[c * LDF + 8] = fmaf(nb * w2.x, acc[nt][2], fa[c * LDF + 8]);
            fa[(c + 1) * LDF + 8] = fmaf(nb * w2.y, acc[nt][3], fa[(c + 1) * LDF + 8]);
        }
        __syncthreads();
        store_tile<VEC>(cur, f, S, site0, NPOP);
        __syncthreads(); // the buffer is refilled by the next iteration's copy
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

using TcKernel = void (*)(Net, CoarseTab, float *, long long, float);

// the specialisations: (N, K) with N_pop a multiple of 8 and at most 80 outputs
template <int VEC>
TcKernel tc_kernel(int N, int K, size_t *smem)
{
    if (N == 2 && K == 24) { *smem = TcGeom<2, 24>::TOTAL; return apply_tc_kernel<2, 24, VEC>; }
    if (N == 2 && K == 16) { *smem = TcGeom<2, 16>::TOTAL; return apply_tc_kernel<2, 16, VEC>; }
    if (N == 3 && K == 16) { *smem = TcGeom<3, 16>::TOTAL; return apply_tc_kernel<3, 16, VEC>; }
    return nullptr;
}

// ---------------------------------------------------------------- tensor-core training
// One training pass (forward, loss, backward, weight gradients) on BF16
// tensor cores, specialised like the correction kernel.  A CTA of TR_WARPS
// warps takes tiles of TR_SITES columns of the feature matrix (persistent
// over the batch); warp w owns rows 16w..16w+15 of the tile.
//
// per warp:  x -> z1 = x W1 + b1 -> h1 = GELU -> z2 -> h2 -> y  (mma.sync, z in
//            registers); dY = 2 (y - t) / (count O); dz2 = (dY W3^T) GELU'(z2);
//            dz1 = (dz2 W2^T) GELU'(z1) (mma.sync; the accumulators of the
//            products share the fragment layout of z, so the derivative is
//            applied in registers).  The layer inputs x, h1, h2 and the deltas
//            dY, dz2, dz1 are rounded to BF16 as they enter a product.
// per CTA:   the weight gradients gW3 = h2^T dY, gW2 = h1^T dz2, gW1 = x^T dz1
//            are reductions over the tile's sites: their 16 x 8 blocks are
//            spread over the warps, fragments taken transposed (ldmatrix.trans)
//            from the row-major tile buffers, and accumulated in registers over
//            all of the CTA's tiles; bias gradients are column sums (FP32) in
//            shared memory.  Both go to the global gradient once per CTA.
constexpr int TR_WARPS = 8;
constexpr int TR_SITES = 16 * TR_WARPS;

__device__ __forceinline__ void ldsm_x4_t(const void *p, unsigned &r0, unsigned &r1, unsigned &r2, unsigned &r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(smem_addr(p)));
}

__device__ __forceinline__ void ldsm_x2_t(const void *p, unsigned &r0, unsigned &r1)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];"
                 : "=r"(r0), "=r"(r1)
                 : "r"(smem_addr(p)));
}

template <int N, int K>
struct TrGeom {
    static constexpr int NPOP = (N + 1) * K, F = 10 + NPOP, O = NPOP;
    static constexpr int KS1 = (F + 15) / 16, FP = 16 * KS1, SX = FP + 8;
    static constexpr int NT3 = O / 8, OP = 16 * ((O + 15) / 16), SO = OP + 8, KS3 = OP / 16;
    static constexpr int NB = 4 * NT3 + 32 + 8 * KS1;     // weight-gradient blocks
    static constexpr int NBW = (NB + TR_WARPS - 1) / TR_WARPS; // per warp
    static constexpr size_t W1T = 0, W2T = W1T + size_t(64) * SX * 2, W2N = W2T + size_t(64) * SH * 2,
                            W3T = W2N + size_t(64) * SH * 2, W3N = W3T + size_t(O) * SH * 2,
                            BIAS = W3N + size_t(64) * SO * 2, GB = BIAS + size_t(128 + OP) * 4,
                            XA = GB + size_t(128 + OP) * 4, H1 = XA + size_t(TR_SITES) * SX * 2,
                            H2 = H1 + size_t(TR_SITES) * SH * 2, DY = H2 + size_t(TR_SITES) * SH * 2,
                            D2 = DY + size_t(TR_SITES) * SO * 2, D1 = D2 + size_t(TR_SITES) * SH * 2,
                            TOTAL = D1 + size_t(TR_SITES) * SH * 2;
};

// rows g, g+8 of a 16 x 64 fragment set, as BF16, into a row-major tile (stride SH);
// FP32 column sums of the 16 rows added to colsum[]
__device__ __forceinline__ void store_rows_colsum(float (*acc)[4], __nv_bfloat16 *h, float *colsum, int lane)
{
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const int c = nt * 8 + t * 2;
        *reinterpret_cast<unsigned *>(h + g * SH + c) = pack_bf16(acc[nt][0], acc[nt][1]);
        *reinterpret_cast<unsigned *>(h + (g + 8) * SH + c) = pack_bf16(acc[nt][2], acc[nt][3]);
        float c0 = acc[nt][0] + acc[nt][2], c1 = acc[nt][1] + acc[nt][3];
#pragma unroll
        for (int o = 4; o < 32; o <<= 1) {
            c0 += __shfl_xor_sync(0xffffffffu, c0, o);
            c1 += __shfl_xor_sync(0xffffffffu, c1, o);
        }
        if (g == 0) {
            atomicAdd(&colsum[c], c0);
            atomicAdd(&colsum[c + 1], c1);
        }
    }
}

template <int N, int K>
__global__ void __launch_bounds__(TR_WARPS * 32, 1)
    train_tc_kernel(Net net, const float *__restrict__ X, const float *__restrict__ T, long long ld, long long off,
                    int count, float inv_count, float *__restrict__ grad, float *__restrict__ loss)
{
    using Gm = TrGeom<N, K>;
    constexpr int F = Gm::F, O = Gm::O, SX = Gm::SX, SO = Gm::SO, NT3 = Gm::NT3, OP = Gm::OP, FP = Gm::FP;
    static_assert(O % 8 == 0 && O <= 128, "output geometry");
    extern __shared__ __align__(16) unsigned char sm[];
    __nv_bfloat16 *w1t = reinterpret_cast<__nv_bfloat16 *>(sm + Gm::W1T); // [64][SX]  W1^T
    __nv_bfloat16 *w2t = reinterpret_cast<__nv_bfloat16 *>(sm + Gm::W2T); // [64][SH]  W2^T
    __nv_bfloat16 *w2n = reinterpret_cast<__nv_bfloat16 *>(sm + Gm::W2N); // [64][SH]  W2
    __nv_bfloat16 *w3t = reinterpret_cast<__nv_bfloat16 *>(sm + Gm::W3T); // [O][SH]   W3^T
    __nv_bfloat16 *w3n = reinterpret_cast<__nv_bfloat16 *>(sm + Gm::W3N); // [64][SO]  W3
    float *bias = reinterpret_cast<float *>(sm + Gm::BIAS);               // b1 | b2 | b3
    float *gbs = reinterpret_cast<float *>(sm + Gm::GB);                  // bias gradients
    __nv_bfloat16 *xa = reinterpret_cast<__nv_bfloat16 *>(sm + Gm::XA);   // [TR_SITES][SX]
    __nv_bfloat16 *h1b = reinterpret_cast<__nv_bfloat16 *>(sm + Gm::H1);  // [TR_SITES][SH]
    __nv_bfloat16 *h2b = reinterpret_cast<__nv_bfloat16 *>(sm + Gm::H2);
    __nv_bfloat16 *dyb = reinterpret_cast<__nv_bfloat16 *>(sm + Gm::DY);  // [TR_SITES][SO]
    __nv_bfloat16 *d2b = reinterpret_cast<__nv_bfloat16 *>(sm + Gm::D2);  // [TR_SITES][SH]
    __nv_bfloat16 *d1b = reinterpret_cast<__nv_bfloat16 *>(sm + Gm::D1);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
    for (int e = tid; e < 64 * SX; e += blockDim.x) {
        const int n = e / SX, k = e % SX;
        w1t[e] = (k < F) ? net.W1[k * H + n] : zero;
    }
    for (int e = tid; e < 64 * SH; e += blockDim.x) {
        const int n = e / SH, k = e % SH;
        w2t[e] = (k < H) ? net.W2[k * H + n] : zero;
        w2n[e] = (k < H) ? net.W2[n * H + k] : zero;
    }
    for (int e = tid; e < O * SH; e += blockDim.x) {
        const int n = e / SH, k = e % SH;
        w3t[e] = (k < H) ? net.W3[k * O + n] : zero;
    }
    for (int e = tid; e < 64 * SO; e += blockDim.x) {
        const int n = e / SO, k = e % SO;
        w3n[e] = (k < O) ? net.W3[n * O + k] : zero;
    }
    for (int e = tid; e < 128 + OP; e += blockDim.x) {
        bias[e] = e < 64 ? net.b1[e] : e < 128 ? net.b2[e - 64] : (e - 128 < O ? net.b3[e - 128] : 0.f);
        gbs[e] = 0.f;
    }
    for (int e = tid; e < TR_SITES * SO; e += blockDim.x) dyb[e] = zero; // columns O..SO-1 stay zero
    __syncthreads();

    float ga[Gm::NBW][4];
#pragma unroll
    for (int i = 0; i < Gm::NBW; ++i)
#pragma unroll
        for (int u = 0; u < 4; ++u) ga[i][u] = 0.f;
    float lsum = 0.f;
    const int g8 = lane >> 2, t4 = lane & 3, mi = lane >> 3, r8 = lane & 7;
    const long long ntile = (count + TR_SITES - 1) / TR_SITES;
    for (long long tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
        const long long s0 = tile * TR_SITES + wid * 16; // the warp's first column (relative to off)
        __nv_bfloat16 *xr = xa + wid * 16 * SX, *h1r = h1b + wid * 16 * SH, *h2r = h2b + wid * 16 * SH;
        __nv_bfloat16 *dyr = dyb + wid * 16 * SO, *d2r = d2b + wid * 16 * SH, *d1r = d1b + wid * 16 * SH;
        {   // input rows (BF16), zero beyond F and beyond the batch
            const int ls = lane & 15, half = lane >> 4;
            const long long sc = s0 + ls;
            const bool v = sc < count;
            for (int f = half; f < FP; f += 2)
                xr[ls * SX + f] = __float2bfloat16_rn(v && f < F ? X[(long long)f * ld + off + sc] : 0.f);
        }
        __syncwarp();
        float z1[8][4], z2[8][4], y[NT3][4];
        bias_init(z1, bias, 8, lane);
        warp_gemm<Gm::KS1, 8>(xr, SX, w1t, SX, z1, lane);
        gelu_rows(z1, h1r, lane);
        __syncwarp();
        bias_init(z2, bias + 64, 8, lane);
        warp_gemm<4, 8>(h1r, SH, w2t, SH, z2, lane);
        gelu_rows(z2, h2r, lane);
        __syncwarp();
        bias_init(y, bias + 128, NT3, lane);
        warp_gemm<4, NT3>(h2r, SH, w3t, SH, y, lane);
        // loss and dY = 2 (y - t) / (count O); rows g8 (u = 0, 1) and g8 + 8 (u = 2, 3)
        const long long sa = s0 + g8, sb = sa + 8;
        const bool va = sa < count, vb = sb < count;
#pragma unroll
        for (int nt = 0; nt < NT3; ++nt) {
            const int c = nt * 8 + 2 * t4;
            const float d0 = va ? y[nt][0] - T[(long long)c * ld + off + sa] : 0.f;
            const float d1 = va ? y[nt][1] - T[(long long)(c + 1) * ld + off + sa] : 0.f;
            const float d2 = vb ? y[nt][2] - T[(long long)c * ld + off + sb] : 0.f;
            const float d3 = vb ? y[nt][3] - T[(long long)(c + 1) * ld + off + sb] : 0.f;
            lsum += d0 * d0 + d1 * d1 + d2 * d2 + d3 * d3;
            const float q = 2.f * inv_count;
            y[nt][0] = q * d0; y[nt][1] = q * d1; y[nt][2] = q * d2; y[nt][3] = q * d3;
            *reinterpret_cast<unsigned *>(dyr + g8 * SO + c) = pack_bf16(y[nt][0], y[nt][1]);
            *reinterpret_cast<unsigned *>(dyr + (g8 + 8) * SO + c) = pack_bf16(y[nt][2], y[nt][3]);
            float c0 = y[nt][0] + y[nt][2], c1 = y[nt][1] + y[nt][3];
#pragma unroll
            for (int o = 4; o < 32; o <<= 1) {
                c0 += __shfl_xor_sync(0xffffffffu, c0, o);
                c1 += __shfl_xor_sync(0xffffffffu, c1, o);
            }
            if (g8 == 0) {
                atomicAdd(&gbs[128 + c], c0);
                atomicAdd(&gbs[128 + c + 1], c1);
            }
        }
        __syncwarp();
        // dz2 = (dY W3^T) GELU'(z2)
        float da[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int u = 0; u < 4; ++u) da[nt][u] = 0.f;
        warp_gemm<Gm::KS3, 8>(dyr, SO, w3n, SO, da, lane);
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int u = 0; u < 4; ++u) da[nt][u] *= gelu_grad(z2[nt][u]);
        store_rows_colsum(da, d2r, gbs + 64, lane);
        __syncwarp();
        // dz1 = (dz2 W2^T) GELU'(z1)
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int u = 0; u < 4; ++u) da[nt][u] = 0.f;
        warp_gemm<4, 8>(d2r, SH, w2n, SH, da, lane);
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int u = 0; u < 4; ++u) da[nt][u] *= gelu_grad(z1[nt][u]);
        store_rows_colsum(da, d1r, gbs, lane);
        __syncthreads();
        // weight-gradient blocks over the tile's TR_SITES sites
#pragma unroll
        for (int i = 0; i < Gm::NBW; ++i) {
            const int b = wid + TR_WARPS * i;
            if (b < Gm::NB) {
                const __nv_bfloat16 *As, *Bs;
                int sa_, sb_, m0, n0;
                if (b < 4 * NT3) {
                    As = h2b; sa_ = SH; Bs = dyb; sb_ = SO; m0 = (b / NT3) * 16; n0 = (b % NT3) * 8;
                } else if (b < 4 * NT3 + 32) {
                    const int bb = b - 4 * NT3;
                    As = h1b; sa_ = SH; Bs = d2b; sb_ = SH; m0 = (bb / 8) * 16; n0 = (bb % 8) * 8;
                } else {
                    const int bb = b - 4 * NT3 - 32;
                    As = xa; sa_ = SX; Bs = d1b; sb_ = SH; m0 = (bb / 8) * 16; n0 = (bb % 8) * 8;
                }
#pragma unroll
                for (int ks = 0; ks < TR_SITES / 16; ++ks) {
                    const int k0 = ks * 16;
                    unsigned a0, a1, a2, a3, b0, b1;
                    ldsm_x4_t(As + (k0 + (mi >> 1) * 8 + r8) * sa_ + m0 + (mi & 1) * 8, a0, a1, a2, a3);
                    ldsm_x2_t(Bs + (k0 + (mi & 1) * 8 + r8) * sb_ + n0, b0, b1);
                    mma_bf16(ga[i], a0, a1, a2, a3, b0, b1);
                }
            }
        }
        __syncthreads(); // the tile buffers are rewritten by the next tile
    }
    // the CTA's contributions to the global gradient (layout W1 [F][H] | b1 | W2 [H][H] | b2 | W3 [H][O] | b3)
    float *gW1 = grad, *gb1 = gW1 + F * H, *gW2 = gb1 + H, *gb2 = gW2 + H * H, *gW3 = gb2 + H, *gb3 = gW3 + H * O;
#pragma unroll
    for (int i = 0; i < Gm::NBW; ++i) {
        const int b = wid + TR_WARPS * i;
        if (b >= Gm::NB) continue;
        int m0, n0, which;
        if (b < 4 * NT3) { which = 3; m0 = (b / NT3) * 16; n0 = (b % NT3) * 8; }
        else if (b < 4 * NT3 + 32) { which = 2; m0 = ((b - 4 * NT3) / 8) * 16; n0 = ((b - 4 * NT3) % 8) * 8; }
        else { which = 1; m0 = ((b - 4 * NT3 - 32) / 8) * 16; n0 = ((b - 4 * NT3 - 32) % 8) * 8; }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int m = m0 + g8 + (u < 2 ? 0 : 8), n = n0 + 2 * t4 + (u & 1);
            if (which == 3) atomicAdd(&gW3[m * O + n], ga[i][u]);
            else if (which == 2) atomicAdd(&gW2[m * H + n], ga[i][u]);
            else if (m < F) atomicAdd(&gW1[m * H + n], ga[i][u]);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
    if (lane == 0) atomicAdd(loss, lsum);
    __syncthreads();
    for (int e = tid; e < 128 + O; e += blockDim.x) {
        if (e < 64) atomicAdd(&gb1[e], gbs[e]);
        else if (e < 128) atomicAdd(&gb2[e - 64], gbs[e]);
        else atomicAdd(&gb3[e - 128], gbs[e]);
    }
}

using TrKernel = void (*)(Net, const float *, const float *, long long, long long, int, float, float *, float *);

TrKernel tr_kernel(int N, int K, size_t *smem)
{
    if (N == 2 && K == 24) { *smem = TrGeom<2, 24>::TOTAL; return train_tc_kernel<2, 24>; }
    if (N == 2 && K == 16) { *smem = TrGeom<2, 16>::TOTAL; return train_tc_kernel<2, 16>; }
    if (N == 3 && K == 16) { *smem = TrGeom<3, 16>::TOTAL; return train_tc_kernel<3, 16>; }
    return nullptr;
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
    bool simt_apply = false;
    bool simt_train = false;
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

bool tc_attributes(const rlbm_closure *c)
{
    size_t trsmem = 0;
    TrKernel tk = tr_kernel(c->N, c->K, &trsmem);
    if (tk && cudaFuncSetAttribute(tk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)trsmem) != cudaSuccess)
        return false;
    for (int v = 0; v < 2; ++v) {
        size_t smem = 0;
        TcKernel k = v ? tc_kernel<4>(c->N, c->K, &smem) : tc_kernel<1>(c->N, c->K, &smem);
        if (k && cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
            return false;
    }
    return true;
}

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
        cudaFuncSetAttribute(mlp_backward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bwd_smem(c)) != cudaSuccess ||
        !tc_attributes(c))
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
    size_t trsmem = 0;
    TrKernel tk = c->simt_train ? nullptr : tr_kernel(c->N, c->K, &trsmem);
    if (tk) {
        // tensor-core path: forward, backward and weight gradients in one persistent kernel
        int dev = 0, sms = 0;
        CL_CUDA(c, cudaGetDevice(&dev));
        CL_CUDA(c, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const long long tiles = (count + TR_SITES - 1) / TR_SITES;
        const int grid = int(std::min<long long>(sms, tiles));
        tk<<<grid, TR_WARPS * 32, trsmem, c->stream>>>(net_of(c), d_x, d_t, ld, off, count,
                                                      1.0f / (float(count) * float(c->O)), c->d_g, c->d_loss);
        CL_CUDA(c, cudaGetLastError());
        if (loss) {
            float l = 0.f;
            CL_CUDA(c, cudaMemcpyAsync(&l, c->d_loss, 4, cudaMemcpyDeviceToHost, c->stream));
            CL_CUDA(c, cudaStreamSynchronize(c->stream));
            *loss = l / (float(count) * float(c->O));
        }
        return RLBM_OK;
    }
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
    size_t smem = 0;
    const bool vec = sites % 4 == 0 && reinterpret_cast<uintptr_t>(d_f) % 16 == 0;
    TcKernel k = c->simt_apply ? nullptr : vec ? tc_kernel<4>(c->N, c->K, &smem) : tc_kernel<1>(c->N, c->K, &smem);
    if (k) {
        // tensor-core path: a persistent grid of one CTA per SM
        int dev = 0, sms = 0;
        CL_CUDA(c, cudaGetDevice(&dev));
        CL_CUDA(c, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        const long long tiles = (sites + TC_SITES - 1) / TC_SITES;
        const int grid = int(std::min<long long>(sms, tiles));
        k<<<grid, TC_WARPS * 32, smem, c->stream>>>(net_of(c), tab_of(c), d_f, sites, float(kn));
        CL_CUDA(c, cudaGetLastError());
        return RLBM_OK;
    }
    const int grid = int(std::min<long long>(4096, (sites + 127) / 128));
    apply_kernel<<<grid, 128, fwd_smem(c, true), c->stream>>>(net_of(c), tab_of(c), d_f, sites, float(kn));
    CL_CUDA(c, cudaGetLastError());
    return RLBM_OK;
}

rlbm_status rlbm_closure_set_train_path(rlbm_closure_t *c, int tensor_cores)
{
    if (!c) return cfail(nullptr, RLBM_ERR_ARG, "NULL closure");
    c->simt_train = !tensor_cores;
    return RLBM_OK;
}

rlbm_status rlbm_closure_set_apply_path(rlbm_closure_t *c, int tensor_cores)
{
    if (!c) return cfail(nullptr, RLBM_ERR_ARG, "NULL closure");
    c->simt_apply = !tensor_cores;
    return RLBM_OK;
}

} // extern "C"
