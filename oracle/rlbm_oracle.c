/*
 * FP64 CPU oracle for the relativistic lattice Boltzmann method of
 * Bazzanini, Gabbana, Simeoni, Succi, Tripiccione (arXiv 2011.06856):
 * a massless gas in (2+1) dimensions, off-lattice product quadrature with
 * shell-rotated angles, bilinear pull streaming, Anderson-Witting collision.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA library is checked against.  Only the test suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * table or constant with the CUDA library, and the library never calls it.
 *
 * Every routine follows one passage of the paper, in the paper's order:
 *   quadrature        Sec. 2.3, Eq. (off-lattice-quad) and the Laguerre rule above it;
 *                     the on-lattice rule of Sec. 2.3 (Eq. mj-orthogonal-conditions,
 *                     stencil vectors of length 5, Fig. 1 left)
 *   equilibrium       Sec. 2.2, Eqs. (mj-feq-expansion), (mj-projection-coefficients),
 *                     (mj-feq-expansion-truncated); the MJ distribution Eq. (feq_dist)
 *   streaming         Sec. 2.2, Eqs. (streaming), (interpolation); on-lattice: the
 *                     exact shift by the stencil vector (Sec. 2.3, perfect streaming)
 *   moments           Sec. 2.2, Eq. (discrete_sum_moments)
 *   Landau frame      Sec. 2.2, the eigenproblem eps U^a = T^{ab} U_b and eps = 2P = 2nT
 *   collision         Sec. 2.2, Eq. (discrete-rbe) (relaxation toward f^eq)
 *
 * Readings where the paper is silent or garbled (each one pinned by a test):
 *   - lattice units dx = dy = dt = 1, c = 1;
 *   - the weighting function is omega(p0) = exp(-p0) (rest-frame MJ at T0 = 1);
 *   - the truncated expansion is the omega-orthogonal projection onto all
 *     polynomials of degree <= N in p^mu restricted to the light cone, built
 *     here from the cone monomials p0^e px^a py^b (e in {0,1}, e+a+b <= N);
 *   - Eq. (interpolation) lacks its "+" signs: the four terms are summed;
 *   - Eq. (collision) prints +omega (f* - f^eq), which anti-relaxes; the
 *     relaxing sign of Eq. (discrete-rbe) and Eq. (boltz_eq) is used;
 *   - boundary conditions: periodic (wrap) or copy-out (clamp the source
 *     index into the grid, i.e. a zero-gradient ghost cell);
 *   - sgn(0) = +1 (the weight of that neighbour is zero either way).
 *
 * Population order is shell-major: i = r*K + j for radial node r, angle j.
 * Population arrays are f[i][y][x] (x fastest).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846264338327950288

/* ------------------------------------------------------------------ */
/* Laguerre polynomials and the Gauss-Laguerre radial rule (Sec. 2.3)   */
/* ------------------------------------------------------------------ */

/* L_n(x) by the three-term recurrence (k+1) L_{k+1} = (2k+1-x) L_k - k L_{k-1}. */
double orc_laguerre(int n, double x)
{
    double lm1 = 1.0, l = 1.0 - x;
    if (n == 0) return 1.0;
    for (int k = 1; k < n; ++k) {
        double lp1 = ((2.0 * k + 1.0 - x) * l - k * lm1) / (k + 1.0);
        lm1 = l;
        l = lp1;
    }
    return l;
}

/* Roots of L_n: scan (0, 4n+4) for sign changes (all roots lie below
 * 4n+2), bisect each bracket until it stops shrinking. */
static int laguerre_roots(int n, double *roots)
{
    const int nscan = 200000;
    const double xmax = 4.0 * n + 4.0;
    int found = 0;
    double xa = 1e-12, fa = orc_laguerre(n, xa);
    for (int s = 1; s <= nscan && found < n; ++s) {
        double xb = xmax * (double)s / nscan;
        double fb = orc_laguerre(n, xb);
        if (fa == 0.0) {
            roots[found++] = xa;
        } else if ((fa < 0.0) != (fb < 0.0)) {
            double lo = xa, hi = xb, flo = fa;
            for (int it = 0; it < 200; ++it) {
                double mid = 0.5 * (lo + hi);
                if (mid <= lo || mid >= hi) break;
                double fm = orc_laguerre(n, mid);
                if (fm == 0.0) { lo = hi = mid; break; }
                if ((fm < 0.0) == (flo < 0.0)) { lo = mid; flo = fm; } else { hi = mid; }
            }
            roots[found++] = 0.5 * (lo + hi);
        }
        xa = xb;
        fa = fb;
    }
    return found;
}

/* Radial nodes p_r = roots of L_{N+1} and weights
 * w^(p)_r = p_r / ((N+2)^2 [L_{N+2}(p_r)]^2)   (Sec. 2.3, Eq. off-lattice-quad).
 * Returns the number of roots found (N+1 on success). */
int orc_radial_rule(int N, double *p, double *wp)
{
    int got = laguerre_roots(N + 1, p);
    for (int r = 0; r < got; ++r) {
        double l = orc_laguerre(N + 2, p[r]);
        wp[r] = p[r] / ((N + 2.0) * (N + 2.0) * l * l);
    }
    return got;
}

/* ------------------------------------------------------------------ */
/* Quadrature context: nodes, weights, projection (Secs. 2.2, 2.3)      */
/* ------------------------------------------------------------------ */

typedef struct {
    int N, K, npop, nb;
    double *p0, *vx, *vy, *w; /* per population, shell-major */
    int *be, *ba, *bb;        /* cone monomial p0^e px^a py^b, one per basis function */
    double *Ginv;             /* nb x nb inverse of the continuous Gram matrix */
    double *Bw;               /* npop x nb: w_i * B_m(p_i) */
    int onlat;                /* on-lattice rule: streaming shifts by (sx, sy) */
    int *sx, *sy;             /* per population, integer stencil vector (on-lattice only) */
} orc_quad;

/* Angular integral of cos^a sin^b over [0, 2pi]: zero unless a and b are
 * even, else 2 pi (a-1)!! (b-1)!! / (a+b)!!. */
double orc_angular_integral(int a, int b)
{
    if ((a & 1) || (b & 1)) return 0.0;
    double num = 1.0, den = 1.0;
    for (int k = a - 1; k > 0; k -= 2) num *= k;
    for (int k = b - 1; k > 0; k -= 2) num *= k;
    for (int k = a + b; k > 0; k -= 2) den *= k;
    return 2.0 * ORC_PI * num / den;
}

static double factorial(int k)
{
    double r = 1.0;
    for (int i = 2; i <= k; ++i) r *= i;
    return r;
}

/* Gauss-Jordan inverse with partial pivoting; returns 0 on success. */
static int invert(int n, const double *A, double *Ainv)
{
    double *M = malloc(sizeof(double) * n * 2 * n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < 2 * n; ++j)
            M[i * 2 * n + j] = j < n ? A[i * n + j] : (j - n == i ? 1.0 : 0.0);
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int i = c + 1; i < n; ++i)
            if (fabs(M[i * 2 * n + c]) > fabs(M[piv * 2 * n + c])) piv = i;
        if (M[piv * 2 * n + c] == 0.0) { free(M); return 1; }
        if (piv != c)
            for (int j = 0; j < 2 * n; ++j) {
                double t = M[c * 2 * n + j];
                M[c * 2 * n + j] = M[piv * 2 * n + j];
                M[piv * 2 * n + j] = t;
            }
        double d = M[c * 2 * n + c];
        for (int j = 0; j < 2 * n; ++j) M[c * 2 * n + j] /= d;
        for (int i = 0; i < n; ++i) {
            if (i == c) continue;
            double f = M[i * 2 * n + c];
            if (f == 0.0) continue;
            for (int j = 0; j < 2 * n; ++j) M[i * 2 * n + j] -= f * M[c * 2 * n + j];
        }
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) Ainv[i * n + j] = M[i * 2 * n + n + j];
    free(M);
    return 0;
}

static double ipow(double x, int e)
{
    double r = 1.0;
    for (int i = 0; i < e; ++i) r *= x;
    return r;
}

void orc_destroy(orc_quad *q)
{
    if (!q) return;
    free(q->p0); free(q->vx); free(q->vy); free(q->w);
    free(q->be); free(q->ba); free(q->bb);
    free(q->Ginv); free(q->Bw);
    free(q->sx); free(q->sy);
    free(q);
}

/* Projection data of the truncated equilibrium (Eqs. mj-projection-coefficients,
 * mj-feq-expansion-truncated) for the nodes and weights already in q: the cone
 * monomial basis, the inverse of its continuous Gram matrix, and w_i B_m(p_i).
 * Returns 0 on success. */
static int build_projection(orc_quad *q)
{
    const int N = q->N;
    /* cone monomials of degree k <= N: e in {0,1}, a + b = k - e */
    q->be = malloc(sizeof(int) * q->nb);
    q->ba = malloc(sizeof(int) * q->nb);
    q->bb = malloc(sizeof(int) * q->nb);
    int m = 0;
    for (int k = 0; k <= N; ++k)
        for (int e = 0; e <= 1 && e <= k; ++e)
            for (int a = k - e; a >= 0; --a) {
                q->be[m] = e;
                q->ba[m] = a;
                q->bb[m] = k - e - a;
                ++m;
            }

    /* continuous Gram matrix G_mn = int exp(-p) B_m B_n d^2p/p0
     *   = (k_m + k_n)! * int cos^(a_m+a_n) sin^(b_m+b_n) dtheta   (d^2p/p0 = dp dtheta) */
    double *G = malloc(sizeof(double) * q->nb * q->nb);
    for (int i = 0; i < q->nb; ++i)
        for (int j = 0; j < q->nb; ++j) {
            int km = q->be[i] + q->ba[i] + q->bb[i];
            int kn = q->be[j] + q->ba[j] + q->bb[j];
            G[i * q->nb + j] = factorial(km + kn) *
                               orc_angular_integral(q->ba[i] + q->ba[j], q->bb[i] + q->bb[j]);
        }
    q->Ginv = malloc(sizeof(double) * q->nb * q->nb);
    int bad = invert(q->nb, G, q->Ginv);
    free(G);
    if (bad) return 1;

    q->Bw = malloc(sizeof(double) * q->npop * q->nb);
    for (int i = 0; i < q->npop; ++i) {
        double p = q->p0[i], px = p * q->vx[i], py = p * q->vy[i];
        for (int b = 0; b < q->nb; ++b)
            q->Bw[i * q->nb + b] = q->w[i] * ipow(p, q->be[b]) * ipow(px, q->ba[b]) * ipow(py, q->bb[b]);
    }
    return 0;
}

/* Build the quadrature of Eq. (off-lattice-quad):
 *   p_ij = p_i (1, cos theta_ij, sin theta_ij),
 *   theta_ij = (j + i/(N+1)) 2 pi / K,   w_ij = w^(p)_i 2 pi / K,
 * for 0 <= i <= N, 0 <= j < K, and the projection data of the truncated
 * equilibrium.  Requires N >= 0 and K >= 2N+1.  Returns NULL on bad input. */
orc_quad *orc_create(int N, int K)
{
    if (N < 0 || N > 12 || K < 2 * N + 1) return NULL;
    orc_quad *q = calloc(1, sizeof(orc_quad));
    q->N = N;
    q->K = K;
    q->npop = K * (N + 1);
    q->nb = (N + 1) * (N + 1);
    q->p0 = malloc(sizeof(double) * q->npop);
    q->vx = malloc(sizeof(double) * q->npop);
    q->vy = malloc(sizeof(double) * q->npop);
    q->w = malloc(sizeof(double) * q->npop);

    double pr[16], wpr[16];
    if (orc_radial_rule(N, pr, wpr) != N + 1) { orc_destroy(q); return NULL; }
    for (int r = 0; r <= N; ++r) {
        for (int j = 0; j < K; ++j) {
            int i = r * K + j;
            double theta = (j + r / (double)(N + 1)) * (2.0 * ORC_PI / K);
            double c = cos(theta), s = sin(theta);
            if (fabs(c) < 1e-15) c = 0.0;
            if (fabs(s) < 1e-15) s = 0.0;
            q->p0[i] = pr[r];
            q->vx[i] = c;
            q->vy[i] = s;
            q->w[i] = wpr[r] * (2.0 * ORC_PI / K);
        }
    }

    if (build_projection(q)) { orc_destroy(q); return NULL; }
    return q;
}

/* On-lattice rule of Sec. 2.3 (Fig. 1, left): the stencil vectors n_i are the
 * integer vectors of length R = 5, (+-5, 0), (0, +-5), (+-3, +-4), (+-4, +-3),
 * the same 12 on every energy shell; the shells are the roots of the radial
 * polynomial of degree N+1 (the Gauss-Laguerre nodes, N = 3); momenta
 * p_i = p_r (1, n_i / |n_i|).  Weights from the orthonormal conditions
 * (Eq. mj-orthogonal-conditions), which for a product rule are the radial
 * Gauss-Laguerre conditions (exact to degree 2N+1) times the angular ones
 * sum_i v_i cos^a sin^b = int cos^a sin^b dtheta for a + b <= 2N.  The angular
 * weights are taken constant on the two symmetry classes of the stencil (on
 * the axes, off the axes) and solved by least squares over all those
 * conditions; the rule is rejected (NULL) unless every condition holds to
 * 1e-12 and both weights are positive.  Populations are shell-major,
 * i = r*12 + j, the vectors ordered by angle from 0.  Only N = 3 (a fourth-order
 * rule needs vectors of length 5 sqrt(13), Sec. 2.3). */
orc_quad *orc_create_onlattice(int N)
{
    if (N != 3) return NULL;
    const int R2 = 25, K = 12;
    int vec[12][2], nv = 0;
    for (int a = -5; a <= 5; ++a)
        for (int b = -5; b <= 5; ++b)
            if (a * a + b * b == R2 && nv < 12) { vec[nv][0] = a; vec[nv][1] = b; ++nv; }
    if (nv != K) return NULL;
    /* order by angle in [0, 2 pi) (insertion sort) */
    for (int i = 1; i < nv; ++i)
        for (int j = i; j > 0; --j) {
            double t0 = atan2(vec[j - 1][1], vec[j - 1][0]), t1 = atan2(vec[j][1], vec[j][0]);
            if (t0 < 0) t0 += 2.0 * ORC_PI;
            if (t1 < 0) t1 += 2.0 * ORC_PI;
            if (t1 < t0) {
                int ta = vec[j][0], tb = vec[j][1];
                vec[j][0] = vec[j - 1][0]; vec[j][1] = vec[j - 1][1];
                vec[j - 1][0] = ta; vec[j - 1][1] = tb;
            }
        }
    /* angular weights: class 0 on the axes, class 1 off the axes */
    int cls[12];
    double c[12], sn[12];
    for (int j = 0; j < K; ++j) {
        cls[j] = (vec[j][0] == 0 || vec[j][1] == 0) ? 0 : 1;
        c[j] = vec[j][0] / 5.0;
        sn[j] = vec[j][1] / 5.0;
    }
    double A[4] = {0, 0, 0, 0}, rhs[2] = {0, 0};
    double Mrow[64][2], brow[64];
    int nc = 0;
    for (int a = 0; a <= 2 * N; ++a)
        for (int b = 0; a + b <= 2 * N; ++b) {
            Mrow[nc][0] = Mrow[nc][1] = 0.0;
            for (int j = 0; j < K; ++j) Mrow[nc][cls[j]] += ipow(c[j], a) * ipow(sn[j], b);
            brow[nc] = orc_angular_integral(a, b);
            ++nc;
        }
    for (int k = 0; k < nc; ++k)
        for (int u = 0; u < 2; ++u) {
            rhs[u] += Mrow[k][u] * brow[k];
            for (int v = 0; v < 2; ++v) A[u * 2 + v] += Mrow[k][u] * Mrow[k][v];
        }
    double Ai[4];
    if (invert(2, A, Ai)) return NULL;
    double vw[2] = {Ai[0] * rhs[0] + Ai[1] * rhs[1], Ai[2] * rhs[0] + Ai[3] * rhs[1]};
    for (int k = 0; k < nc; ++k)
        if (fabs(Mrow[k][0] * vw[0] + Mrow[k][1] * vw[1] - brow[k]) > 1e-12) return NULL;
    if (!(vw[0] > 0.0) || !(vw[1] > 0.0)) return NULL;

    orc_quad *q = calloc(1, sizeof(orc_quad));
    q->N = N;
    q->K = K;
    q->npop = K * (N + 1);
    q->nb = (N + 1) * (N + 1);
    q->onlat = 1;
    q->p0 = malloc(sizeof(double) * q->npop);
    q->vx = malloc(sizeof(double) * q->npop);
    q->vy = malloc(sizeof(double) * q->npop);
    q->w = malloc(sizeof(double) * q->npop);
    q->sx = malloc(sizeof(int) * q->npop);
    q->sy = malloc(sizeof(int) * q->npop);
    double pr[16], wpr[16];
    if (orc_radial_rule(N, pr, wpr) != N + 1) { orc_destroy(q); return NULL; }
    for (int r = 0; r <= N; ++r)
        for (int j = 0; j < K; ++j) {
            int i = r * K + j;
            q->p0[i] = pr[r];
            q->vx[i] = c[j];
            q->vy[i] = sn[j];
            q->w[i] = wpr[r] * vw[cls[j]];
            q->sx[i] = vec[j][0];
            q->sy[i] = vec[j][1];
        }
    if (build_projection(q)) { orc_destroy(q); return NULL; }
    return q;
}

/* Integer stencil vectors of an on-lattice rule (0 for an off-lattice one). */
int orc_shifts(const orc_quad *q, int *sx, int *sy)
{
    if (!q->onlat) return 0;
    memcpy(sx, q->sx, sizeof(int) * q->npop);
    memcpy(sy, q->sy, sizeof(int) * q->npop);
    return 1;
}

int orc_npop(const orc_quad *q) { return q->npop; }
int orc_nbasis(const orc_quad *q) { return q->nb; }

void orc_tables(const orc_quad *q, double *p0, double *vx, double *vy, double *w)
{
    memcpy(p0, q->p0, sizeof(double) * q->npop);
    memcpy(vx, q->vx, sizeof(double) * q->npop);
    memcpy(vy, q->vy, sizeof(double) * q->npop);
    memcpy(w, q->w, sizeof(double) * q->npop);
}

void orc_basis(const orc_quad *q, int *e, int *a, int *b)
{
    memcpy(e, q->be, sizeof(int) * q->nb);
    memcpy(a, q->ba, sizeof(int) * q->nb);
    memcpy(b, q->bb, sizeof(int) * q->nb);
}

/* ------------------------------------------------------------------ */
/* Maxwell-Juttner moments (Sec. 2.1, Eqs. feq_dist, moments)           */
/* ------------------------------------------------------------------ */

/* One component of the rank-k moment tensor of the MJ distribution
 *   f^MJ = n / (2 pi T^2) exp(-U_a p^a / T)
 * (normalised so that N^a = n U^a and eps = 2 n T, the ideal-gas EOS of
 * Sec. 2.2).  idx[0..k-1] in {0,1,2} = (t, x, y).  In the rest frame,
 *   M_rest^{a1..ak} = n k! T^(k-1) / (2 pi) int n^a1 ... n^ak dtheta,
 * n = (1, cos, sin); the lab tensor is the boost of it by U:
 *   L^0_0 = U^0, L^0_j = L^j_0 = U^j, L^i_j = delta_ij + U^i U^j / (1 + U^0). */
double orc_mj_moment(int k, const int *idx, double n, double T, double Ux, double Uy)
{
    double U0 = sqrt(1.0 + Ux * Ux + Uy * Uy);
    double U[3] = {U0, Ux, Uy};
    double L[3][3];
    L[0][0] = U0;
    for (int j = 1; j < 3; ++j) { L[0][j] = U[j]; L[j][0] = U[j]; }
    for (int i = 1; i < 3; ++i)
        for (int j = 1; j < 3; ++j) L[i][j] = (i == j ? 1.0 : 0.0) + U[i] * U[j] / (1.0 + U0);

    /* sum over rest-frame index choices alpha_1..alpha_k, 3^k terms */
    long nterms = 1;
    for (int j = 0; j < k; ++j) nterms *= 3;
    double sum = 0.0;
    for (long t = 0; t < nterms; ++t) {
        long code = t;
        double coef = 1.0;
        int na = 0, nb = 0;
        for (int j = 0; j < k; ++j) {
            int alpha = (int)(code % 3);
            code /= 3;
            coef *= L[idx[j]][alpha];
            if (alpha == 1) ++na;
            if (alpha == 2) ++nb;
        }
        if (coef != 0.0) sum += coef * orc_angular_integral(na, nb);
    }
    return n * factorial(k) * pow(T, k - 1) / (2.0 * ORC_PI) * sum;
}

/* Truncated discrete equilibrium, Eq. (mj-feq-expansion-truncated):
 *   f^eq_i = w_i sum_{k<=N} a^(k) J^(k)(p_i) = w_i [Pi_N (f^MJ / omega)](p_i)
 *          = w_i B(p_i)^T G^{-1} M,   M_m = int f^MJ B_m d^2p/p0 (Eq. mj-projection-coefficients).
 * (Ux, Uy) are the spatial components of U^a; U^0 = sqrt(1 + |U|^2). */
void orc_feq(const orc_quad *q, double n, double T, double Ux, double Uy, double *feq)
{
    double M[169], x[169];
    int idx[32];
    for (int b = 0; b < q->nb; ++b) {
        int k = 0;
        for (int t = 0; t < q->be[b]; ++t) idx[k++] = 0;
        for (int t = 0; t < q->ba[b]; ++t) idx[k++] = 1;
        for (int t = 0; t < q->bb[b]; ++t) idx[k++] = 2;
        M[b] = orc_mj_moment(k, idx, n, T, Ux, Uy);
    }
    for (int a = 0; a < q->nb; ++a) {
        double s = 0.0;
        for (int b = 0; b < q->nb; ++b) s += q->Ginv[a * q->nb + b] * M[b];
        x[a] = s;
    }
    for (int i = 0; i < q->npop; ++i) {
        double s = 0.0;
        for (int b = 0; b < q->nb; ++b) s += q->Bw[i * q->nb + b] * x[b];
        feq[i] = s;
    }
}

/* ------------------------------------------------------------------ */
/* Discrete moments (Eq. discrete_sum_moments) and the Landau frame      */
/* ------------------------------------------------------------------ */

/* Neumaier-compensated accumulator */
typedef struct { double s, c; } nsum;
static void nadd(nsum *a, double v)
{
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
    else a->c += (v - t) + a->s;
    a->s = t;
}

/* mom[0..2] = N^t, N^x, N^y;  mom[3..8] = T^tt, T^tx, T^ty, T^xx, T^xy, T^yy.
 * f is read with stride `stride` between populations. */
void orc_moments(const orc_quad *q, const double *f, long stride, double *mom)
{
    nsum acc[9];
    memset(acc, 0, sizeof(acc));
    for (int i = 0; i < q->npop; ++i) {
        double fi = f[(long)i * stride];
        double pt = q->p0[i], px = q->p0[i] * q->vx[i], py = q->p0[i] * q->vy[i];
        nadd(&acc[0], pt * fi);
        nadd(&acc[1], px * fi);
        nadd(&acc[2], py * fi);
        nadd(&acc[3], pt * pt * fi);
        nadd(&acc[4], pt * px * fi);
        nadd(&acc[5], pt * py * fi);
        nadd(&acc[6], px * px * fi);
        nadd(&acc[7], px * py * fi);
        nadd(&acc[8], py * py * fi);
    }
    for (int k = 0; k < 9; ++k) mom[k] = acc[k].s + acc[k].c;
}

/* Landau frame: eps U^a = T^{ab} U_b (Sec. 2.2).  With A = T eta
 * (A^a_b = T^{ac} eta_cb, eta = diag(+,-,-)), eps is the largest real
 * eigenvalue of A and U its eigenvector, normalised to U^a U_a = 1, U^0 > 0.
 * Then n = U_a N^a and T = eps / (2n) from eps = 2P = 2nT.
 * out = (n, eps, T, U^0, U^x, U^y).  Returns 0, or 1 when the state has no
 * timelike eigenvector or a non-positive n or eps (out then holds a rest
 * state with the same N^0 so that a caller can continue). */
int orc_landau(const double *mom, double *out)
{
    const double Nt = mom[0], Nx = mom[1], Ny = mom[2];
    const double Ttt = mom[3], Ttx = mom[4], Tty = mom[5];
    const double Txx = mom[6], Txy = mom[7], Tyy = mom[8];
    double A[3][3] = {{Ttt, -Ttx, -Tty}, {Ttx, -Txx, -Txy}, {Tty, -Txy, -Tyy}};

    /* characteristic polynomial lambda^3 - c2 lambda^2 + c1 lambda - c0 */
    double c2 = A[0][0] + A[1][1] + A[2][2];
    double c1 = A[0][0] * A[1][1] - A[0][1] * A[1][0] + A[0][0] * A[2][2] - A[0][2] * A[2][0] +
                A[1][1] * A[2][2] - A[1][2] * A[2][1];
    double c0 = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
                A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
                A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
    /* depressed cubic t^3 + p t + q, lambda = t + c2/3; largest root by Viete */
    double p = c1 - c2 * c2 / 3.0;
    double qq = -2.0 * c2 * c2 * c2 / 27.0 + c1 * c2 / 3.0 - c0;
    double lam;
    int status = 0;
    if (p < 0.0) {
        double r = sqrt(-p / 3.0);
        double arg = (3.0 * qq / (2.0 * p)) * sqrt(-3.0 / p);
        if (arg > 1.0) arg = 1.0;
        if (arg < -1.0) arg = -1.0;
        lam = 2.0 * r * cos(acos(arg) / 3.0) + c2 / 3.0;
    } else {
        status = 1; /* no three real roots: not a physical T^{ab} */
        lam = c2 / 3.0 + cbrt(-qq);
    }
    for (int it = 0; it < 2; ++it) {
        double P = ((lam - c2) * lam + c1) * lam - c0;
        double dP = (3.0 * lam - 2.0 * c2) * lam + c1;
        if (dP != 0.0) lam -= P / dP;
    }
    const double eps = lam;

    /* eigenvector: orthogonal to every row of A - eps I; largest cross product */
    double R[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) R[i][j] = A[i][j] - (i == j ? eps : 0.0);
    double best[3] = {0, 0, 0}, bestn = -1.0;
    for (int a = 0; a < 3; ++a) {
        int b = (a + 1) % 3;
        double cx = R[a][1] * R[b][2] - R[a][2] * R[b][1];
        double cy = R[a][2] * R[b][0] - R[a][0] * R[b][2];
        double cz = R[a][0] * R[b][1] - R[a][1] * R[b][0];
        double nn = cx * cx + cy * cy + cz * cz;
        if (nn > bestn) { bestn = nn; best[0] = cx; best[1] = cy; best[2] = cz; }
    }
    double mink = best[0] * best[0] - best[1] * best[1] - best[2] * best[2];
    double U0, Ux, Uy;
    if (mink > 0.0 && bestn > 0.0) {
        double s = 1.0 / sqrt(mink);
        if (best[0] < 0.0) s = -s;
        U0 = best[0] * s;
        Ux = best[1] * s;
        Uy = best[2] * s;
    } else {
        status = 1;
        U0 = 1.0; Ux = 0.0; Uy = 0.0;
    }
    double n = U0 * Nt - Ux * Nx - Uy * Ny;
    if (!(n > 0.0) || !(eps > 0.0)) {
        status = 1;
        if (!(n > 0.0)) n = Nt > 0.0 ? Nt : 1e-300;
    }
    out[0] = n;
    out[1] = eps;
    out[2] = eps / (2.0 * n);
    out[3] = U0;
    out[4] = Ux;
    out[5] = Uy;
    return status;
}

/* ------------------------------------------------------------------ */
/* One time step: stream, moments, Landau, equilibrium, collide          */
/* ------------------------------------------------------------------ */

enum { ORC_BC_PERIODIC = 0, ORC_BC_COPYOUT = 1 };

static int src_index(int i, int L, int bc)
{
    if (bc == ORC_BC_PERIODIC) return ((i % L) + L) % L;
    return i < 0 ? 0 : (i >= L ? L - 1 : i);
}

/* Streaming, Eqs. (streaming) and (interpolation), dt = dx = dy = 1:
 *   f*_i(x) = (1-ax)(1-ay) f_i(x) + ax(1-ay) f_i(x - rx) + (1-ax) ay f_i(x - ry)
 *           + ax ay f_i(x - rx - ry),
 *   ax = |v_x|, ay = |v_y|, rx = sgn(v_x) e_x, ry = sgn(v_y) e_y, sgn(0) = +1. */
void orc_stream(const orc_quad *q, int nx, int ny, int bcx, int bcy, const double *f, double *fs)
{
    long S = (long)nx * ny;
    if (q->onlat) { /* perfect streaming: f*_i(x) = f_i(x - n_i) */
#pragma omp parallel for schedule(static)
        for (int y = 0; y < ny; ++y)
            for (int i = 0; i < q->npop; ++i) {
                int ys = src_index(y - q->sy[i], ny, bcy);
                for (int x = 0; x < nx; ++x)
                    fs[(long)i * S + (long)y * nx + x] =
                        f[(long)i * S + (long)ys * nx + src_index(x - q->sx[i], nx, bcx)];
            }
        return;
    }
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y) {
        for (int i = 0; i < q->npop; ++i) {
            double ax = fabs(q->vx[i]), ay = fabs(q->vy[i]);
            int sx = q->vx[i] >= 0.0 ? 1 : -1, sy = q->vy[i] >= 0.0 ? 1 : -1;
            int ys = src_index(y - sy, ny, bcy);
            const double *fi = f + (long)i * S;
            for (int x = 0; x < nx; ++x) {
                int xs = src_index(x - sx, nx, bcx);
                fs[(long)i * S + (long)y * nx + x] =
                    (1.0 - ax) * (1.0 - ay) * fi[(long)y * nx + x] +
                    ax * (1.0 - ay) * fi[(long)y * nx + xs] +
                    (1.0 - ax) * ay * fi[(long)ys * nx + x] +
                    ax * ay * fi[(long)ys * nx + xs];
            }
        }
    }
}

/* Collision at every site of fs (in place), Eq. (discrete-rbe) with the
 * relaxing sign:  f_i <- f*_i - (dt/tau) (p_i^a U_a / p_i^0) (f*_i - f^eq_i),
 * p^a U_a / p^0 = U^0 - U^x v_x - U^y v_y.  tau = +inf skips it.
 * Returns the number of sites flagged non-physical by the Landau solve. */
long orc_collide(const orc_quad *q, int nx, int ny, double tau, double *fs)
{
    if (isinf(tau)) return 0;
    long S = (long)nx * ny;
    long flagged = 0;
    const double inv_tau = 1.0 / tau;
#pragma omp parallel reduction(+ : flagged)
    {
        double *feq = malloc(sizeof(double) * q->npop);
#pragma omp for schedule(static)
        for (long s = 0; s < S; ++s) {
            double mom[9], mac[6];
            orc_moments(q, fs + s, S, mom);
            flagged += orc_landau(mom, mac);
            orc_feq(q, mac[0], mac[2], mac[4], mac[5], feq);
            for (int i = 0; i < q->npop; ++i) {
                double om = inv_tau * (mac[3] - mac[4] * q->vx[i] - mac[5] * q->vy[i]);
                double fsi = fs[(long)i * S + s];
                fs[(long)i * S + s] = fsi - om * (fsi - feq[i]);
            }
        }
        free(feq);
    }
    return flagged;
}

static void set_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* nsteps full time steps; f (npop x ny x nx) is updated in place.
 * Returns the total number of flagged site-steps. */
long orc_run(const orc_quad *q, int nx, int ny, int bcx, int bcy, double tau, int nsteps,
             double *f, int nthreads)
{
    set_threads(nthreads);
    long S = (long)nx * ny;
    double *fs = malloc(sizeof(double) * S * q->npop);
    long flagged = 0;
    for (int t = 0; t < nsteps; ++t) {
        orc_stream(q, nx, ny, bcx, bcy, f, fs);
        flagged += orc_collide(q, nx, ny, tau, fs);
        memcpy(f, fs, sizeof(double) * S * q->npop);
    }
    free(fs);
    return flagged;
}

/* Equilibrium initial state from macroscopic fields n, T, beta_x, beta_y
 * (each [ny][nx]); U^a = gamma (1, beta). */
void orc_init(const orc_quad *q, int nx, int ny, const double *n, const double *T,
              const double *bx, const double *by, double *f, int nthreads)
{
    set_threads(nthreads);
    long S = (long)nx * ny;
#pragma omp parallel
    {
        double *feq = malloc(sizeof(double) * q->npop);
#pragma omp for schedule(static)
        for (long s = 0; s < S; ++s) {
            double g = 1.0 / sqrt(1.0 - bx[s] * bx[s] - by[s] * by[s]);
            orc_feq(q, n[s], T[s], g * bx[s], g * by[s], feq);
            for (int i = 0; i < q->npop; ++i) f[(long)i * S + s] = feq[i];
        }
        free(feq);
    }
}

/* Landau-frame fields of stored populations (no streaming):
 * out[k*S + s] for k = n, eps, T, U^0, U^x, U^y.  Returns flagged sites. */
long orc_macro(const orc_quad *q, int nx, int ny, const double *f, double *out, int nthreads)
{
    set_threads(nthreads);
    long S = (long)nx * ny;
    long flagged = 0;
#pragma omp parallel for schedule(static) reduction(+ : flagged)
    for (long s = 0; s < S; ++s) {
        double mom[9], mac[6];
        orc_moments(q, f + s, S, mom);
        flagged += orc_landau(mom, mac);
        for (int k = 0; k < 6; ++k) out[k * S + s] = mac[k];
    }
    return flagged;
}
