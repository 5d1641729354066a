"""FP64 numpy reference of the learned angular closure (TEST INFRASTRUCTURE ONLY).

The closure is not in the paper; it is the learned correction the build adds on
top of the method (a coarse angular quadrature corrected toward a fine one).
Everything here is the plain definition, used to check the CUDA kernels:

* :func:`restriction` -- per energy shell, the angular function g = f / w of
  the fine rule is expanded in its discrete Fourier modes, truncated below the
  coarse rule's Nyquist mode (|m| <= (Kc - 1) / 2) and evaluated at the coarse
  angles; f_coarse = w_coarse g.  Exact for every trigonometric polynomial of
  degree <= (Kc - 1) / 2 in theta (all equilibria of order N < Kc / 2); it
  keeps the m = 0 and m = 1 modes, hence N^0, N^x, N^y, T^00, T^0x, T^0y.
* :func:`features` -- per site: the nine moments N^a, T^ab divided by N^0, the
  Knudsen number, and the populations divided by w_i N^0.
* :func:`mlp_forward` / :func:`mlp_loss_and_grad` -- Linear, GELU, Linear,
  GELU, Linear; GELU(x) = x Phi(x) (exact, erf form); loss = mean over sites and
  outputs of (y - target)^2.
* :func:`conservative_projection` -- the correction minus its weighted
  least-squares component along p^0, p^0 p^0, p^0 p^x, p^0 p^y, so that adding
  it leaves N^0, T^00, T^0x, T^0y of the site unchanged.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf


def restriction(N: int, Kf: int, Kc: int) -> np.ndarray:
    """R[r, k, j]: weight of fine population j on coarse population k in shell r,
    R = (w_c / w_f) (1/Kf) sum_{|m| <= M} exp(i m (theta_k - theta_j)), M = (Kc - 1) // 2."""
    R = np.zeros((N + 1, Kc, Kf))
    M = (Kc - 1) // 2
    for r in range(N + 1):
        off = r / (N + 1)
        thf = (np.arange(Kf) + off) * 2 * math.pi / Kf
        thc = (np.arange(Kc) + off) * 2 * math.pi / Kc
        d = thc[:, None] - thf[None, :]
        ker = np.ones_like(d)
        for m in range(1, M + 1):
            ker += 2.0 * np.cos(m * d)
        R[r] = ker / Kc  # (w_c / w_f) / Kf = (Kf / Kc) / Kf
    return R


def restrict(f_fine: np.ndarray, N: int, Kf: int, Kc: int) -> np.ndarray:
    """f_fine[(N+1)Kf, ...] -> f_coarse[(N+1)Kc, ...] (shell-major populations)."""
    R = restriction(N, Kf, Kc)
    shp = f_fine.shape[1:]
    ff = f_fine.reshape(N + 1, Kf, -1)
    out = np.einsum("rkj,rjs->rks", R, ff)
    return out.reshape((N + 1) * Kc, *shp)


def moments9(f, p0, vx, vy):
    """(9, S): N^t, N^x, N^y, T^tt, T^tx, T^ty, T^xx, T^xy, T^yy of f[npop, S]."""
    px, py = p0 * vx, p0 * vy
    return np.stack([p0 @ f, px @ f, py @ f, (p0 * p0) @ f, (p0 * px) @ f, (p0 * py) @ f,
                     (px * px) @ f, (px * py) @ f, (py * py) @ f])


def features(f, p0, vx, vy, w, kn):
    """X[S, 10 + npop] from populations f[npop, S]."""
    m = moments9(f, p0, vx, vy)
    n0 = m[0]
    return np.concatenate([(m / n0).T, np.full((f.shape[1], 1), kn), (f / (w[:, None] * n0)).T],
                          axis=1)


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2 * math.pi)


def mlp_forward(params, X):
    W1, b1, W2, b2, W3, b3 = params
    z1 = X @ W1 + b1
    h1 = gelu(z1)
    z2 = h1 @ W2 + b2
    h2 = gelu(z2)
    return h2 @ W3 + b3, (z1, h1, z2, h2)


def mlp_loss_and_grad(params, X, T):
    """Mean squared error over all entries and its gradient (W1, b1, W2, b2, W3, b3)."""
    W1, b1, W2, b2, W3, b3 = params
    Y, (z1, h1, z2, h2) = mlp_forward(params, X)
    cnt = Y.size
    dY = 2.0 * (Y - T) / cnt
    gW3 = h2.T @ dY
    gb3 = dY.sum(0)
    dz2 = (dY @ W3.T) * gelu_grad(z2)
    gW2 = h1.T @ dz2
    gb2 = dz2.sum(0)
    dz1 = (dz2 @ W2.T) * gelu_grad(z1)
    gW1 = X.T @ dz1
    gb1 = dz1.sum(0)
    return float(((Y - T) ** 2).mean()), (gW1, gb1, gW2, gb2, gW3, gb3)


def conservative_projection(d, p0, vx, vy, w):
    """d[npop, S] -> d - W C^T (C W C^T)^-1 C d, C rows = p^0, p^0 p^0, p^0 p^x, p^0 p^y."""
    C = np.stack([p0, p0 * p0, p0 * p0 * vx, p0 * p0 * vy])
    A = (C * w) @ C.T
    lam = np.linalg.solve(A, C @ d)
    return d - (w[:, None] * (C.T @ lam))
