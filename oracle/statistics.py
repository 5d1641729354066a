"""Fermi-Dirac and Bose-Einstein equilibria, FP64 (TEST INFRASTRUCTURE ONLY).

Eq. (feq_dist) with the statistic eps = +1 (Fermi-Dirac) or -1 (Bose-Einstein):
    f^eq = g / (z^-1 exp(U_a p^a / T) + eps),   z = exp(mu / T),
g a fixed normalisation (degeneracy); eps = 0 is the Maxwell-Juttner form
g z exp(-U.p/T) of the rest of the oracle.  The paper restricts itself to
Maxwell-Juttner and states that its quadratures apply to the other two
statistics as well (Sec. 2.1); everything here follows the same steps as the
Maxwell-Juttner oracle with the rest-frame radial integrals replaced:

    I_k = int_0^inf f(p) p^k dp = g T^(k+1) k! phi_{k+1}(z),
    phi_s(z) = (1/Gamma(s)) int_0^inf x^(s-1) / (z^-1 e^x + eps) dx,

so that (massless, 2+1 dimensions, d^2p/p^0 = dp dtheta)
    n = 2 pi I_1 = 2 pi g T^2 phi_2(z),   e = 2 pi I_2 = 4 pi g T^3 phi_3(z),   P = e/2.

phi_s is evaluated from its definition by adaptive quadrature (scipy), the
only library step; (T, z) from (n, e) by bracketing root finding on
ln phi_3 - 3/2 ln phi_2, which is monotone in ln z.  Moments of f^eq of rank
k are I_k times the boosted angular integral of the rest-frame directions
(obtained from the Maxwell-Juttner moment routine at n = T = 1, whose radial
factor is k!/(2 pi)), and the truncated equilibrium is the omega-orthogonal
projection of Eq. (mj-feq-expansion-truncated) onto the cone monomials, as in
the C oracle.  Bose-Einstein states need z < 1 (2D: phi_1 diverges at z = 1).
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate, optimize

from . import Quadrature, angular_integral, landau, mj_moment

FD, BE, MJ = 1, -1, 0


def phi(s: int, z: float, eps: int) -> float:
    """phi_s(z) from its integral definition (eps = 0: z)."""
    if eps == 0:
        return float(z)
    if eps == BE and not z < 1.0 and s <= 1:
        return math.inf

    def f(x):
        ez = z * math.exp(-x)  # z^-1 e^x + eps = (1 + eps z e^-x) / (z e^-x)
        return x ** (s - 1) * ez / (1.0 + eps * ez)

    pts = [0.0]
    if eps == FD and z > 1.0:
        pts.append(math.log(z))  # the Fermi edge
    pts.append(pts[-1] + 60.0)
    total = 0.0
    for a, b in zip(pts[:-1], pts[1:]):
        v, _ = integrate.quad(f, a, b, epsabs=0.0, epsrel=2e-14, limit=400)
        total += v
    v, _ = integrate.quad(f, pts[-1], math.inf, epsabs=0.0, epsrel=2e-14, limit=400)
    return (total + v) / math.gamma(s)


def density_energy(T: float, z: float, eps: int, g: float):
    """(n, e) of the rest-frame equilibrium."""
    return 2 * math.pi * g * T * T * phi(2, z, eps), 4 * math.pi * g * T ** 3 * phi(3, z, eps)


def solve_Tz(n: float, e: float, eps: int, g: float):
    """(T, z) with density_energy(T, z) = (n, e)."""
    if eps == 0:
        T = e / (2 * n)
        return T, n / (2 * math.pi * g * T * T)
    target = math.log(e * math.sqrt(2 * math.pi * g) / (2 * n ** 1.5))

    def h(eta):
        z = math.exp(eta)
        return math.log(phi(3, z, eps)) - 1.5 * math.log(phi(2, z, eps)) - target

    lo, hi = -60.0, (60.0 if eps == FD else -1e-12)
    if h(lo) * h(hi) > 0:
        raise ValueError("no equilibrium of this statistic has these (n, e)")
    eta = optimize.brentq(h, lo, hi, xtol=1e-15, rtol=1e-15, maxiter=400)
    z = math.exp(eta)
    return math.sqrt(n / (2 * math.pi * g * phi(2, z, eps))), z


def radial(k: int, T: float, z: float, eps: int, g: float) -> float:
    """I_k = int f p^k dp in the rest frame."""
    return g * T ** (k + 1) * math.factorial(k) * phi(k + 1, z, eps)


def moment(idx, T: float, z: float, Ux: float, Uy: float, eps: int, g: float) -> float:
    """Lab-frame moment int f^eq p^idx1 ... p^idxk d^2p/p^0."""
    k = len(idx)
    boost = mj_moment(idx, 1.0, 1.0, Ux, Uy) * 2 * math.pi / math.factorial(k)
    return radial(k, T, z, eps, g) * boost


def feq(q: Quadrature, T: float, z: float, Ux: float, Uy: float, eps: int, g: float) -> np.ndarray:
    """Eq. (mj-feq-expansion-truncated): w_i B(p_i)^T G^-1 M for this statistic."""
    e, a, b = q.basis()
    k = e + a + b
    nb = len(e)
    G = np.array([[math.factorial(int(k[m] + k[n])) * angular_integral(int(a[m] + a[n]), int(b[m] + b[n]))
                   for n in range(nb)] for m in range(nb)])
    M = np.array([moment((0,) * int(e[m]) + (1,) * int(a[m]) + (2,) * int(b[m]), T, z, Ux, Uy, eps, g)
                  for m in range(nb)])
    B = np.stack([q.p0 ** ee * (q.p0 * q.vx) ** aa * (q.p0 * q.vy) ** bb for ee, aa, bb in zip(e, a, b)], 1)
    return q.w * (B @ np.linalg.solve(G, M))


def site_state(q: Quadrature, f_site, eps: int, g: float):
    """(status, n, e, T, z, U0, Ux, Uy) of one site: Landau frame, then (T, z)."""
    st, mac = landau(q.moments(f_site))
    n, e = mac[0], mac[1]
    T, z = solve_Tz(n, e, eps, g)
    return st, n, e, T, z, mac[3], mac[4], mac[5]


def collide(q: Quadrature, fs, tau: float, eps: int, g: float):
    """Eq. (discrete-rbe), relaxing sign, toward this statistic's f^eq."""
    out = np.array(fs, dtype=np.float64, copy=True)
    if math.isinf(tau):
        return out
    _, ny, nx = out.shape
    for y in range(ny):
        for x in range(nx):
            st, n, e, T, z, U0, Ux, Uy = site_state(q, out[:, y, x], eps, g)
            fe = feq(q, T, z, Ux, Uy, eps, g)
            om = (U0 - Ux * q.vx - Uy * q.vy) / tau
            out[:, y, x] = out[:, y, x] - om * (out[:, y, x] - fe)
    return out


def run(q: Quadrature, f, tau: float, nsteps: int, bcx, bcy, eps: int, g: float):
    """nsteps of stream (the oracle's streaming) then collide."""
    for _ in range(nsteps):
        f = collide(q, q.stream(f, bcx, bcy), tau, eps, g)
    return f


def init(q: Quadrature, n, T, bx, by, eps: int, g: float) -> np.ndarray:
    """Equilibrium populations of fields (n, T, beta): z from n = 2 pi g T^2 phi_2(z)."""
    ny, nx = n.shape
    f = np.zeros((q.npop, ny, nx))
    for y in range(ny):
        for x in range(nx):
            t = float(T[y, x])
            z = fugacity(float(n[y, x]), t, eps, g)
            gam = 1.0 / math.sqrt(1.0 - bx[y, x] ** 2 - by[y, x] ** 2)
            f[:, y, x] = feq(q, t, z, gam * bx[y, x], gam * by[y, x], eps, g)
    return f


def fugacity(n: float, T: float, eps: int, g: float) -> float:
    """z with 2 pi g T^2 phi_2(z) = n."""
    target = n / (2 * math.pi * g * T * T)
    if eps == 0:
        return target
    hi = 60.0 if eps == FD else -1e-12
    eta = optimize.brentq(lambda t: math.log(phi(2, math.exp(t), eps)) - math.log(target), -60.0, hi,
                          xtol=1e-15, rtol=1e-15, maxiter=400)
    return math.exp(eta)
