"""Free-streaming solutions of the 1D Sod problem, FP64 numpy (TEST INFRASTRUCTURE ONLY).

Two forms, both for an initial step between a left MJ state (x < 0) and a right
one (x > 0), fluid at rest on both sides:

* :func:`continuum_moments` -- the analytic solution of Appendix A (continuous
  velocities, continuous space).  The printed T^tt = P_L + i_0 (P_R - P_L)/pi
  does not reduce to the left energy density eps_L = 2 P_L for w < -1; the
  component is read as T^tt = 2 P_L + i_0(w) (P_R - P_L)/pi, which gives
  eps_L at w = -1 and eps_R = 2 P_R at w = 1.  All other components are used
  as printed.

* :func:`discrete_velocity_moments` -- the same free-streaming problem for a
  finite set of discrete velocities (continuous space): f_i(x, t) = f_i(x - v_i t, 0),
  with moment sums of Eq. (discrete_sum_moments).  As K grows it approaches the
  continuum form; at finite K it is the limit the lattice scheme approaches as
  the grid is refined.
"""
from __future__ import annotations

import numpy as np


def i0(w):
    w = np.clip(w, -1.0, 1.0)
    return 2.0 * np.pi - 2.0 * np.arccos(w)


def i1(w):
    w = np.clip(w, -1.0, 1.0)
    return -2.0 * np.sqrt(1.0 - w * w)


def i2(w):
    w = np.clip(w, -1.0, 1.0)
    return np.pi - w * np.sqrt(1.0 - w * w) - np.arccos(w)


def continuum_moments(w, nL, PL, nR, PR):
    """(N^t, N^x, N^y, T^tt, T^tx, T^ty, T^xx, T^xy, T^yy) at self-similar w = x/t.

    For |w| > 1 the unperturbed states follow from the same formulas (the
    i-functions saturate at w = -1 and w = 1)."""
    w = np.asarray(w, dtype=np.float64)
    a0, a1, a2 = i0(w), i1(w), i2(w)
    dn = (nR - nL) / (2.0 * np.pi)
    dP = (PR - PL) / np.pi
    z = np.zeros_like(w)
    Nt = nL + a0 * dn
    Nx = a1 * dn
    Ttt = 2.0 * PL + a0 * dP
    Ttx = a1 * dP
    Txx = PL + a2 * dP
    Tyy = PL + (a0 - a2) * dP
    return np.stack([Nt, Nx, z, Ttt, Ttx, z, Txx, z, Tyy])


def printed_Ttt(w, PL, PR):
    """T^tt exactly as printed in Appendix A (kept for the misprint test)."""
    return PL + i0(np.asarray(w, dtype=np.float64)) * (PR - PL) / np.pi


def discrete_velocity_moments(x, t, p0, vx, vy, fL, fR):
    """Moment sums of the discrete-velocity free-streaming solution at positions x, time t.

    fL, fR: equilibrium populations of the left/right states on the nodes
    (p0, vx, vy).  A population i at x came from x - vx_i t."""
    x = np.asarray(x, dtype=np.float64)
    src = x[None, :] - vx[:, None] * t
    f = np.where(src < 0.0, fL[:, None], fR[:, None])
    px, py = p0 * vx, p0 * vy
    out = np.stack([
        (p0[:, None] * f).sum(0), (px[:, None] * f).sum(0), (py[:, None] * f).sum(0),
        ((p0 * p0)[:, None] * f).sum(0), ((p0 * px)[:, None] * f).sum(0),
        ((p0 * py)[:, None] * f).sum(0), ((px * px)[:, None] * f).sum(0),
        ((px * py)[:, None] * f).sum(0), ((py * py)[:, None] * f).sum(0)])
    return out
