"""Pins of the Fermi-Dirac / Bose-Einstein oracle (oracle/statistics.py) against
closed forms, an independent polylogarithm, the Maxwell-Juttner limit and the
conservation laws.  CPU only."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import statistics as S
from paper_2011_06856_gb300 import workloads as W

ZETA3 = 1.2020569031595942853997


def test_phi_closed_forms():
    for z in (0.05, 0.7, 0.999):
        assert abs(S.phi(1, z, S.FD) - math.log1p(z)) < 1e-15
        assert abs(S.phi(1, z, S.BE) + math.log1p(-z)) < 1e-14 * abs(math.log1p(-z))
    assert abs(S.phi(2, 1.0, S.FD) - math.pi ** 2 / 12) < 1e-15
    assert abs(S.phi(2, 1.0, S.BE) - math.pi ** 2 / 6) < 1e-15
    assert abs(S.phi(3, 1.0, S.FD) - 0.75 * ZETA3) < 1e-15
    assert abs(S.phi(3, 1.0, S.BE) - ZETA3) < 1e-15
    # degenerate Fermi gas: F_2(eta) + F_2(-eta) = eta^2 / 2 + pi^2 / 6
    for z in (3.0, 40.0, 1e4):
        eta = math.log(z)
        lhs = S.phi(2, z, S.FD) + S.phi(2, 1.0 / z, S.FD)
        assert abs(lhs - (eta * eta / 2 + math.pi ** 2 / 6)) < 1e-13 * lhs


def test_phi_against_series():
    """Against the defining series of the polylogarithm (z <= 0.5, 200 terms)."""
    for s in range(1, 7):
        for z in (1e-4, 0.1, 0.5):
            li_m = sum((-z) ** k / k ** s for k in range(1, 200))
            li_p = sum(z ** k / k ** s for k in range(1, 200))
            assert abs(S.phi(s, z, S.FD) + li_m) < 1e-15 * abs(li_m)
            assert abs(S.phi(s, z, S.BE) - li_p) < 1e-15 * abs(li_p)


def test_phi_against_mpmath():
    mp = pytest.importorskip("mpmath")
    for s in range(2, 7):
        for z in (0.3, 0.95, 7.0, 500.0):
            ref = -float(mp.polylog(s, -z))
            assert abs(S.phi(s, z, S.FD) - ref) < 1e-14 * ref
            if z < 1:
                ref = float(mp.polylog(s, z))
                assert abs(S.phi(s, z, S.BE) - ref) < 1e-13 * ref


def test_maxwell_juttner_limits():
    """eps = 0 is the Maxwell-Juttner equilibrium of the C oracle; at small z both
    quantum statistics approach it (phi_s = z - eps z^2 / 2^s + ...)."""
    q = O.Quadrature(3, 12)
    T, z, Ux, Uy = 1.1, 0.3, 0.25, -0.15
    n = 2 * math.pi * T * T * z
    fm, fc = S.feq(q, T, z, Ux, Uy, S.MJ, 1.0), q.feq(n, T, Ux, Uy)
    assert np.abs(fm - fc).max() < 1e-13 * np.abs(fc).max()
    for eps in (S.FD, S.BE):
        zz = 1e-6
        assert abs(S.phi(3, zz, eps) / zz - (1 - eps * zz / 8)) < 1e-12
        fe = S.feq(q, T, zz, Ux, Uy, eps, 1.0)
        fm = q.feq(2 * math.pi * T * T * zz, T, Ux, Uy)
        assert np.abs(fe - fm).max() / np.abs(fm).max() < 2e-6


@pytest.mark.parametrize("eps", [S.FD, S.BE])
def test_solve_round_trip_and_feq_moments(eps):
    """(T, z) -> (n, e) -> (T, z); the discrete f^eq carries N^a = n U^a and the
    ideal-fluid T^ab with P = e/2 (quadrature exactness + projection)."""
    q = O.Quadrature(3, 12)
    for T, z in ((0.8, 0.3), (1.3, 0.9), (0.6, 4.0) if eps == S.FD else (0.6, 0.97)):
        n, e = S.density_energy(T, z, eps, 1.0)
        T2, z2 = S.solve_Tz(n, e, eps, 1.0)
        assert abs(T2 - T) < 1e-13 * T and abs(z2 - z) < 1e-12 * z
        assert abs(S.fugacity(n, T, eps, 1.0) - z) < 1e-12 * z
        Ux, Uy = 0.3, -0.2
        U = np.array([math.sqrt(1 + Ux * Ux + Uy * Uy), Ux, Uy])
        m = q.moments(S.feq(q, T, z, Ux, Uy, eps, 1.0))
        np.testing.assert_allclose(m[:3], n * U, rtol=1e-12)
        P = e / 2
        eta = np.diag([1.0, -1.0, -1.0])
        Tab = (e + P) * np.outer(U, U) - P * eta
        got = [m[3], m[4], m[5], m[6], m[7], m[8]]
        want = [Tab[0, 0], Tab[0, 1], Tab[0, 2], Tab[1, 1], Tab[1, 2], Tab[2, 2]]
        np.testing.assert_allclose(got, want, rtol=1e-11, atol=1e-12 * e)


@pytest.mark.parametrize("eps", [S.FD, S.BE])
def test_statistics_collision_conserves(eps):
    q = O.Quadrature(3, 12)
    fl = W.random_fields(3, 2, seed=5, beta_max=0.3)
    f = S.init(q, fl.n * 0.3, fl.T, fl.bx, fl.by, eps, 1.0)
    f = f * (1 + 0.05 * W.random_populations(q.npop, 2, 3, seed=6))
    fn = S.collide(q, f, 1.7, eps, 1.0)
    d = (fn - f).reshape(q.npop, -1)
    for wgt in [q.p0, q.p0 * q.p0, q.p0 * q.p0 * q.vx, q.p0 * q.p0 * q.vy]:
        scale = (np.abs(wgt)[:, None] * f.reshape(q.npop, -1)).sum(0)
        assert (np.abs((wgt[:, None] * d).sum(0)) / scale).max() < 1e-12
