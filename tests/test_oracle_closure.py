"""Pins of the closure reference (oracle/closure.py) against definitions:
finite differences for the backpropagated gradient, exact sums for the
restriction, and the null-space property of the conservative projection."""
import math

import numpy as np

import oracle as O
from oracle import closure as C


def small_params(F, H, Oo, seed=0):
    g = np.random.default_rng(seed)
    return [g.normal(0, 0.3, (F, H)), g.normal(0, 0.1, H), g.normal(0, 0.3, (H, H)),
            g.normal(0, 0.1, H), g.normal(0, 0.3, (H, Oo)), g.normal(0, 0.1, Oo)]


def test_mlp_gradient_matches_finite_differences():
    F, H, Oo, S = 7, 5, 4, 11
    g = np.random.default_rng(1)
    X = g.normal(size=(S, F))
    T = g.normal(size=(S, Oo))
    params = small_params(F, H, Oo)
    loss, grads = C.mlp_loss_and_grad(params, X, T)
    h = 1e-6
    for pi, (P, G) in enumerate(zip(params, grads)):
        it = np.nditer(P, flags=["multi_index"])
        for _ in it:
            idx = it.multi_index
            old = P[idx]
            P[idx] = old + h
            lp, _ = C.mlp_loss_and_grad(params, X, T)
            P[idx] = old - h
            lm, _ = C.mlp_loss_and_grad(params, X, T)
            P[idx] = old
            assert abs((lp - lm) / (2 * h) - G[idx]) < 1e-7 * max(1.0, abs(G[idx])), (pi, idx)


def test_gelu_is_x_times_normal_cdf():
    from scipy.stats import norm
    x = np.linspace(-5, 5, 41)
    np.testing.assert_allclose(C.gelu(x), x * norm.cdf(x), atol=1e-15)
    h = 1e-6
    np.testing.assert_allclose(C.gelu_grad(x), (C.gelu(x + h) - C.gelu(x - h)) / (2 * h), atol=1e-8)


def test_restriction_is_exact_for_equilibria_and_keeps_conserved_moments():
    N, Kf, Kc = 2, 128, 24
    R = C.restriction(N, Kf, Kc)
    np.testing.assert_allclose(R.sum(1), 1.0, atol=1e-13)      # shell sums kept
    qf, qc = O.Quadrature(N, Kf), O.Quadrature(N, Kc)
    # every equilibrium is a trig polynomial of degree N in theta per shell: mapped exactly
    for (n, T, ux, uy) in [(0.7, 1.0, 0.0, 0.0), (0.4, 0.6, 0.3, -0.2), (1.2, 1.4, -0.1, 0.45)]:
        got = C.restrict(qf.feq(n, T, ux, uy)[:, None], N, Kf, Kc)[:, 0]
        np.testing.assert_allclose(got, qc.feq(n, T, ux, uy), rtol=1e-11, atol=1e-15)
    # arbitrary fine states: N^a, T^00, T^0x, T^0y are kept (modes m = 0, 1 survive)
    f = np.random.default_rng(2).uniform(size=(qf.npop, 5)) * qf.w[:, None]
    fc = C.restrict(f, N, Kf, Kc)
    mf, mc = C.moments9(f, qf.p0, qf.vx, qf.vy), C.moments9(fc, qc.p0, qc.vx, qc.vy)
    np.testing.assert_allclose(mc[:6], mf[:6], rtol=1e-12, atol=1e-14)


def test_conservative_projection_null_space():
    q = O.Quadrature(2, 24)
    d = np.random.default_rng(3).normal(size=(q.npop, 6))
    dp = C.conservative_projection(d, q.p0, q.vx, q.vy, q.w)
    Cm = np.stack([q.p0, q.p0 ** 2, q.p0 ** 2 * q.vx, q.p0 ** 2 * q.vy])
    assert np.abs(Cm @ dp).max() < 1e-12 * np.abs(Cm @ d).max()
    np.testing.assert_allclose(C.conservative_projection(dp, q.p0, q.vx, q.vy, q.w), dp, atol=1e-14)


def test_features_of_rest_equilibrium():
    q = O.Quadrature(2, 24)
    n, T = 0.8, 1.0
    f = q.feq(n, T, 0.0, 0.0)[:, None]
    X = C.features(f, q.p0, q.vx, q.vy, q.w, 0.5)[0]
    np.testing.assert_allclose(X[:9], [1, 0, 0, 2 * T, 0, 0, T, 0, T], atol=1e-12)
    assert X[9] == 0.5
    np.testing.assert_allclose(X[10:], 1.0 / (2 * math.pi), rtol=1e-12)
