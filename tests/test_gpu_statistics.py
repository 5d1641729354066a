"""GPU parity of the quantum statistics (Eq. feq_dist with eps = +1 Fermi-Dirac,
-1 Bose-Einstein) against the FP64 oracle (oracle/statistics.py).

The oracle evaluates phi_s(z) from its integral definition and solves (T, z)
by bracketing; the library by accelerated series and safeguarded Newton steps
(rlbm_stat.cuh).  FP64: 1e-12 normwise; FP32 storage (FP64 per-site part): the
FP32 bound of the other parity tests.
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle import statistics as S
from paper_2011_06856_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2011_06856_gb300 import build as B  # noqa: E402
from paper_2011_06856_gb300 import rlbm as R  # noqa: E402

B.build()

NAMES = {S.FD: "fd", S.BE: "be"}


def relerr(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def fields(nx, ny, seed):
    fl = W.random_fields(nx, ny, seed=seed, beta_max=0.3)
    fl.n[:] = fl.n * 0.5  # z = n / (2 pi T^2 ...) stays below 1 for the Bose-Einstein runs
    return fl


@pytest.mark.parametrize("stat", [S.FD, S.BE])
@pytest.mark.parametrize("N,K,nx,ny,bcx,bcy", [(3, 12, 24, 3, W.BC_COPYOUT, W.BC_PERIODIC),
                                               (2, 16, 33, 2, W.BC_PERIODIC, W.BC_COPYOUT)])
def test_quantum_fp64_parity(stat, N, K, nx, ny, bcx, bcy):
    g, tau, steps = 1.0, 2.0, 3
    q = O.Quadrature(N, K)
    fl = fields(nx, ny, seed=nx + N)
    f0 = S.init(q, fl.n, fl.T, fl.bx, fl.by, stat, g)
    sim = R.Simulation(nx, ny, N, K, tau, "fp64", bcx, bcy)
    sim.set_statistics(NAMES[stat], g)
    assert sim.statistics == NAMES[stat] and sim.step_kernel == "per-tile"
    sim.init_fields(fl)
    assert relerr(sim.get_populations(), f0) < 1e-12
    ref = S.run(q, f0, tau, steps, bcx, bcy, stat, g)
    sim.step(steps)
    assert relerr(sim.get_populations(), ref) < 1e-12
    mac = sim.moments()
    for y in range(ny):
        for x in range(0, nx, 7):
            st, n, e, T, z, U0, Ux, Uy = S.site_state(q, ref[:, y, x], stat, g)
            assert abs(mac[0, y, x] - n) < 1e-12 * n
            assert abs(mac[2, y, x] - T) < 1e-12 * T


@pytest.mark.parametrize("stat", [S.FD, S.BE])
def test_quantum_fp32_storage(stat):
    g, tau, steps, N, K, nx, ny = 0.7, 3.0, 10, 3, 12, 40, 2
    q = O.Quadrature(N, K)
    fl = fields(nx, ny, seed=3)
    ref = S.run(q, S.init(q, fl.n, fl.T, fl.bx, fl.by, stat, g), tau, steps, W.BC_COPYOUT, W.BC_PERIODIC, stat, g)
    sim = R.Simulation(nx, ny, N, K, tau, "fp32", W.BC_COPYOUT, W.BC_PERIODIC)
    sim.set_statistics(NAMES[stat], g)
    sim.init_fields(fl)
    sim.step(steps)
    tol = 1e-5
    assert relerr(sim.get_populations().astype(np.float64), ref) < tol


def test_degenerate_fermi_gas():
    """z up to ~1e3 (n / T^2 large): the inversion branch of the Fermi-Dirac integrals."""
    g, tau, N, K, nx = 1.0, 2.0, 3, 12, 16
    q = O.Quadrature(N, K)
    fl = W.shock_tube(nx, 1, (40.0, 0.5), (5.0, 0.6))
    f0 = S.init(q, fl.n, fl.T, fl.bx, fl.by, S.FD, g)
    sim = R.Simulation(nx, 1, N, K, tau, "fp64", W.BC_COPYOUT, W.BC_PERIODIC)
    sim.set_statistics("fd", g)
    sim.init_fields(fl)
    assert relerr(sim.get_populations(), f0) < 1e-12
    sim.step(2)
    assert relerr(sim.get_populations(), S.run(q, f0, tau, 2, W.BC_COPYOUT, W.BC_PERIODIC, S.FD, g)) < 1e-12


def test_statistics_refusals_and_round_trip():
    sim = R.Simulation(16, 2, 3, 12, 2.0, "fp16n")
    with pytest.raises(R.RLBMError) as e:
        sim.set_statistics("fd")
    assert e.value.status == R.ERR_UNSUPPORTED
    with pytest.raises(R.RLBMError) as e:
        R.Simulation(16, 2, 4, 12, 2.0, "fp64").set_statistics("be")
    assert e.value.status == R.ERR_UNSUPPORTED
    with pytest.raises(R.RLBMError) as e:
        R.Simulation(16, 16, 3, 12, 2.0, "fp64", onlattice=True).set_statistics("fd")
    assert e.value.status == R.ERR_UNSUPPORTED
    sim = R.Simulation(32, 2, 3, 12, 2.0, "fp64")
    with pytest.raises(R.RLBMError) as e:
        sim.set_statistics("fd", 0.0)
    assert e.value.status == R.ERR_ARG
    # Bose-Einstein beyond condensation: n / (2 pi g T^2) > zeta(2)
    sim.set_statistics("be", 1.0)
    sim.init_fields(W.uniform(32, 2, 20.0, 1.0))
    with pytest.raises(R.Unphysical):
        sim.moments()
    # back to Maxwell-Juttner: the plain kernel again, same result as a fresh handle
    fl = W.shock_tube(32, 2)
    sim.set_statistics("mj")
    sim.init_fields(fl)
    sim.step(4)
    ref = R.Simulation(32, 2, 3, 12, 2.0, "fp64")
    ref.init_fields(fl)
    ref.step(4)
    np.testing.assert_array_equal(sim.get_populations(), ref.get_populations())
