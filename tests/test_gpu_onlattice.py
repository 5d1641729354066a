"""GPU parity of the on-lattice rule (Sec. 2.3: 12 integer stencil vectors of
length 5 on the 4 shells of N = 3, perfect streaming) against the FP64 oracle.

Free streaming is an exact copy, so it is compared bit for bit; steps with a
collision to 1e-12 normwise in FP64 and to the FP32 bound of the other parity
tests, 1e-5.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2011_06856_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2011_06856_gb300 import build as B  # noqa: E402
from paper_2011_06856_gb300 import rlbm as R  # noqa: E402

B.build()


def relerr(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def lattice(nx, ny, tau, precision="fp64", bcx=W.BC_PERIODIC, bcy=W.BC_PERIODIC):
    return R.Simulation(nx, ny, 3, 12, tau, precision, bcx, bcy, onlattice=True)


def test_onlattice_quadrature_tables_match_oracle():
    """Same nodes, directions and weights as the oracle's rule (the library
    solves its angular weights in closed form, the oracle by least squares)."""
    q = O.Quadrature(3, onlattice=True)
    sim = lattice(8, 8, 2.0)
    assert R.lib().rlbm_is_onlattice(sim._h) == 1
    assert sim.npop == 48 and sim.step_kernel == "per-tile" and sim.tile_populations == 12
    # the equilibrium of a rest state is n w_i / (2 pi): read the weights back through init
    fl = W.uniform(8, 8, 1.0, 1.0)
    sim.init_fields(fl)
    f = sim.get_populations()[:, 0, 0]
    np.testing.assert_allclose(f, q.w / (2 * math.pi), rtol=1e-13)


@pytest.mark.parametrize("nx,ny,bcx,bcy", [(13, 11, W.BC_PERIODIC, W.BC_PERIODIC),
                                           (40, 1, W.BC_COPYOUT, W.BC_PERIODIC),
                                           (3, 4, W.BC_PERIODIC, W.BC_COPYOUT),
                                           (70, 37, W.BC_COPYOUT, W.BC_COPYOUT)])
def test_onlattice_free_streaming_bitwise(nx, ny, bcx, bcy):
    """tau = inf: every population moves by its stencil vector (shifts larger
    than the grid included), bit for bit."""
    q = O.Quadrature(3, onlattice=True)
    f0 = W.random_populations(q.npop, ny, nx, seed=nx + ny) * q.w[:, None, None]
    ref, _ = q.run(f0, math.inf, 7, bcx, bcy)
    sim = lattice(nx, ny, math.inf, bcx=bcx, bcy=bcy)
    sim.set_populations(f0)
    sim.step(7)
    np.testing.assert_array_equal(sim.get_populations(), ref)


@pytest.mark.parametrize("nx,ny,bcx,bcy", [(70, 37, W.BC_COPYOUT, W.BC_COPYOUT),
                                           (64, 1, W.BC_COPYOUT, W.BC_PERIODIC),
                                           (33, 20, W.BC_PERIODIC, W.BC_PERIODIC)])
def test_onlattice_fp64_parity(nx, ny, bcx, bcy):
    """Random smooth fields, 8 steps with a collision: fields and populations."""
    steps, tau = 8, 2.5
    q = O.Quadrature(3, onlattice=True)
    fl = W.random_fields(nx, ny, seed=3 + nx)
    ref, flagged = q.run(q.init(fl.n, fl.T, fl.bx, fl.by), tau, steps, bcx, bcy)
    assert flagged == 0
    mac_ref, _ = q.macro(ref)
    sim = lattice(nx, ny, tau, bcx=bcx, bcy=bcy)
    sim.init_fields(fl)
    sim.step(steps)
    assert relerr(sim.get_populations(), ref) < 1e-12
    mac = sim.moments()
    for i in range(4):
        assert relerr(mac[i], mac_ref[i]) < 1e-12, i


def test_onlattice_fp32_paper_2d_states():
    """The paper's 2D four-quadrant states on 64x64 in FP32, 20 steps."""
    L, steps, tau = 64, 20, 3.0
    q = O.Quadrature(3, onlattice=True)
    fl = W.riemann_2d(L, L, W.PAPER_SOD2D_STATES)
    ref, flagged = q.run(q.init(fl.n, fl.T, fl.bx, fl.by), tau, steps, W.BC_COPYOUT, W.BC_COPYOUT)
    assert flagged == 0
    mac_ref, _ = q.macro(ref)
    sim = lattice(L, L, tau, "fp32", W.BC_COPYOUT, W.BC_COPYOUT)
    sim.init_fields(fl)
    sim.autotune(2)
    sim.step(steps)
    mac = sim.moments()
    tol = 1e-5
    for i in range(4):
        assert relerr(mac[i], mac_ref[i]) < tol, i


def test_onlattice_refusals():
    for prec in ("fp16n", "bf16", "fp16"):
        with pytest.raises(R.RLBMError) as e:
            lattice(16, 16, 2.0, prec)
        assert e.value.status == R.ERR_UNSUPPORTED
    sim = lattice(64, 8, 2.0, "fp32")
    for P, kind in ((16, "per-tile"), (12, "pair"), (12, "tma")):
        with pytest.raises(R.RLBMError) as e:
            sim.set_tiling(P, kind)
        assert e.value.status == R.ERR_UNSUPPORTED
    sim.set_tiling(12, "per-tile")
    with pytest.raises(ValueError):
        R.Simulation(8, 8, 2, 12, 2.0, onlattice=True)
