"""GPU parity for quadrature orders N = 4, 5 and for many angles (several
groups of populations per warp), against the FP64 oracle.

The paper's 1D runs (Sec. 3.1) use N = 3 with K up to 120 on 2000x1, N = 5 with
K = 12, and a K = 600 (N_pop = 2400) reference on 4000x1.  K beyond 64
floor(16 / (N+1)) angles per shell makes every warp own several groups of
populations (rlbm_population_groups > 1).  Tolerances as in the other parity
tests: 1e-12 normwise in FP64, the FP32 bound max(1e-5, b omega_max steps).
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle import appendix_a as A
from paper_2011_06856_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2011_06856_gb300 import build as B  # noqa: E402
from paper_2011_06856_gb300 import rlbm as R  # noqa: E402

B.build()

FP64_TOL = 1e-12
FP32_TOL = 1e-5


def relerr(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def fields_err(got, ref):
    """Largest normwise error over n, eps, T, U^0 and the spatial U (one shared scale)."""
    e = [relerr(got[i], ref[i]) for i in range(4)]
    us = max(np.abs(ref[4:6]).max(), 1e-300)
    e.append(np.abs(got[4:6] - ref[4:6]).max() / us)
    return max(e)


def oracle_run(N, K, fl, tau, steps, bcx, bcy):
    q = O.Quadrature(N, K)
    f, flagged = q.run(q.init(fl.n, fl.T, fl.bx, fl.by), tau, steps, bcx, bcy)
    assert flagged == 0
    mac, _ = q.macro(f)
    return f, mac


def gpu_run(N, K, fl, tau, steps, bcx, bcy, precision="fp64", P=None, kind="per-tile"):
    ny, nx = fl.shape
    sim = R.Simulation(nx, ny, N, K, tau, precision, bcx, bcy)
    if P is not None:
        sim.set_tiling(P, kind)
    sim.init_fields(fl)
    sim.step(steps)
    return sim, sim.moments()


# ------------------------------------------------------------ N = 4, 5

@pytest.mark.parametrize("N,K", [(4, 9), (4, 16), (4, 40), (5, 12), (5, 24), (5, 100)])
def test_fp64_higher_orders_2d_ragged(N, K):
    """Random smooth fields on 70x37 (ragged x tail), copy-out, 6 steps."""
    nx, ny, steps, tau = 70, 37, 6, 3.0
    fl = W.random_fields(nx, ny, seed=11 + K + N)
    f_ref, mac_ref = oracle_run(N, K, fl, tau, steps, W.BC_COPYOUT, W.BC_COPYOUT)
    sim, mac = gpu_run(N, K, fl, tau, steps, W.BC_COPYOUT, W.BC_COPYOUT)
    assert sim.population_groups == 1
    assert sim.step_kernel == "per-tile"
    assert fields_err(mac, mac_ref) < FP64_TOL
    assert relerr(sim.get_populations(), f_ref) < FP64_TOL


@pytest.mark.parametrize("precision", ["fp32", "fp16n", "bf16n"])
def test_higher_order_reduced_precision(precision):
    """N = 5, K = 12 in FP32 and 16-bit storage (tolerances of the other parity tests)."""
    nx, ny, N, K, steps, tau = 96, 5, 5, 12, 20, 4.0
    fl = W.shock_tube(nx, ny, (1.5, 1.5), (0.1, 0.5))
    _, mac_ref = oracle_run(N, K, fl, tau, steps, W.BC_COPYOUT, W.BC_PERIODIC)
    _, mac = gpu_run(N, K, fl, tau, steps, W.BC_COPYOUT, W.BC_PERIODIC, precision)
    tol = {"fp32": FP32_TOL, "fp16n": 3e-3, "bf16n": 2.4e-2}[precision]
    for i in range(3):
        assert relerr(mac[i], mac_ref[i]) < tol, (precision, i)


def test_higher_order_free_streaming():
    """N = 5, K = 12, tau = inf: every population shifts by its own bilinear pull."""
    nx, ny, N, K, steps = 130, 3, 5, 12, 40
    q = O.Quadrature(N, K)
    f0 = W.random_populations(q.npop, ny, nx, seed=9) * q.w[:, None, None]
    ref, _ = q.run(f0, math.inf, steps, W.BC_COPYOUT, W.BC_PERIODIC)
    sim = R.Simulation(nx, ny, N, K, math.inf, "fp64", W.BC_COPYOUT, W.BC_PERIODIC)
    sim.set_populations(f0)
    sim.step(steps)
    assert relerr(sim.get_populations(), ref) < FP64_TOL


# ------------------------------------------------------------ several groups per warp

GROUP_CASES = [  # N, K, nx, ny, bcx, bcy
    (3, 600, 40, 1, W.BC_COPYOUT, W.BC_PERIODIC),   # the paper's reference rule, N_pop = 2400
    (3, 300, 33, 3, W.BC_PERIODIC, W.BC_COPYOUT),   # ragged tile, empty trailing groups
    (2, 400, 20, 5, W.BC_COPYOUT, W.BC_COPYOUT),
    (5, 200, 17, 2, W.BC_PERIODIC, W.BC_PERIODIC),
    (3, 257, 64, 2, W.BC_COPYOUT, W.BC_PERIODIC),   # one angle beyond one group per warp
]


@pytest.mark.parametrize("N,K,nx,ny,bcx,bcy", GROUP_CASES)
def test_fp64_population_groups(N, K, nx, ny, bcx, bcy):
    steps, tau = 5, 2.5
    fl = W.random_fields(nx, ny, seed=K + nx)
    f_ref, mac_ref = oracle_run(N, K, fl, tau, steps, bcx, bcy)
    sim, mac = gpu_run(N, K, fl, tau, steps, bcx, bcy)
    assert sim.population_groups > 1
    assert fields_err(mac, mac_ref) < FP64_TOL
    assert relerr(sim.get_populations(), f_ref) < FP64_TOL


@pytest.mark.parametrize("P", [8, 16, 24, 32, 48, 64])
def test_fp64_population_groups_every_tiling(P):
    """K = 600, N = 3 with every group size; groups = ceil(600 / (4 P))."""
    N, K, nx, ny, steps, tau = 3, 600, 24, 2, 3, 1.5
    fl = W.random_fields(nx, ny, seed=5)
    f_ref, _ = oracle_run(N, K, fl, tau, steps, W.BC_COPYOUT, W.BC_PERIODIC)
    sim, _ = gpu_run(N, K, fl, tau, steps, W.BC_COPYOUT, W.BC_PERIODIC, P=P)
    assert sim.tile_populations == P
    assert sim.population_groups == -(-K // (4 * P))
    assert relerr(sim.get_populations(), f_ref) < FP64_TOL


def test_fp32_population_groups():
    N, K, nx, ny, steps = 3, 600, 64, 2, 30
    tau = 3.0
    fl = W.shock_tube(nx, ny, (1.5, 1.5), (0.1, 0.5))
    _, mac_ref = oracle_run(N, K, fl, tau, steps, W.BC_COPYOUT, W.BC_PERIODIC)
    sim, mac = gpu_run(N, K, fl, tau, steps, W.BC_COPYOUT, W.BC_PERIODIC, "fp32")
    assert sim.population_groups > 1
    tol = FP32_TOL
    for i in range(3):
        assert relerr(mac[i], mac_ref[i]) < tol, i


def test_population_groups_free_streaming_and_init():
    """tau = inf stores every group in pass 1; init and moments run the group loop too."""
    N, K, nx, ny, steps = 3, 600, 50, 1, 25
    q = O.Quadrature(N, K)
    f0 = W.random_populations(q.npop, ny, nx, seed=21) * q.w[:, None, None]
    ref, _ = q.run(f0, math.inf, steps, W.BC_COPYOUT, W.BC_PERIODIC)
    sim = R.Simulation(nx, ny, N, K, math.inf, "fp64", W.BC_COPYOUT, W.BC_PERIODIC)
    assert sim.population_groups > 1
    sim.set_populations(f0)
    sim.step(steps)
    assert relerr(sim.get_populations(), ref) < FP64_TOL
    fl = W.random_fields(nx, ny, seed=2, beta_max=0.5)
    sim.init_fields(fl)
    assert relerr(sim.get_populations(), q.init(fl.n, fl.T, fl.bx, fl.by)) < 1e-13
    mac = sim.moments()
    np.testing.assert_allclose(mac[0], fl.n, rtol=1e-12)
    np.testing.assert_allclose(mac[2], fl.T, rtol=1e-12)


def test_population_groups_refusals_and_autotune():
    with pytest.raises(R.RLBMError) as e:
        R.Simulation(32, 1, 3, 600, 2.0, "fp16n")
    assert e.value.status == R.ERR_UNSUPPORTED
    sim = R.Simulation(64, 2, 3, 600, 2.0, "fp32")
    with pytest.raises(R.RLBMError) as e:
        sim.set_tiling(32, "pair")
    assert e.value.status == R.ERR_UNSUPPORTED
    assert sim.step_kernel == "per-tile"
    fl = W.shock_tube(64, 2, (1.5, 1.5), (0.1, 0.5))
    sim.init_fields(fl)
    sim.autotune(2)
    assert sim.step_kernel in ("per-tile", "pair") and sim.population_groups > 1
    sim.step(4)
    sim.moments()
    with pytest.raises(R.RLBMError) as e:
        sim.set_tiling(24, "pair-bulk")
    assert e.value.status == R.ERR_UNSUPPORTED


@pytest.mark.parametrize("N,K,nx,ny,P", [(3, 600, 130, 3, 24), (3, 600, 64, 1, 8), (2, 480, 66, 4, 12),
                                         (3, 384, 128, 2, 32)])
def test_fp32_pair_kernel_population_groups(N, K, nx, ny, P):
    """Two sites per lane with several population groups per warp (FP32): the
    oracle's fields within the FP32 bound; ragged tiles, warps with one group
    fewer (K = 600, P = 8 and 24), 1D and 2D."""
    steps, tau = 10, 3.0
    fl = W.random_fields(nx, ny, seed=K + P)
    _, mac_ref = oracle_run(N, K, fl, tau, steps, W.BC_COPYOUT, W.BC_PERIODIC)
    sim, mac = gpu_run(N, K, fl, tau, steps, W.BC_COPYOUT, W.BC_PERIODIC, "fp32", P=P, kind="pair")
    assert sim.step_kernel == "pair" and sim.population_groups > 1
    tol = FP32_TOL
    for i in range(4):
        assert relerr(mac[i], mac_ref[i]) < tol, i
    us = np.abs(mac_ref[4:6]).max()
    assert np.abs(mac[4:6] - mac_ref[4:6]).max() / us < tol


# ------------------------------------------------------------ the paper's Fig. 2 runs

def appendix_a_beta(nx, steps):
    x = np.arange(nx) + 0.5 - nx / 2
    cont = A.continuum_moments(x / steps, 1.5, 2.25, 0.1, 0.05)
    return np.array([(lambda m: m[4] / m[3])(O.landau(cont[:, s])[1]) for s in range(nx)])


@pytest.mark.parametrize("N,K", [(3, 12), (5, 12), (3, 120)])
def test_fig2_sod_free_streaming_2000x1(N, K):
    """Sec. 3.1, Fig. 2: 2000x1, tau -> inf, 900 steps (t/t_max = 0.9): the
    library equals the oracle (FP64), and the FP32 run gives the same error
    against Appendix A (Eq. rel_err) to 1e-4."""
    nx, steps = 2000, 900
    fl = W.shock_tube(nx, 1, (1.5, 1.5), (0.1, 0.5))
    f_ref, mac_ref = oracle_run(N, K, fl, math.inf, steps, W.BC_COPYOUT, W.BC_PERIODIC)
    sim, mac = gpu_run(N, K, fl, math.inf, steps, W.BC_COPYOUT, W.BC_PERIODIC)
    assert fields_err(mac, mac_ref) < FP64_TOL
    bref = appendix_a_beta(nx, steps)
    e_ref = np.linalg.norm(mac_ref[4, 0] / mac_ref[3, 0] - bref) / np.linalg.norm(bref)
    _, mac32 = gpu_run(N, K, fl, math.inf, steps, W.BC_COPYOUT, W.BC_PERIODIC, "fp32")
    e32 = np.linalg.norm(mac32[4, 0] / mac32[3, 0] - bref) / np.linalg.norm(bref)
    assert abs(e32 - e_ref) < 1e-4, (e32, e_ref)


# ------------------------------------------------------------ the paper's Fig. 3 K-sweep

def test_ksweep_matches_oracle_at_L200():
    """The sweep driver (library, FP64) gives the oracle's errors (Eq. rel_err)
    for a 400x1, K = 600 reference (groups of populations) and K in {12, 120}."""
    from paper_2011_06856_gb300 import ksweep
    L, steps = 200, 90
    rows = ksweep.sweep([0.02, 10.0], [12, 120], L=L, k_ref=600, precision="fp64")
    for row, kn in zip(rows, (0.02, 10.0)):
        q = O.Quadrature(3, 600)
        fl = W.shock_tube(2 * L, 1, W.PAPER_SOD_LEFT, W.PAPER_SOD_RIGHT)
        f, _ = q.run(q.init(fl.n, fl.T, fl.bx, fl.by), W.tau_from_kn(kn, 2 * L), 2 * steps)
        mac, _ = q.macro(f)
        bf = mac[4, 0] / mac[3, 0]
        bref = 0.5 * (bf[0::2] + bf[1::2])
        for K, e in zip(row["K"], row["eps"]):
            qk = O.Quadrature(3, K)
            flk = W.shock_tube(L, 1, W.PAPER_SOD_LEFT, W.PAPER_SOD_RIGHT)
            fk, _ = qk.run(qk.init(flk.n, flk.T, flk.bx, flk.by), W.tau_from_kn(kn, L), steps)
            mk, _ = qk.macro(fk)
            e_ref = np.linalg.norm(mk[4, 0] / mk[3, 0] - bref) / np.linalg.norm(bref)
            assert abs(e - e_ref) < 1e-9 * max(1.0, e_ref), (kn, K, e, e_ref)


def test_ksweep_full_size_kinetic_regime():
    """Fig. 3 at the paper's size (2000x1 against 4000x1, K_ref = 600), Kn = 10:
    the error falls with K (no parity: the paper prints no values)."""
    from paper_2011_06856_gb300 import ksweep
    row = ksweep.sweep([10.0], [12, 48, 120], L=2000, k_ref=600, precision="fp32")[0]
    e12, e48, e120 = row["eps"]
    assert e12 > e48 > e120, row["eps"]
    assert e12 > 5 * e120, row["eps"]


# ------------------------------------------------------------ the paper's 2D problem (Sec. 3.2)

def test_fp64_paper_2d_states_population_groups():
    """The four boosted quadrants of Sec. 3.2 with the K = 600 rule (groups of
    populations), 48x48, copy-out walls, Kn = 0.1: fields and populations."""
    N, K, L, steps = 3, 600, 48, 5
    fl = W.riemann_2d(L, L, W.PAPER_SOD2D_STATES)
    tau = W.tau_from_kn(0.1, L)
    f_ref, mac_ref = oracle_run(N, K, fl, tau, steps, W.BC_COPYOUT, W.BC_COPYOUT)
    sim, mac = gpu_run(N, K, fl, tau, steps, W.BC_COPYOUT, W.BC_COPYOUT)
    assert sim.population_groups > 1
    assert fields_err(mac, mac_ref) < FP64_TOL
    assert relerr(sim.get_populations(), f_ref) < FP64_TOL


def test_ksweep_2d_matches_oracle():
    """The 2D sweep (coarse L x L against a 4L x 4L reference with K = 600, 4x4
    block means, both velocity components) gives the oracle's errors; L = 16."""
    from paper_2011_06856_gb300 import ksweep
    L, kn = 16, 1.0
    steps = int(round(0.9 * L / 2))
    row = ksweep.sweep([kn], [12, 48], L=L, k_ref=600, precision="fp64", dim=2)[0]

    def beta(Lg, K, st):
        q = O.Quadrature(3, K)
        fl = W.riemann_2d(Lg, Lg, W.PAPER_SOD2D_STATES)
        f, flagged = q.run(q.init(fl.n, fl.T, fl.bx, fl.by), W.tau_from_kn(kn, Lg), st,
                           W.BC_COPYOUT, W.BC_COPYOUT)
        assert flagged == 0
        mac, _ = q.macro(f)
        return mac[4:6] / mac[3]

    bf = beta(4 * L, 600, 4 * steps)
    bref = bf.reshape(2, L, 4, L, 4).mean((2, 4))
    for K, e in zip(row["K"], row["eps"]):
        b = beta(L, K, steps)
        e_ref = np.linalg.norm(b - bref) / np.linalg.norm(bref)
        assert abs(e - e_ref) < 1e-9 * max(1.0, e_ref), (K, e, e_ref)


def test_fig5_2d_sod_k12_against_k600():
    """Sec. 3.2, Fig. 5 (t/t_max = 0.9): the 500^2, K = 12 density agrees with the
    1000^2, K = 600 one (2x2 block means) in the hydrodynamic regime and departs
    from it in the almost ballistic one (no parity: the paper prints no values)."""
    err = {}
    for kn in (0.002, 100.0):
        dens = {}
        for L, K in ((500, 12), (1000, 600)):
            fl = W.riemann_2d(L, L, W.PAPER_SOD2D_STATES)
            sim = R.Simulation(L, L, 3, K, W.tau_from_kn(kn, L), "fp32", W.BC_COPYOUT, W.BC_COPYOUT)
            sim.init_fields(fl)
            sim.autotune(2)
            sim.step(int(round(0.9 * L / 2)))
            dens[L] = sim.moments()[0]
            sim.close()
        fine = dens[1000].reshape(500, 2, 500, 2).mean((1, 3))
        err[kn] = np.linalg.norm(dens[500] - fine) / np.linalg.norm(fine)
    assert err[100.0] > 3 * err[0.002], err


def test_convergence_driver_matches_oracle():
    """Fig. 4 driver (grids 40, 80 against a 240x1, K = 600 reference, Kn = 10)
    gives the oracle's errors."""
    from paper_2011_06856_gb300 import ksweep
    Lr, grids, kn = 240, [40, 80], 10.0
    row = ksweep.convergence([kn], grids, [12, 60], L_ref=Lr, precision="fp64")[0]

    def beta(L, K):
        q = O.Quadrature(3, K)
        fl = W.shock_tube(L, 1, W.PAPER_SOD_LEFT, W.PAPER_SOD_RIGHT)
        f, _ = q.run(q.init(fl.n, fl.T, fl.bx, fl.by), W.tau_from_kn(kn, L), 9 * L // 20)
        mac, _ = q.macro(f)
        return mac[4, 0] / mac[3, 0]

    bf = beta(Lr, 600)
    for K in (12, 60):
        for L, e in zip(grids, row["eps_by_K"][str(K)]):
            bref = bf.reshape(L, Lr // L).mean(1)
            e_ref = np.linalg.norm(beta(L, K) - bref) / np.linalg.norm(bref)
            assert abs(e - e_ref) < 1e-9 * max(1.0, e_ref), (K, L, e, e_ref)

