"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances (normwise, max|gpu - oracle| / max|oracle| per field; the two
spatial velocity components share the scale max |U^i|):

* FP64 storage and arithmetic: 1e-12.
* FP32 storage: 1e-5, the bound stated for the FP32 path.  Its per-site part
  (moment fold, Landau frame, equilibrium coefficients) runs at FP64-class
  accuracy; in FP32 it would carry the conserved moments to a relative bias
  of about 4e-7 per step, which the collision accumulates linearly (conserved
  quantities do not relax) and which would exceed 1e-5 within a few hundred
  steps at tau ~ 4.
* 16-bit storage with stochastic rounding: 1e-3 for n and eps with FP16
  (unit roundoff u = 2^-11), 8e-3 with BF16 (u = 2^-8); beta 3x that.
  Stochastic rounding makes the per-store error zero-mean, so conserved
  moments random-walk: about u sqrt(steps / N_pop) per site.
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

TOL = {"fp64": 1e-12, "fp32": 1e-5, "fp16": 1e-3, "bf16": 8e-3, "fp16n": 1e-3, "bf16n": 8e-3}


def relerr(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def field_errors(got, ref):
    """Normwise errors; the spatial velocity components share one scale,
    max |U^i| over both components (the rotated shells make U^y of a 1D tube
    small but not zero)."""
    errs = {k: relerr(got[i], ref[i]) for i, k in enumerate(["n", "eps", "T", "U0"])}
    uscale = max(np.abs(ref[4:6]).max(), 1e-300)
    errs["Ux"] = np.abs(got[4] - ref[4]).max() / uscale
    errs["Uy"] = np.abs(got[5] - ref[5]).max() / uscale
    bscale = max(np.abs(ref[4:6] / ref[3]).max(), 1e-300)
    errs["beta_x"] = np.abs(got[4] / got[3] - ref[4] / ref[3]).max() / bscale
    return errs


def assert_fields_close(got, ref, tol, what=""):
    errs = field_errors(got, ref)
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, f"{what}: {bad} (tol {tol})"
    return errs


def oracle_run(N, K, fields, tau, steps, bcx, bcy):
    q = O.Quadrature(N, K)
    f = q.init(fields.n, fields.T, fields.bx, fields.by)
    f, flagged = q.run(f, tau, steps, bcx, bcy)
    mac, _ = q.macro(f)
    return q, f, mac, flagged


def gpu_run(N, K, fields, tau, steps, bcx, bcy, precision="fp64"):
    ny, nx = fields.shape
    sim = R.Simulation(nx, ny, N, K, tau, precision, bcx, bcy)
    sim.init_fields(fields)
    sim.step(steps)
    return sim, sim.moments()


# ------------------------------------------------------------ FP64 parity

def test_fp64_shock_tube_400x1_full_config():
    """400x1, N=2 (3 radial nodes) x K=16 angles, Kn=0.01 -> tau = 4, 400 steps,
    copy-out in x, periodic in y: n, eps, u_x profiles vs the oracle."""
    nx, N, K, steps = 400, 2, 16, 400
    tau = W.tau_from_kn(0.01, nx)
    fl = W.shock_tube(nx, 1, (1.0, 1.0), (0.2, 0.5))
    q, f_ref, mac_ref, flagged = oracle_run(N, K, fl, tau, steps, W.BC_COPYOUT, W.BC_PERIODIC)
    assert flagged == 0
    sim, mac = gpu_run(N, K, fl, tau, steps, W.BC_COPYOUT, W.BC_PERIODIC)
    assert_fields_close(mac, mac_ref, TOL["fp64"], "fields")
    f = sim.get_populations()
    assert relerr(f, f_ref) < TOL["fp64"]
    assert sim.steps_done == steps


@pytest.mark.parametrize("nx,ny", [(1, 1), (2, 1), (3, 2), (5, 4), (33, 3)])
@pytest.mark.parametrize("bcx,bcy", [(W.BC_PERIODIC, W.BC_PERIODIC), (W.BC_COPYOUT, W.BC_COPYOUT),
                                     (W.BC_COPYOUT, W.BC_PERIODIC)])
def test_fp64_tiny_grids_random_populations(nx, ny, bcx, bcy):
    N, K, steps, tau = 2, 16, 3, 2.5
    q = O.Quadrature(N, K)
    f0 = W.random_populations(q.npop, ny, nx, seed=100 + nx * 7 + ny) * q.w[:, None, None]
    ref, flagged = q.run(f0, tau, steps, bcx, bcy)
    assert flagged == 0
    sim = R.Simulation(nx, ny, N, K, tau, "fp64", bcx, bcy)
    sim.set_populations(f0)
    sim.step(steps)
    got = sim.get_populations()
    assert relerr(got, ref) < TOL["fp64"]


@pytest.mark.parametrize("N,K", [(2, 16), (3, 12), (3, 64), (2, 48), (2, 24), (2, 20), (3, 7)])
def test_fp64_2d_ragged_random_fields(N, K):
    """Random smooth (n, T, beta) fields on a 70x37 grid (ragged x tail: 70 = 2*32 + 6),
    copy-out in both directions, 12 steps; covers every tiling the dispatcher picks."""
    nx, ny, steps, tau = 70, 37, 12, 3.0
    fl = W.random_fields(nx, ny, seed=7 + K)
    _, f_ref, mac_ref, flagged = oracle_run(N, K, fl, tau, steps, W.BC_COPYOUT, W.BC_COPYOUT)
    assert flagged == 0
    sim, mac = gpu_run(N, K, fl, tau, steps, W.BC_COPYOUT, W.BC_COPYOUT)
    assert_fields_close(mac, mac_ref, TOL["fp64"], f"N={N} K={K}")
    assert relerr(sim.get_populations(), f_ref) < TOL["fp64"]


def test_fp64_init_and_moments_recover_input_fields():
    """init then moments: the stored equilibrium carries exactly the input
    n, T, U (moment exactness of the truncated expansion, N >= 2)."""
    nx, ny = 45, 19
    fl = W.random_fields(nx, ny, seed=3, beta_max=0.6)
    sim = R.Simulation(nx, ny, 3, 64, 5.0, "fp64", W.BC_PERIODIC, W.BC_PERIODIC)
    sim.init_fields(fl)
    mac = sim.moments()
    g = 1 / np.sqrt(1 - fl.bx ** 2 - fl.by ** 2)
    np.testing.assert_allclose(mac[0], fl.n, rtol=1e-12)
    np.testing.assert_allclose(mac[2], fl.T, rtol=1e-12)
    np.testing.assert_allclose(mac[1], 2 * fl.n * fl.T, rtol=1e-12)
    np.testing.assert_allclose(mac[3], g, rtol=1e-12)
    np.testing.assert_allclose(mac[4], g * fl.bx, atol=1e-12)
    np.testing.assert_allclose(mac[5], g * fl.by, atol=1e-12)
    q = O.Quadrature(3, 64)
    assert relerr(sim.get_populations(), q.init(fl.n, fl.T, fl.bx, fl.by)) < 1e-13


def test_fp64_uniform_equilibrium_fixed_point():
    fl = W.uniform(50, 9, 0.8, 0.7, 0.3, -0.2)
    sim = R.Simulation(50, 9, 2, 16, 2.0, "fp64", W.BC_COPYOUT, W.BC_COPYOUT)
    sim.init_fields(fl)
    f0 = sim.get_populations()
    sim.step(10)
    assert relerr(sim.get_populations(), f0) < 1e-13


def binomial_site(f0_i, ax, ay, sx, sy, n, x, y):
    """Exact n-step ballistic value at one site of a periodic grid (tensor
    product of two binomial upwind operators)."""
    ny, nx = f0_i.shape
    from math import comb
    acc = 0.0
    for k in range(n + 1):
        cx = comb(n, k) * ax ** k * (1 - ax) ** (n - k)
        if cx < 1e-30:
            continue
        for l in range(n + 1):
            cy = comb(n, l) * ay ** l * (1 - ay) ** (n - l)
            if cy < 1e-30:
                continue
            acc += cx * cy * f0_i[(y - sy * l) % ny, (x - sx * k) % nx]
    return acc


def test_fp64_ballistic_binomial_sampled():
    """tau = inf: the exact discrete solution at sampled sites (computed one by one)."""
    nx, ny, N, K, steps = 200, 40, 2, 16, 60
    q = O.Quadrature(N, K)
    f0 = W.random_populations(q.npop, ny, nx, seed=5)
    sim = R.Simulation(nx, ny, N, K, math.inf, "fp64", W.BC_PERIODIC, W.BC_PERIODIC)
    sim.set_populations(f0)
    sim.step(steps)
    got = sim.get_populations()
    rng = np.random.default_rng(1)
    for _ in range(12):
        i, y, x = rng.integers(q.npop), rng.integers(ny), rng.integers(nx)
        ref = binomial_site(f0[i], abs(q.vx[i]), abs(q.vy[i]), 1 if q.vx[i] >= 0 else -1,
                            1 if q.vy[i] >= 0 else -1, steps, x, y)
        assert abs(got[i, y, x] - ref) <= 1e-12 * abs(ref)


# ------------------------------------------------------------ full-size launch configurations

_SHOCK_STATE = {}


def oracle_shock_state(steps, kn):
    """The 8192x4 N=3 K=64 shock tube after `steps` oracle steps (cached)."""
    key = (steps, kn)
    if key not in _SHOCK_STATE:
        nx, ny, N, K = 8192, 4, 3, 64
        q = O.Quadrature(N, K)
        fl = W.shock_tube(nx, ny)
        f0 = q.init(fl.n, fl.T, fl.bx, fl.by)
        _SHOCK_STATE[key] = q.run(f0, W.tau_from_kn(kn, nx), steps, W.BC_COPYOUT, W.BC_PERIODIC)[0]
    return _SHOCK_STATE[key]


def test_fp64_full_size_8192x4_one_step_parity():
    """8192x4, N=3 x K=64 (256 populations), the launch configuration the benchmark
    times: from the oracle's state after 50 steps (uploaded), one GPU step equals
    one oracle step."""
    nx, ny, N, K = 8192, 4, 3, 64
    tau = W.tau_from_kn(0.01, nx)
    f50 = oracle_shock_state(50, 0.01)
    sim = R.Simulation(nx, ny, N, K, tau, "fp64", W.BC_COPYOUT, W.BC_PERIODIC)
    sim.set_populations(f50, step=50)
    sim.step(1)
    got = sim.get_populations()
    q = O.Quadrature(N, K)
    ref, flagged = q.run(f50, tau, 1, W.BC_COPYOUT, W.BC_PERIODIC)
    assert flagged == 0
    assert relerr(got, ref) < TOL["fp64"]


@pytest.mark.parametrize("precision", ["fp32"])
def test_full_size_8192x4_one_step_parity_fp32(precision):
    nx, ny, N, K = 8192, 4, 3, 64
    tau = W.tau_from_kn(0.1, nx)
    f40 = oracle_shock_state(40, 0.1).astype(np.float32)  # the FP32 state the GPU holds
    sim = R.Simulation(nx, ny, N, K, tau, precision, W.BC_COPYOUT, W.BC_PERIODIC)
    sim.set_populations(f40, step=40)
    sim.step(1)
    got = sim.get_populations().astype(np.float64)
    q = O.Quadrature(N, K)
    ref, _ = q.run(f40.astype(np.float64), tau, 1, W.BC_COPYOUT, W.BC_PERIODIC)
    assert relerr(got, ref) < 1e-6


def test_fp64_2048sq_sampled_one_step():
    """2048^2, N=2 x K=48 at full size: one GPU step from an oracle-initialised
    random state, checked on sampled rows (the oracle steps only the rows it needs)."""
    nx = ny = 2048
    N, K, tau = 2, 48, 102.4
    fl = W.random_fields(nx, ny, seed=11)
    q = O.Quadrature(N, K)
    f0 = q.init(fl.n, fl.T, fl.bx, fl.by)
    sim = R.Simulation(nx, ny, N, K, tau, "fp64", W.BC_COPYOUT, W.BC_COPYOUT)
    sim.set_populations(f0)
    sim.step(1)
    got = sim.get_populations()
    for y in (0, 1, 777, 2046, 2047):
        lo, hi = max(0, y - 1), min(ny, y + 2)
        sub = np.ascontiguousarray(f0[:, lo:hi, :])
        # a row band with its own copy-out edges reproduces the interior row y exactly
        # when y has both neighbours inside the band or is a true boundary row
        ref, _ = q.run(sub, tau, 1, W.BC_COPYOUT, W.BC_COPYOUT)
        assert relerr(got[:, y, :], ref[:, y - lo, :]) < TOL["fp64"], y


# ------------------------------------------------------------ FP32 and 16-bit storage

def gpu_run_kernel(N, K, fields, tau, steps, bcx, bcy, precision, kernel, P):
    """gpu_run in a chosen step kernel: "default" (the handle's kernel after
    rlbm_create: TMA-staged or per-tile, FP64 per-site part for FP32 storage)
    or "pair" (two sites per lane, double-float per-site part) with P."""
    ny, nx = fields.shape
    sim = R.Simulation(nx, ny, N, K, tau, precision, bcx, bcy)
    if kernel != "default":
        sim.set_tiling(P, kernel)
    sim.init_fields(fields)
    sim.step(steps)
    return sim, sim.moments()


@pytest.mark.parametrize("kernel", ["default", "pair"])
def test_fp32_shock_tube_400x1(kernel):
    """The 400x1 shock tube (N=2 x K=16, Kn = 0.01 -> tau = 4, 400 steps) in FP32
    storage within 1e-5 of the FP64 oracle: at tau = 4 an FP32 per-site part
    would drift past 1e-5 (bias about 4e-7 per step times omega ~ 1/4)."""
    nx, N, K, steps = 400, 2, 16, 400
    tau = W.tau_from_kn(0.01, nx)
    fl = W.shock_tube(nx, 1)
    _, _, mac_ref, _ = oracle_run(N, K, fl, tau, steps, W.BC_COPYOUT, W.BC_PERIODIC)
    _, mac = gpu_run_kernel(N, K, fl, tau, steps, W.BC_COPYOUT, W.BC_PERIODIC, "fp32", kernel, 16)
    errs = assert_fields_close(mac, mac_ref, TOL["fp32"], f"fp32 400x1 {kernel}")
    print("fp32 400x1", kernel, {k: f"{v:.2e}" for k, v in errs.items()})


@pytest.mark.parametrize("kernel", ["default", "pair"])
@pytest.mark.parametrize("kn", [0.01, 0.1, 1.0, 10.0])
def test_fp32_8192x4_N3K64_reduced_steps(kn, kernel):
    """Config shape 8192x4, N=3 x K=64, each Kn, 200 steps (the full 4000 at
    Kn = 0.01 in test_gpu_configs)."""
    nx, ny, N, K, steps = 8192, 4, 3, 64, 200
    tau = W.tau_from_kn(kn, nx)
    fl = W.shock_tube(nx, ny)
    if ("mac200", kn) not in _SHOCK_STATE:
        _, _, mac_ref, flagged = oracle_run(N, K, fl, tau, steps, W.BC_COPYOUT, W.BC_PERIODIC)
        assert flagged == 0
        _SHOCK_STATE["mac200", kn] = mac_ref
    mac_ref = _SHOCK_STATE["mac200", kn]
    _, mac = gpu_run_kernel(N, K, fl, tau, steps, W.BC_COPYOUT, W.BC_PERIODIC, "fp32", kernel, 32)
    assert_fields_close(mac, mac_ref, TOL["fp32"], f"fp32 Kn={kn} {kernel}")


@pytest.mark.parametrize("precision", ["fp16", "bf16", "fp16n", "bf16n"])
def test_16bit_deviation_storage_riemann(precision):
    """Four-quadrant Riemann states (n, T) = (1,1), (0.5,0.8), (0.25,0.6), (0.5,0.8),
    jitter 1%, N=2 x K=48, Kn = 0.05 at 96^2, 150 steps, copy-out both axes."""
    nx = ny = 96
    N, K, steps = 2, 48, 150
    w = W.WORKLOADS["riemann2d_2048_N2K48"]
    fl = W.workload_fields(w, nx, ny)
    tau = W.tau_from_kn(0.05, nx)
    _, _, mac_ref, flagged = oracle_run(N, K, fl, tau, steps, W.BC_COPYOUT, W.BC_COPYOUT)
    assert flagged == 0
    _, mac = gpu_run(N, K, fl, tau, steps, W.BC_COPYOUT, W.BC_COPYOUT, precision)
    errs = field_errors(mac, mac_ref)
    print(precision, {k: f"{v:.2e}" for k, v in errs.items()})
    for k in ("n", "eps"):
        assert errs[k] <= TOL[precision], (k, errs)
    assert errs["beta_x"] <= 3 * TOL[precision], errs


# ------------------------------------------------------------ runtime behaviour

def test_graph_replay_equals_single_launches():
    fl = W.random_fields(64, 8, seed=21)
    a = R.Simulation(64, 8, 2, 16, 3.0, "fp64", W.BC_COPYOUT, W.BC_PERIODIC)
    b = R.Simulation(64, 8, 2, 16, 3.0, "fp64", W.BC_COPYOUT, W.BC_PERIODIC)
    a.init_fields(fl)
    b.init_fields(fl)
    a.step(70)  # two graph replays of 32 steps + 6 single launches
    for _ in range(70):
        b.step(1)
    np.testing.assert_array_equal(a.get_populations(), b.get_populations())
    assert a.kernel_launches == b.kernel_launches == 71


@pytest.mark.parametrize("precision", ["fp32", "fp16n", "bf16"])
def test_checkpoint_resume_is_bit_identical(precision):
    """Resume = set_populations(step) + step: equal to the uninterrupted run,
    including the stochastic rounding of 16-bit storage (seeded by the step)."""
    fl = W.shock_tube(128, 4)
    a = R.Simulation(128, 4, 3, 12, 6.0, precision, W.BC_COPYOUT, W.BC_PERIODIC)
    a.init_fields(fl)
    a.step(37)
    ck = a.get_populations()
    a.step(41)
    b = R.Simulation(128, 4, 3, 12, 6.0, precision, W.BC_COPYOUT, W.BC_PERIODIC)
    b.set_populations(ck, step=37)
    b.step(41)
    assert b.steps_done == 78
    np.testing.assert_array_equal(a.get_populations(), b.get_populations())


def test_device_entry_points_match_host_ones():
    nx, ny = 77, 5
    fl = W.random_fields(nx, ny, seed=8)
    a = R.Simulation(nx, ny, 2, 24, 4.0, "fp64", W.BC_COPYOUT, W.BC_PERIODIC)
    a.init_fields(fl)
    b = R.Simulation(nx, ny, 2, 24, 4.0, "fp64", W.BC_COPYOUT, W.BC_PERIODIC, own_buffers=True)
    dev = [torch.tensor(x, dtype=torch.float64, device="cuda").contiguous()
           for x in (fl.n, fl.T, fl.bx, fl.by)]
    with torch.cuda.stream(b.stream):
        b.init_device(*dev)
    a.step(9)
    b.step(9)
    out = torch.empty((6, ny, nx), dtype=torch.float64, device="cuda")
    b.moments_device(out)
    b.stream.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), a.moments())


def test_unphysical_state_is_reported_not_trapped():
    q = O.Quadrature(2, 16)
    f0 = W.random_populations(q.npop, 2, 8, seed=2) * q.w[:, None, None]
    f0[:, 1, 3] *= -1.0  # negative populations: no physical Landau frame at that site
    sim = R.Simulation(8, 2, 2, 16, 3.0, "fp64", W.BC_PERIODIC, W.BC_PERIODIC)
    sim.set_populations(f0)
    with pytest.raises(R.Unphysical):
        sim.moments()
    sim.set_populations(np.abs(f0))
    sim.moments()  # flag was cleared
    sim.step(2)
    sim.sync()


def test_many_handles_and_unsupported_order():
    with pytest.raises(R.RLBMError) as e:
        R.Simulation(16, 1, 6, 16, 1.0)
    assert e.value.status == R.ERR_UNSUPPORTED
    sims = [R.Simulation(32, 2, 2, 16, 2.0, "fp32") for _ in range(8)]
    for s in sims:
        s.close()


# ------------------------------------------------------------ both step kernels

@pytest.fixture(params=["tma", "per_tile"])
def kernel_variant(request, monkeypatch):
    if request.param == "per_tile":
        monkeypatch.setenv("RLBM_NO_TMA", "1")
    else:
        monkeypatch.delenv("RLBM_NO_TMA", raising=False)
    return request.param


@pytest.mark.parametrize("nx,ny,N,K,bcx,bcy", [
    (96, 1, 2, 16, W.BC_COPYOUT, W.BC_PERIODIC),     # 1D, three tiles
    (100, 1, 3, 64, W.BC_PERIODIC, W.BC_PERIODIC),   # ragged last tile
    (64, 5, 2, 24, W.BC_COPYOUT, W.BC_COPYOUT),      # 2D copy-out corners
    (72, 6, 3, 12, W.BC_PERIODIC, W.BC_PERIODIC),    # 2D periodic wrap
    (40, 3, 2, 24, W.BC_PERIODIC, W.BC_COPYOUT),
])
def test_fp64_both_kernels_match_oracle(kernel_variant, nx, ny, N, K, bcx, bcy):
    steps, tau = 9, 2.5
    fl = W.random_fields(nx, ny, seed=nx + ny + K)
    _, f_ref, _, flagged = oracle_run(N, K, fl, tau, steps, bcx, bcy)
    assert flagged == 0
    sim = R.Simulation(nx, ny, N, K, tau, "fp64", bcx, bcy)
    assert sim.uses_tma == (kernel_variant == "tma")
    sim.init_fields(fl)
    sim.step(steps)
    assert relerr(sim.get_populations(), f_ref) < TOL["fp64"]


@pytest.mark.parametrize("precision", ["fp32", "fp16n", "bf16n", "fp16", "bf16"])
def test_both_kernels_agree_for_every_storage(precision):
    """The TMA-staged and the per-tile kernel compute the same arithmetic in the
    same order: equal results for every storage type (2D, copy-out)."""
    import os
    nx, ny, N, K = 96, 7, 2, 48
    fl = W.random_fields(nx, ny, seed=5)
    out = {}
    for v in ("tma", "per_tile"):
        if v == "per_tile":
            os.environ["RLBM_NO_TMA"] = "1"
        try:
            s = R.Simulation(nx, ny, N, K, 3.0, precision, W.BC_COPYOUT, W.BC_COPYOUT)
            assert s.uses_tma == (v == "tma")
            s.init_fields(fl)
            s.step(6)
            out[v] = s.moments()
        finally:
            os.environ.pop("RLBM_NO_TMA", None)
    # same formulas; 16-bit stores may round one unit apart where contraction differs
    assert relerr(out["tma"], out["per_tile"]) < (1e-6 if precision == "fp32" else 2e-3)


def test_autotuned_tiling_matches_oracle():
    """The autotuner may pick any compiled tiling; the result stays at parity
    and the state it was tuned on is unchanged."""
    nx, ny, N, K, steps, tau = 128, 6, 2, 48, 7, 2.0
    fl = W.random_fields(nx, ny, seed=12)
    q = O.Quadrature(N, K)
    f0 = q.init(fl.n, fl.T, fl.bx, fl.by)
    sim = R.Simulation(nx, ny, N, K, tau, "fp64", W.BC_COPYOUT, W.BC_PERIODIC)
    sim.set_populations(f0)
    ms = sim.autotune(3)
    assert ms > 0 and sim.tile_populations in (8, 12, 16, 24, 32, 48, 64)
    np.testing.assert_array_equal(sim.get_populations(), f0)
    sim.step(steps)
    ref, _ = q.run(f0, tau, steps, W.BC_COPYOUT, W.BC_PERIODIC)
    assert relerr(sim.get_populations(), ref) < TOL["fp64"]
    # a second handle of the same problem reuses the cached choice
    sim2 = R.Simulation(nx, ny, N, K, tau, "fp64", W.BC_COPYOUT, W.BC_PERIODIC)
    sim2.init_fields(fl)
    sim2.autotune(3)
    assert (sim2.tile_populations, sim2.uses_tma) == (sim.tile_populations, sim.uses_tma)
