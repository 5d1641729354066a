"""GPU parity of the two-sites-per-lane step kernel (packed f32x2 arithmetic,
64-site tiles, per-site solve once per site) against the FP64 oracle and
against the per-tile kernel, through the C ABI.

FP32 tolerance as in test_gpu_parity: 1e-5 (the per-site part runs in
double-float);
16-bit storage: the TOL of test_gpu_parity (stochastic rounding, u of the
format), and agreement with the per-tile kernel within 2e-3 (the rounding
draws differ between the kernels).
"""
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

TOL = {"fp16": 1e-3, "bf16": 8e-3, "fp16n": 1e-3, "bf16n": 8e-3}


FP32_TOL = 1e-5


def relerr(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


ES = {"fp32": 4, "fp16": 2, "bf16": 2, "fp16n": 2, "bf16n": 2}


def bulk_ok(nx, precision):
    """The bulk-staged form copies rows of whole 16-byte chunks."""
    return (nx * ES[precision]) % 16 == 0


def pair_sim(nx, ny, N, K, tau, precision, bcx, bcy, P, kind="pair"):
    sim = R.Simulation(nx, ny, N, K, tau, precision, bcx, bcy)
    sim.set_tiling(P, kind)
    assert sim.step_kernel == kind and sim.tile_populations == P
    return sim


@pytest.mark.parametrize("nx,ny,N,K,P,bcx,bcy", [
    (128, 1, 2, 16, 16, W.BC_COPYOUT, W.BC_PERIODIC),   # 1D, two full tiles
    (100, 1, 3, 64, 32, W.BC_PERIODIC, W.BC_PERIODIC),  # ragged last tile (36 of 64 sites)
    (2, 3, 2, 24, 24, W.BC_PERIODIC, W.BC_PERIODIC),    # one pair per row: both neighbours wrap
    (4, 4, 2, 24, 8, W.BC_COPYOUT, W.BC_PERIODIC),
    (66, 5, 2, 48, 16, W.BC_COPYOUT, W.BC_COPYOUT),     # 2D copy-out corners, 2 sites in the last tile
    (68, 5, 2, 48, 12, W.BC_PERIODIC, W.BC_COPYOUT),    # 4 sites in the last tile, halo wraps
    (70, 6, 3, 32, 32, W.BC_PERIODIC, W.BC_PERIODIC),   # 2D periodic wrap
    (64, 4, 2, 48, 24, W.BC_PERIODIC, W.BC_COPYOUT),
    (132, 3, 2, 24, 12, W.BC_COPYOUT, W.BC_COPYOUT),
    (196, 3, 3, 16, 8, W.BC_COPYOUT, W.BC_PERIODIC),
    (130, 1, 3, 32, 8, W.BC_PERIODIC, W.BC_PERIODIC),
    (200, 1, 2, 16, 8, W.BC_PERIODIC, W.BC_PERIODIC),   # interior tiles at x0 = 64, 128; ragged edge tile
    (256, 3, 2, 24, 12, W.BC_COPYOUT, W.BC_COPYOUT),    # interior tiles at x0 = 64, 128
    (320, 4, 3, 16, 16, W.BC_PERIODIC, W.BC_PERIODIC),
])
@pytest.mark.parametrize("kind", ["pair", "pair-bulk"])
def test_pair_kernel_fp32_matches_oracle(nx, ny, N, K, P, bcx, bcy, kind):
    if kind == "pair-bulk" and not bulk_ok(nx, "fp32"):
        pytest.skip("row pitch not a whole number of 16-byte chunks")
    steps, tau = 9, 2.5
    fl = W.random_fields(nx, ny, seed=nx + 7 * ny + K)
    q = O.Quadrature(N, K)
    f0 = q.init(fl.n, fl.T, fl.bx, fl.by)
    ref, flagged = q.run(f0, tau, steps, bcx, bcy)
    assert flagged == 0
    sim = pair_sim(nx, ny, N, K, tau, "fp32", bcx, bcy, P, kind)
    sim.init_fields(fl)
    sim.step(steps)
    got = sim.get_populations().astype(np.float64)
    assert relerr(got, ref) < FP32_TOL
    mac, _ = q.macro(ref)
    m = sim.moments()
    for k in range(4):
        assert relerr(m[k], mac[k]) < FP32_TOL, k


_STATE = {}


def shock_state_40(q):
    """The 8192x4 shock tube after 40 oracle steps at Kn = 0.1 (cached)."""
    if "s40" not in _STATE:
        nx, ny = 8192, 4
        fl = W.shock_tube(nx, ny)
        _STATE["s40"] = q.run(q.init(fl.n, fl.T, fl.bx, fl.by), W.tau_from_kn(0.1, nx), 40,
                              W.BC_COPYOUT, W.BC_PERIODIC)[0]
    return _STATE["s40"]


@pytest.mark.parametrize("P,kind", [(16, "pair"), (32, "pair"), (32, "pair-bulk"), (16, "pair-bulk"),
                                    (32, "pair-tma"), (16, "pair-tma")])
def test_pair_kernel_full_size_8192x4_one_step(P, kind):
    """The benchmark problem (8192 x 4, N=3, K=64, FP32) one step at full size."""
    nx, ny, N, K = 8192, 4, 3, 64
    tau = W.tau_from_kn(0.1, nx)
    q = O.Quadrature(N, K)
    f40 = shock_state_40(q).astype(np.float32)  # oracle state, as the FP32 buffer holds it
    sim = pair_sim(nx, ny, N, K, tau, "fp32", W.BC_COPYOUT, W.BC_PERIODIC, P, kind)
    sim.set_populations(f40, step=40)
    sim.step(1)
    got = sim.get_populations().astype(np.float64)
    ref, _ = q.run(f40.astype(np.float64), tau, 1, W.BC_COPYOUT, W.BC_PERIODIC)
    assert relerr(got, ref) < 1e-6


@pytest.mark.parametrize("precision", ["fp32", "fp16n", "bf16n", "fp16", "bf16"])
def test_pair_and_per_tile_kernels_agree(precision):
    nx, ny, N, K = 96, 7, 2, 48
    fl = W.random_fields(nx, ny, seed=5)
    out = {}
    for kind, P in (("pair", 24), ("pair", 12), ("pair-bulk", 12), ("per-tile", 24)):
        s = R.Simulation(nx, ny, N, K, 3.0, precision, W.BC_COPYOUT, W.BC_COPYOUT)
        s.set_tiling(P, kind)
        s.init_fields(fl)
        s.step(6)
        out[kind, P] = s.moments()
    tol = 1e-6 if precision == "fp32" else 2e-3
    assert relerr(out["pair", 24], out["per-tile", 24]) < tol
    assert relerr(out["pair", 12], out["per-tile", 24]) < tol
    assert relerr(out["pair-bulk", 12], out["per-tile", 24]) < tol


@pytest.mark.parametrize("kind", ["pair", "pair-bulk"])
@pytest.mark.parametrize("precision", ["fp16n", "bf16n"])
def test_pair_kernel_16bit_riemann_matches_oracle(precision, kind):
    """Four-quadrant Riemann problem, N=2 x K=48 at 96^2, Kn = 0.05, 150 steps."""
    nx = ny = 96
    N, K, steps = 2, 48, 150
    fl = W.workload_fields(W.WORKLOADS["riemann2d_2048_N2K48"], nx, ny)
    tau = W.tau_from_kn(0.05, nx)
    q = O.Quadrature(N, K)
    ref, flagged = q.run(q.init(fl.n, fl.T, fl.bx, fl.by), tau, steps, W.BC_COPYOUT, W.BC_COPYOUT)
    assert flagged == 0
    mac, _ = q.macro(ref)
    sim = pair_sim(nx, ny, N, K, tau, precision, W.BC_COPYOUT, W.BC_COPYOUT, 24, kind)
    sim.init_fields(fl)
    sim.step(steps)
    m = sim.moments()
    for k in (0, 1):  # n, eps
        assert relerr(m[k], mac[k]) <= TOL[precision], (k, relerr(m[k], mac[k]))


def test_pair_kernel_graph_replay_and_resume_are_exact():
    """32-step graph replays equal single launches bit for bit (FP32), and a
    16-bit run resumed from a checkpoint continues bit-identically (the launch
    counter that seeds the rounding is restored with the step count)."""
    nx, ny, N, K = 128, 6, 2, 16
    fl = W.random_fields(nx, ny, seed=3)
    a = pair_sim(nx, ny, N, K, 3.0, "fp32", W.BC_COPYOUT, W.BC_PERIODIC, 16)
    b = pair_sim(nx, ny, N, K, 3.0, "fp32", W.BC_COPYOUT, W.BC_PERIODIC, 16)
    a.init_fields(fl)
    b.init_fields(fl)
    a.step(40)
    for _ in range(40):
        b.step(1)
    np.testing.assert_array_equal(a.get_populations(), b.get_populations())
    c = pair_sim(nx, ny, N, K, 3.0, "fp16n", W.BC_COPYOUT, W.BC_PERIODIC, 16)
    c.init_fields(fl)
    c.step(10)
    ck = c.get_populations()
    c.step(7)
    d = pair_sim(nx, ny, N, K, 3.0, "fp16n", W.BC_COPYOUT, W.BC_PERIODIC, 16)
    d.set_populations(ck, step=10)
    d.step(7)
    np.testing.assert_array_equal(c.get_populations(), d.get_populations())


def test_pair_kernel_refused_where_it_does_not_apply():
    cases = [
        dict(nx=64, ny=2, precision="fp64", tau=2.0, P=16),          # FP64 arithmetic
        dict(nx=65, ny=2, precision="fp32", tau=2.0, P=16),          # odd row length
        dict(nx=64, ny=2, precision="fp32", tau=float("inf"), P=16),  # no collision
        dict(nx=64, ny=2, precision="fp32", tau=2.0, P=48),          # P not compiled for it
        dict(nx=64, ny=2, precision="fp32", tau=2.0, P=8),           # 18 warps: more than 16
    ]
    for c in cases:
        s = R.Simulation(c["nx"], c["ny"], 2, 48, c["tau"], c["precision"], W.BC_COPYOUT, W.BC_PERIODIC)
        with pytest.raises(R.RLBMError):
            s.set_tiling(c["P"], "pair")
        assert s.step_kernel != "pair"
        s.close()


def test_autotune_with_pair_candidates_stays_at_parity():
    nx, ny, N, K, steps, tau = 256, 4, 3, 32, 7, 2.0
    fl = W.random_fields(nx, ny, seed=31)
    q = O.Quadrature(N, K)
    f0 = q.init(fl.n, fl.T, fl.bx, fl.by).astype(np.float32)
    sim = R.Simulation(nx, ny, N, K, tau, "fp32", W.BC_COPYOUT, W.BC_PERIODIC)
    sim.set_populations(f0)
    sim.autotune(3)
    np.testing.assert_array_equal(sim.get_populations(), f0)
    sim.step(steps)
    ref, _ = q.run(f0.astype(np.float64), tau, steps, W.BC_COPYOUT, W.BC_PERIODIC)
    assert relerr(sim.get_populations().astype(np.float64), ref) < FP32_TOL
    print("autotuned:", sim.step_kernel, sim.tile_populations)


@pytest.mark.parametrize("P", [12, 16])
def test_pair_kernel_fp16n_2048sq_sampled_one_step(P):
    """The 16-bit benchmark problem at full size (2048^2, N=2 x K=48, normalised
    FP16 storage) in the benchmark's kernel: the oracle's initial state, encoded
    by this test (s = f / f_rest, rounded to FP16) and uploaded, one GPU step,
    checked on sampled rows against one oracle step of the same stored state.
    The result is stored with stochastic rounding: within 2 units of FP16
    rounding (2^-10) of the largest value, normwise."""
    nx = ny = 2048
    N, K = 2, 48
    fl = W.workload_fields(W.WORKLOADS["riemann2d_2048_N2K48"], nx, ny)
    tau = W.tau_from_kn(0.05, nx)
    q = O.Quadrature(N, K)
    frest = (q.w / (2.0 * np.pi))[:, None, None]
    raw = (q.init(fl.n, fl.T, fl.bx, fl.by) / frest).astype(np.float16)
    f0 = R.decode_populations(raw, "fp16n", q.w)
    sim = pair_sim(nx, ny, N, K, tau, "fp16n", W.BC_COPYOUT, W.BC_COPYOUT, P)
    sim.set_populations(raw)
    sim.step(1)
    got = R.decode_populations(sim.get_populations(), "fp16n", q.w)
    for y in (0, 1, 1000, 1023, 1024, 2046, 2047):
        lo, hi = max(0, y - 1), min(ny, y + 2)
        ref, _ = q.run(np.ascontiguousarray(f0[:, lo:hi, :]), tau, 1, W.BC_COPYOUT, W.BC_COPYOUT)
        assert relerr(got[:, y, :], ref[:, y - lo, :]) < 2e-3, y


# ------------------------------------------------------------ tile-staged form (TMA)

@pytest.mark.parametrize("nx,ny,N,K,P,bcx,bcy", [
    (128, 1, 2, 16, 16, W.BC_COPYOUT, W.BC_PERIODIC),   # 1D, two full tiles, right halo beyond nx
    (100, 1, 3, 64, 32, W.BC_PERIODIC, W.BC_PERIODIC),  # ragged last tile (36 of 64 sites), wrap
    (88, 5, 2, 48, 16, W.BC_COPYOUT, W.BC_COPYOUT),     # 2D copy-out corners, 24 sites in the last tile
    (136, 6, 3, 32, 32, W.BC_PERIODIC, W.BC_PERIODIC),  # 2D periodic wrap in both axes
    (200, 3, 2, 24, 12, W.BC_PERIODIC, W.BC_COPYOUT),   # pull rows in chunks of 4 populations
    (256, 4, 3, 16, 16, W.BC_COPYOUT, W.BC_PERIODIC),   # interior tiles
    (192, 2, 2, 64, 32, W.BC_COPYOUT, W.BC_COPYOUT),    # 192 populations in one centre box
])
@pytest.mark.parametrize("precision", ["fp32", "fp16n", "bf16"])
def test_pair_tma_kernel_matches_oracle(nx, ny, N, K, P, bcx, bcy, precision):
    """The tile-staged form against the FP64 oracle (FP32: 1e-5; 16-bit: the
    storage tolerance) and against the plain pair kernel (FP32: 1e-6, the
    same arithmetic; 16-bit: the storage tolerance, other rounding draws)."""
    if precision != "fp32" and nx % 8:
        pytest.skip("16-bit rows need nx a multiple of 8 (16-byte TMA pitch)")
    steps, tau = 9, 2.5
    fl = W.random_fields(nx, ny, seed=nx + 7 * ny + K)
    q = O.Quadrature(N, K)
    ref, flagged = q.run(q.init(fl.n, fl.T, fl.bx, fl.by), tau, steps, bcx, bcy)
    assert flagged == 0
    mac, _ = q.macro(ref)
    out = {}
    for kind in ("pair-tma", "pair"):
        sim = pair_sim(nx, ny, N, K, tau, precision, bcx, bcy, P, kind)
        sim.init_fields(fl)
        sim.step(steps)
        out[kind] = sim.moments()
    tol = {"fp32": FP32_TOL, "fp16n": TOL["fp16n"], "bf16": TOL["bf16"]}[precision]
    for k in range(4):
        assert relerr(out["pair-tma"][k], mac[k]) < tol, k
    assert relerr(out["pair-tma"], out["pair"]) < (1e-6 if precision == "fp32" else tol)


def test_pair_tma_refused_where_it_does_not_apply():
    cases = [
        dict(nx=66, ny=2, precision="fp32", K=48, P=16),   # row pitch not a whole number of 16-byte chunks
        dict(nx=64, ny=2, precision="fp32", K=48, P=16),   # narrower than one box (64 + 2 x 4 sites)
        dict(nx=128, ny=2, precision="fp32", K=12, P=12),  # pull rows do not chunk by sgn(v_y)
    ]
    for c in cases:
        s = R.Simulation(c["nx"], c["ny"], 3, c["K"], 2.0, c["precision"], W.BC_COPYOUT, W.BC_PERIODIC)
        with pytest.raises(R.RLBMError):
            s.set_tiling(c["P"], "pair-tma")
        assert s.step_kernel != "pair-tma"
        s.close()


def test_pair_tma_graph_replay_and_resume_are_exact():
    nx, ny, N, K = 128, 6, 2, 16
    fl = W.random_fields(nx, ny, seed=3)
    a = pair_sim(nx, ny, N, K, 3.0, "fp32", W.BC_COPYOUT, W.BC_PERIODIC, 16, "pair-tma")
    b = pair_sim(nx, ny, N, K, 3.0, "fp32", W.BC_COPYOUT, W.BC_PERIODIC, 16, "pair-tma")
    a.init_fields(fl)
    b.init_fields(fl)
    a.step(40)
    for _ in range(40):
        b.step(1)
    np.testing.assert_array_equal(a.get_populations(), b.get_populations())
    c = pair_sim(nx, ny, N, K, 3.0, "fp16n", W.BC_COPYOUT, W.BC_PERIODIC, 16, "pair-tma")
    c.init_fields(fl)
    c.step(10)
    ck = c.get_populations()
    c.step(7)
    d = pair_sim(nx, ny, N, K, 3.0, "fp16n", W.BC_COPYOUT, W.BC_PERIODIC, 16, "pair-tma")
    d.set_populations(ck, step=10)
    d.step(7)
    np.testing.assert_array_equal(c.get_populations(), d.get_populations())


@pytest.mark.parametrize("P", [12, 16])
def test_pair_tma_fp16n_2048sq_sampled_one_step(P):
    """The benchmark problem at full size in the tile-staged kernel (as
    test_pair_kernel_fp16n_2048sq_sampled_one_step)."""
    nx = ny = 2048
    N, K = 2, 48
    fl = W.workload_fields(W.WORKLOADS["riemann2d_2048_N2K48"], nx, ny)
    tau = W.tau_from_kn(0.05, nx)
    q = O.Quadrature(N, K)
    frest = (q.w / (2.0 * np.pi))[:, None, None]
    raw = (q.init(fl.n, fl.T, fl.bx, fl.by) / frest).astype(np.float16)
    f0 = R.decode_populations(raw, "fp16n", q.w)
    sim = pair_sim(nx, ny, N, K, tau, "fp16n", W.BC_COPYOUT, W.BC_COPYOUT, P, "pair-tma")
    sim.set_populations(raw)
    sim.step(1)
    got = R.decode_populations(sim.get_populations(), "fp16n", q.w)
    for y in (0, 1, 1000, 1023, 1024, 2046, 2047):
        lo, hi = max(0, y - 1), min(ny, y + 2)
        ref, _ = q.run(np.ascontiguousarray(f0[:, lo:hi, :]), tau, 1, W.BC_COPYOUT, W.BC_COPYOUT)
        assert relerr(got[:, y, :], ref[:, y - lo, :]) < 2e-3, y
