"""CPU checks of the C ABI: the library builds, loads and exports every symbol
declared in include/rlbm.h; host-only entry points (quadrature tables,
buffer sizes, argument validation) behave as documented.  No compute call
needs a GPU here."""
import math
import os
import re
import subprocess

import numpy as np
import pytest

import oracle as O
from paper_2011_06856_gb300 import build as B
from paper_2011_06856_gb300 import rlbm as R

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return R.lib()


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names.update(re.findall(r"\b(rlbm_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for s in ["rlbm_create", "rlbm_init", "rlbm_step", "rlbm_moments", "rlbm_destroy"]:
        assert s in syms
    assert set(syms) <= set(R.EXPORTS) | set(syms)


def test_library_exports_every_declared_symbol(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", R.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (rlbm_[a-z0-9_]+)", out))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing
    for s in declared_symbols():
        assert hasattr(lib, s)


def test_binding_covers_every_declared_symbol():
    assert set(declared_symbols()) == set(R.EXPORTS)


@pytest.mark.parametrize("N,K", [(2, 16), (3, 64), (2, 48), (3, 12), (5, 12), (2, 5)])
def test_library_quadrature_matches_oracle(lib, N, K):
    """Row a0 (Sec. 2.3): the library's host tables, computed by a different
    root finder (Sturm bisection on the Jacobi matrix), equal the oracle's."""
    p0, vx, vy, w = R.quadrature(N, K)
    q = O.Quadrature(N, K)
    np.testing.assert_allclose(p0, q.p0, rtol=2e-15)
    np.testing.assert_allclose(w, q.w, rtol=1e-13)
    np.testing.assert_allclose(vx, q.vx, atol=2e-16)
    np.testing.assert_allclose(vy, q.vy, atol=2e-16)


def test_quadrature_rejects_bad_order(lib):
    n = 6
    bufs = [np.zeros(n) for _ in range(4)]
    with pytest.raises(R.RLBMError) as e:
        R._check(lib.rlbm_quadrature(3, 6, *[R._dptr(b) for b in bufs]))
    assert e.value.status == R.ERR_ARG


def test_population_bytes(lib):
    g = R.Grid(400, 1, 1, 0)
    assert lib.rlbm_population_bytes(g, 2, 16, 0) == 48 * 400 * 8
    assert lib.rlbm_population_bytes(R.Grid(2048, 2048, 1, 1), 2, 48, 2) == 144 * 2048 * 2048 * 2
    assert lib.rlbm_population_bytes(R.Grid(0, 1, 0, 0), 2, 16, 0) == 0


@pytest.mark.parametrize("args,needle", [
    ((R.Grid(0, 1, 0, 0), 2, 16, 1.0, 0), "grid"),
    ((R.Grid(8, 1, 0, 0), 1, 16, 1.0, 0), "order N"),
    ((R.Grid(8, 1, 0, 0), 3, 6, 1.0, 0), "K must be"),
    ((R.Grid(8, 1, 0, 0), 2, 16, -1.0, 0), "tau"),
    ((R.Grid(8, 1, 0, 0), 2, 16, float("nan"), 0), "tau"),
    ((R.Grid(8, 1, 3, 0), 2, 16, 1.0, 0), "boundary"),
    ((R.Grid(8, 1, 0, 0), 2, 16, 1.0, 9), "precision"),
])
def test_create_validates_arguments_without_touching_the_gpu(lib, args, needle):
    h = R._vp()
    st = lib.rlbm_create(R.ctypes.byref(h), *args, None, None, 0)
    assert st == R.ERR_ARG
    assert not h.value
    assert needle in lib.rlbm_last_error(None).decode()


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.rlbm_step(None, 1) == R.ERR_ARG
    assert lib.rlbm_sync(None) == R.ERR_ARG
    assert lib.rlbm_steps_done(None) == -1
    lib.rlbm_destroy(None)


def test_binding_fails_loudly_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(RuntimeError):
        R.Simulation(8, 1, 2, 16, 1.0)


def test_batch_arena_and_validation(lib):
    probs = [(100, 1, 1, 0, 16, 4.0), (64, 3, 1, 1, 48, 2.0)]
    arr = R.problems_array(probs)
    want = sum((2 * K * 3 * nx * ny * 4 + 255) // 256 * 256 for (nx, ny, _, _, K, _) in probs)
    assert lib.rlbm_batch_arena_bytes(arr, 2, 2, 1) == want
    h = R._vp()
    # N = 3 has no 6-warp batched tiling; K > 64 neither; bad tau is an argument error
    assert lib.rlbm_batch_create(R.ctypes.byref(h), arr, 2, 3, 1, None, None, 0) == R.ERR_UNSUPPORTED
    bad = R.problems_array([(100, 1, 1, 0, 96, 4.0)])
    assert lib.rlbm_batch_create(R.ctypes.byref(h), bad, 1, 2, 1, None, None, 0) == R.ERR_UNSUPPORTED
    bad = R.problems_array([(100, 1, 1, 0, 16, -1.0)])
    assert lib.rlbm_batch_create(R.ctypes.byref(h), bad, 1, 2, 1, None, None, 0) == R.ERR_ARG
    assert lib.rlbm_batch_create(R.ctypes.byref(h), arr, 2, 2, 2, None, None, 0) == R.ERR_UNSUPPORTED
    assert not h.value


def test_quantum_phi_matches_oracle(lib):
    """The kernels' Fermi-Dirac / Bose-Einstein integrals phi_s (rlbm_stat.cuh,
    compiled into the host library) against the oracle's integral definition."""
    from oracle import statistics as S
    worst = 0.0
    for s in range(1, 7):
        for z in (1e-6, 0.02, 0.4, 0.5, 0.6, 0.95, 1.0, 3.0, 80.0, 1e5):
            for stat in (S.FD, S.BE):
                if stat == S.BE and z >= 1.0:
                    continue
                got = R.quantum_phi(s, z, "fd" if stat == S.FD else "be")
                ref = S.phi(s, z, stat)
                worst = max(worst, abs(got - ref) / abs(ref))
    assert worst < 1e-13, worst
    assert math.isnan(lib.rlbm_quantum_phi(2, 0.1, -1))  # Bose-Einstein needs z < 1
    assert math.isnan(lib.rlbm_quantum_phi(9, -0.1, 1))


def test_quantum_solve_matches_oracle(lib):
    """The kernels' (eta, T) solve (FP32 Newton steps from the start, then FP64
    Newton steps to the storage's stopping rule; rlbm_stat.cuh compiled into the
    host library) against the oracle's bracketed root of the same equations
    (scipy's Brent method on the integral definition of phi), from a cold start
    and from a start near the root (the previous step's eta in the kernels).
    FP64 rule within 1e-12.  FP32-storage rule within 1e-9: it accepts a Newton
    step below 1e-5 (1 + |eta|), and a cold Bose-Einstein start (no FP32 steps
    for that statistic) can accept one near that size, leaving an error of its
    square order (2.5e-10 measured), far below the FP32 rounding of 6e-8."""
    from oracle import statistics as S
    worst = {"fp64": 0.0, "fp32": 0.0}
    cases = 0
    for stat in (S.FD, S.BE):
        for n in (0.05, 1.0, 7.0):
            for ratio in (2.0005, 2.01, 2.3, 3.0, 10.0, 100.0):
                for g in (0.1, 1.0, 4.0):
                    e = ratio * n ** 1.5
                    try:
                        T_ref, z_ref = S.solve_Tz(n, e, stat, g)
                    except ValueError:  # no equilibrium of this statistic
                        continue
                    eta_ref = math.log(z_ref)
                    for storage in ("fp64", "fp32"):
                        for eta0 in (float("nan"), eta_ref + 1e-3):
                            eta, T, ok = R.quantum_solve(n, e, g, "fd" if stat == S.FD else "be", eta0, storage)
                            assert ok, (stat, n, ratio, g, storage)
                            err = max(abs(eta - eta_ref) / (1.0 + abs(eta_ref)), abs(T - T_ref) / T_ref)
                            worst[storage] = max(worst[storage], err)
                            cases += 1
    assert cases > 100
    assert worst["fp64"] < 1e-12 and worst["fp32"] < 1e-9, worst
    # no equilibrium: Bose-Einstein beyond condensation (with g = 1, e / n^1.5 below
    # 2 zeta(3) / (zeta(2)^1.5 sqrt(2 pi)) = 0.455), bad input
    with pytest.raises(ValueError):
        S.solve_Tz(1.0, 0.3, S.BE, 1.0)
    eta, T, ok = R.quantum_solve(1.0, 0.3, 1.0, "be")
    assert not ok
    assert R.quantum_solve(1.0, 0.5, 1.0, "be")[2]
    assert R.quantum_solve(-1.0, 2.0, 1.0, "fd")[2] is False
    assert lib.rlbm_quantum_solve(1.0, 2.0, 1.0, 2, float("nan"), 0, R.ctypes.byref(R.ctypes.c_double()),
                                  R.ctypes.byref(R.ctypes.c_double())) == 0


@pytest.mark.parametrize("args,status,needle", [
    ((R.Grid(8, 1, 0, 0), 6, 16, 1.0, 0), R.ERR_UNSUPPORTED, "N = 2..5"),
    ((R.Grid(8, 1, 0, 0), 5, 10, 1.0, 0), R.ERR_ARG, "K must be"),
    ((R.Grid(8, 1, 0, 0), 3, 600, 1.0, 2), R.ERR_UNSUPPORTED, "population groups"),
    ((R.Grid(8, 1, 0, 0), 2, 400, 1.0, 3), R.ERR_UNSUPPORTED, "population groups"),
])
def test_create_refuses_unbuilt_forms_without_touching_the_gpu(lib, args, status, needle):
    """N > 5, and K beyond one population group per warp in 16-bit storage."""
    h = R._vp()
    assert lib.rlbm_create(R.ctypes.byref(h), *args, None, None, 0) == status
    assert not h.value
    assert needle in lib.rlbm_last_error(None).decode()


def test_onlattice_and_statistics_validation_without_gpu(lib):
    h = R._vp()
    for prec in (2, 3, 4, 5):  # the 16-bit forms
        assert lib.rlbm_create_onlattice(R.ctypes.byref(h), R.Grid(8, 8, 0, 0), 2.0, prec, None, None, 0) \
            == R.ERR_UNSUPPORTED
        assert "FP32 and FP64" in lib.rlbm_last_error(None).decode()
    assert lib.rlbm_create_onlattice(R.ctypes.byref(h), R.Grid(0, 8, 0, 0), 2.0, 0, None, None, 0) == R.ERR_ARG
    assert lib.rlbm_create_onlattice(R.ctypes.byref(h), R.Grid(8, 8, 0, 0), -1.0, 0, None, None, 0) == R.ERR_ARG
    assert not h.value
    assert lib.rlbm_set_statistics(None, 1, 1.0) == R.ERR_ARG
    assert lib.rlbm_statistics(None) == -2
    assert lib.rlbm_is_onlattice(None) == -1
    assert lib.rlbm_population_groups(None) == -1


def test_noalloc_binding_checks_tensors_before_any_launch():
    """The allocation-free step cannot see buffer sizes on the C side: the
    binding refuses a wrong dtype, a wrong element count, a non-contiguous
    tensor or host memory before it calls into the library (no GPU needed)."""
    torch = pytest.importorskip("torch")
    from paper_2011_06856_gb300 import rlbm as R
    nx, ny, N, K = 8, 2, 2, 16
    count = K * (N + 1) * nx * ny
    good = torch.zeros(count, dtype=torch.float32)
    cases = [
        (torch.zeros(count, dtype=torch.float64), good, "dtype"),
        (torch.zeros(count - 1, dtype=torch.float32), good, "elements"),
        (torch.zeros(2 * count, dtype=torch.float32)[::2], good, "contiguous"),
        (good, good.clone(), "CUDA"),
    ]
    for fin, fout, needle in cases:
        with pytest.raises(R.RLBMError) as e:
            R.step_noalloc(nx, ny, N, K, 1.0, "fp32", fin, fout)
        assert e.value.status == R.ERR_ARG and needle in str(e.value), (needle, str(e.value))
    with pytest.raises(R.RLBMError) as e:
        R.step_noalloc(nx, ny, N, K, 1.0, "fp16", good, good.clone())
    assert e.value.status == R.ERR_UNSUPPORTED
