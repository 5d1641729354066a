"""ctypes binding of librlbm.so (C ABI in include/rlbm.h).

Argument marshalling only: every step of the method runs in the CUDA library.
PyTorch supplies device memory (the population buffers, device-side fields)
and the CUDA stream.  There is no CPU fallback: if the library is missing or
no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librlbm.so")

OK, ERR_ARG, ERR_CUDA, ERR_OOM, ERR_UNPHYSICAL, ERR_TIMEOUT, ERR_UNSUPPORTED = range(7)

# fp16 / bf16: s = f / f^rest - 1 (deviation from the rest equilibrium at n = 1, T = 1);
# fp16n / bf16n: s = f / f^rest (normalised); f^rest_i = w_i / (2 pi).
PRECISIONS = {"fp64": 0, "fp32": 1, "fp16": 2, "bf16": 3, "fp16n": 4, "bf16n": 5}
STORAGE_BYTES = {"fp64": 8, "fp32": 4, "fp16": 2, "bf16": 2, "fp16n": 2, "bf16n": 2}
BC_PERIODIC, BC_COPYOUT = 0, 1

# Symbols declared in include/rlbm.h (checked by the CPU test suite).
EXPORTS = [
    "rlbm_quadrature", "rlbm_population_bytes", "rlbm_create", "rlbm_create_onlattice",
    "rlbm_is_onlattice", "rlbm_set_statistics", "rlbm_statistics", "rlbm_quantum_phi", "rlbm_quantum_solve",
    "rlbm_destroy",
    "rlbm_last_error", "rlbm_init", "rlbm_init_device", "rlbm_step", "rlbm_moments",
    "rlbm_moments_device", "rlbm_get_populations", "rlbm_set_populations",
    "rlbm_current_buffer", "rlbm_steps_done", "rlbm_sync", "rlbm_kernel_launches",
    "rlbm_step_kernel_variant", "rlbm_set_wait_limit", "rlbm_test_stall_next_step",
    "rlbm_tile_populations", "rlbm_population_groups", "rlbm_autotune", "rlbm_set_tiling",
    "rlbm_batch_arena_bytes", "rlbm_batch_create", "rlbm_batch_destroy", "rlbm_batch_last_error",
    "rlbm_batch_count", "rlbm_batch_problem", "rlbm_batch_step", "rlbm_batch_sync",
    "rlbm_batch_kernel_launches", "rlbm_batch_autotune", "rlbm_batch_set_wait_limit",
    "rlbm_batch_test_stall_next_step", "rlbm_step_noalloc", "rlbm_noalloc_last_error",
    "rlbm_closure_create", "rlbm_closure_destroy", "rlbm_closure_last_error",
    "rlbm_closure_param_count", "rlbm_closure_get_params", "rlbm_closure_set_params",
    "rlbm_closure_features", "rlbm_closure_target", "rlbm_closure_restrict",
    "rlbm_closure_forward", "rlbm_closure_work_floats", "rlbm_closure_gradient",
    "rlbm_closure_train_step", "rlbm_closure_apply_buffer", "rlbm_closure_set_apply_path", "rlbm_closure_set_train_path", "rlbm_batch_set_mode", "rlbm_batch_mode",
]


class RLBMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"[rlbm status {status}] {msg}")
        self.status = status


class Unphysical(RLBMError):
    pass


class DeviceTimeout(RLBMError):
    pass


class Problem(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("bc_x", ctypes.c_int),
                ("bc_y", ctypes.c_int), ("angles_K", ctypes.c_int), ("tau", ctypes.c_double)]


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("bc_x", ctypes.c_int),
                ("bc_y", ctypes.c_int)]


_dp = ctypes.POINTER(ctypes.c_double)
_vp = ctypes.c_void_p
_lib = None


def lib(path: str = LIB_PATH):
    """Load librlbm.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -m paper_2011_06856_gb300.build`")
    L = ctypes.CDLL(path)
    st = ctypes.c_int
    L.rlbm_quadrature.restype = st
    L.rlbm_quadrature.argtypes = [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp]
    L.rlbm_population_bytes.restype = ctypes.c_size_t
    L.rlbm_population_bytes.argtypes = [Grid, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.rlbm_create.restype = st
    L.rlbm_create.argtypes = [ctypes.POINTER(_vp), Grid, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                              ctypes.c_int, _vp, _vp, ctypes.c_size_t]
    L.rlbm_create_onlattice.restype = st
    L.rlbm_create_onlattice.argtypes = [ctypes.POINTER(_vp), Grid, ctypes.c_double, ctypes.c_int, _vp, _vp,
                                        ctypes.c_size_t]
    L.rlbm_is_onlattice.restype = ctypes.c_int
    L.rlbm_is_onlattice.argtypes = [_vp]
    L.rlbm_set_statistics.restype = st
    L.rlbm_set_statistics.argtypes = [_vp, ctypes.c_int, ctypes.c_double]
    L.rlbm_statistics.restype = ctypes.c_int
    L.rlbm_statistics.argtypes = [_vp]
    L.rlbm_quantum_phi.restype = ctypes.c_double
    L.rlbm_quantum_phi.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int]
    L.rlbm_quantum_solve.restype = ctypes.c_int
    L.rlbm_quantum_solve.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                     ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double)]
    L.rlbm_destroy.restype = None
    L.rlbm_destroy.argtypes = [_vp]
    L.rlbm_last_error.restype = ctypes.c_char_p
    L.rlbm_last_error.argtypes = [_vp]
    L.rlbm_init.restype = st
    L.rlbm_init.argtypes = [_vp, _dp, _dp, _dp, _dp]
    L.rlbm_init_device.restype = st
    L.rlbm_init_device.argtypes = [_vp, _vp, _vp, _vp, _vp]
    L.rlbm_step.restype = st
    L.rlbm_step.argtypes = [_vp, ctypes.c_int]
    L.rlbm_moments.restype = st
    L.rlbm_moments.argtypes = [_vp] + [_dp] * 6
    L.rlbm_moments_device.restype = st
    L.rlbm_moments_device.argtypes = [_vp] + [_vp] * 6
    L.rlbm_get_populations.restype = st
    L.rlbm_get_populations.argtypes = [_vp, _vp, ctypes.c_size_t]
    L.rlbm_set_populations.restype = st
    L.rlbm_set_populations.argtypes = [_vp, _vp, ctypes.c_size_t, ctypes.c_longlong]
    L.rlbm_current_buffer.restype = _vp
    L.rlbm_current_buffer.argtypes = [_vp]
    L.rlbm_steps_done.restype = ctypes.c_longlong
    L.rlbm_steps_done.argtypes = [_vp]
    L.rlbm_sync.restype = st
    L.rlbm_sync.argtypes = [_vp]
    L.rlbm_kernel_launches.restype = ctypes.c_longlong
    L.rlbm_kernel_launches.argtypes = [_vp]
    L.rlbm_step_kernel_variant.restype = ctypes.c_int
    L.rlbm_step_kernel_variant.argtypes = [_vp]
    L.rlbm_set_wait_limit.restype = st
    L.rlbm_set_wait_limit.argtypes = [_vp, ctypes.c_longlong]
    L.rlbm_test_stall_next_step.restype = st
    L.rlbm_test_stall_next_step.argtypes = [_vp]
    L.rlbm_tile_populations.restype = ctypes.c_int
    L.rlbm_tile_populations.argtypes = [_vp]
    L.rlbm_population_groups.restype = ctypes.c_int
    L.rlbm_population_groups.argtypes = [_vp]
    L.rlbm_set_tiling.restype = st
    L.rlbm_set_tiling.argtypes = [_vp, ctypes.c_int, ctypes.c_int]
    L.rlbm_autotune.restype = st
    L.rlbm_autotune.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_float)]
    _pp = ctypes.POINTER(Problem)
    L.rlbm_batch_arena_bytes.restype = ctypes.c_size_t
    L.rlbm_batch_arena_bytes.argtypes = [_pp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.rlbm_batch_create.restype = st
    L.rlbm_batch_create.argtypes = [ctypes.POINTER(_vp), _pp, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_int, _vp, _vp, ctypes.c_size_t]
    L.rlbm_batch_destroy.restype = None
    L.rlbm_batch_destroy.argtypes = [_vp]
    L.rlbm_batch_last_error.restype = ctypes.c_char_p
    L.rlbm_batch_last_error.argtypes = [_vp]
    L.rlbm_batch_count.restype = ctypes.c_int
    L.rlbm_batch_count.argtypes = [_vp]
    L.rlbm_batch_problem.restype = _vp
    L.rlbm_batch_problem.argtypes = [_vp, ctypes.c_int]
    L.rlbm_batch_step.restype = st
    L.rlbm_batch_step.argtypes = [_vp, ctypes.c_int]
    L.rlbm_batch_sync.restype = st
    L.rlbm_batch_sync.argtypes = [_vp]
    L.rlbm_batch_kernel_launches.restype = ctypes.c_longlong
    L.rlbm_batch_kernel_launches.argtypes = [_vp]
    L.rlbm_batch_autotune.restype = st
    L.rlbm_batch_autotune.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_float)]
    L.rlbm_batch_set_wait_limit.restype = st
    L.rlbm_batch_set_wait_limit.argtypes = [_vp, ctypes.c_longlong]
    L.rlbm_batch_test_stall_next_step.restype = st
    L.rlbm_batch_test_stall_next_step.argtypes = [_vp]
    L.rlbm_step_noalloc.restype = st
    L.rlbm_step_noalloc.argtypes = [Grid, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                    _vp, _vp, _vp]
    L.rlbm_noalloc_last_error.restype = ctypes.c_char_p
    L.rlbm_noalloc_last_error.argtypes = []
    ll, fp = ctypes.c_longlong, ctypes.POINTER(ctypes.c_float)
    L.rlbm_closure_create.restype = st
    L.rlbm_closure_create.argtypes = [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_int,
                                      ctypes.c_ulonglong, _vp]
    L.rlbm_closure_destroy.restype = None
    L.rlbm_closure_destroy.argtypes = [_vp]
    L.rlbm_closure_last_error.restype = ctypes.c_char_p
    L.rlbm_closure_last_error.argtypes = [_vp]
    L.rlbm_closure_param_count.restype = ctypes.c_size_t
    L.rlbm_closure_param_count.argtypes = [_vp]
    L.rlbm_closure_get_params.restype = st
    L.rlbm_closure_get_params.argtypes = [_vp, fp, ctypes.c_size_t]
    L.rlbm_closure_set_params.restype = st
    L.rlbm_closure_set_params.argtypes = [_vp, fp, ctypes.c_size_t]
    L.rlbm_closure_features.restype = st
    L.rlbm_closure_features.argtypes = [_vp, _vp, ll, ctypes.c_double, _vp, ll, ll]
    L.rlbm_closure_target.restype = st
    L.rlbm_closure_target.argtypes = [_vp, _vp, _vp, ll, _vp, ll, ll]
    L.rlbm_closure_restrict.restype = st
    L.rlbm_closure_restrict.argtypes = [_vp, ctypes.c_int, _vp, ll, _vp]
    L.rlbm_closure_forward.restype = st
    L.rlbm_closure_forward.argtypes = [_vp, _vp, ll, ll, ctypes.c_int, _vp]
    L.rlbm_closure_work_floats.restype = ctypes.c_size_t
    L.rlbm_closure_work_floats.argtypes = [_vp, ll]
    L.rlbm_closure_gradient.restype = st
    L.rlbm_closure_gradient.argtypes = [_vp, _vp, _vp, ll, ll, ctypes.c_int, _vp, fp, fp]
    L.rlbm_closure_train_step.restype = st
    L.rlbm_closure_train_step.argtypes = [_vp, _vp, _vp, ll, ll, ctypes.c_int, ctypes.c_float,
                                          _vp, fp]
    L.rlbm_closure_apply_buffer.restype = st
    L.rlbm_closure_apply_buffer.argtypes = [_vp, _vp, ll, ctypes.c_double]
    L.rlbm_batch_set_mode.restype = st
    L.rlbm_batch_set_mode.argtypes = [_vp, ctypes.c_int]
    L.rlbm_batch_mode.restype = ctypes.c_int
    L.rlbm_batch_mode.argtypes = [_vp]
    L.rlbm_closure_set_train_path.restype = st
    L.rlbm_closure_set_train_path.argtypes = [_vp, ctypes.c_int]
    L.rlbm_closure_set_apply_path.restype = st
    L.rlbm_closure_set_apply_path.argtypes = [_vp, ctypes.c_int]
    _lib = L
    return L


def _check(status: int, handle=None):
    if status == OK:
        return
    msg = lib().rlbm_last_error(handle).decode(errors="replace")
    cls = {ERR_UNPHYSICAL: Unphysical, ERR_TIMEOUT: DeviceTimeout}.get(status, RLBMError)
    raise cls(status, msg)


def _dptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def quadrature(N: int, K: int):
    """(p0, vx, vy, w) of the off-lattice rule, computed by the library."""
    n = K * (N + 1)
    out = [np.zeros(n) for _ in range(4)]
    _check(lib().rlbm_quadrature(N, K, *[_dptr(a) for a in out]))
    return tuple(out)


def quantum_phi(s: int, z: float, statistics: str) -> float:
    """phi_s(z) as the kernels evaluate it (rlbm_quantum_phi): -Li_s(-z) for 'fd',
    Li_s(z) for 'be'; runs on the host."""
    import math
    return lib().rlbm_quantum_phi(int(s), math.log(z), {"fd": 1, "be": -1}[statistics])


def quantum_solve(n: float, e: float, g: float, statistics: str, eta0: float = float("nan"),
                  storage: str = "fp64"):
    """(eta, T, ok) of the equilibrium with density n and energy density e, as the
    kernels solve it (rlbm_quantum_solve; storage 'fp32' selects the FP32-storage
    stopping rule); runs on the host."""
    eta = ctypes.c_double()
    T = ctypes.c_double()
    ok = lib().rlbm_quantum_solve(float(n), float(e), float(g), {"fd": 1, "be": -1}[statistics], float(eta0),
                                  1 if storage == "fp32" else 0, ctypes.byref(eta), ctypes.byref(T))
    return eta.value, T.value, bool(ok)


def population_bytes(nx, ny, N, K, precision="fp64", bcx=BC_COPYOUT, bcy=BC_PERIODIC) -> int:
    return lib().rlbm_population_bytes(Grid(nx, ny, bcx, bcy), N, K, PRECISIONS[precision])


class Simulation:
    """One RLBM problem on the current CUDA device.

    The population buffers are a torch uint8 tensor (two ping-pong halves)
    unless ``own_buffers`` is set, in which case the library allocates them."""

    def __init__(self, nx: int, ny: int, N: int, K: int, tau: float, precision: str = "fp64",
                 bcx: int = BC_COPYOUT, bcy: int = BC_PERIODIC, stream=None,
                 own_buffers: bool = False, onlattice: bool = False):
        """onlattice: the on-lattice rule of Sec. 2.3 (rlbm_create_onlattice;
        needs N = 3, and K is set to its 12 stencil vectors)."""
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("librlbm needs a CUDA GPU")
        if onlattice:
            if int(N) != 3:
                raise ValueError("the on-lattice rule has order N = 3")
            K = 12
        self.onlattice = bool(onlattice)
        self.nx, self.ny, self.N, self.K = int(nx), int(ny), int(N), int(K)
        self.npop = self.K * (self.N + 1)
        self.precision = precision
        self.tau = float(tau)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        grid = Grid(self.nx, self.ny, bcx, bcy)
        self.pop_bytes = lib().rlbm_population_bytes(grid, self.N, self.K, PRECISIONS[precision])
        self._buf = None
        ptr, nbytes = None, 0
        if not own_buffers:
            self._buf = torch.empty(2 * self.pop_bytes, dtype=torch.uint8, device="cuda")
            ptr, nbytes = self._buf.data_ptr(), 2 * self.pop_bytes
        h = _vp()
        if onlattice:
            status = lib().rlbm_create_onlattice(ctypes.byref(h), grid, self.tau, PRECISIONS[precision],
                                                 _vp(self.stream.cuda_stream), _vp(ptr), nbytes)
        else:
            status = lib().rlbm_create(ctypes.byref(h), grid, self.N, self.K, self.tau,
                                       PRECISIONS[precision], _vp(self.stream.cuda_stream), _vp(ptr),
                                       nbytes)
        _check(status, None)
        self._h = h

    # ---- lifetime
    def close(self):
        if getattr(self, "_h", None):
            lib().rlbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---- API
    @property
    def sites(self) -> int:
        return self.nx * self.ny

    def init(self, n, T, bx, by):
        """Equilibrium state from host fields ([ny][nx] float64 each)."""
        arrs = [np.ascontiguousarray(a, dtype=np.float64).reshape(-1) for a in (n, T, bx, by)]
        for a in arrs:
            assert a.size == self.sites
        _check(lib().rlbm_init(self._h, *[_dptr(a) for a in arrs]), self._h)

    def init_fields(self, fields):
        self.init(fields.n, fields.T, fields.bx, fields.by)

    def init_device(self, n, T, bx, by):
        """Equilibrium state from device float64 tensors (asynchronous)."""
        for t in (n, T, bx, by):
            assert t.is_cuda and t.is_contiguous() and t.numel() == self.sites
        _check(lib().rlbm_init_device(self._h, *[_vp(t.data_ptr()) for t in (n, T, bx, by)]),
               self._h)

    def step(self, nsteps: int = 1):
        _check(lib().rlbm_step(self._h, int(nsteps)), self._h)

    def moments(self) -> np.ndarray:
        """(6, ny, nx) float64: n, eps, T, U^0, U^x, U^y of the stored populations."""
        out = np.zeros((6, self.ny, self.nx))
        _check(lib().rlbm_moments(self._h, *[_dptr(out[k]) for k in range(6)]), self._h)
        return out

    def moments_device(self, out):
        """Write the six fields into a contiguous (6, ny, nx) float64 CUDA tensor."""
        assert out.is_cuda and out.is_contiguous() and out.numel() == 6 * self.sites
        S = self.sites
        base = out.data_ptr()
        _check(lib().rlbm_moments_device(self._h, *[_vp(base + 8 * k * S) for k in range(6)]),
               self._h)

    def get_populations(self) -> np.ndarray:
        """Raw stored populations, shape (npop, ny, nx), storage dtype."""
        dt = {"fp64": np.float64, "fp32": np.float32, "fp16": np.float16, "bf16": np.uint16,
              "fp16n": np.float16, "bf16n": np.uint16}[self.precision]
        out = np.empty((self.npop, self.ny, self.nx), dtype=dt)
        _check(lib().rlbm_get_populations(self._h, _vp(out.ctypes.data), out.nbytes), self._h)
        return out

    def set_populations(self, arr: np.ndarray, step: int = 0):
        arr = np.ascontiguousarray(arr)
        _check(lib().rlbm_set_populations(self._h, _vp(arr.ctypes.data), arr.nbytes, int(step)),
               self._h)

    def sync(self):
        _check(lib().rlbm_sync(self._h), self._h)

    @property
    def steps_done(self) -> int:
        return lib().rlbm_steps_done(self._h)

    @property
    def kernel_launches(self) -> int:
        return lib().rlbm_kernel_launches(self._h)

    def current_buffer_ptr(self) -> int:
        return lib().rlbm_current_buffer(self._h)

    @property
    def uses_tma(self) -> bool:
        """True when steps run the persistent TMA-staged kernel."""
        return lib().rlbm_step_kernel_variant(self._h) == 1

    @property
    def tile_populations(self) -> int:
        return lib().rlbm_tile_populations(self._h)

    STATISTICS = {"mj": 0, "fd": 1, "be": -1}

    def set_statistics(self, kind: str, g: float = 1.0):
        """Equilibrium statistic: 'mj' (Maxwell-Juttner), 'fd' (Fermi-Dirac) or
        'be' (Bose-Einstein), f^eq = g / (z^-1 exp(U.p/T) + eps); see
        rlbm_set_statistics."""
        _check(lib().rlbm_set_statistics(self._h, self.STATISTICS[kind], float(g)), self._h)

    @property
    def statistics(self) -> str:
        v = lib().rlbm_statistics(self._h)
        return {0: "mj", 1: "fd", -1: "be"}[v]

    @property
    def population_groups(self) -> int:
        """Groups of tile_populations populations per warp (> 1 only for K beyond
        one group per warp, see rlbm_population_groups)."""
        return lib().rlbm_population_groups(self._h)

    KERNELS = ("per-tile", "tma", "pair", "pair-bulk", "pair-tma")

    @property
    def step_kernel(self) -> str:
        """'per-tile', 'tma', 'pair' (two sites per lane) or 'pair-bulk' (two
        sites per lane, first pass staged by bulk copies)."""
        return self.KERNELS[lib().rlbm_step_kernel_variant(self._h)]

    def set_tiling(self, P: int, kind: str):
        """Select P populations per warp and the step kernel (one of KERNELS);
        raises RLBMError if that kernel is not possible here."""
        k = self.KERNELS.index(kind)
        _check(lib().rlbm_set_tiling(self._h, int(P), k), self._h)

    def autotune(self, launches_per_trial: int = 8) -> float:
        """Pick the fastest compiled tiling for this problem (see rlbm_autotune);
        returns the time of one step launch in ms.  Call after init."""
        ms = ctypes.c_float(0.0)
        _check(lib().rlbm_autotune(self._h, int(launches_per_trial), ctypes.byref(ms)), self._h)
        return ms.value

    def set_wait_limit(self, cycles: int):
        _check(lib().rlbm_set_wait_limit(self._h, int(cycles)), self._h)

    def test_stall_next_step(self):
        _check(lib().rlbm_test_stall_next_step(self._h), self._h)


def decode_populations(raw: np.ndarray, precision: str, w: np.ndarray) -> np.ndarray:
    """Stored values -> f_i: identity for fp64/fp32; f = f^rest (s + beta) for
    16-bit storage, f^rest_i = w_i / (2 pi), beta = 1 (deviation) or 0 (normalised)."""
    if precision in ("fp64", "fp32"):
        return raw.astype(np.float64)
    if precision.startswith("fp16"):
        s = raw.astype(np.float64)
    else:
        s = (raw.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    beta = 0.0 if precision.endswith("n") else 1.0
    return (w / (2.0 * math.pi))[:, None, None] * (s + beta)


def _bcheck(status: int, b=None):
    if status == OK:
        return
    msg = lib().rlbm_batch_last_error(b).decode(errors="replace")
    cls = {ERR_UNPHYSICAL: Unphysical, ERR_TIMEOUT: DeviceTimeout}.get(status, RLBMError)
    raise cls(status, msg)


def problems_array(problems):
    """ctypes array of Problem from (nx, ny, bc_x, bc_y, K, tau) tuples or Problem objects."""
    arr = (Problem * len(problems))()
    for i, p in enumerate(problems):
        arr[i] = p if isinstance(p, Problem) else Problem(*p)
    return arr


def batch_arena_bytes(problems, N: int, precision: str = "fp32") -> int:
    arr = problems_array(problems)
    return lib().rlbm_batch_arena_bytes(arr, len(problems), N, PRECISIONS[precision])


class _View(Simulation):
    """A problem of a batch: the Simulation API on a handle the batch owns."""

    def __init__(self, handle, nx, ny, N, K, tau, precision, stream):
        self._h = handle
        self.nx, self.ny, self.N, self.K = nx, ny, N, K
        self.npop = K * (N + 1)
        self.precision = precision
        self.tau = tau
        self.stream = stream
        self._buf = None

    def close(self):
        self._h = None  # owned by the batch

    def step(self, nsteps: int = 1):
        raise RuntimeError("step a batch with Batch.step")


class Batch:
    """Many independent problems (N shared) advanced by one persistent launch."""

    def __init__(self, problems, N: int = 2, precision: str = "fp32", stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("librlbm needs a CUDA GPU")
        self.N = int(N)
        self.precision = precision
        self.stream = stream if stream is not None else torch.cuda.Stream()
        arr = problems_array(problems)
        self.specs = [(p.nx, p.ny, p.bc_x, p.bc_y, p.angles_K, p.tau) for p in arr]
        nbytes = lib().rlbm_batch_arena_bytes(arr, len(arr), self.N, PRECISIONS[precision])
        self._arena = torch.empty(max(nbytes, 1), dtype=torch.uint8, device="cuda")
        h = _vp()
        _bcheck(lib().rlbm_batch_create(ctypes.byref(h), arr, len(arr), self.N,
                                        PRECISIONS[precision], _vp(self.stream.cuda_stream),
                                        _vp(self._arena.data_ptr()), nbytes))
        self._b = h
        self.problems = []
        for i, (nx, ny, bcx, bcy, K, tau) in enumerate(self.specs):
            ph = lib().rlbm_batch_problem(self._b, i)
            self.problems.append(_View(_vp(ph), nx, ny, self.N, K, tau, precision, self.stream))

    def __len__(self):
        return len(self.problems)

    def __getitem__(self, i) -> Simulation:
        return self.problems[i]

    def step(self, nsteps: int = 1):
        _bcheck(lib().rlbm_batch_step(self._b, int(nsteps)), self._b)

    def sync(self):
        _bcheck(lib().rlbm_batch_sync(self._b), self._b)

    def autotune(self, steps_per_trial: int = 4) -> float:
        ms = ctypes.c_float(0.0)
        _bcheck(lib().rlbm_batch_autotune(self._b, int(steps_per_trial), ctypes.byref(ms)), self._b)
        return ms.value

    MODES = ("persistent", "streams")

    def set_mode(self, mode: str):
        """'persistent' (one cooperative launch per call) or 'streams' (each
        problem's own step kernel on a pool of streams)."""
        _bcheck(lib().rlbm_batch_set_mode(self._b, self.MODES.index(mode)), self._b)

    @property
    def mode(self) -> str:
        return self.MODES[lib().rlbm_batch_mode(self._b)]

    def set_wait_limit(self, cycles: int):
        _bcheck(lib().rlbm_batch_set_wait_limit(self._b, int(cycles)), self._b)

    def test_stall_next_step(self):
        _bcheck(lib().rlbm_batch_test_stall_next_step(self._b), self._b)

    @property
    def kernel_launches(self) -> int:
        return lib().rlbm_batch_kernel_launches(self._b)

    @property
    def population_updates_per_step(self) -> int:
        return sum(nx * ny * K * (self.N + 1) for (nx, ny, _, _, K, _) in self.specs)

    def close(self):
        if getattr(self, "_b", None):
            for p in self.problems:
                p.close()
            lib().rlbm_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _check_noalloc_tensors(nx, ny, N, K, precision, fin, fout):
    """The C entry point cannot see buffer sizes: check the tensors here, on
    the host, before anything is launched (dtype and size first, so that the
    checks also run without a GPU)."""
    import torch
    want = {"fp64": torch.float64, "fp32": torch.float32}.get(precision)
    if want is None:
        raise RLBMError(ERR_UNSUPPORTED, f"rlbm_step_noalloc supports fp64 and fp32 storage, not {precision}")
    count = int(K) * (int(N) + 1) * int(nx) * int(ny)
    for name, t in (("fin", fin), ("fout", fout)):
        if not isinstance(t, torch.Tensor):
            raise RLBMError(ERR_ARG, f"{name} must be a torch tensor")
        if t.dtype != want:
            raise RLBMError(ERR_ARG, f"{name} has dtype {t.dtype}, {precision} storage needs {want}")
        if t.numel() != count:
            raise RLBMError(ERR_ARG, f"{name} holds {t.numel()} elements, need K (N+1) nx ny = {count}")
        if not t.is_contiguous():
            raise RLBMError(ERR_ARG, f"{name} must be contiguous")
        if not t.is_cuda or t.device.index != torch.cuda.current_device():
            raise RLBMError(ERR_ARG, f"{name} must be a CUDA tensor on the current device")


def step_noalloc(nx, ny, N, K, tau, precision, fin, fout, bcx=BC_COPYOUT, bcy=BC_PERIODIC,
                 stream=None):
    """One step from device tensor fin to device tensor fout through the
    allocation-free entry point (the library allocates no device memory).
    fin and fout: contiguous CUDA tensors on the current device, float64 for
    'fp64' / float32 for 'fp32', of K (N+1) nx ny elements each."""
    _check_noalloc_tensors(nx, ny, N, K, precision, fin, fout)
    st = lib().rlbm_step_noalloc(Grid(nx, ny, bcx, bcy), int(N), int(K), float(tau),
                                 PRECISIONS[precision], _vp(fin.data_ptr()), _vp(fout.data_ptr()),
                                 _vp(stream.cuda_stream if stream is not None else 0))
    if st != OK:
        msg = lib().rlbm_noalloc_last_error().decode(errors="replace")
        cls = {ERR_UNPHYSICAL: Unphysical}.get(st, RLBMError)
        raise cls(st, msg)


class Closure:
    """Learned angular closure (MLP) for a coarse FP32 problem of order N with K angles.

    Arrays are torch CUDA float32 tensors: populations (npop, sites), features
    (F, ld), targets and outputs (npop, ld)."""

    HIDDEN = 64

    def __init__(self, N: int, K: int, seed: int = 0, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("librlbm needs a CUDA GPU")
        self.N, self.K = int(N), int(K)
        self.npop = self.K * (self.N + 1)
        self.F = 10 + self.npop
        # one explicit stream for the closure and the simulations it works with
        self.stream = stream if stream is not None else torch.cuda.Stream()
        h = _vp()
        st = lib().rlbm_closure_create(ctypes.byref(h), self.N, self.K, int(seed),
                                       _vp(self.stream.cuda_stream))
        self._c = h
        self._check(st)

    def _check(self, status: int):
        if status != OK:
            msg = lib().rlbm_closure_last_error(self._c if self._c else None).decode(errors="replace")
            raise RLBMError(status, msg)

    def close(self):
        if getattr(self, "_c", None):
            lib().rlbm_closure_destroy(self._c)
            self._c = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def param_count(self) -> int:
        return lib().rlbm_closure_param_count(self._c)

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.param_count, dtype=np.float32)
        self._check(lib().rlbm_closure_get_params(self._c, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                                  out.size))
        return out

    def set_params(self, p: np.ndarray):
        p = np.ascontiguousarray(p, dtype=np.float32)
        self._check(lib().rlbm_closure_set_params(self._c, p.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                                  p.size))

    def split_params(self, p: np.ndarray):
        """(W1 [F][64], b1, W2 [64][64], b2, W3 [64][npop], b3) views of a flat array."""
        H, F, O = self.HIDDEN, self.F, self.npop
        sizes = [F * H, H, H * H, H, H * O, O]
        shapes = [(F, H), (H,), (H, H), (H,), (H, O), (O,)]
        out, o = [], 0
        for n, shp in zip(sizes, shapes):
            out.append(p[o:o + n].reshape(shp))
            o += n
        return out

    def features(self, f, kn: float, X, off: int = 0):
        self._check(lib().rlbm_closure_features(self._c, _vp(f.data_ptr()), f.shape[1], float(kn),
                                                _vp(X.data_ptr()), X.shape[1], int(off)))

    def target(self, fr, fc, T, off: int = 0):
        self._check(lib().rlbm_closure_target(self._c, _vp(fr.data_ptr()), _vp(fc.data_ptr()),
                                              fr.shape[1], _vp(T.data_ptr()), T.shape[1], int(off)))

    def restrict(self, fine_K: int, ff, fc):
        self._check(lib().rlbm_closure_restrict(self._c, int(fine_K), _vp(ff.data_ptr()), ff.shape[1],
                                                _vp(fc.data_ptr())))

    def forward(self, X, off: int, count: int, Y):
        self._check(lib().rlbm_closure_forward(self._c, _vp(X.data_ptr()), X.shape[1], int(off),
                                               int(count), _vp(Y.data_ptr())))

    def work(self, ld: int):
        import torch
        n = lib().rlbm_closure_work_floats(self._c, int(ld))
        return torch.empty(n, dtype=torch.float32, device="cuda")

    def gradient(self, X, T, off: int, count: int, work):
        g = np.zeros(self.param_count, dtype=np.float32)
        loss = ctypes.c_float(0.0)
        self._check(lib().rlbm_closure_gradient(self._c, _vp(X.data_ptr()), _vp(T.data_ptr()),
                                                X.shape[1], int(off), int(count), _vp(work.data_ptr()),
                                                g.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                                ctypes.byref(loss)))
        return g, loss.value

    def train_step(self, X, T, off: int, count: int, lr: float, work) -> float:
        loss = ctypes.c_float(0.0)
        self._check(lib().rlbm_closure_train_step(self._c, _vp(X.data_ptr()), _vp(T.data_ptr()),
                                                  X.shape[1], int(off), int(count), float(lr),
                                                  _vp(work.data_ptr()), ctypes.byref(loss)))
        return loss.value

    def apply_buffer(self, f_ptr: int, sites: int, kn: float):
        self._check(lib().rlbm_closure_apply_buffer(self._c, _vp(f_ptr), int(sites), float(kn)))

    def set_train_path(self, tensor_cores: bool):
        self._check(lib().rlbm_closure_set_train_path(self._c, 1 if tensor_cores else 0))

    def set_apply_path(self, tensor_cores: bool):
        self._check(lib().rlbm_closure_set_apply_path(self._c, 1 if tensor_cores else 0))

    def apply(self, sim, kn: float):
        """Correct the current populations of a coarse FP32 Simulation in place."""
        assert sim.precision == "fp32" and sim.K == self.K and sim.N == self.N
        self.apply_buffer(sim.current_buffer_ptr(), sim.sites, kn)
