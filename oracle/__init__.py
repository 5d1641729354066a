"""FP64 CPU oracle for the relativistic lattice Boltzmann method (arXiv 2011.06856).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg of
``bench.py`` load this package; the product library never does.  The arithmetic
lives in ``rlbm_oracle.c`` (plain C, FP64, OpenMP over sites); this module only
compiles it with gcc and marshals numpy arrays through ctypes.  It shares no
code with the CUDA library.

Each wrapper names the passage of the paper it follows:

* :func:`radial_rule`, :class:`Quadrature` -- Sec. 2.3, Eq. (off-lattice-quad)
* :meth:`Quadrature.feq` -- Sec. 2.2, Eqs. (mj-feq-expansion-truncated),
  (mj-projection-coefficients); MJ moments of Sec. 2.1, Eq. (moments)
* :meth:`Quadrature.stream` -- Sec. 2.2, Eqs. (streaming), (interpolation)
* :meth:`Quadrature.moments`, :func:`landau` -- Sec. 2.2, Eq.
  (discrete_sum_moments) and the Landau eigenproblem
* :meth:`Quadrature.collide`, :meth:`Quadrature.run` -- Sec. 2.2, Eq. (discrete-rbe)
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rlbm_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "librlbm_oracle.so")

BC_PERIODIC = 0
BC_COPYOUT = 1

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags: no -march, no FMA contraction)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call([
            "gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
            _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        L.orc_laguerre.restype = ctypes.c_double
        L.orc_laguerre.argtypes = [ctypes.c_int, ctypes.c_double]
        L.orc_radial_rule.restype = ctypes.c_int
        L.orc_radial_rule.argtypes = [ctypes.c_int, _dp, _dp]
        L.orc_angular_integral.restype = ctypes.c_double
        L.orc_angular_integral.argtypes = [ctypes.c_int, ctypes.c_int]
        L.orc_create.restype = ctypes.c_void_p
        L.orc_create.argtypes = [ctypes.c_int, ctypes.c_int]
        L.orc_create_onlattice.restype = ctypes.c_void_p
        L.orc_create_onlattice.argtypes = [ctypes.c_int]
        L.orc_shifts.restype = ctypes.c_int
        L.orc_shifts.argtypes = [ctypes.c_void_p, _ip, _ip]
        L.orc_destroy.restype = None
        L.orc_destroy.argtypes = [ctypes.c_void_p]
        L.orc_npop.restype = ctypes.c_int
        L.orc_npop.argtypes = [ctypes.c_void_p]
        L.orc_nbasis.restype = ctypes.c_int
        L.orc_nbasis.argtypes = [ctypes.c_void_p]
        L.orc_tables.restype = None
        L.orc_tables.argtypes = [ctypes.c_void_p, _dp, _dp, _dp, _dp]
        L.orc_basis.restype = None
        L.orc_basis.argtypes = [ctypes.c_void_p, _ip, _ip, _ip]
        L.orc_mj_moment.restype = ctypes.c_double
        L.orc_mj_moment.argtypes = [ctypes.c_int, _ip, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_double]
        L.orc_feq.restype = None
        L.orc_feq.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                              ctypes.c_double, ctypes.c_double, _dp]
        L.orc_moments.restype = None
        L.orc_moments.argtypes = [ctypes.c_void_p, _dp, ctypes.c_long, _dp]
        L.orc_landau.restype = ctypes.c_int
        L.orc_landau.argtypes = [_dp, _dp]
        L.orc_stream.restype = None
        L.orc_stream.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 ctypes.c_int, _dp, _dp]
        L.orc_collide.restype = ctypes.c_long
        L.orc_collide.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp]
        L.orc_run.restype = ctypes.c_long
        L.orc_run.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                              ctypes.c_int, ctypes.c_double, ctypes.c_int, _dp, ctypes.c_int]
        L.orc_init.restype = None
        L.orc_init.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp,
                               _dp, ctypes.c_int]
        L.orc_macro.restype = ctypes.c_long
        L.orc_macro.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, _dp, _dp, ctypes.c_int]
        L.orc_max_threads.restype = ctypes.c_int
        L.orc_max_threads.argtypes = []
        _lib = L
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def _c(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def laguerre(n: int, x: float) -> float:
    """L_n(x) by its three-term recurrence."""
    return lib().orc_laguerre(n, float(x))


def radial_rule(N: int):
    """(p_r, w^(p)_r): roots of L_{N+1} and the weights of Sec. 2.3."""
    p = np.zeros(N + 1)
    w = np.zeros(N + 1)
    got = lib().orc_radial_rule(N, _p(p), _p(w))
    if got != N + 1:
        raise RuntimeError(f"found {got} Laguerre roots, expected {N + 1}")
    return p, w


def angular_integral(a: int, b: int) -> float:
    """Closed-form integral of cos^a sin^b over [0, 2 pi]."""
    return lib().orc_angular_integral(a, b)


def mj_moment(idx, n: float, T: float, Ux: float, Uy: float) -> float:
    """Component idx (tuple over {0,1,2}) of the rank-len(idx) MJ moment tensor."""
    arr = (ctypes.c_int * max(1, len(idx)))(*idx)
    return lib().orc_mj_moment(len(idx), arr, n, T, Ux, Uy)


def landau(mom):
    """Landau frame of 9 moments (N^t,N^x,N^y,T^tt,T^tx,T^ty,T^xx,T^xy,T^yy).

    Returns (status, array[n, eps, T, U0, Ux, Uy])."""
    m = _c(mom)
    out = np.zeros(6)
    st = lib().orc_landau(_p(m), _p(out))
    return st, out


class Quadrature:
    """Quadrature context of order N with K angles per shell (N_pop = K (N+1)).

    With onlattice=True: the on-lattice rule of Sec. 2.3 (N = 3, the 12 integer
    stencil vectors of length 5 on every shell, N_pop = 48; K is ignored), with
    perfect streaming; sx, sy hold the integer stencil vectors."""

    def __init__(self, N: int, K: int = 0, onlattice: bool = False):
        self.N = int(N)
        self.onlattice = bool(onlattice)
        if onlattice:
            self._h = lib().orc_create_onlattice(self.N)
            if not self._h:
                raise ValueError(f"no on-lattice rule for N={N} (only N = 3)")
            self.K = lib().orc_npop(self._h) // (self.N + 1)
        else:
            self.K = int(K)
            self._h = lib().orc_create(self.N, self.K)
            if not self._h:
                raise ValueError(f"invalid quadrature N={N}, K={K} (need K >= 2N+1)")
        self.npop = lib().orc_npop(self._h)
        self.nbasis = lib().orc_nbasis(self._h)
        self.p0 = np.zeros(self.npop)
        self.vx = np.zeros(self.npop)
        self.vy = np.zeros(self.npop)
        self.w = np.zeros(self.npop)
        lib().orc_tables(self._h, _p(self.p0), _p(self.vx), _p(self.vy), _p(self.w))
        self.sx = self.sy = None
        if onlattice:
            self.sx = np.zeros(self.npop, dtype=np.int32)
            self.sy = np.zeros(self.npop, dtype=np.int32)
            lib().orc_shifts(self._h, self.sx.ctypes.data_as(_ip), self.sy.ctypes.data_as(_ip))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_destroy(h)
            self._h = None

    def basis(self):
        e = np.zeros(self.nbasis, dtype=np.int32)
        a = np.zeros(self.nbasis, dtype=np.int32)
        b = np.zeros(self.nbasis, dtype=np.int32)
        ip = lambda v: v.ctypes.data_as(_ip)
        lib().orc_basis(self._h, ip(e), ip(a), ip(b))
        return e, a, b

    def feq(self, n: float, T: float, Ux: float, Uy: float) -> np.ndarray:
        """Discrete equilibrium for U^a = (sqrt(1+|U|^2), Ux, Uy)."""
        out = np.zeros(self.npop)
        lib().orc_feq(self._h, n, T, Ux, Uy, _p(out))
        return out

    def moments(self, f_site) -> np.ndarray:
        f = _c(f_site)
        out = np.zeros(9)
        lib().orc_moments(self._h, _p(f), 1, _p(out))
        return out

    def stream(self, f, bcx=BC_COPYOUT, bcy=BC_PERIODIC) -> np.ndarray:
        f = _c(f)
        npop, ny, nx = f.shape
        assert npop == self.npop
        out = np.zeros_like(f)
        lib().orc_stream(self._h, nx, ny, bcx, bcy, _p(f), _p(out))
        return out

    def collide(self, fs, tau: float):
        """Collision in place on a copy; returns (f_new, flagged_sites)."""
        f = _c(fs).copy()
        npop, ny, nx = f.shape
        flagged = lib().orc_collide(self._h, nx, ny, float(tau), _p(f))
        return f, flagged

    def init(self, n, T, bx, by, nthreads: int = 0) -> np.ndarray:
        n, T, bx, by = (_c(a) for a in (n, T, bx, by))
        ny, nx = n.shape
        f = np.zeros((self.npop, ny, nx))
        lib().orc_init(self._h, nx, ny, _p(n), _p(T), _p(bx), _p(by), _p(f), nthreads)
        return f

    def run(self, f, tau: float, nsteps: int, bcx=BC_COPYOUT, bcy=BC_PERIODIC, nthreads: int = 0):
        """nsteps full steps on a copy of f; returns (f_new, flagged site-steps)."""
        f = _c(f).copy()
        npop, ny, nx = f.shape
        flagged = lib().orc_run(self._h, nx, ny, bcx, bcy, float(tau), int(nsteps), _p(f), nthreads)
        return f, flagged

    def macro(self, f, nthreads: int = 0):
        """Landau fields (n, eps, T, U0, Ux, Uy) of stored populations; (array[6,ny,nx], flagged)."""
        f = _c(f)
        npop, ny, nx = f.shape
        out = np.zeros((6, ny, nx))
        flagged = lib().orc_macro(self._h, nx, ny, _p(f), _p(out), nthreads)
        return out, flagged


def max_threads() -> int:
    return lib().orc_max_threads()
