"""Seeded synthetic inputs: macroscopic initial fields and random populations.

This module holds no arithmetic of the lattice Boltzmann method itself (no
quadrature, no equilibrium, no moments): it only draws the piecewise-constant
Maxwell-Juttner states (n, T, beta) of shock-tube and Riemann problems and
random positive arrays.  Both the CUDA library and the FP64 oracle turn these
fields into populations with their own code.

The problems have the structure of the paper's workloads: the 1D Sod tube of
Sec. 3.1 (two states at rest, a sharp step at x = 0 in the middle of the
domain) and the 2D four-quadrant problem of Sec. 3.2.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MASTER_SEED = 2011_06856

BC_PERIODIC = 0
BC_COPYOUT = 1


class SplitMix64:
    """SplitMix64 (Steele, Lea, Flood 2014): state += 0x9E3779B97F4A7C15, then mix."""

    MASK = (1 << 64) - 1

    def __init__(self, seed: int):
        self.state = seed & self.MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & self.MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & self.MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & self.MASK
        return z ^ (z >> 31)

    def uniform(self, lo: float = 0.0, hi: float = 1.0) -> float:
        return lo + (hi - lo) * ((self.next_u64() >> 11) * (1.0 / (1 << 53)))


@dataclass
class Fields:
    """Initial macroscopic fields, each [ny][nx] float64: n, T, beta_x, beta_y."""
    n: np.ndarray
    T: np.ndarray
    bx: np.ndarray
    by: np.ndarray

    @property
    def shape(self):
        return self.n.shape


def shock_tube(nx: int, ny: int, left=(1.0, 1.0), right=(0.2, 0.5)) -> Fields:
    """Two states (n, T) at rest; cell ix < nx/2 (centre x = ix + 1/2 - nx/2 < 0) is left."""
    n = np.empty((ny, nx))
    T = np.empty((ny, nx))
    is_left = (np.arange(nx) + 0.5 - nx / 2.0) < 0.0
    n[:, :] = np.where(is_left, left[0], right[0])[None, :]
    T[:, :] = np.where(is_left, left[1], right[1])[None, :]
    z = np.zeros((ny, nx))
    return Fields(n, T, z, z.copy())


def riemann_2d(nx: int, ny: int, states, jitter: float = 0.0, seed: int = MASTER_SEED) -> Fields:
    """Four quadrants, listed in the order (x<0,y<0), (x>0,y<0), (x<0,y>0), (x>0,y>0).

    Each state is (n, T, beta_x, beta_y).  With jitter > 0, n and T of each
    quadrant are multiplied by (1 + U(-jitter, jitter)), drawn from SplitMix64
    in quadrant-major order, n then T; velocities are not jittered."""
    rng = SplitMix64(seed)
    st = []
    for (n0, T0, bx0, by0) in states:
        if jitter > 0.0:
            n0 = n0 * (1.0 + rng.uniform(-jitter, jitter))
            T0 = T0 * (1.0 + rng.uniform(-jitter, jitter))
        st.append((n0, T0, bx0, by0))
    xl = (np.arange(nx) + 0.5 - nx / 2.0) < 0.0
    yl = (np.arange(ny) + 0.5 - ny / 2.0) < 0.0
    out = [np.empty((ny, nx)) for _ in range(4)]
    for q, (xs, ys) in enumerate([(True, True), (False, True), (True, False), (False, False)]):
        mask = (yl[:, None] == ys) & (xl[None, :] == xs)
        for k in range(4):
            out[k][mask] = st[q][k]
    return Fields(*out)


def uniform(nx: int, ny: int, n: float, T: float, bx: float = 0.0, by: float = 0.0) -> Fields:
    return Fields(np.full((ny, nx), n), np.full((ny, nx), T), np.full((ny, nx), bx),
                  np.full((ny, nx), by))


def random_fields(nx: int, ny: int, seed: int, beta_max: float = 0.3) -> Fields:
    """Smoothly varying random (n, T, beta) fields for parity tests."""
    g = np.random.default_rng(seed)
    n = g.uniform(0.3, 1.2, (ny, nx))
    T = g.uniform(0.4, 1.2, (ny, nx))
    r = g.uniform(0.0, beta_max, (ny, nx))
    phi = g.uniform(0.0, 2.0 * math.pi, (ny, nx))
    return Fields(n, T, r * np.cos(phi), r * np.sin(phi))


def random_populations(npop: int, ny: int, nx: int, seed: int, lo=0.05, hi=1.0) -> np.ndarray:
    """Random positive populations f[npop][ny][nx]."""
    return np.random.default_rng(seed).uniform(lo, hi, (npop, ny, nx))


def tau_from_kn(kn: float, L: int, c: float = 1.0) -> float:
    """Kn = c tau / L (Sec. 3.1); c = 1 cell per step off lattice, 5 cells per
    step for the on-lattice rule (stencil vectors of length 5)."""
    return math.inf if math.isinf(kn) else kn * L / c


# --------------------------------------------------------------------------
# The synthetic workloads (grid, quadrature, Kn, steps, precision)
# --------------------------------------------------------------------------

# The paper's 1D Sod states (Sec. 3.1, Eq. initial-cond-macro), (n, T) of
# (P, n, T) = (2.25, 1.5, 1.5) for x < 0 and (0.05, 0.1, 0.5) for x > 0.
PAPER_SOD_LEFT = (1.5, 1.5)
PAPER_SOD_RIGHT = (0.1, 0.5)
_PAPER_SOD = {"left": PAPER_SOD_LEFT, "right": PAPER_SOD_RIGHT}
# The paper's 2D problem (Sec. 3.2, second Eq. initial-cond-macro), (n, T, beta_x, beta_y)
# per quadrant in the order (x<0,y<0), (x>0,y<0), (x<0,y>0), (x>0,y>0).
PAPER_SOD2D_STATES = [(0.5, 1.0, 0.0, 0.0), (0.5, 2.0, 0.0, 0.1), (0.5, 2.0, 0.1, 0.0),
                      (1.0, 1.0, 0.0, 0.0)]

@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    N: int
    K: int
    kn: tuple
    steps: int
    precision: str
    bcx: int = BC_COPYOUT
    bcy: int = BC_PERIODIC
    extra: dict = field(default_factory=dict)

    @property
    def npop(self) -> int:
        return self.K * (self.N + 1)

    @property
    def sites(self) -> int:
        return self.nx * self.ny


WORKLOADS = {
    # 1D shock tube, 400 x 1, 3 radial x 16 angles, Kn 0.01, 400 steps, FP64
    "shock1d_400x1_N2K16": Workload("shock1d_400x1_N2K16", 400, 1, 2, 16, (0.01,), 400, "fp64"),
    # scaled 1D shock tube, 8192 x 4, 4 radial x 64 angles, four Kn, 4000 steps
    "shock1d_8192x4_N3K64": Workload("shock1d_8192x4_N3K64", 8192, 4, 3, 64,
                                     (0.01, 0.1, 1.0, 10.0), 4000, "fp32"),
    # 2D Riemann problem 2048^2, 3 radial x 48 angles, Kn 0.05, 2000 steps, 16-bit storage
    "riemann2d_2048_N2K48": Workload("riemann2d_2048_N2K48", 2048, 2048, 2, 48, (0.05,), 2000,
                                     "fp16n", BC_COPYOUT, BC_COPYOUT,
                                     {"states": [(1.0, 1.0, 0.0, 0.0), (0.5, 0.8, 0.0, 0.0),
                                                 (0.25, 0.6, 0.0, 0.0), (0.5, 0.8, 0.0, 0.0)],
                                      "jitter": 0.01}),
    # the paper's Fig. 2 runs: 2000 x 1, tau -> inf, t = 0.9 t_max = 900 steps
    "sod1d_2000x1_N3K120": Workload("sod1d_2000x1_N3K120", 2000, 1, 3, 120, (math.inf,), 900, "fp32",
                                    extra=dict(_PAPER_SOD)),
    "sod1d_2000x1_N5K12": Workload("sod1d_2000x1_N5K12", 2000, 1, 5, 12, (math.inf,), 900, "fp32",
                                   extra=dict(_PAPER_SOD)),
    # the paper's reference rule of Fig. 3: N = 3, K = 600 (2400 populations), 4000 x 1,
    # t = 0.9 t_max = 1800 steps, three Kn of the figure's range
    "sod1d_4000x1_N3K600": Workload("sod1d_4000x1_N3K600", 4000, 1, 3, 600, (0.05, 1.0, 10.0), 1800,
                                    "fp32", extra=dict(_PAPER_SOD)),
    # the paper's Fig. 5 runs (2D Sod, copy-out walls, t = 0.9 t_max, t_max = L/2): 500^2 with
    # K = 12 at the three Kn, and 1000^2 with K = 600 (N_pop = 2400, 19 GB of FP32
    # populations) at the transition Kn
    "sod2d_500sq_N3K12": Workload("sod2d_500sq_N3K12", 500, 500, 3, 12, (0.002, 0.1, 100.0), 225, "fp32",
                                  BC_COPYOUT, BC_COPYOUT, {"states": PAPER_SOD2D_STATES}),
    "sod2d_1000sq_N3K600": Workload("sod2d_1000sq_N3K600", 1000, 1000, 3, 600, (0.1,), 450, "fp32",
                                    BC_COPYOUT, BC_COPYOUT, {"states": PAPER_SOD2D_STATES}),
    # the on-lattice rule of Sec. 2.3 (N = 3, 12 stencil vectors of length 5, N_pop = 48, perfect
    # streaming at 5 cells per step) on the paper's 2D problem: t = 0.9 t_max, t_max = L/10 steps;
    # tau = Kn L / 5, so the hydrodynamic end is Kn = 0.02 (tau = 4; Kn = 0.002 would over-relax)
    "onlattice2d_1000sq_N3": Workload("onlattice2d_1000sq_N3", 1000, 1000, 3, 12, (0.02, 0.1, 100.0), 90,
                                      "fp32", BC_COPYOUT, BC_COPYOUT,
                                      {"states": PAPER_SOD2D_STATES, "onlattice": True}),
    # the Fermi-Dirac statistic (Eq. feq_dist, eps = +1) on the paper's 2D problem; g = 0.1 puts
    # the fugacity near 1 (between the classical and the degenerate gas)
    "fermi2d_500sq_N3K12": Workload("fermi2d_500sq_N3K12", 500, 500, 3, 12, (0.1,), 225, "fp32",
                                    BC_COPYOUT, BC_COPYOUT,
                                    {"states": PAPER_SOD2D_STATES, "statistics": "fd", "g": 0.1}),
}


def statistics(w: Workload):
    """(kind, g) of the workload's equilibrium statistic ('mj' unless it names another)."""
    return w.extra.get("statistics", "mj"), w.extra.get("g", 1.0)


def light_speed(w: Workload) -> float:
    """Cells per time step a massless particle moves (5 for the on-lattice rule)."""
    return 5.0 if w.extra.get("onlattice") else 1.0

SHOCK_LEFT = (1.0, 1.0)
SHOCK_RIGHT = (0.2, 0.5)


def workload_fields(w: Workload, nx: int | None = None, ny: int | None = None,
                    seed: int = MASTER_SEED) -> Fields:
    nx = nx or w.nx
    ny = ny or w.ny
    if "states" in w.extra:
        return riemann_2d(nx, ny, w.extra["states"], w.extra.get("jitter", 0.0), seed)
    return shock_tube(nx, ny, w.extra.get("left", SHOCK_LEFT), w.extra.get("right", SHOCK_RIGHT))


@dataclass
class BatchProblem:
    nx: int
    ny: int
    K: int
    kn: float
    left: tuple
    right: tuple
    bcx: int
    bcy: int


def batch_problems(count: int = 256, seed: int = MASTER_SEED, nx_range=(256, 8192),
                   ny_choices=(1, 64, 256), k_choices=(16, 32, 48, 64),
                   kn_range=(0.01, 10.0)):
    """Uneven independent shock problems (N = 2): Nx log-uniform, Ny, K uniform
    from the choices, Kn log-uniform, left/right n in [0.1, 1], T in [0.3, 1], u = 0."""
    rng = SplitMix64(seed ^ 0xB47C4)
    out = []
    for _ in range(count):
        nx = int(round(math.exp(rng.uniform(math.log(nx_range[0]), math.log(nx_range[1])))))
        ny = ny_choices[min(len(ny_choices) - 1, int(rng.uniform() * len(ny_choices)))]
        K = k_choices[min(len(k_choices) - 1, int(rng.uniform() * len(k_choices)))]
        kn = math.exp(rng.uniform(math.log(kn_range[0]), math.log(kn_range[1])))
        left = (rng.uniform(0.1, 1.0), rng.uniform(0.3, 1.0))
        right = (rng.uniform(0.1, 1.0), rng.uniform(0.3, 1.0))
        bcy = BC_PERIODIC
        out.append(BatchProblem(nx, ny, K, kn, left, right, BC_COPYOUT, bcy))
    return out
