"""K-sweeps against a finely resolved reference: the 1D Sod tube (Sec. 3.1,
Fig. 3) and the 2D Sod problem (Sec. 3.2, Fig. 6); and the grid-convergence
study of the tube (Sec. 3.1, Fig. 4, --convergence).

For each Knudsen number Kn = c tau / L the tube of L x 1 cells is run with the
N = 3 rule at several K, and compared with a reference on 2L x 1 cells with
K_ref = 600 angles (N_pop = 2400), both at t = 0.9 t_max (t_max = L/2 time
steps on the coarse grid, the front moving at c = 1 from the middle to the
edge; 2x the steps, and tau, on the fine grid).  The error is the relative L2
difference of the velocity profile (Eq. rel_err),
    eps = || beta - beta_ref ||_2 / || beta_ref ||_2,
with beta_ref at a coarse cell the mean of the two fine cells it covers (the
linear interpolation to the coarse cell centre).  Everything runs through the
library on the GPU; the initial states are the paper's (Eq. initial-cond-macro).

    python -m paper_2011_06856_gb300.ksweep [--L 2000] [--kn 0.05 0.2 1 10]
        [--K 12 24 48 96 120 240 480] [--kref 600] [--precision fp64]

With --dim 2 the problem is the paper's four-quadrant one on L x L cells (copy-out
walls), the reference on (4L) x (4L) cells (Fig. 6: 250^2 against 1000^2), the
coarse run takes round(0.9 L/2) steps and the reference 4x as many, beta_ref is
the mean over the 4 x 4 fine cells of a coarse cell, and the norm runs over both
velocity components.

With --convergence the tube runs on several grids L (each dividing the
reference grid L_ref = 12000, with 0.9 L/2 a whole number of steps) for several
K, against one L_ref x 1, K = 600 reference per Kn at the same physical time
(Fig. 4: N_pop = 48, 240, 480 against N_pop = 2400).

Prints one JSON object per Kn.  A run that reaches a cell without a physical
Landau frame (the library raises Unphysical; at Kn = 0.002 on 2000 x 1, tau = 4,
the 45:1 pressure jump drives populations negative, as in the FP64 oracle) is
reported as "unstable" for that Kn and K.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import workloads as W


def problem(L: int, dim: int):
    """Initial fields and boundary conditions of the paper's 1D (L x 1) or 2D (L x L) problem."""
    if dim == 1:
        return W.shock_tube(L, 1, W.PAPER_SOD_LEFT, W.PAPER_SOD_RIGHT), W.BC_COPYOUT, W.BC_PERIODIC
    return W.riemann_2d(L, L, W.PAPER_SOD2D_STATES), W.BC_COPYOUT, W.BC_COPYOUT


def run_profile(L: int, N: int, K: int, kn: float, steps: int, precision: str, dim: int = 1,
                stream=None):
    """Velocity field (beta_x, beta_y) [2][ny][nx] of the paper's problem after
    `steps` steps, and the population updates per second of the run."""
    from . import rlbm as R
    import torch
    fl, bcx, bcy = problem(L, dim)
    ny = fl.shape[0]
    sim = R.Simulation(L, ny, N, K, W.tau_from_kn(kn, L), precision, bcx, bcy, stream=stream)
    try:
        sim.init_fields(fl)
        sim.autotune(2)
        sim.sync()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.step(steps)
        mac = sim.moments()
        dt = time.perf_counter() - t0
    finally:
        sim.close()
    return mac[4:6] / mac[3], L * ny * (N + 1) * K * steps / dt


def coarsen(beta_fine: np.ndarray, s: int, dim: int) -> np.ndarray:
    """Mean over the s fine cells (1D) or s x s fine cells (2D) of each coarse cell."""
    c, ny, nx = beta_fine.shape
    if dim == 1:
        return beta_fine.reshape(c, ny, nx // s, s).mean(-1)
    return beta_fine.reshape(c, ny // s, s, nx // s, s).mean((2, 4))


def rel_err(beta: np.ndarray, beta_ref: np.ndarray) -> float:
    """Eq. rel_err."""
    return float(np.linalg.norm(beta - beta_ref) / np.linalg.norm(beta_ref))


def sweep(kn_list, k_list, L: int = 2000, N: int = 3, k_ref: int = 600, precision: str = "fp64",
          dim: int = 1):
    from .rlbm import Unphysical
    s = 2 if dim == 1 else 4
    steps = int(round(0.9 * L / 2))
    out = []
    for kn in kn_list:
        try:
            bref_f, rate_ref = run_profile(s * L, N, k_ref, kn, s * steps, precision, dim)
        except Unphysical:
            out.append({"kn": kn, "L": L, "N": N, "steps": steps, "reference": "unstable"})
            continue
        bref = coarsen(bref_f, s, dim)
        if dim == 1:
            bref = bref[0]  # the tube's velocity is beta_x
        eps, rates = [], []
        for K in k_list:
            try:
                b, rate = run_profile(L, N, K, kn, steps, precision, dim)
                if dim == 1:
                    b = b[0]
                eps.append(rel_err(b, bref))
                rates.append(rate)
            except Unphysical:
                eps.append("unstable")
                rates.append(None)
        out.append({"kn": kn if math.isfinite(kn) else "inf", "dim": dim, "L": L, "N": N,
                    "steps": steps, "K": list(k_list), "npop": [(N + 1) * k for k in k_list], "eps": eps,
                    "reference": {"L": s * L, "K": k_ref, "npop": (N + 1) * k_ref,
                                  "steps": s * steps, "updates_per_s": rate_ref},
                    "updates_per_s": rates, "precision": precision})
    return out


def convergence(kn_list, L_list, k_list, L_ref: int = 12000, N: int = 3, k_ref: int = 600,
                precision: str = "fp64"):
    """Fig. 4: eps(L, K) for each Kn against one L_ref x 1 reference."""
    from .rlbm import Unphysical
    for L in L_list:
        if L_ref % L or (9 * L) % 20:
            raise ValueError(f"L = {L} must divide {L_ref} and make 0.9 L/2 a whole number of steps")
    ref_steps = 9 * L_ref // 20
    out = []
    for kn in kn_list:
        try:
            bref_f, rate_ref = run_profile(L_ref, N, k_ref, kn, ref_steps, precision)
        except Unphysical:
            out.append({"kn": kn, "L_ref": L_ref, "reference": "unstable"})
            continue
        eps = {}
        for K in k_list:
            row = []
            for L in L_list:
                bref = coarsen(bref_f, L_ref // L, 1)[0]
                try:
                    b, _ = run_profile(L, N, K, kn, 9 * L // 20, precision)
                    row.append(rel_err(b[0], bref))
                except Unphysical:
                    row.append("unstable")
            eps[str(K)] = row
        out.append({"kn": kn, "N": N, "L": list(L_list), "K": list(k_list),
                    "npop": [(N + 1) * k for k in k_list], "eps_by_K": eps,
                    "reference": {"L": L_ref, "K": k_ref, "npop": (N + 1) * k_ref, "steps": ref_steps,
                                  "updates_per_s": rate_ref}, "precision": precision})
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--dim", type=int, default=1, choices=[1, 2])
    ap.add_argument("--L", type=int, default=None, help="coarse grid (default 2000 in 1D, 250 in 2D)")
    ap.add_argument("--kn", type=float, nargs="+", default=[0.05, 0.2, 1.0, 10.0])
    ap.add_argument("--K", type=int, nargs="+", default=[12, 24, 48, 96, 120, 240, 480])
    ap.add_argument("--kref", type=int, default=600)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"])
    ap.add_argument("--convergence", action="store_true", help="Fig. 4 instead of a K-sweep")
    ap.add_argument("--grids", type=int, nargs="+", default=[500, 1000, 1500, 2000, 3000, 4000, 6000])
    ap.add_argument("--lref", type=int, default=12000)
    args = ap.parse_args()
    from . import build as B
    B.build()
    if args.convergence:
        K = args.K if args.K != ap.get_default("K") else [12, 60, 120]
        for row in convergence(args.kn, args.grids, K, args.lref, 3, args.kref, args.precision):
            print(json.dumps(row), flush=True)
        return
    L = args.L or (2000 if args.dim == 1 else 250)
    for row in sweep(args.kn, args.K, L, 3, args.kref, args.precision, args.dim):
        print(json.dumps(row), flush=True)


if __name__ == "__main__":
    main()
