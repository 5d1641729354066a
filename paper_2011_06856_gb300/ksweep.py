"""K-sweep of the 1D Sod tube against a finely resolved reference (Sec. 3.1, Fig. 3).

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


def run_profile(L: int, N: int, K: int, kn: float, steps: int, precision: str, stream=None):
    """beta_x profile of the paper's Sod tube on L x 1 cells after `steps` steps,
    and the population updates per second of the run."""
    from . import rlbm as R
    import torch
    fl = W.shock_tube(L, 1, W.PAPER_SOD_LEFT, W.PAPER_SOD_RIGHT)
    sim = R.Simulation(L, 1, N, K, W.tau_from_kn(kn, L), precision, W.BC_COPYOUT, W.BC_PERIODIC,
                       stream=stream)
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
    return mac[4, 0] / mac[3, 0], L * (N + 1) * K * steps / dt


def coarsen(beta_fine: np.ndarray) -> np.ndarray:
    """Mean of fine cells 2i, 2i+1 (coarse cell i)."""
    return 0.5 * (beta_fine[0::2] + beta_fine[1::2])


def rel_err(beta: np.ndarray, beta_ref: np.ndarray) -> float:
    """Eq. rel_err."""
    return float(np.linalg.norm(beta - beta_ref) / np.linalg.norm(beta_ref))


def sweep(kn_list, k_list, L: int = 2000, N: int = 3, k_ref: int = 600, precision: str = "fp64"):
    from .rlbm import Unphysical
    steps = int(round(0.9 * L / 2))
    out = []
    for kn in kn_list:
        try:
            bref_f, rate_ref = run_profile(2 * L, N, k_ref, kn, 2 * steps, precision)
        except Unphysical:
            out.append({"kn": kn, "L": L, "N": N, "steps": steps, "reference": "unstable"})
            continue
        bref = coarsen(bref_f)
        eps, rates = [], []
        for K in k_list:
            try:
                b, rate = run_profile(L, N, K, kn, steps, precision)
                eps.append(rel_err(b, bref))
                rates.append(rate)
            except Unphysical:
                eps.append("unstable")
                rates.append(None)
        out.append({"kn": kn if math.isfinite(kn) else "inf", "L": L, "N": N, "steps": steps,
                    "K": list(k_list), "npop": [(N + 1) * k for k in k_list], "eps": eps,
                    "reference": {"L": 2 * L, "K": k_ref, "npop": (N + 1) * k_ref,
                                  "steps": 2 * steps, "updates_per_s": rate_ref},
                    "updates_per_s": rates, "precision": precision})
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--L", type=int, default=2000)
    ap.add_argument("--kn", type=float, nargs="+", default=[0.05, 0.2, 1.0, 10.0])
    ap.add_argument("--K", type=int, nargs="+", default=[12, 24, 48, 96, 120, 240, 480])
    ap.add_argument("--kref", type=int, default=600)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "fp32"])
    args = ap.parse_args()
    from . import build as B
    B.build()
    for row in sweep(args.kn, args.K, args.L, 3, args.kref, args.precision):
        print(json.dumps(row), flush=True)


if __name__ == "__main__":
    main()
