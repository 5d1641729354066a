"""Command-line runner: one problem, equilibrium initial state, n steps, fields.

    python -m paper_2011_06856_gb300.run --nx 8192 --ny 4 --N 3 --K 64 \\
        --precision fp32 --kn 0.01 --steps 100 [--tile-p 32] [--autotune] [--out fields.npz]
        [--closure]

The initial state is the shock tube of the named workload shape (a 2D
four-quadrant Riemann problem when --riemann is given).  Prints the tiling
used and the step count; with --out writes n, eps, T, U^0, U^x, U^y.  With
--closure (FP32) the learned correction, with its initial random weights,
is applied after every step.
Used for ncu captures of single kernels.
"""
from __future__ import annotations

import argparse
import os
import sys

import numpy as np

from . import rlbm as R
from . import workloads as W


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--nx", type=int, required=True)
    ap.add_argument("--ny", type=int, default=1)
    ap.add_argument("--N", type=int, default=2)
    ap.add_argument("--K", type=int, default=16)
    ap.add_argument("--precision", default="fp32", choices=sorted(R.PRECISIONS))
    ap.add_argument("--kn", type=float, default=0.05)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--riemann", action="store_true")
    ap.add_argument("--paper2d", action="store_true", help="the paper's 2D four-quadrant states (Sec. 3.2)")
    ap.add_argument("--bcx", type=int, default=W.BC_COPYOUT)
    ap.add_argument("--bcy", type=int, default=None)
    ap.add_argument("--tile-p", type=int, default=None, help="populations per warp")
    ap.add_argument("--per-tile", action="store_true", help="do not use the TMA-staged kernel")
    ap.add_argument("--kernel", choices=R.Simulation.KERNELS, default=None,
                    help="step kernel (with --tile-p as its populations per warp)")
    ap.add_argument("--autotune", action="store_true")
    ap.add_argument("--out", default=None)
    ap.add_argument("--closure", action="store_true", help="fused learned correction after each step")
    a = ap.parse_args(argv)
    if a.tile_p:
        os.environ["RLBM_TILE_P"] = str(a.tile_p)
    if a.per_tile:
        os.environ["RLBM_NO_TMA"] = "1"
    bcy = a.bcy if a.bcy is not None else (W.BC_COPYOUT if (a.riemann or a.paper2d) else W.BC_PERIODIC)
    if a.paper2d:
        fl = W.riemann_2d(a.nx, a.ny, W.PAPER_SOD2D_STATES)
    elif a.riemann:
        fl = W.workload_fields(W.WORKLOADS["riemann2d_2048_N2K48"], a.nx, a.ny)
    else:
        fl = W.shock_tube(a.nx, a.ny)
    cl = R.Closure(a.N, a.K, seed=1) if a.closure else None
    sim = R.Simulation(a.nx, a.ny, a.N, a.K, W.tau_from_kn(a.kn, a.nx), a.precision, a.bcx, bcy,
                       stream=cl.stream if cl else None)
    sim.init_fields(fl)
    if a.kernel:
        sim.set_tiling(a.tile_p or sim.tile_populations, a.kernel)
    if a.autotune:
        sim.autotune(8)
    if cl:
        for _ in range(a.steps):
            sim.step(1)
            cl.apply(sim, a.kn)
        cl.stream.synchronize()
    else:
        sim.step(a.steps)
    sim.sync()
    print(f"tiling P={sim.tile_populations} groups={sim.population_groups} kernel={sim.step_kernel} "
          f"steps={sim.steps_done} launches={sim.kernel_launches}")
    if a.out:
        m = sim.moments()
        np.savez(a.out, n=m[0], eps=m[1], T=m[2], U0=m[3], Ux=m[4], Uy=m[5])
    sim.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
