"""Training and deployment driver of the learned angular closure.

Everything numeric runs in librlbm kernels (LB steps, restriction, features,
targets, network forward/backward/Adam, fused correction); this module only
orders the calls and holds the device arrays (torch tensors).

* :func:`generate` -- fine-angle runs of four-quadrant Riemann problems; at
  every step t: f_c = R f_fine(t) in a coarse handle, one coarse step,
  features of the result, and the target R f_fine(t+1) minus that result.
* :func:`train` -- Adam on random contiguous column blocks.
* :func:`deploy` -- a coarse run with the correction applied after every
  step, next to the plain coarse run and the fine run it is judged against.
"""
from __future__ import annotations

import math

import numpy as np

from . import rlbm as R
from . import workloads as W

RIEMANN = [(1.0, 1.0, 0.0, 0.0), (0.5, 0.8, 0.0, 0.0), (0.25, 0.6, 0.0, 0.0), (0.5, 0.8, 0.0, 0.0)]


def kn_feature(tau: float, train_n: int) -> float:
    """The network's scalar input for a run with relaxation time tau (in time
    steps): tau / train_n, the Knudsen number that tau has on the n x n grid
    the network was trained on.

    The correction the network predicts is the coarse rule's error over one
    time step, which scales with the field's gradients in lattice units.  Its
    inputs are local, and near equilibrium the non-equilibrium part of f is
    about tau times those gradients (Chapman-Enskog), so the relaxation time
    in steps, not the grid-independent Kn = tau / L, is what ties the local
    state to the size of the correction.  On the training grid the two agree;
    on a finer grid (same Kn, larger tau) the gradients per cell are smaller
    and so is the correction.
    """
    return float(tau) / float(train_n)


def generate(closure: R.Closure, n: int, K_fine: int, kns, steps: int, seed: int = 1,
             every: int = 1):
    """Training pairs from runs at each Kn on an n x n Riemann problem; returns (X, T) tensors.
    The scalar feature is kn_feature(tau, n) = Kn."""
    import torch
    N, K = closure.N, closure.K
    S = n * n
    cols = len(kns) * ((steps + every - 1) // every) * S
    X = torch.empty((closure.F, cols), dtype=torch.float32, device="cuda")
    T = torch.empty((closure.npop, cols), dtype=torch.float32, device="cuda")
    tmp = torch.empty((closure.npop, S), dtype=torch.float32, device="cuda")
    off = 0
    for r, kn in enumerate(kns):
        tau = W.tau_from_kn(kn, n)
        fl = W.riemann_2d(n, n, RIEMANN, jitter=0.01, seed=seed + r)
        fine = R.Simulation(n, n, N, K_fine, tau, "fp32", W.BC_COPYOUT, W.BC_COPYOUT,
                            stream=closure.stream)
        coarse = R.Simulation(n, n, N, K, tau, "fp32", W.BC_COPYOUT, W.BC_COPYOUT,
                              stream=closure.stream)
        fine.init_fields(fl)
        coarse.init_fields(fl)
        for t in range(steps):
            fview = _view(fine)
            if t % every == 0:
                cview = _view(coarse)
                closure.restrict(K_fine, fview, cview)      # coarse state := R f_fine(t)
                coarse.step(1)
                cview = _view(coarse)
                closure.features(cview, kn_feature(tau, n), X, off)
            fine.step(1)
            if t % every == 0:
                closure.restrict(K_fine, _view(fine), tmp)  # R f_fine(t+1)
                closure.target(tmp, cview, T, off)
                off += S
        fine.sync()
        coarse.sync()
        fine.close()
        coarse.close()
    return X[:, :off], T[:, :off]


def _view(sim: R.Simulation):
    """The current population buffer of an FP32 Simulation as a (npop, sites) tensor view."""
    import torch
    base = sim._buf
    off = sim.current_buffer_ptr() - base.data_ptr()
    return base[off:off + sim.pop_bytes].view(torch.float32).view(sim.npop, sim.sites)


def train(closure: R.Closure, X, T, iters: int = 300, batch: int = 4096, lr: float = 2e-3,
          seed: int = 0, log_every: int = 0, decay: bool = False):
    """Adam on random contiguous column blocks; with decay the step size
    follows a half cosine from lr down to 0 over the iterations."""
    cols = X.shape[1]
    batch = min(batch, cols)
    work = closure.work(X.shape[1])
    rng = np.random.default_rng(seed)
    losses = []
    for it in range(iters):
        off = int(rng.integers(0, cols - batch + 1))
        lr_it = lr * 0.5 * (1.0 + math.cos(math.pi * it / iters)) if decay else lr
        losses.append(closure.train_step(X, T, off, batch, max(lr_it, 1e-7), work))
        if log_every and it % log_every == 0:
            print(f"iter {it} loss {losses[-1]:.4e}")
    return losses


def deploy(closure: R.Closure, n: int, K_fine: int, kn: float, steps: int, seed: int = 99,
           train_n: int | None = None):
    """Fine, plain coarse and corrected coarse runs of one Riemann problem; returns
    (moments fine, moments coarse, moments corrected), each (6, n, n).  train_n:
    the side of the training grid (default n)."""
    N, K = closure.N, closure.K
    tau = W.tau_from_kn(kn, n)
    feat = kn_feature(tau, train_n or n)
    fl = W.riemann_2d(n, n, RIEMANN, jitter=0.01, seed=seed)
    out = []
    for (k, corrected) in ((K_fine, False), (K, False), (K, True)):
        sim = R.Simulation(n, n, N, k, tau, "fp32", W.BC_COPYOUT, W.BC_COPYOUT, stream=closure.stream)
        sim.init_fields(fl)
        if corrected:
            for _ in range(steps):
                sim.step(1)
                closure.apply(sim, feat)
        else:
            sim.step(steps)
        out.append(sim.moments())
        sim.close()
    return tuple(out)


def rel_l2(a, b):
    """Relative L2 error, Eq. (rel_err)."""
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
