"""Batched form: every problem of a mixed batch, stepped by one persistent
launch (mode 'persistent') or by its own kernels on a pool of streams (mode
'streams'), equals the FP64 oracle run of that problem alone."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import oracle as O  # noqa: E402
from paper_2011_06856_gb300 import build as B  # noqa: E402
from paper_2011_06856_gb300 import rlbm as R  # noqa: E402
from paper_2011_06856_gb300 import workloads as W  # noqa: E402

B.build()

MIXED = [  # nx, ny, bc_x, bc_y, K, tau
    (100, 1, 1, 0, 16, 4.0), (70, 3, 1, 1, 48, 2.5), (33, 1, 0, 0, 64, math.inf),
    (64, 5, 1, 0, 32, 1.5), (130, 2, 0, 1, 24, 3.0), (40, 1, 1, 0, 48, 6.0),
    (96, 4, 0, 0, 16, 2.0), (31, 2, 1, 1, 64, 2.2),
]


def relerr(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def run_oracle(spec, fl, steps):
    nx, ny, bcx, bcy, K, tau = spec
    q = O.Quadrature(2, K)
    f = q.init(fl.n, fl.T, fl.bx, fl.by)
    return q.run(f, tau, steps, bcx, bcy)[0]


@pytest.mark.parametrize("mode,autotune", [("persistent", False), ("persistent", True), ("streams", False)])
def test_mixed_batch_matches_oracle_per_problem(mode, autotune):
    b = R.Batch(MIXED, N=2, precision="fp64")
    if autotune:
        b.autotune(2)
    else:
        b.set_mode(mode)
    assert b.mode in R.Batch.MODES
    fields = [W.random_fields(s[0], s[1], seed=40 + i) for i, s in enumerate(MIXED)]
    for p, fl in zip(b.problems, fields):
        p.init_fields(fl)
    steps = 7
    b.step(3)
    b.step(4)  # two launches: the buffer parity carries over
    b.sync()
    assert b.kernel_launches >= 2
    for i, (p, fl) in enumerate(zip(b.problems, fields)):
        ref = run_oracle(MIXED[i], fl, steps)
        assert p.steps_done == steps
        assert relerr(p.get_populations(), ref) < 1e-12, i


@pytest.mark.parametrize("mode", ["persistent", "streams", "autotuned"])
def test_batch_fp32_matches_oracle(mode):
    b = R.Batch(MIXED, N=2, precision="fp32")
    if mode == "autotuned":
        b.autotune(2)
    else:
        b.set_mode(mode)
    fields = [W.random_fields(s[0], s[1], seed=7 + i) for i, s in enumerate(MIXED)]
    for p, fl in zip(b.problems, fields):
        p.init_fields(fl)
    b.step(20)
    b.step(13)  # 32-step graphs and single launches per problem in the streams mode
    b.sync()
    for i, (p, fl) in enumerate(zip(b.problems, fields)):
        ref = run_oracle(MIXED[i], fl, 33)
        assert p.steps_done == 33
        assert relerr(p.get_populations().astype(np.float64), ref) < 3e-5, i


@pytest.mark.parametrize("mode", ["persistent", "streams"])
def test_batch_reinit_one_problem_midway(mode):
    b = R.Batch(MIXED[:3], N=2, precision="fp64")
    b.set_mode(mode)
    fields = [W.random_fields(s[0], s[1], seed=3 + i) for i, s in enumerate(MIXED[:3])]
    for p, fl in zip(b.problems, fields):
        p.init_fields(fl)
    b.step(5)
    b.problems[1].init_fields(fields[1])  # back to step 0 on buffer 0 for this one
    b.step(4)
    b.sync()
    assert relerr(b.problems[0].get_populations(), run_oracle(MIXED[0], fields[0], 9)) < 1e-12
    assert relerr(b.problems[1].get_populations(), run_oracle(MIXED[1], fields[1], 4)) < 1e-12


def test_batch_barrier_timeout_is_reported():
    b = R.Batch(MIXED[:2], N=2, precision="fp32")
    for i, p in enumerate(b.problems):
        p.init_fields(W.random_fields(MIXED[i][0], MIXED[i][1], seed=i))
    b.set_wait_limit(2_000_000)
    b.test_stall_next_step()
    b.step(3)  # the barrier waits for one CTA more than the grid: every wait runs out
    with pytest.raises(R.DeviceTimeout):
        b.sync()
    b.step(2)  # the context and the batch still work
    b.sync()


def test_batch_mode_switch_keeps_the_state():
    """Switching modes between calls re-tiles the problems but keeps their state."""
    b = R.Batch(MIXED[:5], N=2, precision="fp32")
    fields = [W.random_fields(s[0], s[1], seed=90 + i) for i, s in enumerate(MIXED[:5])]
    for p, fl in zip(b.problems, fields):
        p.init_fields(fl)
    b.step(6)
    b.set_mode("streams")
    b.step(5)
    b.set_mode("persistent")
    b.step(4)
    b.sync()
    for i, (p, fl) in enumerate(zip(b.problems, fields)):
        assert relerr(p.get_populations().astype(np.float64), run_oracle(MIXED[i], fl, 15)) < 3e-5, i
    b.set_mode("streams")
    with pytest.raises(R.RLBMError):
        b.test_stall_next_step()  # no barrier to stall in this mode


@pytest.mark.parametrize("mode", ["streams", "persistent"])
def test_full_batch_256_sampled_problems_one_step(mode):
    """The batched benchmark workload at full size (256 uneven problems, FP32,
    61.7 GB of populations) in both execution modes: four problems (the
    smallest, the largest, a 64-row and a long 1D one) start from the oracle's
    initial state (uploaded), the rest from the GPU initialisation; after one
    batched step the four are checked against one oracle step, on whole 1D
    problems and on interior rows of 2D ones (a three-row band reproduces its
    middle row exactly)."""
    probs = W.batch_problems(256)
    specs = [(p.nx, p.ny, p.bcx, p.bcy, p.K, W.tau_from_kn(p.kn, p.nx)) for p in probs]
    b = R.Batch(specs, N=2, precision="fp32")
    b.set_mode(mode)
    size = [nx * ny * K for (nx, ny, _, _, K, _) in specs]
    picks = {int(np.argmin(size)), int(np.argmax(size))}
    picks.add(next(i for i, s in enumerate(specs) if s[1] == 64))
    picks.add(max((i for i, s in enumerate(specs) if s[1] == 1), key=lambda i: specs[i][0]))
    states = {}
    for i, (p, pb) in enumerate(zip(b.problems, probs)):
        fl = W.shock_tube(pb.nx, pb.ny, pb.left, pb.right)
        if i in picks:
            q = O.Quadrature(2, pb.K)
            f0 = q.init(fl.n, fl.T, fl.bx, fl.by).astype(np.float32)
            p.set_populations(f0)
            states[i] = (q, f0)
        else:
            p.init_fields(fl)
    b.step(1)
    b.sync()
    for i, (q, f0) in states.items():
        nx, ny, bcx, bcy, K, tau = specs[i]
        got = b.problems[i].get_populations().astype(np.float64)
        if ny == 1:
            ref, _ = q.run(f0.astype(np.float64), tau, 1, bcx, bcy)
            assert relerr(got, ref) < 2e-6, i
        else:
            for y in (1, ny // 2, ny - 2):
                band = np.ascontiguousarray(f0[:, y - 1:y + 2, :].astype(np.float64))
                ref, _ = q.run(band, tau, 1, bcx, bcy)
                assert relerr(got[:, y, :], ref[:, 1, :]) < 2e-6, (i, y)
    b.close()
