"""Failure detection on the GPU without a GPU fault: a bounded device wait is
made to run out (its barrier expects bytes that never arrive) and the host
reads the error status; the context stays usable."""
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


def test_stalled_wait_reports_timeout_and_context_survives():
    nx, ny, N, K, tau = 128, 4, 2, 16, 3.0
    sim = R.Simulation(nx, ny, N, K, tau, "fp64", W.BC_COPYOUT, W.BC_PERIODIC)
    assert sim.uses_tma
    fl = W.random_fields(nx, ny, seed=1)
    sim.init_fields(fl)
    sim.set_wait_limit(2_000_000)  # about 1 ms
    sim.test_stall_next_step()
    sim.step(1)
    with pytest.raises(R.DeviceTimeout):
        sim.sync()
    # the status is cleared and the context still works: a fresh state steps correctly
    q = O.Quadrature(N, K)
    f0 = q.init(fl.n, fl.T, fl.bx, fl.by)
    sim.set_populations(f0)
    sim.step(5)
    sim.sync()
    ref, _ = q.run(f0, tau, 5, W.BC_COPYOUT, W.BC_PERIODIC)
    got = sim.get_populations()
    assert np.abs(got - ref).max() / np.abs(ref).max() < 1e-12


def test_wait_limit_validation():
    sim = R.Simulation(64, 1, 2, 16, 1.0, "fp32")
    with pytest.raises(R.RLBMError):
        sim.set_wait_limit(10)


def test_stall_hook_needs_the_tma_kernel(monkeypatch):
    monkeypatch.setenv("RLBM_NO_TMA", "1")
    sim = R.Simulation(64, 1, 2, 16, 1.0, "fp32")
    assert not sim.uses_tma
    with pytest.raises(R.RLBMError) as e:
        sim.test_stall_next_step()
    assert e.value.status == R.ERR_UNSUPPORTED


def test_bulk_staged_pair_kernel_timeout_reports_and_context_survives():
    """The bulk-staged form of the two-sites-per-lane kernel: its slot
    barriers expect 16 bytes more than the copies bring, every bounded wait
    runs out, the warps drain their copies (bounded), skip their stores and
    meet the CTA barriers; the host reads RLBM_ERR_TIMEOUT and the handle
    keeps working."""
    nx, ny, N, K, tau = 256, 3, 2, 16, 3.0
    sim = R.Simulation(nx, ny, N, K, tau, "fp32", W.BC_COPYOUT, W.BC_PERIODIC)
    sim.set_tiling(8, "pair-bulk")
    assert sim.step_kernel == "pair-bulk"
    fl = W.random_fields(nx, ny, seed=2)
    sim.init_fields(fl)
    sim.set_wait_limit(2_000_000)
    sim.test_stall_next_step()
    sim.step(1)
    with pytest.raises(R.DeviceTimeout):
        sim.sync()
    q = O.Quadrature(N, K)
    f0 = q.init(fl.n, fl.T, fl.bx, fl.by)
    sim.set_populations(f0.astype(np.float32))
    sim.step(5)
    sim.sync()
    ref, _ = q.run(f0, tau, 5, W.BC_COPYOUT, W.BC_PERIODIC)
    got = sim.get_populations().astype(np.float64)
    assert np.abs(got - ref).max() / np.abs(ref).max() < 1e-5
    sim.set_tiling(8, "pair")  # no device waits in this form
    with pytest.raises(R.RLBMError):
        sim.test_stall_next_step()


def test_tile_staged_pair_kernel_timeout_reports_and_context_survives():
    """The tile-staged form: its mbarrier expects 16 bytes more than the TMA
    brings, the bounded wait runs out, the CTA drains (bounded) and returns
    without storing; the host reads RLBM_ERR_TIMEOUT and the handle keeps
    working."""
    nx, ny, N, K, tau = 256, 3, 2, 16, 3.0
    sim = R.Simulation(nx, ny, N, K, tau, "fp32", W.BC_COPYOUT, W.BC_PERIODIC)
    sim.set_tiling(16, "pair-tma")
    assert sim.step_kernel == "pair-tma"
    fl = W.random_fields(nx, ny, seed=2)
    sim.init_fields(fl)
    sim.set_wait_limit(2_000_000)
    sim.test_stall_next_step()
    sim.step(1)
    with pytest.raises(R.DeviceTimeout):
        sim.sync()
    q = O.Quadrature(N, K)
    f0 = q.init(fl.n, fl.T, fl.bx, fl.by)
    sim.set_populations(f0.astype(np.float32))
    sim.step(5)
    sim.sync()
    ref, _ = q.run(f0, tau, 5, W.BC_COPYOUT, W.BC_PERIODIC)
    got = sim.get_populations().astype(np.float64)
    assert np.abs(got - ref).max() / np.abs(ref).max() < 1e-5
