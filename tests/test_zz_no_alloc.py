"""The allocation-free entry point against the FP64 oracle and the ordinary one.

rlbm_step_noalloc serves callers that cannot let the library allocate device
memory (their memory comes from their own pool or allocator, or a fixed
budget): it keeps its tables and status word in a static device array and
writes into buffers the caller owns.  Here the caller's buffers are torch
tensors; two calls in a row must reproduce two oracle steps and two steps of
a handle created with rlbm_create, within the parity tolerances of the other
GPU tests.  This file is collected last, and it also runs alone in a fresh
process."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2011_06856_gb300 import build as B  # noqa: E402
from paper_2011_06856_gb300 import rlbm as R  # noqa: E402
from paper_2011_06856_gb300 import workloads as W  # noqa: E402

B.build()

TOL = {"fp64": 1e-12, "fp32": 1e-6}
DT = {"fp64": torch.float64, "fp32": torch.float32}


def relerr(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("precision,nx,ny,N,K,bcx,bcy", [
    ("fp64", 150, 1, 2, 16, W.BC_COPYOUT, W.BC_PERIODIC),
    ("fp64", 70, 9, 3, 64, W.BC_COPYOUT, W.BC_COPYOUT),
    ("fp32", 96, 5, 2, 48, W.BC_PERIODIC, W.BC_PERIODIC),
    ("fp32", 90, 4, 2, 20, W.BC_COPYOUT, W.BC_PERIODIC),   # P = 24 for K = 20: a partly filled warp
    ("fp32", 77, 6, 3, 32, W.BC_PERIODIC, W.BC_COPYOUT),   # N = 3, ragged tile
])
def test_noalloc_two_steps_match_oracle_and_handle(precision, nx, ny, N, K, bcx, bcy):
    tau = 2.5
    fl = W.random_fields(nx, ny, seed=nx + K)
    q = O.Quadrature(N, K)
    f0 = q.init(fl.n, fl.T, fl.bx, fl.by)
    if precision == "fp32":
        f0 = f0.astype(np.float32).astype(np.float64)  # the state the FP32 buffer holds
    o1, _ = q.run(f0, tau, 1, bcx, bcy)
    o2, _ = q.run(f0, tau, 2, bcx, bcy)

    sim = R.Simulation(nx, ny, N, K, tau, precision, bcx, bcy)
    sim.set_populations(f0.astype(np.float32) if precision == "fp32" else f0)  # raw storage bytes
    sim.step(1)
    h1 = sim.get_populations()
    sim.step(1)
    h2 = sim.get_populations()

    a = torch.tensor(f0, dtype=DT[precision], device="cuda").contiguous()
    b = torch.empty_like(a)
    c = torch.empty_like(a)
    torch.cuda.synchronize()
    R.step_noalloc(nx, ny, N, K, tau, precision, a, b, bcx, bcy)
    R.step_noalloc(nx, ny, N, K, tau, precision, b, c, bcx, bcy)
    g1 = b.cpu().numpy().astype(np.float64)
    g2 = c.cpu().numpy().astype(np.float64)
    for got, orc, hnd in ((g1, o1, h1), (g2, o2, h2)):
        assert relerr(got, orc) < TOL[precision]
        assert relerr(got, hnd.astype(np.float64)) < TOL[precision]


def test_noalloc_on_a_stream():
    nx, ny, N, K, tau = 64, 3, 2, 16, 3.0
    fl = W.random_fields(nx, ny, seed=4)
    q = O.Quadrature(N, K)
    f0 = q.init(fl.n, fl.T, fl.bx, fl.by)
    ref, _ = q.run(f0, tau, 1, W.BC_COPYOUT, W.BC_PERIODIC)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        a = torch.tensor(f0, dtype=torch.float64, device="cuda")
        b = torch.empty_like(a)
        R.step_noalloc(nx, ny, N, K, tau, "fp64", a, b, stream=s)
        got = b.cpu().numpy()
    assert relerr(got, ref) < TOL["fp64"]


def test_noalloc_reports_an_unphysical_state_then_recovers():
    nx, ny, N, K, tau = 16, 2, 2, 16, 3.0
    q = O.Quadrature(N, K)
    f0 = W.random_populations(q.npop, ny, nx, seed=9) * q.w[:, None, None]
    bad = -f0  # negative populations everywhere: no streamed site has a physical Landau frame
    a = torch.tensor(bad, dtype=torch.float64, device="cuda")
    b = torch.empty_like(a)
    with pytest.raises(R.Unphysical):
        R.step_noalloc(nx, ny, N, K, tau, "fp64", a, b, W.BC_PERIODIC, W.BC_PERIODIC)
    # the next call clears the status word and steps a physical state correctly
    a = torch.tensor(f0, dtype=torch.float64, device="cuda")
    R.step_noalloc(nx, ny, N, K, tau, "fp64", a, b, W.BC_PERIODIC, W.BC_PERIODIC)
    ref, _ = q.run(f0, tau, 1, W.BC_PERIODIC, W.BC_PERIODIC)
    assert relerr(b.cpu().numpy(), ref) < TOL["fp64"]


def test_noalloc_rejects_overlapping_buffers():
    nx, ny, N, K = 32, 1, 2, 16
    count = K * (N + 1) * nx * ny
    buf = torch.zeros(2 * count, dtype=torch.float32, device="cuda")
    with pytest.raises(R.RLBMError) as e:  # fout starts inside fin
        R.step_noalloc(nx, ny, N, K, 1.0, "fp32", buf[:count], buf[count // 2: count // 2 + count])
    assert e.value.status == R.ERR_ARG


def test_noalloc_rejects_sizes_beyond_its_scratch():
    nx, ny, N, K = 8, 1, 3, 96  # 384 populations > 256
    a = torch.zeros(K * (N + 1) * nx * ny, device="cuda")
    with pytest.raises(R.RLBMError) as e:
        R.step_noalloc(nx, ny, N, K, 1.0, "fp32", a, a.clone())
    assert e.value.status == R.ERR_ARG
    assert "256" in str(e.value)
