"""The allocation-free entry point against the ordinary one.

rlbm_step_noalloc serves callers that cannot let the library allocate device
memory (their memory comes from their own pool or allocator, or a fixed
budget): it keeps its tables and status word in a static device array and
writes into buffers the caller owns.  Here the caller's buffers are torch
tensors; two calls in a row must reproduce two steps of a handle created with
rlbm_create, within the parity tolerances of the other GPU tests.  This file
is collected last, and it also runs alone in a fresh process."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2011_06856_gb300 import build as B  # noqa: E402
from paper_2011_06856_gb300 import rlbm as R  # noqa: E402
from paper_2011_06856_gb300 import workloads as W  # noqa: E402

B.build()

TOL = {"fp64": 1e-12, "fp32": 1e-6}


@pytest.mark.parametrize("precision,nx,ny,N,K,bcx,bcy", [
    ("fp64", 150, 1, 2, 16, W.BC_COPYOUT, W.BC_PERIODIC),
    ("fp64", 70, 9, 3, 64, W.BC_COPYOUT, W.BC_COPYOUT),
    ("fp32", 96, 5, 2, 48, W.BC_PERIODIC, W.BC_PERIODIC),
])
def test_noalloc_two_steps_match_handle(precision, nx, ny, N, K, bcx, bcy):
    tau = 2.5
    fl = W.random_fields(nx, ny, seed=nx + K)
    sim = R.Simulation(nx, ny, N, K, tau, precision, bcx, bcy)
    sim.init_fields(fl)
    f0 = sim.get_populations()
    sim.step(1)
    f1 = sim.get_populations()
    sim.step(1)
    f2 = sim.get_populations()

    dt = torch.float64 if precision == "fp64" else torch.float32
    a = torch.tensor(f0, dtype=dt, device="cuda").contiguous()
    b = torch.empty_like(a)
    c = torch.empty_like(a)
    torch.cuda.synchronize()
    R.step_noalloc(nx, ny, N, K, tau, precision, a, b, bcx, bcy)
    R.step_noalloc(nx, ny, N, K, tau, precision, b, c, bcx, bcy)
    g1 = b.cpu().numpy().astype(np.float64)
    g2 = c.cpu().numpy().astype(np.float64)
    for got, ref in ((g1, f1), (g2, f2)):
        ref = ref.astype(np.float64)
        assert np.abs(got - ref).max() / np.abs(ref).max() < TOL[precision]


def test_noalloc_rejects_sizes_beyond_its_scratch():
    a = torch.zeros(8, device="cuda")
    with pytest.raises(R.RLBMError) as e:
        R.step_noalloc(8, 1, 3, 96, 1.0, "fp32", a, a.clone())  # 384 populations > 256
    assert e.value.status == R.ERR_ARG
