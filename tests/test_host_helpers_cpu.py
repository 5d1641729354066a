"""CPU checks of host-side helpers: the sweep driver's coarsening and error,
its argument checks, the workload definitions of the paper's runs, and the
benchmark's JSON helpers.  No GPU."""
import math
import sys

import numpy as np
import pytest

from paper_2011_06856_gb300 import ksweep
from paper_2011_06856_gb300 import workloads as W


def test_coarsen_block_means():
    f = np.arange(2 * 1 * 8, dtype=float).reshape(2, 1, 8)
    c = ksweep.coarsen(f, 2, 1)
    np.testing.assert_array_equal(c, 0.5 * (f[..., 0::2] + f[..., 1::2]))
    g = np.random.default_rng(0).random((2, 8, 12))
    c2 = ksweep.coarsen(g, 4, 2)
    assert c2.shape == (2, 2, 3)
    assert abs(c2[1, 1, 2] - g[1, 4:8, 8:12].mean()) < 1e-15


def test_rel_err_is_eq_rel_err():
    b = np.array([0.1, 0.2, -0.3])
    assert ksweep.rel_err(b, b) == 0.0
    assert abs(ksweep.rel_err(2 * b, b) - 1.0) < 1e-15


def test_convergence_rejects_grids_before_any_run():
    with pytest.raises(ValueError):
        ksweep.convergence([1.0], [700], [12], L_ref=12000)   # 700 does not divide 12000
    with pytest.raises(ValueError):
        ksweep.convergence([1.0], [750], [12], L_ref=12000)   # 0.9 * 750 / 2 is not whole


def test_paper_workloads():
    w = W.WORKLOADS["sod1d_4000x1_N3K600"]
    assert w.npop == 2400 and w.steps == int(0.9 * w.nx / 2)
    fl = W.workload_fields(w)
    assert fl.n[0, 0] == 1.5 and fl.T[0, 0] == 1.5 and fl.n[0, -1] == 0.1 and fl.T[0, -1] == 0.5
    w2 = W.WORKLOADS["sod2d_1000sq_N3K600"]
    fl2 = W.workload_fields(w2)
    assert fl2.by[0, -1] == 0.1 and fl2.bx[-1, 0] == 0.1 and fl2.n[-1, -1] == 1.0
    wl = W.WORKLOADS["onlattice2d_1000sq_N3"]
    assert W.light_speed(wl) == 5.0 and W.light_speed(w) == 1.0
    assert W.tau_from_kn(0.1, 1000, W.light_speed(wl)) == 20.0
    assert math.isinf(W.tau_from_kn(math.inf, 100))
    assert W.statistics(W.WORKLOADS["fermi2d_500sq_N3K12"]) == ("fd", 0.1)
    assert W.statistics(w) == ("mj", 1.0)


def test_bench_json_helpers():
    sys.argv = ["bench.py"]
    import bench
    assert bench.kn_json([0.1, math.inf]) == [0.1, "inf"]
    # streaming 9 + sums 9 + equilibrium 13 + omega 4 + relaxation 3, plus 500 once per site / 256
    assert abs(bench.fp64_flops_per_update(3, True, 256) - (38 + 500 / 256)) < 1e-12
    # the L2 label: the default workload streams from HBM, the 8192 x 4 tube stays in L2
    big = W.WORKLOADS["riemann2d_2048_N2K48"]
    small = W.WORKLOADS["shock1d_8192x4_N3K64"]
    assert 2 * 2 * big.sites * big.npop > bench.L2_BYTES > 2 * 4 * small.sites * small.npop
