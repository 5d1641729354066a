"""GB300-native relativistic lattice Boltzmann hot path (arXiv 2011.06856).

The compute path is the CUDA library ``librlbm.so`` (sources in ``csrc/``),
reached through the C ABI declared in ``include/rlbm.h``; :mod:`.rlbm` is the
thin ctypes binding.  :mod:`.workloads` draws seeded synthetic inputs.
"""
__all__ = ["rlbm", "workloads"]
