"""GB300-native (sm_103a) D2V16 MRT flux-limiter finite-difference lattice Boltzmann step.

The compute path is the C-ABI library ``liblbm.so`` (CUDA kernels in ``csrc/``);
``lbm.py`` is its thin ctypes binding, ``workloads.py`` the seeded input
generators.  Importing this package loads nothing; ``lbm.load()`` loads the
library and raises if it has not been built.
"""
__all__ = ["lbm", "workloads", "build"]
