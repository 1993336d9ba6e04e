"""GB300 (sm_103a) implementation of the coupled lattice Boltzmann / discrete
element step for discrete particle simulations (Rettinger & Ruede,
arXiv:1711.00336).

The compute path is the CUDA library ``_build/libdps.so`` behind the C ABI of
``include/dps.h``; :mod:`.dps` is its thin ctypes binding and :mod:`.build`
compiles it.  Importing this package does not load the library; ``dps.lib()``
does, and raises if it has not been built.
"""
from . import workloads  # noqa: F401  (seeded synthetic inputs, no method arithmetic)

__all__ = ["build", "dps", "workloads"]
