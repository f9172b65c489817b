"""GB300-native qubit lattice algorithm (QLA) for 2D Maxwell scattering.

The compute path is the CUDA library ``libqla.so`` (built from ``csrc/``)
behind the C ABI declared in ``include/qla.h``; ``qla`` is its thin ctypes
binding and ``inputs`` the seeded workload generators.  Importing the
package loads nothing; ``qla`` loads the library on first use and raises if
it is missing.
"""
__all__ = ["qla", "inputs"]
