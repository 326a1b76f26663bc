"""GB300-native Monte Carlo dust radiative transfer hot path.

The photon-packet life cycle of arXiv:1705.04702 (launch, peel-off,
continuous absorption, forced Henyey-Greenstein scattering) runs in
hand-written sm_103a CUDA kernels behind the C ABI in ``include/skirt.h``
(``lib/libskirt.so``).  ``skirt`` is its ctypes binding; ``workloads``
describes seeded synthetic problems; ``build`` compiles the library.
"""
__all__ = ["build", "workloads", "skirt"]
