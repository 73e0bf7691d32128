"""GB300-native (sm_103a) WCSPH(-RANS) time step with the improved
bidirectional buffer of Wang & Hu (arXiv 2510.25702).

The compute path is the C-ABI library built from csrc/ (see include/sph.h);
this package holds its thin ctypes binding (``sph``), the build step
(``build``) and the seeded input generators (``cases``).  Submodules are
imported lazily so that ``cases`` works on machines without a GPU.
"""
__all__ = ["cases", "sph", "build"]
