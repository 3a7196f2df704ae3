"""GB300-native SPH neighbour-interaction hot path (density with smoothing-length
iteration, hydro force, kick-drift-kick) after Schaller et al., PASC '16.

The compute path is the CUDA library `libsph` (C ABI, declared in
include/sph.h); `paper_1606_02738_gb300.sph` is its thin ctypes binding and
`paper_1606_02738_gb300.inputs` holds the seeded synthetic particle sets.
Importing the package loads nothing; the library is loaded on first use.
"""
__all__ = ["inputs", "sph"]
