"""GB300 (sm_103a) implementation of the per-time-step bond loop of updated
Lagrangian unsaturated periporomechanics (Menon & Song, arXiv:2203.05562).

The compute path is the CUDA library ``_lib/libppm.so`` behind the C ABI of
``include/ppm.h``; :mod:`.ppm` is a thin ctypes binding over it that uses
PyTorch only for the device workspace and the current stream.
"""
from .ppm import (FIELD, MIXED, FP64, STANDARD, SUBHORIZON, SUBHORIZON_CONJUGATE, PPMError,
                  Simulation, library, make_params)

__all__ = ["Simulation", "PPMError", "library", "make_params", "FIELD", "FP64", "MIXED",
           "SUBHORIZON", "STANDARD", "SUBHORIZON_CONJUGATE"]
