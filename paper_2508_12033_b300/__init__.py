"""B300-native LRDMC hot path: CUDA library behind a C ABI plus a thin binding.

    from paper_2508_12033_b300 import Lrdmc, LOAD_BALANCED, CONVENTIONAL

The binding only marshals arguments; every step runs in the CUDA kernels of
``liblrdmc.so`` (built by ``paper_2508_12033_b300.build.build()``).  Importing
this package does not load the library; the first use does, and raises if the
library is missing -- there is no CPU fallback.
"""
from .binding import (CONVENTIONAL, LOAD_BALANCED, LrdmcError, Lrdmc, LrdmcBatch, estimate, extrapolate_a,
                      load_library,
                      local_energy,
                      philox4x32, reconfigure_indices)

__all__ = ["Lrdmc", "LrdmcBatch", "LrdmcError", "local_energy", "LOAD_BALANCED", "CONVENTIONAL", "estimate", "extrapolate_a", "load_library",
           "philox4x32", "reconfigure_indices"]
