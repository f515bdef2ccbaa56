"""GB300-native soft-sphere DEM hot path (Yade documentation, chapter 2).

The compute path is the CUDA library ``libdem.so`` (C ABI in
``include/dem.h``); this package is its thin Python binding.  Import is
cheap: the library is loaded on first use, and a missing library raises.
"""
from .dem import (DEM_FP64, DEM_LAW_HERTZ_MINDLIN, DEM_LAW_LINEAR, DEM_MIXED, DemError, Scene,
                  Server, exported_symbols, find_pairs, load_library, version)

__all__ = ["Scene", "Server", "DemError", "find_pairs", "load_library", "exported_symbols",
           "version", "DEM_FP64", "DEM_MIXED", "DEM_LAW_LINEAR", "DEM_LAW_HERTZ_MINDLIN"]
