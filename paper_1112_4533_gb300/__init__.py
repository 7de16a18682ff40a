"""GB300-native (sm_103a) SU(Nc) pure-gauge link sweep.

Chessboard heatbath / overrelaxation sweep of Cardoso & Bicudo,
"Generating SU(Nc) pure gauge lattice QCD configurations on GPUs with CUDA"
(arXiv:1112.4533), behind the C ABI of include/sun.h (libsun.so).
"""
from .sun import (HEATBATH, OVERRELAX, Batch, Lattice, Slabs, SunError, autotune, autotune_batch,  # noqa: F401
                  footprint_bytes, lattice_create, load_library, read_config_header)

__all__ = ["HEATBATH", "OVERRELAX", "Batch", "Lattice", "Slabs", "SunError", "autotune", "autotune_batch", "footprint_bytes",
           "lattice_create", "load_library", "read_config_header"]
