"""GB300 (sm_103a) library for the fluctuating two-species lattice Boltzmann
update of arXiv 1410.5584 (Sec. V B): a C-ABI CUDA library (``libflbm.so``,
``include/flbm.h``) and this thin Python binding."""
from .flbm import (D2Q9, D3Q19, Batch, FlbmError, Lattice, MultiLattice, lib, library_path, version)  # noqa: F401
