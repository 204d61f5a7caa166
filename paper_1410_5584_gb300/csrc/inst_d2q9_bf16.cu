// Kernel instances for the D2Q9 lattice with BF16 population storage.
#include "flbm_kernels.cuh"

template struct flbm::Launch<flbm::D2Q9, flbm::StoreBF16>;
