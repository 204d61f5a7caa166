// Kernel instances for the D3Q19 lattice with BF16 population storage.
#include "flbm_kernels.cuh"

template struct flbm::Launch<flbm::D3Q19, flbm::StoreBF16>;
