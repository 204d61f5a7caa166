// Kernel instances for the D3Q19 lattice with F32 population storage.
#include "flbm_kernels.cuh"

template struct flbm::Launch<flbm::D3Q19, flbm::StoreF32>;
