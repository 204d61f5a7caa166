// Kernel instances for the D2Q9 lattice with F16 population storage.
#include "flbm_kernels.cuh"

template struct flbm::Launch<flbm::D2Q9, flbm::StoreF16>;
