#include "flbm_multi.cuh"
namespace flbm {
template struct MLaunch<D3Q19, 2>;
template struct MLaunch<D3Q19, 3>;
template struct MLaunch<D3Q19, 4>;
} // namespace flbm
