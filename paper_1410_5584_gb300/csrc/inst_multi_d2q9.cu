#include "flbm_multi.cuh"
namespace flbm {
template struct MLaunch<D2Q9, 2>;
template struct MLaunch<D2Q9, 3>;
template struct MLaunch<D2Q9, 4>;
} // namespace flbm
