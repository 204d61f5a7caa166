#include "flbm_multi.cuh"
namespace flbm {
template struct MLaunch<D2Q9, 2>;
template struct MLaunch<D2Q9, 3>;
template struct MLaunch<D2Q9, 4>;
} // namespace flbm

namespace flbm {
cudaError_t launch_msf_snapshot(int ns, const MStepParams &p, int axis, const float4 *drho, double *prof,
                                double *acc, cudaStream_t st)
{
    const int n = axis == 0 ? p.nx : (axis == 1 ? p.ny : p.nz);
    const int nk = n / 2;
    const unsigned kb = (unsigned)((nk + 63) / 64);
    const double inv = 1.0 / (double)p.N;
    switch (ns) {
    case 2:
        mkern::k_mprofile<2><<<n, mkern::kObsBlock, 0, st>>>(p, axis, drho, prof);
        mkern::k_msf_accumulate<2><<<kb, 64, 0, st>>>(prof, n, inv, acc);
        break;
    case 3:
        mkern::k_mprofile<3><<<n, mkern::kObsBlock, 0, st>>>(p, axis, drho, prof);
        mkern::k_msf_accumulate<3><<<kb, 64, 0, st>>>(prof, n, inv, acc);
        break;
    case 4:
        mkern::k_mprofile<4><<<n, mkern::kObsBlock, 0, st>>>(p, axis, drho, prof);
        mkern::k_msf_accumulate<4><<<kb, 64, 0, st>>>(prof, n, inv, acc);
        break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}
} // namespace flbm
