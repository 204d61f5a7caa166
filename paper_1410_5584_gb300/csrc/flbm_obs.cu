// flbm_obs.cu -- observables of the current state, off the per-step loop:
// densities, baricentric velocity (Eq. lattice-vb), FP64 conservation totals
// and the axis structure factors of Sec. VI A.  All reductions run in a fixed
// order, so repeated calls on the same state give bit-identical results.
#include "flbm_internal.h"

namespace flbm {

namespace {

// fixed-order block reduction of NV doubles per thread; result valid in thread 0
template <int NV, int NT>
__device__ __forceinline__ void block_sum(double (&v)[NV], double (*sh)[NV])
{
    const int t = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
#pragma unroll
    for (int k = 0; k < NV; k++) sh[t][k] = v[k];
    __syncthreads();
    for (int stride = NT / 2; stride > 0; stride >>= 1) {
        if (t < stride)
#pragma unroll
            for (int k = 0; k < NV; k++) sh[t][k] += sh[t + stride][k];
        __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < NV; k++) v[k] = sh[0][k];
}

__global__ void __launch_bounds__(256) k_sum_partials(const double *__restrict__ partials, int nblocks,
                                                      double *__restrict__ out)
{
    __shared__ double sh[256][5];
    double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += 256)
#pragma unroll
        for (int k = 0; k < 5; k++) v[k] += partials[(size_t)b * 5 + k];
    block_sum<5, 256>(v, sh);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < 5; k++) out[k] = v[k];
}

// profile[c][pcoord] = sum over the sites with that coordinate along `axis`
__global__ void __launch_bounds__(256) k_profile(int nx, int ny, int nz, int axis, const double *__restrict__ obs,
                                                 double *__restrict__ profile)
{
    __shared__ double sh[256][1];
    const int pc = blockIdx.x, c = blockIdx.y;
    const int n_axis = axis == 0 ? nx : (axis == 1 ? ny : nz);
    const size_t N = (size_t)nx * ny * nz;
    const size_t M = N / n_axis;
    double v[1] = {0.0};
    for (size_t q = threadIdx.x; q < M; q += 256) {
        size_t site;
        if (axis == 0) site = q * nx + pc;
        else if (axis == 1) site = ((q / nx) * ny + pc) * nx + (q % nx);
        else site = (size_t)pc * nx * ny + q;
        v[0] += obs[(size_t)c * N + site];
    }
    block_sum<1, 256>(v, sh);
    if (threadIdx.x == 0) profile[(size_t)c * n_axis + pc] = v[0];
}

// one block per m: Fourier coefficients of the profiles, accumulated |.|^2 / N
__global__ void __launch_bounds__(256) k_dft_accumulate(int D, int n_axis, double inv_n, const double *__restrict__ profile,
                                                        double *__restrict__ acc)
{
    __shared__ double sh[256][10];
    const int m = blockIdx.x + 1;
    const int C = 2 + D;
    double v[10];
#pragma unroll
    for (int k = 0; k < 10; k++) v[k] = 0.0;
    for (int pc = threadIdx.x; pc < n_axis; pc += 256) {
        const long long r = ((long long)m * pc) % n_axis;
        double sn, cs;
        sincospi(2.0 * (double)r / (double)n_axis, &sn, &cs);
        for (int c = 0; c < C; c++) {
            const double P = profile[(size_t)c * n_axis + pc];
            v[2 * c] += P * cs;
            v[2 * c + 1] -= P * sn;
        }
    }
    block_sum<10, 256>(v, sh);
    if (threadIdx.x == 0) {
        const int nk = n_axis / 2;
        const double are = v[0], aim = v[1], bre = v[2], bim = v[3];
        acc[0 * nk + m - 1] += (are * are + aim * aim) * inv_n;
        acc[1 * nk + m - 1] += (are * bre + aim * bim) * inv_n;
        acc[2 * nk + m - 1] += (bre * bre + bim * bim) * inv_n;
        double uu = 0.0;
        for (int d = 0; d < D; d++) uu += v[4 + 2 * d] * v[4 + 2 * d] + v[5 + 2 * d] * v[5 + 2 * d];
        acc[3 * nk + m - 1] += uu / D * inv_n;
    }
}

// Float densities of both species from the caller's double arrays, read
// straight from host memory (NULL: uniform rho0); the smallest index of a
// value that is not positive and finite goes to *bad (left as it is when
// there is none).
__global__ void k_densities_from_host(const double *__restrict__ ra, const double *__restrict__ rb, double r0a,
                                      double r0b, long long n, float *__restrict__ out,
                                      unsigned long long *__restrict__ bad)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const double a = ra ? ra[k] : r0a, b = rb ? rb[k] : r0b;
        const bool oka = a > 0.0 && isfinite(a), okb = b > 0.0 && isfinite(b);
        if (!oka) atomicMin(bad, (unsigned long long)k);
        if (!okb) atomicMin(bad + 1, (unsigned long long)k);
        out[k] = (float)a;
        out[n + k] = (float)b;
    }
}

__global__ void k_add_u32(unsigned *p, unsigned v) { *p += v; }
__global__ void k_set_u32(unsigned *p, unsigned v) { *p = v; }

} // namespace

cudaError_t launch_add_u32(unsigned *p, unsigned v, cudaStream_t stream)
{
    k_add_u32<<<1, 1, 0, stream>>>(p, v);
    return cudaGetLastError();
}

cudaError_t launch_densities_from_host(const double *rho_a, const double *rho_b, double rho0_a, double rho0_b,
                                       int64_t n, float *out, unsigned long long *bad, cudaStream_t stream)
{
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const long long want = (n + 255) / 256, most = (long long)sms * 8;
    k_densities_from_host<<<(unsigned)(want < most ? (want > 0 ? want : 1) : most), 256, 0, stream>>>(
        rho_a, rho_b, rho0_a, rho0_b, (long long)n, out, bad);
    return cudaGetLastError();
}

cudaError_t launch_set_u32(unsigned *p, unsigned v, cudaStream_t stream)
{
    k_set_u32<<<1, 1, 0, stream>>>(p, v);
    return cudaGetLastError();
}

cudaError_t launch_sum_partials(const double *partials, int nblocks, double *out, cudaStream_t stream)
{
    k_sum_partials<<<1, 256, 0, stream>>>(partials, nblocks, out);
    return cudaGetLastError();
}

cudaError_t launch_sf_accumulate(int D, int nx, int ny, int nz, int axis, const double *obs, double *profile,
                                 double *acc, cudaStream_t stream)
{
    const int n_axis = axis == 0 ? nx : (axis == 1 ? ny : nz);
    k_profile<<<dim3(n_axis, 2 + D), 256, 0, stream>>>(nx, ny, nz, axis, obs, profile);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const double inv_n = 1.0 / ((double)nx * ny * nz);
    k_dft_accumulate<<<n_axis / 2, 256, 0, stream>>>(D, n_axis, inv_n, profile, acc);
    return cudaGetLastError();
}

} // namespace flbm
