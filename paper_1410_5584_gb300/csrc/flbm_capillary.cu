// flbm_capillary.cu -- capillary fluctuations of a flat interface (Sec. VI B,
// Eq. predictionspectrum): heights of the two interfaces of a stripe and the
// spectrum of their fluctuations, accumulated on the device.  D2Q9 boxes.
//
// One snapshot, in four or five launches:
//   fields   rho_A - rho0_A per site in float (the fluctuation-fields kernel);
//   track    (when the columns are not given) the stripe's middle column x_l
//            and the column x_g half a box away, found on the device;
//   bulk     means over y of that field at the liquid-bulk column x_l and the
//            gas-bulk column x_g (one block, fixed order, FP64);
//   heights  per row y (one warp): the liquid fractions
//            L(y) = sum_x (rho_A - rho_g) / (rho_l - rho_g) of the windows of
//            columns [x_g, x_l) and [x_l, x_g) (periodic) place the two
//            dividing surfaces h1 = x_l - 1/2 - L1 and h2 = x_l - 1/2 + L2, in
//            the frame of x_l, column x covering [x - 1/2, x + 1/2); with
//            tracked columns each snapshot uses its own frame;
//   spectrum each interface's mean height is removed and, for k_m = 2 pi m /
//            n_y, |sum_y dh(y) exp(-i k_m y)|^2 / n_y of the two interfaces is
//            averaged and added to an FP64 accumulator (twiddles from a table
//            indexed by m y mod n_y); the mean heights are accumulated too.
#include <cmath>
#include <vector>

#include "flbm_ctx.h"

using namespace flbm;
using namespace flbm::host;

namespace {

__device__ __forceinline__ int wrap_col(int x, int nx) { return x >= nx ? x - nx : x; }

// Columns of a stripe that may have moved: with C(x) the mean over y of
// rho_A - rho0_A, the window of nx/2 columns with the largest sum of C holds
// the A-rich stripe; its middle column is the liquid-bulk column and the one
// half a box away the gas-bulk column (ties: the lowest x).  One block;
// cols[0] = x_l, cols[1] = x_g.  colsum: nx doubles of scratch.
__global__ void __launch_bounds__(256) k_cap_track(const float2 *__restrict__ z, int nx, int ny,
                                                   double *__restrict__ colsum, int *__restrict__ cols)
{
    __shared__ double best_v[256];
    __shared__ int best_x[256];
    for (int x = threadIdx.x; x < nx; x += 256) {
        double c = 0.0;
        for (int y = 0; y < ny; y++) c += (double)z[(size_t)y * nx + x].x;
        colsum[x] = c;
    }
    __syncthreads();
    const int w = nx / 2;
    double bv = -1e300;
    int bx = nx;
    for (int x0 = threadIdx.x; x0 < nx; x0 += 256) {
        double s = 0.0;
        for (int k = 0; k < w; k++) s += colsum[wrap_col(x0 + k, nx)];
        if (s > bv) {
            bv = s;
            bx = x0;
        }
    }
    best_v[threadIdx.x] = bv;
    best_x[threadIdx.x] = bx;
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) {
            const double v2 = best_v[threadIdx.x + st];
            const int x2 = best_x[threadIdx.x + st];
            if (v2 > best_v[threadIdx.x] || (v2 == best_v[threadIdx.x] && x2 < best_x[threadIdx.x])) {
                best_v[threadIdx.x] = v2;
                best_x[threadIdx.x] = x2;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const int xl = wrap_col(best_x[0] + w / 2, nx);
        cols[0] = xl;
        cols[1] = wrap_col(xl + nx / 2, nx);
    }
}

// columns from the caller (fixed) or from k_cap_track (cols)
__device__ __forceinline__ void cap_cols(int xl_in, int xg_in, const int *cols, int &xl, int &xg)
{
    if (xl_in >= 0) {
        xl = xl_in;
        xg = xg_in;
    } else {
        xl = cols[0];
        xg = cols[1];
    }
}

__global__ void __launch_bounds__(256) k_cap_bulk(const float2 *__restrict__ z, int nx, int ny, int xl_in, int xg_in,
                                                  const int *__restrict__ cols, double *__restrict__ bulk)
{
    __shared__ double sh[256][2];
    int xl, xg;
    cap_cols(xl_in, xg_in, cols, xl, xg);
    double l = 0.0, g = 0.0;
    for (int y = threadIdx.x; y < ny; y += 256) {
        l += (double)z[(size_t)y * nx + xl].x;
        g += (double)z[(size_t)y * nx + xg].x;
    }
    sh[threadIdx.x][0] = l;
    sh[threadIdx.x][1] = g;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            sh[threadIdx.x][0] += sh[threadIdx.x + s][0];
            sh[threadIdx.x][1] += sh[threadIdx.x + s][1];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        bulk[0] = sh[0][0] / ny;
        bulk[1] = sh[0][1] / ny;
    }
}

// one warp per row; h[0][y] and h[1][y]
__global__ void __launch_bounds__(128) k_cap_heights(const float2 *__restrict__ z, int nx, int ny, int xl_in,
                                                     int xg_in, const int *__restrict__ cols,
                                                     const double *__restrict__ bulk, double *__restrict__ h)
{
    const int lane = threadIdx.x & 31;
    const int y = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (y >= ny) return;
    int xl, xg;
    cap_cols(xl_in, xg_in, cols, xl, xg);
    const double rl = bulk[0], rg = bulk[1], inv = 1.0 / (rl - rg);
    const int n1 = xl - xg >= 0 ? xl - xg : xl - xg + nx; // window [x_g, x_l)
    const int n2 = nx - n1;                               // window [x_l, x_g)
    const float2 *row = z + (size_t)y * nx;
    double s1 = 0.0, s2 = 0.0;
    for (int k = lane; k < n1; k += 32) s1 += ((double)row[wrap_col(xg + k, nx)].x - rg) * inv;
    for (int k = lane; k < n2; k += 32) s2 += ((double)row[wrap_col(xl + k, nx)].x - rg) * inv;
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_down_sync(0xffffffffu, s1, o);
        s2 += __shfl_down_sync(0xffffffffu, s2, o);
    }
    if (lane == 0) {
        h[y] = xl - 0.5 - s1;
        h[ny + y] = xl - 0.5 + s2;
    }
}

// one block: mean heights, then the spectrum of both interfaces for m = 1..nk
__global__ void __launch_bounds__(256) k_cap_spectrum(const double *__restrict__ h, int ny, int nk,
                                                      const double2 *__restrict__ tw, double *__restrict__ acc,
                                                      double *__restrict__ hsum)
{
    __shared__ double sh[256][2];
    __shared__ double mean[2];
    double a = 0.0, b = 0.0;
    for (int y = threadIdx.x; y < ny; y += 256) {
        a += h[y];
        b += h[ny + y];
    }
    sh[threadIdx.x][0] = a;
    sh[threadIdx.x][1] = b;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            sh[threadIdx.x][0] += sh[threadIdx.x + s][0];
            sh[threadIdx.x][1] += sh[threadIdx.x + s][1];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        mean[0] = sh[0][0] / ny;
        mean[1] = sh[0][1] / ny;
        hsum[0] += mean[0];
        hsum[1] += mean[1];
    }
    __syncthreads();
    for (int m = 1 + (int)threadIdx.x; m <= nk; m += 256) {
        double r0 = 0.0, i0 = 0.0, r1 = 0.0, i1 = 0.0;
        int idx = 0; // m y mod ny
        for (int y = 0; y < ny; y++) {
            const double2 w = tw[idx]; // (cos, -sin)(2 pi idx / ny)
            const double d0 = h[y] - mean[0], d1 = h[ny + y] - mean[1];
            r0 += d0 * w.x;
            i0 += d0 * w.y;
            r1 += d1 * w.x;
            i1 += d1 * w.y;
            idx += m;
            if (idx >= ny) idx -= ny;
        }
        acc[m - 1] += 0.5 * (r0 * r0 + i0 * i0 + r1 * r1 + i1 * i1) / ny;
    }
}

} // namespace

namespace flbm {
void free_cap(flbm_ctx *c)
{
    if (c->d_cap_z) cudaFree(c->d_cap_z);
    if (c->d_cap_h) cudaFree(c->d_cap_h);
    if (c->d_cap_tw) cudaFree(c->d_cap_tw);
    c->d_cap_z = nullptr;
    c->d_cap_h = nullptr;
    c->d_cap_tw = nullptr;
    c->cap_count = 0;
}
} // namespace flbm

extern "C" {

flbm_status flbm_cap_sample(flbm_ctx *c, int x_liquid, int x_gas)
{
    if (!c) return FLBM_EINVAL;
    if (is_batch(c)) return fail(c, FLBM_EINVAL, "a batch has one spectrum per replica: use flbm_batch_replica");
    if (c->lat != FLBM_D2Q9) return fail(c, FLBM_EUNSUPPORTED, "interface heights are defined for D2Q9 stripes");
    if (!c->initialised) return fail(c, FLBM_ESTATE, "flbm_cap_sample before flbm_init");
    const bool track = x_liquid < 0 && x_gas < 0;
    if (!track && (x_liquid < 0 || x_liquid >= c->nx || x_gas < 0 || x_gas >= c->nx || x_liquid == x_gas))
        return fail(c, FLBM_EINVAL, "bulk columns must be two different columns of the box, or both negative");
    if (track) x_liquid = x_gas = -1;
    if (c->cap_count > 0 && (x_liquid != c->cap_xl || x_gas != c->cap_xg))
        return fail(c, FLBM_EINVAL, "bulk columns differ from the accumulated snapshots; reset first");
    flbm_status st = ensure_obs(c); // block partials of the fields kernel
    if (st != FLBM_OK) return st;
    const int ny = c->ny, nk = ny / 2;
    if (!c->d_cap_z) {
        // layout of d_cap_h: heights [2][ny], spectrum sums [nk], mean-height sums [2], bulk [2],
        // column sums [nx], tracked columns (2 ints in one double)
        if (cudaMalloc((void **)&c->d_cap_z, (size_t)c->N * sizeof(float2)) != cudaSuccess ||
            cudaMalloc((void **)&c->d_cap_h, (size_t)(2 * ny + nk + 5 + c->nx) * sizeof(double)) != cudaSuccess ||
            cudaMalloc((void **)&c->d_cap_tw, (size_t)ny * sizeof(double2)) != cudaSuccess) {
            cudaGetLastError();
            free_cap(c);
            return fail(c, FLBM_ENOMEM, "capillary-spectrum buffers do not fit");
        }
        std::vector<double2> tw((size_t)ny);
        for (int j = 0; j < ny; j++) {
            const double a = 2.0 * M_PI * (double)j / (double)ny;
            tw[j] = make_double2(std::cos(a), -std::sin(a));
        }
        FLBM_CUDA(c, cudaMemcpy(c->d_cap_tw, tw.data(), tw.size() * sizeof(double2), cudaMemcpyHostToDevice),
                  "H2D twiddles");
        FLBM_CUDA(c, cudaMemsetAsync(c->d_cap_h, 0, (size_t)(2 * ny + nk + 5 + c->nx) * sizeof(double), c->stream),
                  "memset");
        c->cap_count = 0;
    }
    double *heights = c->d_cap_h, *spec = heights + 2 * ny, *hsum = spec + nk, *bulk = hsum + 2;
    double *colsum = bulk + 2;
    int *cols = reinterpret_cast<int *>(colsum + c->nx);
    const StepParams p = make_params(c);
    int nb = 0;
    FLBM_CUDA(c, launch_sfk_fields(c->lat, c->storage, layout_parity(c), p, cur_pop(c), c->d_cap_z, c->d_partials, &nb, c->stream),
              "fields kernel launch");
    if (x_liquid < 0) k_cap_track<<<1, 256, 0, c->stream>>>(c->d_cap_z, c->nx, ny, colsum, cols);
    k_cap_bulk<<<1, 256, 0, c->stream>>>(c->d_cap_z, c->nx, ny, x_liquid, x_gas, cols, bulk);
    k_cap_heights<<<(ny + 3) / 4, 128, 0, c->stream>>>(c->d_cap_z, c->nx, ny, x_liquid, x_gas, cols, bulk, heights);
    k_cap_spectrum<<<1, 256, 0, c->stream>>>(heights, ny, nk, c->d_cap_tw, spec, hsum);
    FLBM_CUDA(c, cudaGetLastError(), "capillary kernel launch");
    c->cap_xl = x_liquid;
    c->cap_xg = x_gas;
    c->cap_count++;
    return FLBM_OK;
}

flbm_status flbm_cap_spectrum(flbm_ctx *c, int nk, double *S_h, double *h_mean, int64_t *nsamples)
{
    if (!c) return FLBM_EINVAL;
    if (nsamples) *nsamples = c->cap_count;
    if (!c->d_cap_h || c->cap_count == 0) return fail(c, FLBM_ESTATE, "no capillary snapshot taken");
    const int ny = c->ny, nmax = ny / 2;
    if (nk < 1 || nk > nmax) return fail(c, FLBM_EINVAL, "nk must lie in [1, %d]", nmax);
    flbm_status st = sync_and_check(c);
    if (st != FLBM_OK) return st;
    std::vector<double> h((size_t)nmax + 2);
    FLBM_CUDA(c, cudaMemcpy(h.data(), c->d_cap_h + 2 * ny, h.size() * sizeof(double), cudaMemcpyDeviceToHost),
              "D2H spectrum");
    if (S_h)
        for (int m = 0; m < nk; m++) S_h[m] = h[m] / (double)c->cap_count;
    if (h_mean) {
        h_mean[0] = h[nmax] / (double)c->cap_count;
        h_mean[1] = h[nmax + 1] / (double)c->cap_count;
    }
    return FLBM_OK;
}

flbm_status flbm_cap_reset(flbm_ctx *c)
{
    if (!c) return FLBM_EINVAL;
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_cap(c);
    return FLBM_OK;
}

} // extern "C"
