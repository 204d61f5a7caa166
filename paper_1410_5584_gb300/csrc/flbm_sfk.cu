// flbm_sfk.cu -- structure factors at every lattice wavevector (the quantities
// of Eq. str-bin-hom, Sec. IV A, over the whole Brillouin zone) and the
// structure functions of Eq. structurefunctions, accumulated on the device.
//
// One snapshot: a fields kernel sums each site's population deviations into
// z = (rho_A - rho0_A) + i (rho_B - rho0_B) in float, with FP64 block partials
// from which the means follow (fixed order).  The first line-FFT pass
// subtracts the means as it loads, so z becomes the fluctuation field
// delta rho_A + i delta rho_B, and every axis is transformed in place by line
// FFTs in shared memory (radix 2 for power-of-two lengths, a direct DFT
// otherwise).  The two real spectra follow
// from Hermitian symmetry, rho_hat_A(k) = (z(k) + conj z(-k)) / 2 and
// rho_hat_B(k) = (z(k) - conj z(-k)) / (2i), and their products are added
// into FP64 accumulators.  The transform is in float because this GPU's FP64
// rate is a small fraction of its FP32 rate; on fluctuation fields its
// relative error is a few float roundings times log2 N, far below the
// statistical error of any structure-factor estimate.
#include <cmath>
#include <vector>

#include "flbm_ctx.h"

using namespace flbm;
using namespace flbm::host;

namespace {

constexpr int kFftThreads = 256;
constexpr int kSmemBudget = 48 * 1024; // bytes of line data per block

__device__ __forceinline__ float2 cmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }

// lines of one axis of an [nz][ny][nx] array
struct Lines {
    int axis, nx, ny;
    int n;        // points per line
    long stride;  // elements between consecutive points
    long count;   // number of lines
    int group;    // lines per block (adjacent in memory for axes y and z)
    int log2n;    // power-of-two lengths only, else -1
    __device__ __forceinline__ long base(long l) const
    {
        if (axis == 0) return l * nx;
        if (axis == 1) return (l / nx) * (long)nx * ny + l % nx;
        return l;
    }
    // element e of the block's tile -> (line in group, point); axis x reads its
    // lines one after the other, axes y and z read a point of every line of
    // the group at once (adjacent addresses)
    __device__ __forceinline__ void split(int e, int &g, int &j) const
    {
        if (axis == 0) {
            g = e / n;
            j = e - g * n;
        } else {
            j = e / group;
            g = e - j * group;
        }
    }
};

// the value a line transform loads: z minus the field means when `mean` is set
// (the first pass), z otherwise
__device__ __forceinline__ float2 load_point(const float2 *data, long idx, const double *mean)
{
    float2 v = data[idx];
    if (mean) {
        v.x -= (float)mean[0];
        v.y -= (float)mean[1];
    }
    return v;
}

__global__ void __launch_bounds__(kFftThreads) k_fft_pow2(float2 *__restrict__ data, const Lines L,
                                                          const float2 *__restrict__ tw, const double *mean)
{
    extern __shared__ float2 sm[];
    const long l0 = (long)blockIdx.x * L.group;
    const int n = L.n, half_n = n >> 1;
    const int tile = L.group * n;
    for (int e = threadIdx.x; e < tile; e += kFftThreads) {
        int g, j;
        L.split(e, g, j);
        if (l0 + g < L.count)
            sm[g * n + (int)(__brev((unsigned)j) >> (32 - L.log2n))] = load_point(data, L.base(l0 + g) + j * L.stride, mean);
    }
    __syncthreads();
    for (int s = 1; s <= L.log2n; s++) {
        const int half = 1 << (s - 1), tstep = n >> s;
        for (int b = threadIdx.x; b < L.group * half_n; b += kFftThreads) {
            const int g = b / half_n, t = b - g * half_n;
            const int grp = t >> (s - 1), pos = t & (half - 1);
            const int i0 = g * n + (grp << s) + pos, i1 = i0 + half;
            const float2 u = sm[i0], v = cmul(sm[i1], tw[pos * tstep]);
            sm[i0] = make_float2(u.x + v.x, u.y + v.y);
            sm[i1] = make_float2(u.x - v.x, u.y - v.y);
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < tile; e += kFftThreads) {
        int g, j;
        L.split(e, g, j);
        if (l0 + g < L.count) data[L.base(l0 + g) + j * L.stride] = sm[g * n + j];
    }
}

// direct DFT of lines of any length: out_k = sum_j in_j exp(-2 pi i j k / n)
__global__ void __launch_bounds__(kFftThreads) k_dft_lines(float2 *__restrict__ data, const Lines L,
                                                           const float2 *__restrict__ tw, const double *mean)
{
    extern __shared__ float2 sm[];
    const long l0 = (long)blockIdx.x * L.group;
    const int n = L.n, tile = L.group * n;
    float2 *in = sm, *out = sm + tile;
    for (int e = threadIdx.x; e < tile; e += kFftThreads) {
        int g, j;
        L.split(e, g, j);
        if (l0 + g < L.count) in[g * n + j] = load_point(data, L.base(l0 + g) + j * L.stride, mean);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < tile; e += kFftThreads) {
        const int g = e / n, k = e - g * n;
        if (l0 + g >= L.count) continue;
        float2 acc = make_float2(0.0f, 0.0f);
        int idx = 0; // j k mod n
        for (int j = 0; j < n; j++) {
            const float2 v = cmul(in[g * n + j], tw[idx]);
            acc.x += v.x;
            acc.y += v.y;
            idx += k;
            if (idx >= n) idx -= n;
        }
        out[g * n + k] = acc;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < tile; e += kFftThreads) {
        int g, j;
        L.split(e, g, j);
        if (l0 + g < L.count) data[L.base(l0 + g) + j * L.stride] = out[g * n + j];
    }
}

// means of the two fields from the [nblocks][2] block partials (one block,
// fixed order): mean[s] = sum / N
__global__ void __launch_bounds__(256) k_sfk_means(const double *__restrict__ partials, int nblocks, long N,
                                                   double *__restrict__ mean)
{
    __shared__ double sh[256][2];
    double a = 0.0, b = 0.0;
    for (int k = threadIdx.x; k < nblocks; k += 256) {
        a += partials[2 * k];
        b += partials[2 * k + 1];
    }
    sh[threadIdx.x][0] = a;
    sh[threadIdx.x][1] = b;
    __syncthreads();
    for (int stride = 128; stride > 0; stride >>= 1) {
        if ((int)threadIdx.x < stride) {
            sh[threadIdx.x][0] += sh[threadIdx.x + stride][0];
            sh[threadIdx.x][1] += sh[threadIdx.x + stride][1];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        mean[0] = sh[0][0] / (double)N;
        mean[1] = sh[0][1] / (double)N;
    }
}

// acc[0..2][k] += |A|^2, Re(A conj B), |B|^2 with A, B the spectra of the real
// and imaginary parts of z (products in float, sums in FP64); grid over
// (x blocks, y, z)
__global__ void __launch_bounds__(128) k_sfk_accumulate(const float2 *__restrict__ z, int nx, int ny, int nz,
                                                        double *__restrict__ acc)
{
    const int mx = blockIdx.x * blockDim.x + threadIdx.x, my = blockIdx.y, mz = blockIdx.z;
    if (mx >= nx) return;
    const size_t N = (size_t)nx * ny * nz;
    const size_t i = ((size_t)mz * ny + my) * nx + mx;
    const size_t im = ((size_t)(mz == 0 ? 0 : nz - mz) * ny + (my == 0 ? 0 : ny - my)) * nx + (mx == 0 ? 0 : nx - mx);
    const float2 a = z[i], b = z[im];
    const float Ar = 0.5f * (a.x + b.x), Ai = 0.5f * (a.y - b.y);
    const float Br = 0.5f * (a.y + b.y), Bi = 0.5f * (b.x - a.x);
    acc[i] += (double)(Ar * Ar + Ai * Ai);
    acc[N + i] += (double)(Ar * Br + Ai * Bi);
    acc[2 * N + i] += (double)(Br * Br + Bi * Bi);
}

// the structure factors (acc scaled) or the structure functions of Eq.
// structurefunctions about (r0a, r0b)
__global__ void k_sfk_out(const double *__restrict__ acc, long N, double scale, int functions, double r0a,
                          double r0b, double *__restrict__ o0, double *__restrict__ o1, double *__restrict__ o2)
{
    const double rt = r0a + r0b, rt2 = rt * rt;
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < N; i += (long)gridDim.x * blockDim.x) {
        const double saa = acc[i] * scale, sab = acc[N + i] * scale, sbb = acc[2 * N + i] * scale;
        if (!functions) {
            o0[i] = saa;
            o1[i] = sab;
            o2[i] = sbb;
        } else {
            o0[i] = saa + 2.0 * sab + sbb;
            o1[i] = (r0b * r0b * saa - 2.0 * r0a * r0b * sab + r0a * r0a * sbb) / (rt2 * rt2);
            o2[i] = (r0b * saa + (r0b - r0a) * sab - r0a * sbb) / rt2;
        }
    }
}

int log2_exact(int n)
{
    int l = 0;
    while ((1 << l) < n) l++;
    return (1 << l) == n ? l : -1;
}

int grid_for(long n) { return (int)std::min<long>((n + 255) / 256, 152L * 16); }

// twiddles exp(-2 pi i j / n): n/2 of them for radix 2, n for the direct DFT
flbm_status ensure_twiddles(flbm_ctx *c, int axis, int n)
{
    if (c->d_sfk_tw[axis] && c->sfk_tw_n[axis] == n) return FLBM_OK;
    if (c->d_sfk_tw[axis]) cudaFree(c->d_sfk_tw[axis]);
    c->d_sfk_tw[axis] = nullptr;
    const int m = log2_exact(n) >= 0 ? n / 2 : n;
    std::vector<float2> h((size_t)(m > 0 ? m : 1));
    for (int j = 0; j < m; j++) {
        const double a = -2.0 * M_PI * (double)j / (double)n;
        h[j] = make_float2((float)std::cos(a), (float)std::sin(a));
    }
    FLBM_CUDA(c, cudaMalloc((void **)&c->d_sfk_tw[axis], h.size() * sizeof(float2)), "cudaMalloc(twiddles)");
    FLBM_CUDA(c, cudaMemcpy(c->d_sfk_tw[axis], h.data(), h.size() * sizeof(float2), cudaMemcpyHostToDevice),
              "H2D twiddles");
    c->sfk_tw_n[axis] = n;
    return FLBM_OK;
}

flbm_status transform_axis(flbm_ctx *c, int axis, const double *mean)
{
    const int n = axis == 0 ? c->nx : (axis == 1 ? c->ny : c->nz);
    if (n == 1) return FLBM_OK;
    flbm_status st = ensure_twiddles(c, axis, n);
    if (st != FLBM_OK) return st;
    Lines L;
    L.axis = axis;
    L.nx = c->nx;
    L.ny = c->ny;
    L.n = n;
    L.stride = axis == 0 ? 1 : (axis == 1 ? c->nx : (long)c->nx * c->ny);
    L.count = c->N / n;
    L.log2n = log2_exact(n);
    const int buffers = L.log2n >= 0 ? 1 : 2;
    L.group = std::max(1, std::min(16, kSmemBudget / (buffers * n * (int)sizeof(float2))));
    const size_t smem = (size_t)buffers * L.group * n * sizeof(float2);
    const unsigned blocks = (unsigned)((L.count + L.group - 1) / L.group);
    if (L.log2n >= 0) k_fft_pow2<<<blocks, kFftThreads, smem, c->stream>>>(c->d_sfk_z, L, c->d_sfk_tw[axis], mean);
    else k_dft_lines<<<blocks, kFftThreads, smem, c->stream>>>(c->d_sfk_z, L, c->d_sfk_tw[axis], mean);
    FLBM_CUDA(c, cudaGetLastError(), "line transform launch");
    return FLBM_OK;
}

flbm_status sfk_supported(flbm_ctx *c)
{
    const int lens[3] = {c->nx, c->ny, c->nz};
    for (int a = 0; a < 3; a++) {
        const int n = lens[a];
        if (n == 1) continue;
        const int cap = log2_exact(n) >= 0 ? kSmemBudget / (int)sizeof(float2) : kSmemBudget / (2 * (int)sizeof(float2));
        if (n > cap)
            return fail(c, FLBM_EUNSUPPORTED, "full-k structure factor: axis length %d exceeds %d (%s)", n, cap,
                        log2_exact(n) >= 0 ? "power of two" : "other lengths");
    }
    return FLBM_OK;
}

} // namespace

namespace flbm {
void free_sfk(flbm_ctx *c)
{
    if (c->d_sfk_z) cudaFree(c->d_sfk_z);
    if (c->d_sfk_acc) cudaFree(c->d_sfk_acc);
    if (c->d_sfk_mean) cudaFree(c->d_sfk_mean);
    c->d_sfk_mean = nullptr;
    for (int a = 0; a < 3; a++) {
        if (c->d_sfk_tw[a]) cudaFree(c->d_sfk_tw[a]);
        c->d_sfk_tw[a] = nullptr;
        c->sfk_tw_n[a] = 0;
    }
    c->d_sfk_z = nullptr;
    c->d_sfk_acc = nullptr;
    c->sfk_count = 0;
}
} // namespace flbm

extern "C" {

flbm_status flbm_sfk_sample(flbm_ctx *c)
{
    if (!c) return FLBM_EINVAL;
    if (is_batch(c)) return fail(c, FLBM_EINVAL, "a batch has one structure factor per replica: use flbm_batch_replica");
    if (!c->initialised) return fail(c, FLBM_ESTATE, "flbm_sfk_sample before flbm_init");
    flbm_status st = sfk_supported(c);
    if (st != FLBM_OK) return st;
    if ((st = ensure_obs(c)) != FLBM_OK) return st; // block partials buffer
    if (!c->d_sfk_acc) {
        if (cudaMalloc((void **)&c->d_sfk_acc, 3 * (size_t)c->N * sizeof(double)) != cudaSuccess ||
            cudaMalloc((void **)&c->d_sfk_z, (size_t)c->N * sizeof(float2)) != cudaSuccess ||
            cudaMalloc((void **)&c->d_sfk_mean, 2 * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            free_sfk(c);
            return fail(c, FLBM_ENOMEM, "full-k structure factor buffers (%zu bytes) do not fit",
                        (size_t)c->N * (3 * sizeof(double) + sizeof(float2)));
        }
        FLBM_CUDA(c, cudaMemsetAsync(c->d_sfk_acc, 0, 3 * (size_t)c->N * sizeof(double), c->stream), "memset");
        c->sfk_count = 0;
    }
    const StepParams p = make_params(c);
    int nb = 0;
    FLBM_CUDA(c, launch_sfk_fields(c->lat, c->storage, layout_parity(c), p, cur_pop(c), c->d_sfk_z, c->d_partials, &nb, c->stream),
              "fields kernel launch");
    k_sfk_means<<<1, 256, 0, c->stream>>>(c->d_partials, nb, (long)c->N, c->d_sfk_mean);
    FLBM_CUDA(c, cudaGetLastError(), "means kernel launch");
    for (int a = 0; a < 3; a++)
        if ((st = transform_axis(c, a, a == 0 ? c->d_sfk_mean : nullptr)) != FLBM_OK) return st;
    const dim3 blk(128), grd((c->nx + 127) / 128, c->ny, c->nz);
    k_sfk_accumulate<<<grd, blk, 0, c->stream>>>(c->d_sfk_z, c->nx, c->ny, c->nz, c->d_sfk_acc);
    FLBM_CUDA(c, cudaGetLastError(), "accumulate kernel launch");
    c->sfk_count++;
    return FLBM_OK;
}

flbm_status flbm_sfk_reset(flbm_ctx *c)
{
    if (!c) return FLBM_EINVAL;
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_sfk(c);
    return FLBM_OK;
}

static flbm_status sfk_out(flbm_ctx *c, int functions, double r0a, double r0b, double *o0, double *o1, double *o2,
                           int64_t *nsamples)
{
    if (!c) return FLBM_EINVAL;
    if (is_batch(c)) return fail(c, FLBM_EINVAL, "a batch has one structure factor per replica: use flbm_batch_replica");
    if (nsamples) *nsamples = c->sfk_count;
    if (!c->d_sfk_acc || c->sfk_count == 0) return fail(c, FLBM_ESTATE, "no full-k structure-factor snapshot taken");
    if (functions && !(r0a > 0.0 && r0b > 0.0)) return fail(c, FLBM_EINVAL, "reference densities must be positive");
    const size_t n = (size_t)c->N;
    double *d_out = nullptr;
    FLBM_CUDA(c, cudaMalloc((void **)&d_out, 3 * n * sizeof(double)), "cudaMalloc(sfk out)");
    k_sfk_out<<<grid_for(c->N), 256, 0, c->stream>>>(c->d_sfk_acc, (long)n, 1.0 / ((double)c->N * c->sfk_count),
                                                     functions, r0a, r0b, d_out, d_out + n, d_out + 2 * n);
    cudaError_t e = cudaGetLastError();
    flbm_status st = e == cudaSuccess ? sync_and_check(c) : cuda_fail(c, e, "sfk output kernel launch");
    double *outs[3] = {o0, o1, o2};
    for (int q = 0; q < 3 && st == FLBM_OK; q++)
        if (outs[q] && cudaMemcpy(outs[q], d_out + q * n, n * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
            st = fail(c, FLBM_ECUDA, "D2H structure factor");
    cudaFree(d_out);
    return st;
}

flbm_status flbm_sfk(flbm_ctx *c, double *S_aa, double *S_ab, double *S_bb, int64_t *nsamples)
{
    return sfk_out(c, 0, 0.0, 0.0, S_aa, S_ab, S_bb, nsamples);
}

flbm_status flbm_sfk_functions(flbm_ctx *c, double rho0_a, double rho0_b, double *S_tt, double *S_cc, double *S_tc)
{
    return sfk_out(c, 1, rho0_a, rho0_b, S_tt, S_cc, S_tc, nullptr);
}

} // extern "C"
