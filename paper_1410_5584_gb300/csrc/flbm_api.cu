// flbm_api.cu -- the C-ABI of include/flbm.h: context, argument checks, buffer
// ownership, the step loop, observables, checkpoints and error reporting.
// Every entry point catches its own failures and returns an flbm_status.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <thread>
#include <unistd.h>
#include <vector>

#include "flbm_ctx.h"
#include "flbm_lattice.cuh"

using namespace flbm;



namespace flbm {
namespace host {

const char *kNoError = "";

flbm_status fail(flbm_ctx *c, flbm_status st, const char *fmt, ...)
{
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
    }
    return st;
}

flbm_status cuda_fail(flbm_ctx *c, cudaError_t e, const char *what)
{
    return fail(c, FLBM_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}


double lat_w(int lat, int i) { return lat == FLBM_D2Q9 ? D2Q9::wd(i) : D3Q19::wd(i); }
double lat_N(int lat, int a) { return lat == FLBM_D2Q9 ? D2Q9::Nd(a) : D3Q19::Nd(a); }
int lat_c(int lat, int i, int d)
{
    if (lat == FLBM_D2Q9) return d == 0 ? D2Q9::cx(i) : (d == 1 ? D2Q9::cy(i) : 0);
    return d == 0 ? D3Q19::cx(i) : (d == 1 ? D3Q19::cy(i) : D3Q19::cz(i));
}
int lat_opp(int lat, int i) { return lat == FLBM_D2Q9 ? D2Q9::opp(i) : D3Q19::opp(i); }

void default_rates(flbm_ctx *c)
{
    const double lam_d = c->tau[0] == c->tau[1] ? 1.0 / c->tau[0] : 2.0 / (c->tau[0] + c->tau[1]);
    for (int s = 0; s < 2; s++)
        for (int a = 0; a < kMaxQ; a++) c->lam[s][a] = a == 0 ? 0.0 : (a <= c->D ? lam_d : 1.0 / c->tau[s]);
}

StepParams make_params(const flbm_ctx *c)
{
    StepParams p;
    std::memset(&p, 0, sizeof(p));
    p.nx = c->nx;
    p.ny = c->ny;
    p.nz = c->nz;
    p.N = (int)c->N;
    p.y0 = p.z0 = 0;
    p.yn = c->ny;
    p.zn = c->nz;
    p.block_x = c->block_x;
    p.block_y = c->block_y;
    p.G = (float)c->G;
    const double mu = 3.0 * c->kT; // k_B T / c_s^2
    const double lb_d = c->lam[0][1];
    p.lam_d = (float)lb_d;
    p.hlam_d = (float)(1.0 - 0.5 * lb_d);
    for (int s = 0; s < 2; s++)
        for (int a = c->D + 1; a < c->Q; a++) {
            const double lb = c->lam[s][a], Na = lat_N(c->lat, a);
            p.cm[s][a] = (float)((1.0 - lb) / Na);
            p.ceq[s][a] = (float)(lb / Na);
            p.cphi[s][a] = (float)((1.0 - 0.5 * lb) / Na);
            p.cxi[s][a] = (float)(std::sqrt((2.0 * lb - lb * lb) * Na * mu) / Na);
        }
    for (int a = 0; a < kMaxQ; a++) {
        p.pair_eq[a] = make_float2(p.ceq[0][a], p.ceq[1][a]);
        p.pair_phi[a] = make_float2(p.cphi[0][a], p.cphi[1][a]);
        p.pair_xi[a] = make_float2(p.cxi[0][a], p.cxi[1][a]);
    }
    p.noise_amp_j = c->sdf ? (float)std::sqrt((2.0 * lb_d - lb_d * lb_d) * c->kT) : 0.0f;
    p.rho0[0] = (float)c->rho0[0];
    p.rho0[1] = (float)c->rho0[1];
    p.noise_ref = c->noise_ref;
    p.force_velocity = c->force_velocity;
    p.ghost_noise = c->ghost_noise;
    p.key0 = (uint32_t)(c->seed & 0xFFFFFFFFu);
    p.key1 = (uint32_t)(c->seed >> 32);
    p.step = (uint32_t)c->step;
    p.general_collide = c->test_general || c->ghost_noise; // the option lives in the general collide
    return p;
}

flbm_status ensure_stream(flbm_ctx *c)
{
    if (!c->stream) {
        FLBM_CUDA(c, cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking), "cudaStreamCreate");
        c->own_stream = true;
    }
    return FLBM_OK;
}

size_t array_bytes_of(const flbm_ctx *c) { return (size_t)2 * c->Q * (size_t)c->N * storage_bytes(c->storage); }
bool two_arrays(const flbm_ctx *c) { return c->streaming == FLBM_STREAM_TWO_ARRAYS; }
// a replica view owns slices of its batch's arrays, not two arrays of its own
size_t pop_bytes_of(const flbm_ctx *c) { return array_bytes_of(c) * (two_arrays(c) && !c->is_view ? 2 : 1); }
static void *second_array(const flbm_ctx *c)
{
    return c->pop_second ? c->pop_second : static_cast<unsigned char *>(c->pop) + array_bytes_of(c);
}
// the same for an explicit parity (a step captured ahead of time)
void *cur_pop_at(const flbm_ctx *c, int parity)
{
    if (!two_arrays(c) || parity == 0) return c->pop;
    return second_array(c);
}
void *next_pop_at(const flbm_ctx *c, int parity)
{
    if (!two_arrays(c)) return c->pop;
    return parity == 0 ? second_array(c) : c->pop;
}
void *cur_pop(const flbm_ctx *c) { return cur_pop_at(c, c->parity); }
void *next_pop(const flbm_ctx *c) { return next_pop_at(c, c->parity); }
int layout_parity(const flbm_ctx *c) { return two_arrays(c) ? 0 : c->parity; }
void drop_step_graphs(flbm_ctx *c)
{
    for (int k = 0; k < 2; k++) {
        if (c->graph[k]) cudaGraphExecDestroy(c->graph[k]);
        c->graph[k] = nullptr;
    }
}
size_t rho_bytes_of(const flbm_ctx *c) { return (size_t)2 * (size_t)c->N * sizeof(float); }

flbm_status ensure_status(flbm_ctx *c)
{
    if (!c->d_status) {
        FLBM_CUDA(c, cudaMalloc(&c->d_status, sizeof(unsigned)), "cudaMalloc(status)");
        FLBM_CUDA(c, cudaMemsetAsync(c->d_status, 0, sizeof(unsigned), c->stream), "cudaMemset(status)");
    }
    return FLBM_OK;
}

flbm_status ensure_buffers(flbm_ctx *c)
{
    flbm_status st = ensure_stream(c);
    if (st != FLBM_OK) return st;
    if (!c->pop) {
        c->pop_bytes = pop_bytes_of(c);
        c->rho_bytes = rho_bytes_of(c);
        cudaError_t e = cudaMalloc(&c->pop, c->pop_bytes);
        if (e != cudaSuccess) {
            c->pop = nullptr;
            return fail(c, FLBM_ENOMEM, "cudaMalloc of %zu population bytes failed: %s", c->pop_bytes, cudaGetErrorString(e));
        }
        e = cudaMalloc((void **)&c->rho, c->rho_bytes);
        if (e != cudaSuccess) {
            cudaFree(c->pop);
            c->pop = nullptr;
            c->rho = nullptr;
            return fail(c, FLBM_ENOMEM, "cudaMalloc of %zu density bytes failed: %s", c->rho_bytes, cudaGetErrorString(e));
        }
        c->own_buffers = true;
    }
    return ensure_status(c);
}

flbm_status ensure_pipe(flbm_ctx *c)
{
    if (!c->d_pipe) {
        const size_t n = 1 + (size_t)pipeline_slices(c->lat, c->ny, c->nz);
        FLBM_CUDA(c, cudaMalloc((void **)&c->d_pipe, n * sizeof(unsigned)), "cudaMalloc(pipeline counters)");
    }
    return FLBM_OK;
}

// f(lo, hi) over [0, n) in contiguous pieces on up to `most` host threads
// (one piece when n is small): the host side of the copies between the
// caller's buffers and the pinned staging buffer, and of mapping pages.
template <class F> void host_parallel(size_t n, F &&f, unsigned most = 8)
{
    const unsigned hw = std::thread::hardware_concurrency();
    const unsigned t = std::min(most, hw ? hw : 1u);
    if (t <= 1 || n < ((size_t)1 << 18)) {
        f((size_t)0, n);
        return;
    }
    const size_t piece = (n + t - 1) / t;
    std::vector<std::thread> pool;
    for (unsigned k = 1; k < t; k++) {
        const size_t lo = k * piece, hi = std::min(n, lo + piece);
        if (lo < hi) pool.emplace_back([&f, lo, hi] { f(lo, hi); });
    }
    f((size_t)0, std::min(n, piece));
    for (auto &th : pool) th.join();
}

// Device -> the caller's (pageable) host memory through the context's pinned
// staging buffer: chunks alternate between its two halves, so the copy of
// one chunk into the caller's buffer (on host threads) runs while the next
// chunk crosses the bus on the context's stream.
flbm_status d2h_staged(flbm_ctx *c, void *dst, const void *src, size_t bytes)
{
    unsigned char *stage = reinterpret_cast<unsigned char *>(c->h_stage);
    const size_t half = (((size_t)2 * c->N * sizeof(float)) / 2) & ~(size_t)255;
    if (half == 0) {
        FLBM_CUDA(c, cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost), "D2H");
        return FLBM_OK;
    }
    cudaEvent_t ev[2] = {nullptr, nullptr};
    for (int k = 0; k < 2; k++)
        if (cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming) != cudaSuccess) {
            if (ev[0]) cudaEventDestroy(ev[0]);
            return fail(c, FLBM_ECUDA, "cudaEventCreate failed");
        }
    const size_t nchunk = (bytes + half - 1) / half;
    auto issue = [&](size_t i) -> cudaError_t {
        const size_t off = i * half, len = std::min(half, bytes - off);
        cudaError_t e = cudaMemcpyAsync(stage + (i & 1) * half, static_cast<const unsigned char *>(src) + off, len,
                                        cudaMemcpyDeviceToHost, c->stream);
        return e == cudaSuccess ? cudaEventRecord(ev[i & 1], c->stream) : e;
    };
    cudaError_t e = issue(0);
    for (size_t i = 0; i < nchunk && e == cudaSuccess; i++) {
        if (i + 1 < nchunk) e = issue(i + 1);
        if (e == cudaSuccess) e = cudaEventSynchronize(ev[i & 1]);
        if (e != cudaSuccess) break;
        const size_t off = i * half, len = std::min(half, bytes - off);
        unsigned char *to = static_cast<unsigned char *>(dst) + off;
        const unsigned char *from = stage + (i & 1) * half;
        host_parallel(len, [&](size_t lo, size_t hi) { std::memcpy(to + lo, from + lo, hi - lo); });
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (e != cudaSuccess) return cuda_fail(c, e, "staged D2H copy");
    return FLBM_OK;
}

// Whether kernels may store straight into the caller's pageable host memory:
// on a CPU-GPU pair that shares page tables (cudaDevAttrPageableMemoryAccess
// with host page tables, as Grace with Blackwell over NVLink-C2C) device
// stores reach any mapped host page coherently.  Queried once per device.
bool pageable_direct()
{
    static std::atomic<int> cached[64]; // 0 not asked yet, 1 no, 2 yes
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return false;
    }
    if (cached[dev].load() == 0) {
        int a = 0, b = 0;
        if (cudaDeviceGetAttribute(&a, cudaDevAttrPageableMemoryAccess, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&b, cudaDevAttrPageableMemoryAccessUsesHostPageTables, dev) != cudaSuccess) {
            cudaGetLastError();
            a = b = 0;
        }
        cached[dev].store(a && b ? 2 : 1);
    }
    return cached[dev].load() == 2;
}

// Map every page of a host output buffer before a kernel stores into it: a
// device store to a page the OS has not mapped yet goes through a slow fault
// path (on GB300 about 50 times slower than into a mapped page), while host
// threads map pages quickly.  One byte a page is written (the buffer is
// output only).
void map_pages(void *buf, size_t bytes)
{
    const long pg = sysconf(_SC_PAGESIZE);
    const size_t page = pg > 0 ? (size_t)pg : 4096;
    volatile unsigned char *b = static_cast<volatile unsigned char *>(buf);
    host_parallel(bytes, [&](size_t lo, size_t hi) {
        // the pages that start in [lo, hi), and the first byte's page
        size_t k = lo == 0 ? 0 : ((lo + page - 1) / page) * page;
        for (; k < hi; k += page) b[k] = 0;
        if (hi == bytes && bytes > 0) b[bytes - 1] = 0; // the last page, when the buffer starts mid-page
    });
}

flbm_status ensure_stage(flbm_ctx *c)
{
    if (!c->h_stage) {
        cudaError_t e = cudaMallocHost((void **)&c->h_stage, (size_t)2 * c->N * sizeof(float));
        if (e != cudaSuccess) {
            c->h_stage = nullptr;
            return fail(c, FLBM_ENOMEM, "cudaMallocHost of the staging buffer failed: %s", cudaGetErrorString(e));
        }
    }
    return FLBM_OK;
}

flbm_status ensure_obs(flbm_ctx *c)
{
    if (!c->d_obs) {
        cudaError_t e = cudaMalloc((void **)&c->d_obs, (size_t)(2 + c->D) * c->N * sizeof(double));
        if (e != cudaSuccess) {
            c->d_obs = nullptr;
            return fail(c, FLBM_ENOMEM, "cudaMalloc of the observables buffer failed: %s", cudaGetErrorString(e));
        }
    }
    if (!c->d_cons) FLBM_CUDA(c, cudaMalloc((void **)&c->d_cons, 5 * sizeof(double)), "cudaMalloc(cons)");
    const size_t nb = (size_t)((c->nx + 127) / 128) * c->ny * c->nz;
    if (c->partials_cap < nb) {
        cudaFree(c->d_partials);
        c->d_partials = nullptr;
        FLBM_CUDA(c, cudaMalloc((void **)&c->d_partials, nb * 5 * sizeof(double)), "cudaMalloc(partials)");
        c->partials_cap = nb;
    }
    return FLBM_OK;
}

int axis_len(const flbm_ctx *c, int axis) { return axis == 0 ? c->nx : (axis == 1 ? c->ny : c->nz); }

flbm_status ensure_sf(flbm_ctx *c)
{
    if (!c->d_sf) {
        const int n = axis_len(c, c->sf_axis);
        FLBM_CUDA(c, cudaMalloc((void **)&c->d_sf, (size_t)4 * (n / 2) * sizeof(double)), "cudaMalloc(sf)");
        FLBM_CUDA(c, cudaMalloc((void **)&c->d_profile, (size_t)(2 + c->D) * n * sizeof(double)), "cudaMalloc(profile)");
        FLBM_CUDA(c, cudaMemsetAsync(c->d_sf, 0, (size_t)4 * (n / 2) * sizeof(double), c->stream), "cudaMemset(sf)");
        c->sf_count = 0;
    }
    return FLBM_OK;
}

void free_sf(flbm_ctx *c)
{
    if (c->d_sf) cudaFree(c->d_sf);
    if (c->d_profile) cudaFree(c->d_profile);
    c->d_sf = nullptr;
    c->d_profile = nullptr;
    c->sf_count = 0;
}

// wait for the stream, then report device-side faults
flbm_status sync_and_check(flbm_ctx *c)
{
    FLBM_CUDA(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    if (c->d_status) {
        unsigned h = 0;
        FLBM_CUDA(c, cudaMemcpy(&h, c->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost), "status read");
        if (h & kStatusNonFinite) c->faulted = true;
        if (h & kStatusTimeout) c->timed_out = true;
    }
    if (c->timed_out)
        return fail(c, FLBM_ETIMEOUT, "a device-side wait of the fused step gave up (state is not valid)");
    if (c->faulted)
        return fail(c, FLBM_ENONFINITE, "a density became non-positive or non-finite on the device (step <= %lld)",
                    (long long)c->step);
    return FLBM_OK;
}

// fold the recorded events into the per-kernel totals and recycle them
flbm_status drain_timing(flbm_ctx *c)
{
    if (c->ev_used == 0) return FLBM_OK;
    FLBM_CUDA(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    if (c->stream_d) FLBM_CUDA(c, cudaStreamSynchronize(c->stream_d), "cudaStreamSynchronize");
    for (const auto &m : c->marks) {
        float ms = 0.0f;
        FLBM_CUDA(c, cudaEventElapsedTime(&ms, c->ev_pool[m.start], c->ev_pool[m.end]), "cudaEventElapsedTime");
        c->kernel_ms[m.kernel] += ms;
    }
    c->marks.clear();
    c->ev_used = 0;
    return FLBM_OK;
}

flbm_status next_event(flbm_ctx *c, cudaEvent_t *ev)
{
    if (c->ev_used == c->ev_pool.size()) {
        cudaEvent_t e;
        FLBM_CUDA(c, cudaEventCreate(&e), "cudaEventCreate");
        c->ev_pool.push_back(e);
    }
    *ev = c->ev_pool[c->ev_used++];
    return FLBM_OK;
}

// Event-timing bracket around one launch on stream st (a no-op unless the
// kernel_timing option is on): begin() records the start event, end() the end
// event and the mark that drain_timing() turns into milliseconds.
struct TimedLaunch {
    flbm_ctx *c;
    cudaStream_t st;
    int kernel;
    size_t start = 0;
    flbm_status begin()
    {
        if (!c->timing) return FLBM_OK;
        if (c->ev_used + 2 > 3 * 4096) {
            flbm_status s = drain_timing(c);
            if (s != FLBM_OK) return s;
        }
        cudaEvent_t e;
        flbm_status s = next_event(c, &e);
        if (s != FLBM_OK) return s;
        start = c->ev_used - 1;
        FLBM_CUDA(c, cudaEventRecord(e, st), "cudaEventRecord");
        return FLBM_OK;
    }
    flbm_status end()
    {
        if (!c->timing) return FLBM_OK;
        cudaEvent_t e;
        flbm_status s = next_event(c, &e);
        if (s != FLBM_OK) return s;
        FLBM_CUDA(c, cudaEventRecord(e, st), "cudaEventRecord");
        c->marks.push_back({start, c->ev_used - 1, kernel});
        return FLBM_OK;
    }
};

flbm_status density_now(flbm_ctx *c, const StepParams &p)
{
    FLBM_CUDA(c, launch_density(c->lat, c->storage, layout_parity(c), p, cur_pop(c), c->rho, c->stream),
              "density kernel launch");
    return FLBM_OK;
}

// natural-layout population f_i(site) of species s from a raw host copy
double raw_to_natural(const flbm_ctx *c, const std::vector<unsigned char> &raw, int s, int i, int64_t site)
{
    int64_t src = site;
    int slot = i;
    if (layout_parity(c) == 1) {
        const int x = (int)(site % c->nx), y = (int)((site / c->nx) % c->ny), z = (int)(site / ((int64_t)c->nx * c->ny));
        const int xs = (x - lat_c(c->lat, i, 0) + c->nx) % c->nx;
        const int ys = (y - lat_c(c->lat, i, 1) + c->ny) % c->ny;
        const int zs = (z - lat_c(c->lat, i, 2) + c->nz) % c->nz;
        src = ((int64_t)zs * c->ny + ys) * c->nx + xs;
        slot = lat_opp(c->lat, i);
    }
    const size_t idx = pop_index(s, slot, (size_t)src, (size_t)c->N);
    const float base = (float)lat_w(c->lat, i) * (float)c->rho0[s];
    if (c->storage == FLBM_STORE_F32) {
        float dev;
        std::memcpy(&dev, raw.data() + idx * 4, 4);
        return (double)base + (double)dev;
    }
    uint16_t bits;
    std::memcpy(&bits, raw.data() + idx * 2, 2);
    float dev;
    if (c->storage == FLBM_STORE_F16) {
        __half_raw hr;
        hr.x = bits;
        dev = __half2float(__half(hr));
    } else {
        __nv_bfloat16_raw br;
        br.x = bits;
        dev = __bfloat162float(__nv_bfloat16(br));
    }
    return (double)base + (double)dev;
}

uint64_t fnv1a(const unsigned char *p, size_t n)
{
    uint64_t h = 1469598103934665603ull;
    for (size_t k = 0; k < n; k++) {
        h ^= p[k];
        h *= 1099511628211ull;
    }
    return h;
}

struct CkptHeader {
    char magic[8];
    uint32_t version;
    int32_t lat, nx, ny, nz, storage, parity, sdf, noise_ref, force_velocity, sf_axis, ghost_noise, pad_;
    int64_t step;
    uint64_t seed;
    double tau[2], kT, G, rho0[2];
    double lam[2][kMaxQ];
    uint64_t payload_bytes;
    uint64_t payload_hash;
};

} // namespace host
} // namespace flbm

using namespace flbm::host;

bool flbm::ctx_view(const flbm_ctx *c, CtxView *out)
{
    if (!c || !out) return false;
    out->lat = c->lat;
    out->storage = c->storage;
    out->D = c->D;
    out->Q = c->Q;
    out->nx = c->nx;
    out->ny = c->ny;
    out->nz = c->nz;
    out->batch = is_batch(c);
    out->N = c->N;
    out->params = make_params(c);
    return true;
}

extern "C" {

const char *flbm_version(void) { return "flbm 0.1 sm_103a"; }

const char *flbm_last_error(const flbm_ctx *ctx) { return ctx ? ctx->err : kNoError; }

flbm_status flbm_create(flbm_lattice lat, int nx, int ny, int nz, double tau_a, double tau_b, double kT,
                        double G, uint64_t seed, flbm_ctx **out)
{
    if (!out) return FLBM_EINVAL;
    *out = nullptr;
    if (lat != FLBM_D2Q9 && lat != FLBM_D3Q19) return FLBM_EINVAL;
    if (nx < 2 || ny < 2 || ny > 65535) return FLBM_EINVAL;
    if (lat == FLBM_D2Q9 ? nz != 1 : (nz < 2 || nz > 65535)) return FLBM_EINVAL;
    if ((int64_t)nx * ny * nz >= (int64_t(1) << 31)) return FLBM_EINVAL;
    if (!(tau_a > 0.5) || !(tau_b > 0.5) || !std::isfinite(tau_a) || !std::isfinite(tau_b)) return FLBM_EINVAL;
    if (!(kT >= 0.0) || !std::isfinite(kT) || !std::isfinite(G)) return FLBM_EINVAL;
    flbm_ctx *c = new (std::nothrow) flbm_ctx();
    if (!c) return FLBM_ENOMEM;
    c->lat = lat;
    c->D = lat == FLBM_D2Q9 ? 2 : 3;
    c->Q = lat == FLBM_D2Q9 ? 9 : 19;
    c->nx = nx;
    c->ny = ny;
    c->nz = nz;
    c->N = (int64_t)nx * ny * nz;
    c->tau[0] = tau_a;
    c->tau[1] = tau_b;
    c->kT = kT;
    c->G = G;
    c->seed = seed;
    default_rates(c);
    *out = c;
    return FLBM_OK;
}

flbm_status flbm_set_option(flbm_ctx *c, int key, double v)
{
    if (!c) return FLBM_EINVAL;
    if (is_batch(c)) return batch_set_option(c, key, v);
    if (c->is_view && key != FLBM_OPT_SF_AXIS && !view_call_allowed(c))
        return fail(c, FLBM_ESTATE, "a replica view can be observed, not changed; use its batch");
    drop_step_graphs(c); // a captured step holds the parameters and launch settings by value
    if (key == FLBM_OPT_GRAPH_STEPS) {
        if (!(v >= 0.0 && v <= 4096.0) || v != (double)(int)v)
            return fail(c, FLBM_EINVAL, "graph steps must be an integer in [0, 4096]");
        c->graph_steps = (int)v;
        return FLBM_OK;
    }
    if (key == FLBM_OPT_STORAGE) {
        if (c->pop) return fail(c, FLBM_ESTATE, "the storage format is fixed once the buffers exist");
        if (v != 0.0 && v != 1.0 && v != 2.0) return fail(c, FLBM_EINVAL, "storage must be 0 (f32), 1 (f16) or 2 (bf16)");
        c->storage = (int)v;
    } else if (key == FLBM_OPT_LAMBDA_D) {
        if (!(v > 0.0 && v < 2.0)) return fail(c, FLBM_EINVAL, "lambda_d must lie in (0, 2)");
        for (int s = 0; s < 2; s++)
            for (int a = 1; a <= c->D; a++) c->lam[s][a] = v;
    } else if (key == FLBM_OPT_SDF) {
        c->sdf = v != 0.0;
    } else if (key == FLBM_OPT_RHO0_A || key == FLBM_OPT_RHO0_B) {
        if (!(v > 0.0) || !std::isfinite(v)) return fail(c, FLBM_EINVAL, "reference densities must be positive");
        if (c->pop) return fail(c, FLBM_ESTATE, "the deviation base is fixed once the buffers exist");
        c->rho0[key == FLBM_OPT_RHO0_A ? 0 : 1] = v;
    } else if (key == FLBM_OPT_NOISE_RHO) {
        c->noise_ref = v != 0.0;
    } else if (key == FLBM_OPT_FORCE_VELOCITY) {
        c->force_velocity = v != 0.0;
    } else if (key == FLBM_OPT_GHOST_NOISE) {
        if (c->batch) return fail(c, FLBM_EUNSUPPORTED, "the population-space noise is for single boxes");
        c->ghost_noise = v != 0.0;
    } else if (key == FLBM_OPT_DIRECT_HOST) {
        if (v != 0.0 && v != 1.0) return fail(c, FLBM_EINVAL, "direct host stores must be 0 or 1");
        c->direct_host = (int)v;
    } else if (key == FLBM_OPT_SF_AXIS) {
        if (v != 0.0 && v != 1.0 && v != 2.0) return fail(c, FLBM_EINVAL, "axis must be 0, 1 or 2");
        if ((int)v >= c->D) return fail(c, FLBM_EINVAL, "axis %d does not exist on this lattice", (int)v);
        if ((int)v != c->sf_axis) {
            free_sf(c);
            c->sf_axis = (int)v;
        }
    } else if (key == FLBM_OPT_STREAMING) {
        if (c->pop) return fail(c, FLBM_ESTATE, "the streaming mode is fixed once the buffers exist");
        if (v != (double)FLBM_STREAM_IN_PLACE && v != (double)FLBM_STREAM_TWO_ARRAYS)
            return fail(c, FLBM_EINVAL, "streaming must be 0 (in place) or 1 (two arrays)");
        c->streaming = (int)v;
    } else if (key == FLBM_OPT_SCHEDULE) {
        if (v != (double)FLBM_SCHEDULE_FUSED && v != (double)FLBM_SCHEDULE_TWO_KERNELS &&
            v != (double)FLBM_SCHEDULE_OVERLAP && v != (double)FLBM_SCHEDULE_TILED)
            return fail(c, FLBM_EINVAL, "schedule must be 0 (fused), 1 (two kernels), 2 (overlap) or 3 (tiled)");
        if ((int)v != c->schedule) drop_step_graphs(c);
        c->schedule = (int)v;
    } else if (key == FLBM_OPT_BLOCK_X || key == FLBM_OPT_BLOCK_Y) {
        const int bx = key == FLBM_OPT_BLOCK_X ? (int)v : c->block_x;
        const int by = key == FLBM_OPT_BLOCK_Y ? (int)v : c->block_y;
        if (v != (double)(int)v || (key == FLBM_OPT_BLOCK_X && bx != 32 && bx != 64 && bx != 128) ||
            (key == FLBM_OPT_BLOCK_Y && by != 1 && by != 2 && by != 4) || bx * by > kSiteBlockMax)
            return fail(c, FLBM_EINVAL, "block shape must be x in {32,64,128}, y in {1,2,4}, x*y <= %d",
                        kSiteBlockMax);
        c->block_x = bx;
        c->block_y = by;
    } else if (key == FLBM_OPT_SLABS) {
        if (!(v >= 3.0 && v <= 256.0) || v != (double)(int)v)
            return fail(c, FLBM_EINVAL, "slabs must be an integer in [3, 256]");
        c->slabs = (int)v;
    } else if (key == FLBM_OPT_WAIT_LIMIT_MS) {
        if (!(v >= 1.0 && v <= 60000.0)) return fail(c, FLBM_EINVAL, "wait limit must lie in [1, 60000] ms");
        c->wait_limit_ms = v;
    } else if (key == FLBM_OPT_PIPE_LAG) {
        if (!(v == 0.0 || (v >= 2.0 && v <= 4096.0)) || v != (double)(int)v)
            return fail(c, FLBM_EINVAL, "pipeline lag must be 0 (automatic) or an integer in [2, 4096]");
        c->pipe_lag = (int)v;
    } else if (key == FLBM_OPT_TEST_STALL) {
        c->test_stall = v != 0.0;
    } else if (key == FLBM_OPT_TEST_GENERAL_COLLIDE) {
        c->test_general = v != 0.0;
    } else if (key == FLBM_OPT_KERNEL_TIMING) {
        if (c->stream) {
            flbm_status st = drain_timing(c);
            if (st != FLBM_OK) return st;
        }
        c->timing = v != 0.0;
        c->kernel_ms[0] = c->kernel_ms[1] = 0.0;
        c->kernel_launches[0] = c->kernel_launches[1] = 0;
    } else if (key >= FLBM_OPT_LAMBDA_MODE && key < FLBM_OPT_LAMBDA_MODE + 200) {
        const int s = (key - FLBM_OPT_LAMBDA_MODE) / 100, a = (key - FLBM_OPT_LAMBDA_MODE) % 100;
        if (a <= c->D || a >= c->Q) return fail(c, FLBM_EINVAL, "mode %d is not a non-conserved mode", a);
        if (!(v > 0.0 && v < 2.0)) return fail(c, FLBM_EINVAL, "rates must lie in (0, 2)");
        c->lam[s][a] = v;
    } else {
        return fail(c, FLBM_EINVAL, "unknown option key %d", key);
    }
    return FLBM_OK;
}

flbm_status flbm_get_option(const flbm_ctx *c, int key, double *value)
{
    if (!c || !value) return FLBM_EINVAL;
    switch (key) {
    case FLBM_OPT_STORAGE: *value = c->storage; break;
    case FLBM_OPT_LAMBDA_D: *value = c->lam[0][1]; break;
    case FLBM_OPT_SDF: *value = c->sdf; break;
    case FLBM_OPT_RHO0_A: *value = c->rho0[0]; break;
    case FLBM_OPT_RHO0_B: *value = c->rho0[1]; break;
    case FLBM_OPT_NOISE_RHO: *value = c->noise_ref; break;
    case FLBM_OPT_FORCE_VELOCITY: *value = c->force_velocity; break;
    case FLBM_OPT_GHOST_NOISE: *value = c->ghost_noise; break;
    case FLBM_OPT_DIRECT_HOST: *value = c->direct_host && pageable_direct() ? 1.0 : 0.0; break; // the route in effect
    case FLBM_OPT_SF_AXIS: *value = c->sf_axis; break;
    case FLBM_OPT_KERNEL_TIMING: *value = c->timing ? 1.0 : 0.0; break;
    case FLBM_OPT_SCHEDULE: *value = c->schedule; break;
    case FLBM_OPT_STREAMING: *value = c->streaming; break;
    case FLBM_OPT_WAIT_LIMIT_MS: *value = c->wait_limit_ms; break;
    case FLBM_OPT_TEST_STALL: *value = c->test_stall; break;
    case FLBM_OPT_TEST_GENERAL_COLLIDE: *value = c->test_general; break;
    case FLBM_OPT_PIPE_LAG: *value = c->pipe_lag; break;
    case FLBM_OPT_GRAPH_STEPS: *value = is_batch(c) ? batch_graph_steps(c) : c->graph_steps; break;
    case FLBM_OPT_SLABS: *value = c->slabs; break;
    case FLBM_OPT_BLOCK_X: *value = c->block_x; break;
    case FLBM_OPT_BLOCK_Y: *value = c->block_y; break;
    default: {
        const int s = (key - FLBM_OPT_LAMBDA_MODE) / 100, a = (key - FLBM_OPT_LAMBDA_MODE) % 100;
        if (key < FLBM_OPT_LAMBDA_MODE || key >= FLBM_OPT_LAMBDA_MODE + 200 || a <= c->D || a >= c->Q)
            return FLBM_EINVAL;
        *value = c->lam[s][a];
    }
    }
    return FLBM_OK;
}

flbm_status flbm_set_stream(flbm_ctx *c, void *stream)
{
    if (!c) return FLBM_EINVAL;
    if (!view_call_allowed(c)) return fail(c, FLBM_ESTATE, "a replica view can be observed, not changed; use its batch");
    drop_step_graphs(c);
    if (c->own_stream && c->stream) {
        cudaStreamSynchronize(c->stream);
        cudaStreamDestroy(c->stream);
    }
    c->stream = static_cast<cudaStream_t>(stream);
    c->own_stream = false;
    if (!stream) {
        flbm_status st = ensure_stream(c);
        if (st != FLBM_OK) return st;
    }
    if (is_batch(c)) return batch_set_stream(c, stream);
    return FLBM_OK;
}

flbm_status flbm_buffer_bytes(const flbm_ctx *c, size_t *pop_bytes, size_t *rho_bytes)
{
    if (!c) return FLBM_EINVAL;
    if (pop_bytes) *pop_bytes = pop_bytes_of(c);
    if (rho_bytes) *rho_bytes = rho_bytes_of(c);
    return FLBM_OK;
}

flbm_status flbm_attach_buffers(flbm_ctx *c, void *pop, size_t pop_bytes, void *rho, size_t rho_bytes)
{
    if (!c) return FLBM_EINVAL;
    if (!view_call_allowed(c)) return fail(c, FLBM_ESTATE, "a replica view can be observed, not changed; use its batch");
    if (c->pop) return fail(c, FLBM_ESTATE, "buffers already exist");
    if (!pop || !rho) return fail(c, FLBM_EINVAL, "NULL buffer");
    if (pop_bytes < pop_bytes_of(c) || rho_bytes < rho_bytes_of(c))
        return fail(c, FLBM_EINVAL, "buffers too small: need %zu and %zu bytes", pop_bytes_of(c), rho_bytes_of(c));
    if (((uintptr_t)pop % 256) != 0 || ((uintptr_t)rho % 256) != 0)
        return fail(c, FLBM_EINVAL, "buffers must be 256-byte aligned");
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, pop) != cudaSuccess || at.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        return fail(c, FLBM_EINVAL, "population buffer is not device memory");
    }
    if (cudaPointerGetAttributes(&at, rho) != cudaSuccess || at.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        return fail(c, FLBM_EINVAL, "density buffer is not device memory");
    }
    c->pop = pop;
    c->pop_bytes = pop_bytes;
    c->rho = static_cast<float *>(rho);
    c->rho_bytes = rho_bytes;
    c->own_buffers = false;
    flbm_status st = ensure_stream(c);
    if (st != FLBM_OK) return st;
    if ((st = ensure_status(c)) != FLBM_OK) return st;
    if (is_batch(c)) return batch_attach_buffers(c, pop, pop_bytes, rho, rho_bytes);
    return FLBM_OK;
}

flbm_status flbm_init(flbm_ctx *c, const double *rho_a, const double *rho_b)
{
    if (!c) return FLBM_EINVAL;
    if (!view_call_allowed(c)) return fail(c, FLBM_ESTATE, "a replica view can be observed, not changed; use its batch");
    if (is_batch(c)) return batch_init(c, rho_a, rho_b);
    flbm_status st = ensure_buffers(c);
    if (st != FLBM_OK) return st;
    if (c->direct_host && pageable_direct()) {
        // the densities read by a kernel straight from the caller's arrays and
        // checked there; nothing of the state changes before they pass
        if (!c->d_bad) FLBM_CUDA(c, cudaMalloc((void **)&c->d_bad, 2 * sizeof(unsigned long long)), "cudaMalloc");
        FLBM_CUDA(c, cudaMemsetAsync(c->d_bad, 0xFF, 2 * sizeof(unsigned long long), c->stream), "cudaMemset");
        FLBM_CUDA(c, launch_densities_from_host(rho_a, rho_b, c->rho0[0], c->rho0[1], c->N, c->rho, c->d_bad, c->stream),
                  "density read kernel launch");
        unsigned long long bad[2];
        FLBM_CUDA(c, cudaMemcpyAsync(bad, c->d_bad, sizeof(bad), cudaMemcpyDeviceToHost, c->stream), "D2H check");
        FLBM_CUDA(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
        for (int s = 0; s < 2; s++)
            if (bad[s] != ~0ull) {
                const double *from = s == 0 ? rho_a : rho_b;
                return fail(c, FLBM_EINVAL, "initial density %g at site %lld is not positive",
                            from ? from[bad[s]] : c->rho0[s], (long long)bad[s]);
            }
        const StepParams p = make_params(c);
        FLBM_CUDA(c, launch_init_rest(c->lat, c->storage, p, c->rho, c->pop, c->stream), "init kernel launch");
        FLBM_CUDA(c, cudaMemsetAsync(c->d_status, 0, sizeof(unsigned), c->stream), "status reset");
        c->step = 0;
        c->parity = 0;
        c->faulted = false;
        c->timed_out = false;
        c->initialised = true;
        return FLBM_OK;
    }
    if ((st = ensure_stage(c)) != FLBM_OK) return st;
    // previous asynchronous work may still read the staging buffer
    FLBM_CUDA(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    const double *in[2] = {rho_a, rho_b};
    for (int s = 0; s < 2; s++) {
        // converted on host threads; the first bad site of each piece is kept
        std::vector<int64_t> bad;
        std::mutex bad_lock;
        float *to = c->h_stage + s * c->N;
        const double *from = in[s];
        const double r0 = c->rho0[s];
        host_parallel((size_t)c->N, [&](size_t lo, size_t hi) {
            for (size_t k = lo; k < hi; k++) {
                const double r = from ? from[k] : r0;
                if (!(r > 0.0) || !std::isfinite(r)) {
                    std::lock_guard<std::mutex> g(bad_lock);
                    bad.push_back((int64_t)k);
                    return;
                }
                to[k] = (float)r;
            }
        }, 16);
        if (!bad.empty()) {
            const int64_t k = *std::min_element(bad.begin(), bad.end());
            return fail(c, FLBM_EINVAL, "initial density %g at site %lld is not positive", from ? from[k] : r0,
                        (long long)k);
        }
    }
    FLBM_CUDA(c, cudaMemcpyAsync(c->rho, c->h_stage, (size_t)2 * c->N * sizeof(float), cudaMemcpyHostToDevice, c->stream), "H2D densities");
    const StepParams p = make_params(c);
    FLBM_CUDA(c, launch_init_rest(c->lat, c->storage, p, c->rho, c->pop, c->stream), "init kernel launch");
    FLBM_CUDA(c, cudaMemsetAsync(c->d_status, 0, sizeof(unsigned), c->stream), "status reset");
    c->step = 0;
    c->parity = 0;
    c->faulted = false;
    c->timed_out = false;
    c->initialised = true;
    return FLBM_OK;
}

// One slab of the overlap schedule: planes (rows for D2Q9) [j n / K, (j + 1) n / K).
StepParams slab_params(const flbm_ctx *c, StepParams p, int j, int K)
{
    const int n = c->lat == FLBM_D2Q9 ? c->ny : c->nz;
    const int lo = (int)((int64_t)j * n / K), hi = (int)((int64_t)(j + 1) * n / K);
    if (c->lat == FLBM_D2Q9) {
        p.y0 = lo;
        p.yn = hi - lo;
    } else {
        p.z0 = lo;
        p.zn = hi - lo;
    }
    return p;
}

int overlap_slabs(const flbm_ctx *c)
{
    const int n = c->lat == FLBM_D2Q9 ? c->ny : c->nz;
    return std::min(c->slabs, n);
}

flbm_status ensure_overlap(flbm_ctx *c, int K)
{
    if (!c->stream_d) {
        int least = 0, greatest = 0;
        FLBM_CUDA(c, cudaDeviceGetStreamPriorityRange(&least, &greatest), "cudaDeviceGetStreamPriorityRange");
        FLBM_CUDA(c, cudaStreamCreateWithPriority(&c->stream_d, cudaStreamNonBlocking, greatest),
                  "cudaStreamCreateWithPriority");
    }
    while ((int)c->ev_dep.size() < 2 * K) {
        cudaEvent_t e;
        FLBM_CUDA(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "cudaEventCreate");
        c->ev_dep.push_back(e);
    }
    return FLBM_OK;
}

// n steps of the overlap schedule.  With the AA layout every array slot belongs
// to the read/write set of exactly one site, so launches over disjoint slabs
// never touch the same slot.  With two arrays a collision reads its own slab of
// one array and pushes into slabs j-1, j, j+1 of the other, which no launch of
// the same step reads.  In both modes the orderings that matter are:
//  - the density of slab j for step t+1 reads the sets of slab j's sites, which
//    the collisions of slabs j-1, j, j+1 at step t filled (streaming moves one
//    plane at most);
//  - the collision of slab j at step t+1 reads the densities of slabs j-1, j,
//    j+1 (the force stencil) and overwrites slab j's sets, after their density
//    pass read them;
//  - a density launch overwrites rho of its slab only after the step-t
//    collisions that read it (slabs j-1, j, j+1) are done.
// The collisions run in slab order on the context's stream, starting at slab 0
// or K/2 on alternate steps so that the two density slabs that wait for the
// last collision of a step are far from the first collisions of the next; the
// densities run on the second stream, each after the collision that completes
// its inputs.  The first step's densities are one launch over the box.
flbm_status step_overlap(flbm_ctx *c, int64_t n, StepParams p)
{
    const int K = overlap_slabs(c);
    flbm_status st = ensure_overlap(c, K);
    if (st != FLBM_OK) return st;
    cudaEvent_t *evC = c->ev_dep.data(), *evD = c->ev_dep.data() + K;
    const bool two = two_arrays(c);
    auto density = [&](cudaStream_t s, const StepParams &q, int parity) -> flbm_status {
        TimedLaunch tl{c, s, 0};
        if ((st = tl.begin()) != FLBM_OK) return st;
        cudaError_t e = two ? launch_density(c->lat, c->storage, 0, q, cur_pop_at(c, parity), c->rho, s)
                            : launch_density(c->lat, c->storage, parity, q, c->pop, c->rho, s);
        if (e != cudaSuccess) return cuda_fail(c, e, "density kernel launch");
        return tl.end();
    };
    auto collide = [&](const StepParams &q) -> flbm_status {
        TimedLaunch tl{c, c->stream, 1};
        if ((st = tl.begin()) != FLBM_OK) return st;
        cudaError_t e = two ? launch_collide(c->lat, c->storage, kStreamPush, q, cur_pop(c), next_pop(c), c->rho,
                                             c->d_status, c->stream)
                            : launch_collide(c->lat, c->storage, c->parity, q, c->pop, c->pop, c->rho, c->d_status,
                                             c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "collide kernel launch");
        return tl.end();
    };
    if ((st = density(c->stream, p, c->parity)) != FLBM_OK) return st;
    for (int64_t t = 0; t < n; t++) {
        p.step = (uint32_t)c->step;
        const int s0 = (c->step & 1) ? K / 2 : 0;
        const bool more = t + 1 < n;
        for (int q = 0; q < K; q++) {
            const int j = (s0 + q) % K;
            if (t > 0)
                for (int d = -1; d <= 1; d++)
                    FLBM_CUDA(c, cudaStreamWaitEvent(c->stream, evD[(j + d + K) % K], 0), "cudaStreamWaitEvent");
            if ((st = collide(slab_params(c, p, j, K))) != FLBM_OK) return st;
            FLBM_CUDA(c, cudaEventRecord(evC[j], c->stream), "cudaEventRecord");
            if (!more) continue;
            // densities of step t+1 whose three input slabs are now collided
            int ready[3], nready = 0;
            if (q >= 2) ready[nready++] = (s0 + q - 1) % K;
            if (q == K - 1) {
                ready[nready++] = (s0 + K - 1) % K;
                ready[nready++] = s0;
            }
            if (nready == 0) continue;
            FLBM_CUDA(c, cudaStreamWaitEvent(c->stream_d, evC[j], 0), "cudaStreamWaitEvent");
            for (int r = 0; r < nready; r++) {
                if ((st = density(c->stream_d, slab_params(c, p, ready[r], K), c->parity ^ 1)) != FLBM_OK) return st;
                FLBM_CUDA(c, cudaEventRecord(evD[ready[r]], c->stream_d), "cudaEventRecord");
            }
        }
        if (c->timing) {
            c->kernel_launches[0]++;
            c->kernel_launches[1]++;
        }
        c->step++;
        c->parity ^= 1;
    }
    return FLBM_OK;
}

// The two-kernel step at full relaxation (every lambdabar_a = 1, the condition
// the collide's full-relaxation instance is chosen on), in either streaming
// mode: the density pass also stores m_0 .. m_D of both species and the
// collide reads those instead of the populations (in place it then only
// writes).  Sets p.mom when that applies.
flbm_status use_moments(flbm_ctx *c, StepParams &p)
{
    p.mom = nullptr;
    if (p.general_collide) return FLBM_OK;
    for (int s = 0; s < 2; s++)
        for (int a = c->D + 1; a < c->Q; a++)
            if (p.cm[s][a] != 0.0f) return FLBM_OK;
    if (!c->d_mom)
        FLBM_CUDA(c, cudaMalloc((void **)&c->d_mom, (size_t)2 * (c->D + 1) * (size_t)c->N * sizeof(float)),
                  "cudaMalloc(moment planes)");
    p.mom = c->d_mom;
    return FLBM_OK;
}

// The tiled schedule runs where it applies: a 2D box with two arrays.
bool tiled_applies(const flbm_ctx *c) { return two_arrays(c) && tiled_step_rows(c->lat) > 0; }

// One CUDA graph of c->graph_steps steps of the two-kernel schedule (or, where
// it applies, the tiled one) starting at `parity`: the step kernels read the
// noise counter as *d_gstep + k, so the graph replays for any starting step
// once d_gstep is set.
flbm_status ensure_step_graph(flbm_ctx *c, int parity)
{
    if (c->graph[parity]) return FLBM_OK;
    if (!c->d_gstep) FLBM_CUDA(c, cudaMalloc((void **)&c->d_gstep, sizeof(unsigned)), "cudaMalloc(graph step counter)");
    StepParams p = make_params(c);
    p.step_dev = c->d_gstep;
    const bool tiled = c->schedule == FLBM_SCHEDULE_TILED && tiled_applies(c);
    if (!tiled)
        if (flbm_status st = use_moments(c, p); st != FLBM_OK) return st;
    cudaGraph_t g = nullptr;
    FLBM_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < c->graph_steps && e == cudaSuccess; k++) {
        const int par = (parity + k) & 1;
        p.step = (uint32_t)k;
        void *cur = cur_pop_at(c, par);
        if (tiled) {
            e = launch_step_tiled(c->lat, c->storage, p, cur, next_pop_at(c, par), c->d_status, c->stream);
            continue;
        }
        e = launch_density(c->lat, c->storage, two_arrays(c) ? 0 : par, p, cur, c->rho, c->stream);
        if (e == cudaSuccess) {
            if (two_arrays(c))
                e = launch_collide(c->lat, c->storage, kStreamPush, p, cur, next_pop_at(c, par), c->rho, c->d_status,
                                   c->stream);
            else
                e = launch_collide(c->lat, c->storage, par, p, c->pop, c->pop, c->rho, c->d_status, c->stream);
        }
    }
    const cudaError_t ee = cudaStreamEndCapture(c->stream, &g);
    if (e != cudaSuccess || ee != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(c, e != cudaSuccess ? e : ee, "step graph capture");
    }
    e = cudaGraphInstantiate(&c->graph[parity], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        c->graph[parity] = nullptr;
        return cuda_fail(c, e, "cudaGraphInstantiate");
    }
    return FLBM_OK;
}

// Full relaxation (every lambdabar_a = 1 on the non-conserved modes, the
// condition of the collide's full-relaxation instance).
bool full_relaxation(const flbm_ctx *c, const StepParams &p)
{
    if (p.general_collide) return false;
    for (int s = 0; s < 2; s++)
        for (int a = c->D + 1; a < c->Q; a++)
            if (p.cm[s][a] != 0.0f) return false;
    return true;
}

// n steps of the pipelined two-array step (the fused schedule with two
// arrays).  *done = false, with nothing launched, when the box has too few
// slices for the pipeline; the caller then runs the two-kernel step.
flbm_status step_pipe(flbm_ctx *c, int64_t n, bool *done)
{
    *done = false;
    StepParams p = make_params(c);
    // the population-space noise reads the density ring again after a tile has
    // released its slots, so it runs the two-kernel step
    if (p.ghost_noise) return FLBM_OK;
    const bool mom = full_relaxation(c, p);
    int lag = 0, slots = 0;
    size_t floats = 0, ncount = 0;
    FLBM_CUDA(c, pipe_geometry(c->lat, c->storage, p, mom, c->pipe_lag, &lag, &slots, &floats, &ncount),
              "pipelined step geometry");
    if (slots == 0) return FLBM_OK;
    if (c->ring_floats < floats) {
        if (c->d_ring) cudaFree(c->d_ring);
        c->d_ring = nullptr;
        c->ring_floats = 0;
        FLBM_CUDA(c, cudaMalloc((void **)&c->d_ring, floats * sizeof(float)), "cudaMalloc(pipeline ring)");
        c->ring_floats = floats;
    }
    if (!c->d_ring_cnt)
        FLBM_CUDA(c, cudaMalloc((void **)&c->d_ring_cnt, ncount * sizeof(unsigned)), "cudaMalloc(pipeline counters)");
    for (int64_t t = 0; t < n; t++) {
        p.step = (uint32_t)c->step;
        TimedLaunch t1{c, c->stream, 1};
        flbm_status st;
        if ((st = t1.begin()) != FLBM_OK) return st;
        const cudaError_t e = launch_step_pipe(c->lat, c->storage, p, cur_pop(c), next_pop(c), c->d_ring,
                                               c->d_ring_cnt, slots, lag, mom, c->d_status, c->wait_limit_ms,
                                               c->test_stall, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "pipelined step kernel launch");
        if ((st = t1.end()) != FLBM_OK) return st;
        if (c->timing) c->kernel_launches[1]++;
        c->step++;
        c->parity ^= 1;
    }
    *done = true;
    return FLBM_OK;
}

// n steps of the tiled schedule (one launch a step)
flbm_status step_tiled(flbm_ctx *c, int64_t n)
{
    StepParams p = make_params(c);
    for (int64_t t = 0; t < n; t++) {
        p.step = (uint32_t)c->step;
        TimedLaunch t1{c, c->stream, 1};
        flbm_status st;
        if ((st = t1.begin()) != FLBM_OK) return st;
        const cudaError_t e = launch_step_tiled(c->lat, c->storage, p, cur_pop(c), next_pop(c), c->d_status, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "tiled step kernel launch");
        if ((st = t1.end()) != FLBM_OK) return st;
        if (c->timing) c->kernel_launches[1]++;
        c->step++;
        c->parity ^= 1;
    }
    return FLBM_OK;
}

flbm_status flbm_step(flbm_ctx *c, int64_t n)
{
    if (!c || n < 0) return fail(c, FLBM_EINVAL, "negative step count");
    if (!view_call_allowed(c)) return fail(c, FLBM_ESTATE, "a replica view can be observed, not changed; use its batch");
    if (is_batch(c)) return batch_step(c, n);
    if (!c->initialised) return fail(c, FLBM_ESTATE, "flbm_step before flbm_init");
    if (n == 0) return FLBM_OK;
    int sched = c->schedule;
    if (two_arrays(c) && sched == FLBM_SCHEDULE_FUSED) {
        bool done = false;
        flbm_status st = step_pipe(c, n, &done);
        if (st != FLBM_OK || done) return st;
        sched = FLBM_SCHEDULE_TWO_KERNELS; // too few slices for the pipeline
    }
    if (sched == FLBM_SCHEDULE_TILED && !tiled_applies(c)) sched = FLBM_SCHEDULE_TWO_KERNELS;
    // whole graphs of graph_steps steps first (two-kernel or tiled schedule, timing off)
    if (c->graph_steps > 0 && (sched == FLBM_SCHEDULE_TWO_KERNELS || sched == FLBM_SCHEDULE_TILED) && !c->timing) {
        while (n >= c->graph_steps) {
            flbm_status st = ensure_step_graph(c, c->parity);
            if (st != FLBM_OK) return st;
            FLBM_CUDA(c, launch_set_u32(c->d_gstep, (unsigned)c->step, c->stream), "graph step counter");
            FLBM_CUDA(c, cudaGraphLaunch(c->graph[c->parity], c->stream), "cudaGraphLaunch");
            c->step += c->graph_steps;
            c->parity = (c->parity + c->graph_steps) & 1;
            n -= c->graph_steps;
        }
        if (n == 0) return FLBM_OK;
    }
    if (sched == FLBM_SCHEDULE_TILED) return step_tiled(c, n);
    StepParams p = make_params(c);
    if (sched == FLBM_SCHEDULE_OVERLAP && overlap_slabs(c) >= 3) {
        // at full relaxation the slabs run the moment-fed pair: a density slab
        // rewrites its moment planes only after the collisions that read them
        // (those of its own slab) are done, as for its densities
        if (flbm_status st = use_moments(c, p); st != FLBM_OK) return st;
        return step_overlap(c, n, p);
    }
    if (sched == FLBM_SCHEDULE_FUSED) {
        flbm_status st = ensure_pipe(c);
        if (st != FLBM_OK) return st;
    } else if (flbm_status st = use_moments(c, p); st != FLBM_OK) {
        return st;
    }
    for (int64_t t = 0; t < n; t++) {
        p.step = (uint32_t)c->step;
        flbm_status st;
        TimedLaunch t0{c, c->stream, 0}, t1{c, c->stream, 1};
        if ((st = t0.begin()) != FLBM_OK) return st;
        if (sched == FLBM_SCHEDULE_FUSED) {
            if ((st = t0.end()) != FLBM_OK) return st;
            if ((st = t1.begin()) != FLBM_OK) return st;
            cudaError_t e = launch_step_fused(c->lat, c->storage, c->parity, p, c->pop, c->rho, c->d_status,
                                              c->d_pipe, c->wait_limit_ms, c->test_stall, c->pipe_lag, c->stream);
            if (e != cudaSuccess) return cuda_fail(c, e, "fused step kernel launch");
        } else {
            cudaError_t e = launch_density(c->lat, c->storage, layout_parity(c), p, cur_pop(c), c->rho, c->stream);
            if (e != cudaSuccess) return cuda_fail(c, e, "density kernel launch");
            if ((st = t0.end()) != FLBM_OK) return st;
            if ((st = t1.begin()) != FLBM_OK) return st;
            if (two_arrays(c))
                e = launch_collide(c->lat, c->storage, kStreamPush, p, cur_pop(c), next_pop(c), c->rho, c->d_status,
                                   c->stream);
            else
                e = launch_collide(c->lat, c->storage, c->parity, p, c->pop, c->pop, c->rho, c->d_status, c->stream);
            if (e != cudaSuccess) return cuda_fail(c, e, "collide kernel launch");
        }
        if ((st = t1.end()) != FLBM_OK) return st;
        if (c->timing) {
            c->kernel_launches[0]++;
            c->kernel_launches[1]++;
        }
        c->step++;
        c->parity ^= 1;
    }
    return FLBM_OK;
}

flbm_status flbm_sync(flbm_ctx *c)
{
    if (!c) return FLBM_EINVAL;
    if (!c->stream) return FLBM_OK;
    return sync_and_check(c);
}

flbm_status flbm_kernel_times(flbm_ctx *c, double ms[2], int64_t launches[2])
{
    if (!c) return FLBM_EINVAL;
    if (c->stream) {
        flbm_status st = drain_timing(c);
        if (st != FLBM_OK) return st;
    }
    for (int k = 0; k < 2; k++) {
        if (ms) ms[k] = c->kernel_ms[k];
        if (launches) launches[k] = c->kernel_launches[k];
    }
    return FLBM_OK;
}

flbm_status flbm_get_step(const flbm_ctx *c, int64_t *step)
{
    if (!c || !step) return FLBM_EINVAL;
    *step = c->step;
    return FLBM_OK;
}

flbm_status flbm_moments(flbm_ctx *c, double *rho_a, double *rho_b, double *u, double *cons)
{
    if (!c) return FLBM_EINVAL;
    if (is_batch(c)) return batch_moments(c, rho_a, rho_b, u, cons);
    if (!c->initialised) return fail(c, FLBM_ESTATE, "flbm_moments before flbm_init");
    flbm_status st = ensure_obs(c);
    if (st != FLBM_OK) return st;
    const StepParams p = make_params(c);
    if ((st = density_now(c, p)) != FLBM_OK) return st;
    double *ra = c->d_obs, *rb = c->d_obs + c->N, *uu = c->d_obs + 2 * c->N;
    // with shared page tables the kernel stores the fields straight into the
    // caller's buffers (their pages mapped first); otherwise into device
    // scratch, copied out through the pinned staging buffer below
    const bool direct = c->direct_host && pageable_direct();
    if (direct) {
        if (rho_a) map_pages(rho_a, c->N * sizeof(double));
        if (rho_b) map_pages(rho_b, c->N * sizeof(double));
        if (u) map_pages(u, (size_t)c->D * c->N * sizeof(double));
        ra = rho_a;
        rb = rho_b;
        uu = u;
    }
    int nb = 0;
    FLBM_CUDA(c, launch_observables(c->lat, c->storage, layout_parity(c), p, cur_pop(c), c->rho, rho_a ? ra : nullptr,
                                    rho_b ? rb : nullptr, u ? uu : nullptr, c->d_partials, &nb, c->stream),
              "observables kernel launch");
    FLBM_CUDA(c, launch_sum_partials(c->d_partials, nb, c->d_cons, c->stream), "reduction kernel launch");
    if ((st = sync_and_check(c)) != FLBM_OK) return st;
    if (direct) {
        if (cons) FLBM_CUDA(c, cudaMemcpy(cons, c->d_cons, 5 * sizeof(double), cudaMemcpyDeviceToHost), "D2H cons");
        return FLBM_OK;
    }
    if ((st = ensure_stage(c)) != FLBM_OK) return st;
    if (rho_a && (st = d2h_staged(c, rho_a, ra, c->N * sizeof(double))) != FLBM_OK) return st;
    if (rho_b && (st = d2h_staged(c, rho_b, rb, c->N * sizeof(double))) != FLBM_OK) return st;
    if (u && (st = d2h_staged(c, u, uu, (size_t)c->D * c->N * sizeof(double))) != FLBM_OK) return st;
    if (cons) FLBM_CUDA(c, cudaMemcpy(cons, c->d_cons, 5 * sizeof(double), cudaMemcpyDeviceToHost), "D2H cons");
    return FLBM_OK;
}

flbm_status flbm_sf_sample(flbm_ctx *c)
{
    if (!c) return FLBM_EINVAL;
    if (is_batch(c)) return batch_sf_sample(c);
    if (!c->initialised) return fail(c, FLBM_ESTATE, "flbm_sf_sample before flbm_init");
    flbm_status st = ensure_obs(c);
    if (st != FLBM_OK) return st;
    if ((st = ensure_sf(c)) != FLBM_OK) return st;
    const StepParams p = make_params(c);
    if ((st = density_now(c, p)) != FLBM_OK) return st;
    int nb = 0;
    FLBM_CUDA(c, launch_observables(c->lat, c->storage, layout_parity(c), p, cur_pop(c), c->rho, c->d_obs, c->d_obs + c->N,
                                    c->d_obs + 2 * c->N, c->d_partials, &nb, c->stream),
              "observables kernel launch");
    FLBM_CUDA(c, launch_sf_accumulate(c->D, c->nx, c->ny, c->nz, c->sf_axis, c->d_obs, c->d_profile, c->d_sf, c->stream),
              "structure-factor kernel launch");
    if ((st = sync_and_check(c)) != FLBM_OK) return st;
    c->sf_count++;
    return FLBM_OK;
}

flbm_status flbm_structure_factor(flbm_ctx *c, int axis, int nk, double *S_aa, double *S_ab, double *S_bb,
                                  double *S_uu, int64_t *nsamples)
{
    if (!c) return FLBM_EINVAL;
    if (is_batch(c)) return fail(c, FLBM_EINVAL, "a batch has one structure factor per replica: use flbm_batch_replica");
    if (axis != c->sf_axis) return fail(c, FLBM_EINVAL, "axis %d differs from the sampled axis %d", axis, c->sf_axis);
    const int half = axis_len(c, axis) / 2;
    if (nk < 1 || nk > half) return fail(c, FLBM_EINVAL, "nk must lie in [1, %d]", half);
    if (nsamples) *nsamples = c->sf_count;
    if (!c->d_sf || c->sf_count == 0) return fail(c, FLBM_ESTATE, "no structure-factor snapshot taken");
    flbm_status st = sync_and_check(c);
    if (st != FLBM_OK) return st;
    std::vector<double> h((size_t)4 * half);
    FLBM_CUDA(c, cudaMemcpy(h.data(), c->d_sf, h.size() * sizeof(double), cudaMemcpyDeviceToHost), "D2H sf");
    double *outs[4] = {S_aa, S_ab, S_bb, S_uu};
    for (int q = 0; q < 4; q++)
        if (outs[q])
            for (int m = 0; m < nk; m++) outs[q][m] = h[(size_t)q * half + m] / (double)c->sf_count;
    return FLBM_OK;
}

flbm_status flbm_sf_reset(flbm_ctx *c)
{
    if (!c) return FLBM_EINVAL;
    if (is_batch(c)) {
        for (int r = 0;; r++) {
            flbm_ctx *v = nullptr;
            if (flbm_batch_replica(c, r, &v) != FLBM_OK) break;
            flbm_sf_reset(v);
        }
        return FLBM_OK;
    }
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_sf(c);
    return FLBM_OK;
}

flbm_status flbm_get_populations(flbm_ctx *c, double *f)
{
    if (!c || !f) return FLBM_EINVAL;
    if (is_batch(c)) return batch_get_populations(c, f);
    if (!c->initialised) return fail(c, FLBM_ESTATE, "no populations before flbm_init");
    flbm_status st = sync_and_check(c);
    if (st != FLBM_OK) return st;
    const size_t bytes = array_bytes_of(c);
    std::vector<unsigned char> raw(bytes);
    FLBM_CUDA(c, cudaMemcpy(raw.data(), cur_pop(c), bytes, cudaMemcpyDeviceToHost), "D2H populations");
    for (int s = 0; s < 2; s++)
        for (int i = 0; i < c->Q; i++)
            for (int64_t site = 0; site < c->N; site++)
                f[((size_t)s * c->Q + i) * c->N + site] = raw_to_natural(c, raw, s, i, site);
    return FLBM_OK;
}

flbm_status flbm_set_populations(flbm_ctx *c, const double *f, int64_t step)
{
    if (!c || !f || step < 0) return FLBM_EINVAL;
    if (!view_call_allowed(c)) return fail(c, FLBM_ESTATE, "a replica view can be observed, not changed; use its batch");
    if (is_batch(c)) return batch_set_populations(c, f, step);
    flbm_status st = ensure_buffers(c);
    if (st != FLBM_OK) return st;
    FLBM_CUDA(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    const size_t n = (size_t)2 * c->Q * c->N;
    std::vector<unsigned char> raw(n * storage_bytes(c->storage));
    for (int s = 0; s < 2; s++)
        for (int i = 0; i < c->Q; i++) {
            const float base = (float)lat_w(c->lat, i) * (float)c->rho0[s];
            for (int64_t site = 0; site < c->N; site++) {
                const size_t idx = ((size_t)s * c->Q + i) * c->N + site;          // caller's [s][i][site]
                const size_t at = pop_index(s, i, (size_t)site, (size_t)c->N); // the device layout
                const double v = f[idx];
                if (!std::isfinite(v)) return fail(c, FLBM_EINVAL, "non-finite population at index %zu", idx);
                if (c->storage == FLBM_STORE_F32) {
                    const float x = (float)(v - (double)base);
                    std::memcpy(raw.data() + at * 4, &x, 4);
                } else if (c->storage == FLBM_STORE_F16) {
                    const __half h = __float2half_rn((float)(v - (double)base));
                    const __half_raw hr = h;
                    std::memcpy(raw.data() + at * 2, &hr.x, 2);
                } else {
                    const __nv_bfloat16 b = __float2bfloat16_rn((float)(v - (double)base));
                    const __nv_bfloat16_raw br = b;
                    std::memcpy(raw.data() + at * 2, &br.x, 2);
                }
            }
        }
    FLBM_CUDA(c, cudaMemcpy(c->pop, raw.data(), raw.size(), cudaMemcpyHostToDevice), "H2D populations");
    FLBM_CUDA(c, cudaMemset(c->d_status, 0, sizeof(unsigned)), "status reset");
    c->step = step;
    c->parity = 0;
    c->faulted = false;
    c->timed_out = false;
    c->initialised = true;
    return FLBM_OK;
}

flbm_status flbm_get_site_populations(flbm_ctx *c, const int64_t *sites, int64_t nsites, double *out)
{
    if (!c || (!sites && nsites) || (!out && nsites) || nsites < 0) return FLBM_EINVAL;
    if (is_batch(c)) return fail(c, FLBM_EINVAL, "site indices are per replica: use flbm_batch_replica");
    if (!c->initialised) return fail(c, FLBM_ESTATE, "no populations before flbm_init");
    for (int64_t k = 0; k < nsites; k++)
        if (sites[k] < 0 || sites[k] >= c->N) return fail(c, FLBM_EINVAL, "site index %lld out of range", (long long)sites[k]);
    flbm_status st = sync_and_check(c);
    if (st != FLBM_OK || nsites == 0) return st;
    int64_t *d_sites = nullptr;
    double *d_out = nullptr;
    const size_t out_n = (size_t)nsites * 2 * c->Q;
    cudaError_t e = cudaMalloc((void **)&d_sites, nsites * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMalloc((void **)&d_out, out_n * sizeof(double));
    if (e == cudaSuccess) e = cudaMemcpy(d_sites, sites, nsites * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_gather_sites(c->lat, c->storage, layout_parity(c), make_params(c), cur_pop(c), d_sites, nsites,
                                                      d_out, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) e = cudaMemcpy(out, d_out, out_n * sizeof(double), cudaMemcpyDeviceToHost);
    cudaFree(d_sites);
    cudaFree(d_out);
    if (e != cudaSuccess) return cuda_fail(c, e, "site gather");
    return FLBM_OK;
}

flbm_status flbm_checkpoint(flbm_ctx *c, void *buf, size_t *bytes)
{
    if (!c || !bytes) return FLBM_EINVAL;
    if (is_batch(c)) return batch_checkpoint(c, buf, bytes);
    const size_t payload = array_bytes_of(c); // the current state only
    const size_t need = sizeof(CkptHeader) + payload;
    if (!buf) {
        *bytes = need;
        return FLBM_OK;
    }
    if (*bytes < need) return fail(c, FLBM_EINVAL, "checkpoint buffer too small: need %zu bytes", need);
    if (!c->initialised) return fail(c, FLBM_ESTATE, "nothing to checkpoint before flbm_init");
    flbm_status st = sync_and_check(c);
    if (st != FLBM_OK) return st;
    CkptHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, "FLBMCKP1", 8);
    h.version = 4; // 2: float storage holds deviations f_i - w_i rho0; 3: with the ghost-noise option;
                   // 4: the two species' words of a slot side by side
    h.lat = c->lat;
    h.nx = c->nx;
    h.ny = c->ny;
    h.nz = c->nz;
    h.storage = c->storage;
    h.parity = layout_parity(c);
    h.sdf = c->sdf;
    h.noise_ref = c->noise_ref;
    h.force_velocity = c->force_velocity;
    h.ghost_noise = c->ghost_noise;
    h.pad_ = 0;
    h.sf_axis = c->sf_axis;
    h.step = c->step;
    h.seed = c->seed;
    std::memcpy(h.tau, c->tau, sizeof(h.tau));
    h.kT = c->kT;
    h.G = c->G;
    std::memcpy(h.rho0, c->rho0, sizeof(h.rho0));
    std::memcpy(h.lam, c->lam, sizeof(h.lam));
    h.payload_bytes = payload;
    unsigned char *dst = static_cast<unsigned char *>(buf);
    FLBM_CUDA(c, cudaMemcpy(dst + sizeof(CkptHeader), cur_pop(c), payload, cudaMemcpyDeviceToHost), "D2H checkpoint");
    h.payload_hash = fnv1a(dst + sizeof(CkptHeader), payload);
    std::memcpy(dst, &h, sizeof(h));
    *bytes = need;
    return FLBM_OK;
}

flbm_status flbm_restore(flbm_ctx *c, const void *buf, size_t bytes)
{
    if (!c || !buf) return FLBM_EINVAL;
    if (!view_call_allowed(c)) return fail(c, FLBM_ESTATE, "a replica view can be observed, not changed; use its batch");
    if (is_batch(c)) return batch_restore(c, buf, bytes);
    if (bytes < sizeof(CkptHeader)) return fail(c, FLBM_EINVAL, "checkpoint image too small");
    CkptHeader h;
    std::memcpy(&h, buf, sizeof(h));
    if (std::memcmp(h.magic, "FLBMCKP1", 8) != 0 || h.version != 4) return fail(c, FLBM_EINVAL, "not a checkpoint image");
    if (h.lat != c->lat || h.nx != c->nx || h.ny != c->ny || h.nz != c->nz)
        return fail(c, FLBM_EINVAL, "checkpoint lattice or box differs from this context");
    if (c->pop && h.storage != c->storage) return fail(c, FLBM_EINVAL, "checkpoint storage format differs");
    const size_t payload = (size_t)2 * c->Q * (size_t)c->N * storage_bytes(h.storage);
    if (h.payload_bytes != payload || bytes < sizeof(CkptHeader) + payload)
        return fail(c, FLBM_EINVAL, "checkpoint image truncated");
    if (two_arrays(c) && h.parity != 0)
        return fail(c, FLBM_EINVAL, "an in-place image in the swapped layout restores into an in-place context only");
    const unsigned char *src = static_cast<const unsigned char *>(buf) + sizeof(CkptHeader);
    if (fnv1a(src, payload) != h.payload_hash) return fail(c, FLBM_EINVAL, "checkpoint image corrupt (hash mismatch)");
    c->storage = h.storage;
    std::memcpy(c->rho0, h.rho0, sizeof(h.rho0));
    flbm_status st = ensure_buffers(c);
    if (st != FLBM_OK) return st;
    FLBM_CUDA(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    FLBM_CUDA(c, cudaMemcpy(c->pop, src, payload, cudaMemcpyHostToDevice), "H2D checkpoint");
    FLBM_CUDA(c, cudaMemset(c->d_status, 0, sizeof(unsigned)), "status reset");
    c->parity = h.parity;
    c->step = h.step;
    c->seed = h.seed;
    c->tau[0] = h.tau[0];
    c->tau[1] = h.tau[1];
    c->kT = h.kT;
    c->G = h.G;
    c->sdf = h.sdf;
    c->noise_ref = h.noise_ref;
    c->force_velocity = h.force_velocity;
    c->ghost_noise = h.ghost_noise;
    std::memcpy(c->lam, h.lam, sizeof(h.lam));
    if (h.sf_axis != c->sf_axis) {
        free_sf(c);
        c->sf_axis = h.sf_axis;
    }
    c->faulted = false;
    c->timed_out = false;
    c->initialised = true;
    return FLBM_OK;
}

void flbm_destroy(flbm_ctx *c)
{
    if (!c) return;
    if (c->is_view && c->batch) return; // replica views belong to their batch
    if (c->batch) batch_destroy(c);
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->own_buffers) {
        if (c->pop) cudaFree(c->pop);
        if (c->rho) cudaFree(c->rho);
    }
    drop_step_graphs(c);
    if (c->d_gstep) cudaFree(c->d_gstep);
    if (c->d_mom) cudaFree(c->d_mom);
    if (c->d_status) cudaFree(c->d_status);
    if (c->d_pipe) cudaFree(c->d_pipe);
    if (c->d_ring) cudaFree(c->d_ring);
    if (c->d_ring_cnt) cudaFree(c->d_ring_cnt);
    if (c->d_obs) cudaFree(c->d_obs);
    if (c->d_partials) cudaFree(c->d_partials);
    if (c->d_cons) cudaFree(c->d_cons);
    free_sf(c);
    free_sfk(c);
    free_cap(c);
    if (c->h_stage) cudaFreeHost(c->h_stage);
    if (c->d_bad) cudaFree(c->d_bad);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    for (cudaEvent_t e : c->ev_dep) cudaEventDestroy(e);
    if (c->stream_d) cudaStreamDestroy(c->stream_d);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

} // extern "C"
