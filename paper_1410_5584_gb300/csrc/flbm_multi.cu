// flbm_multi.cu -- the flbm_m* C-ABI: N-species mixtures (arXiv 1410.5584,
// App. C-D) on one GPU.  Kernels in flbm_multi.cuh.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "flbm_ctx.h"
#include "flbm_multi.cuh"

struct flbm_mctx {
    int lat = 0, D = 2, Q = 9, ns = 0;
    int nx = 0, ny = 0, nz = 1;
    int64_t N = 0;
    double tau[flbm::kMaxSpecies] = {}, kT = 0.0, G[flbm::kMaxSpecies][flbm::kMaxSpecies] = {};
    double rho0[flbm::kMaxSpecies] = {1.0, 1.0, 1.0, 1.0};
    double lam_d = 1.0;
    uint64_t seed = 0;
    int block_x = 128, block_y = 1;
    int streaming = FLBM_STREAM_TWO_ARRAYS; // FLBM_OPT_STREAMING
    // CUDA graphs of graph_steps steps, one per starting parity (FLBM_OPT_GRAPH_STEPS)
    int graph_steps = 0;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    unsigned *d_gstep = nullptr; // noise counter at the start of a replay
    // state
    int64_t step = 0;
    int parity = 0; // in place: 0 natural layout, 1 swapped layout (after an odd number of steps);
                    // two arrays: which of the two holds the current (natural-layout) state
    bool initialised = false, faulted = false;
    // device buffers
    float *pop = nullptr;
    float4 *drho = nullptr;
    float *d_mom = nullptr; // ns (D + 1) planes: the moment-fed pair's m_0 .. m_D (MStepParams::mom)
    unsigned *d_status = nullptr;
    double *d_obs = nullptr;      // ns * N + D * N doubles
    double *d_partials = nullptr; // per-block totals
    size_t partials_cap = 0;
    // axis structure factors (flbm_msf_*): per axis ns * ns * (n_axis / 2) FP64 sums
    double *d_sf_acc[3] = {nullptr, nullptr, nullptr};
    int64_t sf_count[3] = {0, 0, 0};
    double *d_sf_prof = nullptr; // ns * max(nx, ny, nz) doubles of scratch
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // per-kernel event timing
    bool timing = false;
    std::vector<cudaEvent_t> ev;  // pairs (start, end), kernel = (index / 2) % 2
    size_t ev_used = 0;
    double kernel_ms[2] = {0.0, 0.0};
    int64_t kernel_launches[2] = {0, 0};
    char err[512] = {0};
};

namespace {

using flbm::MStepParams;

const char kNoError[] = "";

flbm_status mfail(flbm_mctx *c, flbm_status st, const char *fmt, ...)
{
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        std::vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
    }
    return st;
}

#define MCUDA(ctx, call, what)                                                                            \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess) return mfail((ctx), FLBM_ECUDA, "%s: %s", what, cudaGetErrorString(e_)); \
    } while (0)

double lat_N(int lat, int a) { return lat == FLBM_D2Q9 ? flbm::D2Q9::Nd(a) : flbm::D3Q19::Nd(a); }

// w_i rho0^s as the kernels form it (float product): the base of the stored deviations
float dev_base(const flbm_mctx *c, int s, int i)
{
    const float w = (float)(c->lat == FLBM_D2Q9 ? flbm::D2Q9::wd(i) : flbm::D3Q19::wd(i));
    return w * (float)c->rho0[s];
}

MStepParams make_mparams(const flbm_mctx *c)
{
    MStepParams p;
    std::memset(&p, 0, sizeof(p));
    p.nx = c->nx;
    p.ny = c->ny;
    p.nz = c->nz;
    p.N = (int)c->N;
    p.block_x = c->block_x;
    p.block_y = c->block_y;
    for (int s = 0; s < c->ns; s++)
        for (int t = 0; t < c->ns; t++) p.G[s][t] = s == t ? 0.0f : (float)c->G[s][t];
    p.lam_d = (float)c->lam_d;
    p.hlam_d = (float)(1.0 - 0.5 * c->lam_d);
    p.amp_d = (float)std::sqrt((2.0 * c->lam_d - c->lam_d * c->lam_d) * c->kT);
    const double mu = 3.0 * c->kT; // k_B T / c_s^2
    for (int s = 0; s < c->ns; s++) {
        const double lb = 1.0 / c->tau[s];
        for (int a = c->D + 1; a < c->Q; a++) {
            const double Na = lat_N(c->lat, a);
            p.cm[s][a] = (float)((1.0 - lb) / Na);
            p.ceq[s][a] = (float)(lb / Na);
            p.cphi[s][a] = (float)((1.0 - 0.5 * lb) / Na);
            p.cxi[s][a] = (float)(std::sqrt((2.0 * lb - lb * lb) * Na * mu) / Na);
        }
        p.rho0[s] = (float)c->rho0[s];
    }
    p.key0 = (uint32_t)(c->seed & 0xFFFFFFFFu);
    p.key1 = (uint32_t)(c->seed >> 32);
    p.step = (uint32_t)c->step;
    return p;
}

// Dispatch over (lattice, species count).
template <class F> cudaError_t dispatch(const flbm_mctx *c, F &&f)
{
    using namespace flbm;
    if (c->lat == FLBM_D2Q9) {
        switch (c->ns) {
        case 2: return f(MLaunch<D2Q9, 2>{});
        case 3: return f(MLaunch<D2Q9, 3>{});
        case 4: return f(MLaunch<D2Q9, 4>{});
        }
    } else {
        switch (c->ns) {
        case 2: return f(MLaunch<D3Q19, 2>{});
        case 3: return f(MLaunch<D3Q19, 3>{});
        case 4: return f(MLaunch<D3Q19, 4>{});
        }
    }
    return cudaErrorInvalidValue;
}

size_t pop_elems(const flbm_mctx *c) { return (size_t)c->ns * c->Q * (size_t)c->N; } // one array
bool two_arrays(const flbm_mctx *c) { return c->streaming == FLBM_STREAM_TWO_ARRAYS; }
// the array holding the current state, the one a two-array step writes, and
// the layout readers see (two arrays: always natural)
float *cur_pop_at(const flbm_mctx *c, int par) { return c->pop + (two_arrays(c) && par ? pop_elems(c) : 0); }
float *next_pop_at(const flbm_mctx *c, int par) { return c->pop + (two_arrays(c) && !par ? pop_elems(c) : 0); }
float *cur_pop(const flbm_mctx *c) { return cur_pop_at(c, c->parity); }
float *next_pop(const flbm_mctx *c) { return next_pop_at(c, c->parity); }
void drop_graphs(flbm_mctx *c)
{
    for (int k = 0; k < 2; k++) {
        if (c->graph[k]) cudaGraphExecDestroy(c->graph[k]);
        c->graph[k] = nullptr;
    }
}
int layout_parity(const flbm_mctx *c) { return two_arrays(c) ? 0 : c->parity; }

flbm_status ensure_buffers(flbm_mctx *c)
{
    if (!c->stream) {
        MCUDA(c, cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking), "cudaStreamCreate");
        c->own_stream = true;
    }
    if (!c->pop) {
        // both buffers or neither: a later call must never find one without the other
        float *pop = nullptr;
        float4 *drho = nullptr;
        cudaError_t e = cudaMalloc((void **)&pop, pop_elems(c) * (two_arrays(c) ? 2 : 1) * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc((void **)&drho, (size_t)c->N * sizeof(float4));
        if (e != cudaSuccess) {
            cudaFree(pop);
            cudaGetLastError(); // clear the allocation error
            return mfail(c, FLBM_ENOMEM, "cudaMalloc of %zu population bytes and the density field failed: %s",
                         pop_elems(c) * sizeof(float), cudaGetErrorString(e));
        }
        c->pop = pop;
        c->drho = drho;
    }
    if (!c->d_status) {
        MCUDA(c, cudaMalloc((void **)&c->d_status, sizeof(unsigned)), "cudaMalloc(status)");
        MCUDA(c, cudaMemsetAsync(c->d_status, 0, sizeof(unsigned), c->stream), "cudaMemset(status)");
    }
    return FLBM_OK;
}

flbm_status sync_and_check(flbm_mctx *c)
{
    MCUDA(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    unsigned st = 0;
    MCUDA(c, cudaMemcpy(&st, c->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost), "status read");
    if (st & flbm::kStatusNonFinite) {
        c->faulted = true;
        return mfail(c, FLBM_ENONFINITE, "a density became non-positive or non-finite on the device");
    }
    return FLBM_OK;
}

flbm_status check_ready(flbm_mctx *c)
{
    if (!c) return FLBM_EINVAL;
    if (!c->initialised) return mfail(c, FLBM_ESTATE, "call flbm_minit or flbm_mset_populations first");
    return FLBM_OK;
}

cudaEvent_t timing_event(flbm_mctx *c)
{
    if (c->ev_used == c->ev.size()) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        c->ev.push_back(e);
    }
    return c->ev[c->ev_used++];
}

flbm_status drain_timing(flbm_mctx *c)
{
    if (c->ev_used == 0) return FLBM_OK;
    MCUDA(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    for (size_t k = 0; k + 1 < c->ev_used; k += 2) {
        float ms = 0.0f;
        MCUDA(c, cudaEventElapsedTime(&ms, c->ev[k], c->ev[k + 1]), "cudaEventElapsedTime");
        const int kernel = (int)((k / 2) % 2);
        c->kernel_ms[kernel] += ms;
        c->kernel_launches[kernel] += 1;
    }
    c->ev_used = 0;
    return FLBM_OK;
}

int axis_len(const flbm_mctx *c, int axis) { return axis == 0 ? c->nx : (axis == 1 ? c->ny : c->nz); }

// The density field of the current state.
flbm_status density_now(flbm_mctx *c, const MStepParams &p)
{
    cudaError_t e = dispatch(c, [&](auto l) {
        return decltype(l)::density(layout_parity(c), p, cur_pop(c), c->drho, c->stream);
    });
    MCUDA(c, e, "density kernel launch");
    return FLBM_OK;
}

} // namespace

extern "C" {

flbm_status flbm_mcreate(flbm_lattice lat, int nspecies, int nx, int ny, int nz, const double *tau, double kT,
                         const double *G, uint64_t seed, flbm_mctx **out)
{
    if (!out) return FLBM_EINVAL;
    *out = nullptr;
    if (lat != FLBM_D2Q9 && lat != FLBM_D3Q19) return FLBM_EINVAL;
    if (nspecies < 2 || nspecies > flbm::kMaxSpecies || !tau || !G) return FLBM_EINVAL;
    if (nx < 2 || ny < 2 || ny > 65535) return FLBM_EINVAL;
    if (lat == FLBM_D2Q9 ? nz != 1 : (nz < 2 || nz > 65535)) return FLBM_EINVAL;
    if ((int64_t)nx * ny * nz >= (int64_t(1) << 31)) return FLBM_EINVAL;
    if (!(kT >= 0.0) || !std::isfinite(kT)) return FLBM_EINVAL;
    double tsum = 0.0;
    for (int s = 0; s < nspecies; s++) {
        if (!(tau[s] > 0.5) || !std::isfinite(tau[s])) return FLBM_EINVAL;
        tsum += tau[s];
    }
    for (int s = 0; s < nspecies; s++)
        for (int t = 0; t < nspecies; t++)
            if (!std::isfinite(G[s * nspecies + t]) || G[s * nspecies + t] != G[t * nspecies + s]) return FLBM_EINVAL;
    flbm_mctx *c = new (std::nothrow) flbm_mctx();
    if (!c) return FLBM_ENOMEM;
    c->lat = lat;
    c->D = lat == FLBM_D2Q9 ? 2 : 3;
    c->Q = lat == FLBM_D2Q9 ? 9 : 19;
    c->ns = nspecies;
    c->nx = nx;
    c->ny = ny;
    c->nz = nz;
    c->N = (int64_t)nx * ny * nz;
    c->kT = kT;
    c->seed = seed;
    for (int s = 0; s < nspecies; s++) {
        c->tau[s] = tau[s];
        for (int t = 0; t < nspecies; t++) c->G[s][t] = s == t ? 0.0 : G[s * nspecies + t];
    }
    c->lam_d = nspecies / tsum;
    *out = c;
    return FLBM_OK;
}

flbm_status flbm_mset_option(flbm_mctx *c, int key, double v)
{
    if (!c) return FLBM_EINVAL;
    drop_graphs(c); // a captured step holds the parameters and launch settings by value
    if (key == FLBM_OPT_GRAPH_STEPS) {
        if (!(v >= 0.0 && v <= 4096.0) || v != (double)(int)v)
            return mfail(c, FLBM_EINVAL, "graph steps must be an integer in [0, 4096]");
        c->graph_steps = (int)v;
        return FLBM_OK;
    }
    if (key == FLBM_OPT_KERNEL_TIMING) {
        if (v != 0.0 && v != 1.0) return mfail(c, FLBM_EINVAL, "kernel timing is 0 or 1");
        if (c->stream) {
            flbm_status st = drain_timing(c);
            if (st != FLBM_OK) return st;
        }
        c->timing = v != 0.0;
        c->kernel_ms[0] = c->kernel_ms[1] = 0.0;
        c->kernel_launches[0] = c->kernel_launches[1] = 0;
        return FLBM_OK;
    }
    if (key == FLBM_OPT_BLOCK_X || key == FLBM_OPT_BLOCK_Y) {
        const int b = (int)v;
        if ((double)b != v) return mfail(c, FLBM_EINVAL, "the block shape is an integer");
        const int bx = key == FLBM_OPT_BLOCK_X ? b : c->block_x, by = key == FLBM_OPT_BLOCK_Y ? b : c->block_y;
        if ((bx != 32 && bx != 64 && bx != 128) || (by != 1 && by != 2 && by != 4) || bx * by > flbm::kSiteBlockMax)
            return mfail(c, FLBM_EINVAL, "block shape %d x %d: x in {32, 64, 128}, y in {1, 2, 4}, x y <= 128", bx, by);
        c->block_x = bx;
        c->block_y = by;
        return FLBM_OK;
    }
    if (key == FLBM_OPT_STREAMING) {
        if (c->pop) return mfail(c, FLBM_ESTATE, "the streaming mode is fixed once the buffers exist");
        if (v != (double)FLBM_STREAM_IN_PLACE && v != (double)FLBM_STREAM_TWO_ARRAYS)
            return mfail(c, FLBM_EINVAL, "streaming must be 0 (in place) or 1 (two arrays)");
        c->streaming = (int)v;
        return FLBM_OK;
    }
    if (key >= FLBM_OPT_RHO0_SPECIES && key < FLBM_OPT_RHO0_SPECIES + c->ns) {
        if (c->initialised) return mfail(c, FLBM_ESTATE, "the reference densities are fixed once the state exists");
        if (!(v > 0.0) || !std::isfinite(v)) return mfail(c, FLBM_EINVAL, "a reference density is positive");
        c->rho0[key - FLBM_OPT_RHO0_SPECIES] = v;
        return FLBM_OK;
    }
    return mfail(c, FLBM_EINVAL, "unknown option %d for an N-species context", key);
}

flbm_status flbm_mget_option(const flbm_mctx *c, int key, double *value)
{
    if (!c || !value) return FLBM_EINVAL;
    if (key == FLBM_OPT_KERNEL_TIMING) *value = c->timing ? 1.0 : 0.0;
    else if (key == FLBM_OPT_BLOCK_X) *value = c->block_x;
    else if (key == FLBM_OPT_BLOCK_Y) *value = c->block_y;
    else if (key == FLBM_OPT_STREAMING) *value = c->streaming;
    else if (key == FLBM_OPT_GRAPH_STEPS) *value = c->graph_steps;
    else if (key >= FLBM_OPT_RHO0_SPECIES && key < FLBM_OPT_RHO0_SPECIES + c->ns) *value = c->rho0[key - FLBM_OPT_RHO0_SPECIES];
    else return FLBM_EINVAL;
    return FLBM_OK;
}

flbm_status flbm_mset_stream(flbm_mctx *c, void *stream)
{
    if (!c) return FLBM_EINVAL;
    drop_graphs(c);
    if (c->initialised) {
        MCUDA(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    }
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    c->stream = (cudaStream_t)stream;
    c->own_stream = false;
    if (!c->stream) {
        MCUDA(c, cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking), "cudaStreamCreate");
        c->own_stream = true;
    }
    return FLBM_OK;
}

flbm_status flbm_minit(flbm_mctx *c, const double *rho)
{
    if (!c) return FLBM_EINVAL;
    flbm_status st = ensure_buffers(c);
    if (st != FLBM_OK) return st;
    const size_t n = (size_t)c->ns * c->N;
    std::vector<float> h(n);
    for (int s = 0; s < c->ns; s++)
        for (int64_t k = 0; k < c->N; k++) {
            const double r = rho ? rho[(size_t)s * c->N + k] : c->rho0[s];
            if (!(r > 0.0) || !std::isfinite(r)) return mfail(c, FLBM_EINVAL, "densities must be positive and finite");
            h[(size_t)s * c->N + k] = (float)r;
        }
    float *d = nullptr;
    MCUDA(c, cudaMallocAsync((void **)&d, n * sizeof(float), c->stream), "cudaMallocAsync");
    cudaError_t e = cudaMemcpyAsync(d, h.data(), n * sizeof(float), cudaMemcpyHostToDevice, c->stream);
    const MStepParams p = make_mparams(c);
    if (e == cudaSuccess) e = dispatch(c, [&](auto l) { return decltype(l)::init_rest(p, d, c->pop, c->stream); });
    cudaFreeAsync(d, c->stream);
    MCUDA(c, e, "rest-state initialisation");
    MCUDA(c, cudaMemsetAsync(c->d_status, 0, sizeof(unsigned), c->stream), "cudaMemset(status)");
    MCUDA(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    c->step = 0;
    c->parity = 0;
    c->faulted = false;
    c->initialised = true;
    return FLBM_OK;
}

// With two arrays and every non-conserved rate 1 (the old non-conserved
// moments drop out of Eq. algorithm) the density pass also stores m_0 .. m_D
// of every species and the collide reads those instead of the populations:
// sets p.mom then.
static flbm_status use_mmoments(flbm_mctx *c, MStepParams &p)
{
    p.mom = nullptr;
    if (!two_arrays(c)) return FLBM_OK;
    for (int s = 0; s < c->ns; s++)
        for (int a = c->D + 1; a < c->Q; a++)
            if (p.cm[s][a] != 0.0f) return FLBM_OK;
    if (!c->d_mom)
        MCUDA(c, cudaMalloc((void **)&c->d_mom, (size_t)c->ns * (c->D + 1) * (size_t)c->N * sizeof(float)),
              "cudaMalloc(moment planes)");
    p.mom = c->d_mom;
    return FLBM_OK;
}

// One CUDA graph of graph_steps steps from `parity`; the collide reads the
// noise counter as *d_gstep + k.
flbm_status ensure_graph(flbm_mctx *c, int parity)
{
    if (c->graph[parity]) return FLBM_OK;
    if (!c->d_gstep) MCUDA(c, cudaMalloc((void **)&c->d_gstep, sizeof(unsigned)), "cudaMalloc(graph step counter)");
    MStepParams p = make_mparams(c);
    p.step_dev = c->d_gstep;
    if (flbm_status st = use_mmoments(c, p); st != FLBM_OK) return st;
    cudaGraph_t g = nullptr;
    MCUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < c->graph_steps && e == cudaSuccess; k++) {
        const int par = (parity + k) & 1;
        p.step = (uint32_t)k;
        float *cur = cur_pop_at(c, par), *nxt = next_pop_at(c, par);
        const int lp = two_arrays(c) ? 0 : par, cp = two_arrays(c) ? flbm::kStreamPush : par;
        e = dispatch(c, [&](auto l) { return decltype(l)::density(lp, p, cur, c->drho, c->stream); });
        if (e == cudaSuccess)
            e = dispatch(c, [&](auto l) { return decltype(l)::collide(cp, p, cur, nxt, c->drho, c->d_status, c->stream); });
    }
    const cudaError_t ee = cudaStreamEndCapture(c->stream, &g);
    if (e != cudaSuccess || ee != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return mfail(c, FLBM_ECUDA, "step graph capture: %s", cudaGetErrorString(e != cudaSuccess ? e : ee));
    }
    e = cudaGraphInstantiate(&c->graph[parity], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        c->graph[parity] = nullptr;
        return mfail(c, FLBM_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
    }
    return FLBM_OK;
}

flbm_status flbm_mstep(flbm_mctx *c, int64_t n)
{
    flbm_status st = check_ready(c);
    if (st != FLBM_OK) return st;
    if (n < 0) return mfail(c, FLBM_EINVAL, "negative step count");
    if (c->graph_steps > 0 && !c->timing) {
        while (n >= c->graph_steps) {
            if ((st = ensure_graph(c, c->parity)) != FLBM_OK) return st;
            MCUDA(c, flbm::launch_set_u32(c->d_gstep, (unsigned)c->step, c->stream), "graph step counter");
            MCUDA(c, cudaGraphLaunch(c->graph[c->parity], c->stream), "cudaGraphLaunch");
            c->step += c->graph_steps;
            c->parity = (c->parity + c->graph_steps) & 1;
            n -= c->graph_steps;
        }
    }
    for (int64_t k = 0; k < n; k++) {
        MStepParams p = make_mparams(c);
        if ((st = use_mmoments(c, p)) != FLBM_OK) return st;
        const int parity = c->parity;
        cudaEvent_t e0 = nullptr, e1 = nullptr, e2 = nullptr, e3 = nullptr;
        if (c->timing) {
            if (c->ev_used + 4 > 4096) {
                st = drain_timing(c);
                if (st != FLBM_OK) return st;
            }
            e0 = timing_event(c);
            e1 = timing_event(c);
            e2 = timing_event(c);
            e3 = timing_event(c);
            if (!e0 || !e1 || !e2 || !e3) return mfail(c, FLBM_ECUDA, "cudaEventCreate failed");
            MCUDA(c, cudaEventRecord(e0, c->stream), "cudaEventRecord");
        }
        float *cur = cur_pop(c), *nxt = next_pop(c);
        const int lp = layout_parity(c), cp = two_arrays(c) ? flbm::kStreamPush : parity;
        cudaError_t e = dispatch(c, [&](auto l) { return decltype(l)::density(lp, p, cur, c->drho, c->stream); });
        MCUDA(c, e, "density kernel launch");
        if (c->timing) {
            MCUDA(c, cudaEventRecord(e1, c->stream), "cudaEventRecord");
            MCUDA(c, cudaEventRecord(e2, c->stream), "cudaEventRecord");
        }
        e = dispatch(c, [&](auto l) {
            return decltype(l)::collide(cp, p, cur, nxt, c->drho, c->d_status, c->stream);
        });
        MCUDA(c, e, "collide kernel launch");
        if (c->timing) MCUDA(c, cudaEventRecord(e3, c->stream), "cudaEventRecord");
        c->parity ^= 1;
        c->step++;
    }
    return FLBM_OK;
}

flbm_status flbm_msync(flbm_mctx *c)
{
    flbm_status st = check_ready(c);
    if (st != FLBM_OK) return st;
    return sync_and_check(c);
}

flbm_status flbm_mkernel_times(flbm_mctx *c, double ms[2], int64_t launches[2])
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

flbm_status flbm_mget_step(const flbm_mctx *c, int64_t *step)
{
    if (!c || !step) return FLBM_EINVAL;
    *step = c->step;
    return FLBM_OK;
}

flbm_status flbm_mmoments(flbm_mctx *c, double *rho, double *u, double *cons)
{
    flbm_status st = check_ready(c);
    if (st != FLBM_OK) return st;
    const MStepParams p = make_mparams(c);
    const int nblk = (int)((c->N + flbm::mkern::kObsBlock - 1) / flbm::mkern::kObsBlock);
    const size_t ncol = (size_t)c->ns + 3;
    if (!c->d_obs) MCUDA(c, cudaMalloc((void **)&c->d_obs, (size_t)(c->ns + c->D) * c->N * sizeof(double)), "cudaMalloc(obs)");
    if (c->partials_cap < (size_t)nblk * ncol) {
        if (c->d_partials) cudaFree(c->d_partials);
        c->d_partials = nullptr;
        MCUDA(c, cudaMalloc((void **)&c->d_partials, (size_t)nblk * ncol * sizeof(double)), "cudaMalloc(partials)");
        c->partials_cap = (size_t)nblk * ncol;
    }
    st = density_now(c, p);
    if (st != FLBM_OK) return st;
    double *d_rho = c->d_obs, *d_u = c->d_obs + (size_t)c->ns * c->N;
    int nb = 0;
    cudaError_t e = dispatch(c, [&](auto l) {
        return decltype(l)::observables(layout_parity(c), p, cur_pop(c), c->drho, rho ? d_rho : nullptr, u ? d_u : nullptr,
                                        c->d_partials, &nb, c->stream);
    });
    MCUDA(c, e, "observables kernel launch");
    st = sync_and_check(c);
    if (st != FLBM_OK) return st;
    if (rho) MCUDA(c, cudaMemcpy(rho, d_rho, (size_t)c->ns * c->N * sizeof(double), cudaMemcpyDeviceToHost), "copy rho");
    if (u) MCUDA(c, cudaMemcpy(u, d_u, (size_t)c->D * c->N * sizeof(double), cudaMemcpyDeviceToHost), "copy u");
    if (cons) {
        // the per-block totals, summed in block order
        std::vector<double> h((size_t)nb * ncol);
        MCUDA(c, cudaMemcpy(h.data(), c->d_partials, h.size() * sizeof(double), cudaMemcpyDeviceToHost), "copy totals");
        for (size_t k = 0; k < ncol; k++) cons[k] = 0.0;
        for (int b = 0; b < nb; b++)
            for (size_t k = 0; k < ncol; k++) cons[k] += h[(size_t)b * ncol + k];
    }
    return FLBM_OK;
}

flbm_status flbm_mget_populations(flbm_mctx *c, double *f)
{
    flbm_status st = check_ready(c);
    if (st != FLBM_OK) return st;
    if (!f) return mfail(c, FLBM_EINVAL, "null output");
    const MStepParams p = make_mparams(c);
    const size_t n = pop_elems(c);
    float *d = nullptr;
    MCUDA(c, cudaMallocAsync((void **)&d, n * sizeof(float), c->stream), "cudaMallocAsync");
    cudaError_t e =
        dispatch(c, [&](auto l) { return decltype(l)::natural(layout_parity(c), p, cur_pop(c), d, c->stream); });
    std::vector<float> h(n);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), d, n * sizeof(float), cudaMemcpyDeviceToHost, c->stream);
    cudaFreeAsync(d, c->stream);
    MCUDA(c, e, "natural-layout copy");
    st = sync_and_check(c);
    if (st != FLBM_OK) return st;
    for (int s = 0; s < c->ns; s++)
        for (int i = 0; i < c->Q; i++) {
            const double base = dev_base(c, s, i);
            const size_t off = ((size_t)s * c->Q + i) * (size_t)c->N;
            for (int64_t k = 0; k < c->N; k++) f[off + k] = base + (double)h[off + k];
        }
    return FLBM_OK;
}

flbm_status flbm_mget_site_populations(flbm_mctx *c, const int64_t *sites, int64_t nsites, double *out)
{
    flbm_status st = check_ready(c);
    if (st != FLBM_OK) return st;
    if (nsites < 0 || (nsites > 0 && (!sites || !out))) return mfail(c, FLBM_EINVAL, "bad site list");
    for (int64_t k = 0; k < nsites; k++)
        if (sites[k] < 0 || sites[k] >= c->N) return mfail(c, FLBM_EINVAL, "site %lld out of range", (long long)sites[k]);
    if (nsites == 0) return FLBM_OK;
    const MStepParams p = make_mparams(c);
    const size_t nout = (size_t)nsites * c->ns * c->Q;
    int64_t *d_sites = nullptr;
    double *d_out = nullptr;
    MCUDA(c, cudaMallocAsync((void **)&d_sites, (size_t)nsites * sizeof(int64_t), c->stream), "cudaMallocAsync");
    cudaError_t e = cudaMallocAsync((void **)&d_out, nout * sizeof(double), c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_sites, sites, (size_t)nsites * sizeof(int64_t), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = dispatch(c, [&](auto l) {
            return decltype(l)::gather(layout_parity(c), p, cur_pop(c), d_sites, nsites, d_out, c->stream);
        });
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d_out, nout * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    cudaFreeAsync(d_sites, c->stream);
    if (d_out) cudaFreeAsync(d_out, c->stream);
    MCUDA(c, e, "site gather");
    return sync_and_check(c);
}

flbm_status flbm_mset_populations(flbm_mctx *c, const double *f, int64_t step)
{
    if (!c) return FLBM_EINVAL;
    if (!f || step < 0) return mfail(c, FLBM_EINVAL, "null input or negative step");
    flbm_status st = ensure_buffers(c);
    if (st != FLBM_OK) return st;
    const size_t n = pop_elems(c);
    std::vector<float> h(n);
    for (int s = 0; s < c->ns; s++)
        for (int i = 0; i < c->Q; i++) {
            const double base = dev_base(c, s, i);
            const size_t off = ((size_t)s * c->Q + i) * (size_t)c->N;
            for (int64_t k = 0; k < c->N; k++) {
                if (!std::isfinite(f[off + k])) return mfail(c, FLBM_EINVAL, "non-finite population");
                h[off + k] = (float)(f[off + k] - base);
            }
        }
    MCUDA(c, cudaMemcpyAsync(c->pop, h.data(), n * sizeof(float), cudaMemcpyHostToDevice, c->stream), "copy populations");
    MCUDA(c, cudaMemsetAsync(c->d_status, 0, sizeof(unsigned), c->stream), "cudaMemset(status)");
    MCUDA(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    c->step = step;
    c->parity = 0;
    c->faulted = false;
    c->initialised = true;
    return FLBM_OK;
}

flbm_status flbm_msf_sample(flbm_mctx *c, int axis)
{
    flbm_status st = check_ready(c);
    if (st != FLBM_OK) return st;
    if (axis < 0 || axis >= c->D) return mfail(c, FLBM_EINVAL, "axis %d of a %dD box", axis, c->D);
    const int n = axis_len(c, axis);
    const size_t nacc = (size_t)c->ns * c->ns * (n / 2);
    if (!c->d_sf_prof) {
        const int nmax = c->nx > c->ny ? (c->nx > c->nz ? c->nx : c->nz) : (c->ny > c->nz ? c->ny : c->nz);
        MCUDA(c, cudaMalloc((void **)&c->d_sf_prof, (size_t)c->ns * nmax * sizeof(double)), "cudaMalloc(profiles)");
    }
    if (!c->d_sf_acc[axis]) {
        MCUDA(c, cudaMalloc((void **)&c->d_sf_acc[axis], nacc * sizeof(double)), "cudaMalloc(S(k) sums)");
        MCUDA(c, cudaMemsetAsync(c->d_sf_acc[axis], 0, nacc * sizeof(double), c->stream), "cudaMemset(S(k) sums)");
        c->sf_count[axis] = 0;
    }
    const MStepParams p = make_mparams(c);
    st = density_now(c, p);
    if (st != FLBM_OK) return st;
    MCUDA(c, flbm::launch_msf_snapshot(c->ns, p, axis, c->drho, c->d_sf_prof, c->d_sf_acc[axis], c->stream),
          "structure-factor kernels");
    st = sync_and_check(c);
    if (st != FLBM_OK) return st;
    c->sf_count[axis]++;
    return FLBM_OK;
}

flbm_status flbm_mstructure_factor(flbm_mctx *c, int axis, int nk, double *S, int64_t *nsamples)
{
    if (!c) return FLBM_EINVAL;
    if (axis < 0 || axis >= c->D) return mfail(c, FLBM_EINVAL, "axis %d of a %dD box", axis, c->D);
    const int n = axis_len(c, axis);
    if (nk < 0 || nk > n / 2) return mfail(c, FLBM_EINVAL, "nk = %d outside 0 .. %d", nk, n / 2);
    if (!c->d_sf_acc[axis] || c->sf_count[axis] == 0)
        return mfail(c, FLBM_ESTATE, "no structure-factor snapshot along axis %d", axis);
    if (nsamples) *nsamples = c->sf_count[axis];
    if (!S || nk == 0) return FLBM_OK;
    const int nh = n / 2;
    std::vector<double> h((size_t)c->ns * c->ns * nh);
    MCUDA(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    MCUDA(c, cudaMemcpy(h.data(), c->d_sf_acc[axis], h.size() * sizeof(double), cudaMemcpyDeviceToHost), "copy S(k)");
    const double inv = 1.0 / (double)c->sf_count[axis];
    for (int st2 = 0; st2 < c->ns * c->ns; st2++)
        for (int m = 0; m < nk; m++) S[(size_t)st2 * nk + m] = h[(size_t)st2 * nh + m] * inv;
    return FLBM_OK;
}

flbm_status flbm_msf_reset(flbm_mctx *c)
{
    if (!c) return FLBM_EINVAL;
    for (int a = 0; a < 3; a++) {
        if (c->d_sf_acc[a]) cudaFree(c->d_sf_acc[a]);
        c->d_sf_acc[a] = nullptr;
        c->sf_count[a] = 0;
    }
    return FLBM_OK;
}

namespace {
// Checkpoint image: this header, then the stored deviations in the current
// (parity-dependent) layout.
struct MCkptHeader {
    char magic[8]; // "FLBMMCK1"
    uint32_t version, lat, ns, parity;
    int32_t nx, ny, nz, pad;
    int64_t step;
    uint64_t seed, payload_bytes, payload_hash;
    double tau[flbm::kMaxSpecies], kT, G[flbm::kMaxSpecies][flbm::kMaxSpecies], rho0[flbm::kMaxSpecies], lam_d;
};
} // namespace

flbm_status flbm_mcheckpoint(flbm_mctx *c, void *buf, size_t *bytes)
{
    if (!c || !bytes) return FLBM_EINVAL;
    const size_t payload = pop_elems(c) * sizeof(float);
    const size_t need = sizeof(MCkptHeader) + payload;
    if (!buf) {
        *bytes = need;
        return FLBM_OK;
    }
    if (*bytes < need) return mfail(c, FLBM_EINVAL, "checkpoint buffer too small: need %zu bytes", need);
    flbm_status st = check_ready(c);
    if (st != FLBM_OK) return st;
    st = sync_and_check(c);
    if (st != FLBM_OK) return st;
    MCkptHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, "FLBMMCK1", 8);
    h.version = 1;
    h.lat = (uint32_t)c->lat;
    h.ns = (uint32_t)c->ns;
    h.parity = (uint32_t)layout_parity(c);
    h.nx = c->nx;
    h.ny = c->ny;
    h.nz = c->nz;
    h.step = c->step;
    h.seed = c->seed;
    std::memcpy(h.tau, c->tau, sizeof(h.tau));
    h.kT = c->kT;
    std::memcpy(h.G, c->G, sizeof(h.G));
    std::memcpy(h.rho0, c->rho0, sizeof(h.rho0));
    h.lam_d = c->lam_d;
    h.payload_bytes = payload;
    unsigned char *dst = static_cast<unsigned char *>(buf);
    MCUDA(c, cudaMemcpy(dst + sizeof(MCkptHeader), cur_pop(c), payload, cudaMemcpyDeviceToHost), "D2H checkpoint");
    h.payload_hash = flbm::host::fnv1a(dst + sizeof(MCkptHeader), payload);
    std::memcpy(dst, &h, sizeof(h));
    *bytes = need;
    return FLBM_OK;
}

flbm_status flbm_mrestore(flbm_mctx *c, const void *buf, size_t bytes)
{
    if (!c || !buf) return FLBM_EINVAL;
    if (bytes < sizeof(MCkptHeader)) return mfail(c, FLBM_EINVAL, "checkpoint image too small");
    MCkptHeader h;
    std::memcpy(&h, buf, sizeof(h));
    if (std::memcmp(h.magic, "FLBMMCK1", 8) != 0 || h.version != 1)
        return mfail(c, FLBM_EINVAL, "not an N-species checkpoint image");
    if ((int)h.lat != c->lat || (int)h.ns != c->ns || h.nx != c->nx || h.ny != c->ny || h.nz != c->nz)
        return mfail(c, FLBM_EINVAL, "checkpoint lattice, species count or box differs from this context");
    const size_t payload = pop_elems(c) * sizeof(float);
    if (h.payload_bytes != payload || bytes < sizeof(MCkptHeader) + payload || h.parity > 1)
        return mfail(c, FLBM_EINVAL, "checkpoint image truncated");
    if (two_arrays(c) && h.parity != 0)
        return mfail(c, FLBM_EINVAL, "an in-place image in the swapped layout restores into an in-place context only");
    const unsigned char *src = static_cast<const unsigned char *>(buf) + sizeof(MCkptHeader);
    if (flbm::host::fnv1a(src, payload) != h.payload_hash)
        return mfail(c, FLBM_EINVAL, "checkpoint image corrupt (hash mismatch)");
    flbm_status st = ensure_buffers(c);
    if (st != FLBM_OK) return st;
    MCUDA(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    MCUDA(c, cudaMemcpy(c->pop, src, payload, cudaMemcpyHostToDevice), "H2D checkpoint");
    MCUDA(c, cudaMemset(c->d_status, 0, sizeof(unsigned)), "status reset");
    std::memcpy(c->tau, h.tau, sizeof(h.tau));
    c->kT = h.kT;
    std::memcpy(c->G, h.G, sizeof(h.G));
    std::memcpy(c->rho0, h.rho0, sizeof(h.rho0));
    c->lam_d = h.lam_d;
    c->seed = h.seed;
    c->step = h.step;
    c->parity = (int)h.parity;
    c->faulted = false;
    c->initialised = true;
    drop_graphs(c); // captured steps hold the old parameters by value
    return FLBM_OK;
}

const char *flbm_mlast_error(const flbm_mctx *c) { return c ? c->err : kNoError; }

void flbm_mdestroy(flbm_mctx *c)
{
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    cudaFree(c->pop);
    cudaFree(c->drho);
    cudaFree(c->d_mom);
    cudaFree(c->d_status);
    drop_graphs(c);
    cudaFree(c->d_gstep);
    cudaFree(c->d_obs);
    cudaFree(c->d_partials);
    cudaFree(c->d_sf_prof);
    for (int a = 0; a < 3; a++) cudaFree(c->d_sf_acc[a]);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

} // extern "C"
