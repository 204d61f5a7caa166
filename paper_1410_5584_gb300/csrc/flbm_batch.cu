// flbm_batch.cu -- many independent two-species boxes of uneven size, stepped
// together: one density launch and one collide launch per step over a work list
// of 128-site tiles that spans every replica, or (tiled schedule, 2D, two
// arrays) one launch per step over a work list of 32 x 16 tiles, replayed from
// CUDA graphs of K steps.  Each replica has its own box, parameters and Philox
// key; its site index (and so its noise) is replica-local, exactly as a lone
// context with the same parameters.
//
// The replicas share the population arrays (two by default, or one updated in
// place) and one density field.  Each replica is also exposed as a *view*: a
// context whose buffers are its slices of the shared ones, on which the
// observation calls (flbm_moments, flbm_sf_sample, flbm_structure_factor,
// flbm_get_populations, ...) work unchanged.
#include <cstring>
#include <new>
#include <vector>

#include "flbm_ctx.h"

namespace flbm {

struct BatchState {
    std::vector<flbm_ctx *> views;
    std::vector<int64_t> site_off; // first site of each replica in the density field
    std::vector<int2> tiles_h;     // (replica, first site) per 128-site tile
    std::vector<int4> tiles2_h;    // (replica, x0, y0, 0) per tile of the tiled step
    RepInfo *d_reps = nullptr;
    int2 *d_tiles = nullptr;
    int4 *d_tiles2 = nullptr;
    int schedule = FLBM_SCHEDULE_TWO_KERNELS; // or FLBM_SCHEDULE_TILED
    unsigned *d_step = nullptr; // noise counter of the next step
    bool reps_dirty = true;
    bool step_dirty = true;
    int graph_steps = 16;                          // steps per CUDA graph (0: launch directly)
    cudaGraphExec_t graph[2] = {nullptr, nullptr}; // per parity at the start of the graph
    int graph_len[2] = {0, 0};
    bool internal = false; // batch code is calling the single-box functions on a view
    bool full = false;     // every replica has rate 1 on all non-conserved modes
    float *d_mom = nullptr; // moment planes of all replicas (full relaxation: the moment-fed collide)
};

using namespace host;

namespace {

BatchState *B(const flbm_ctx *c) { return c->batch; }

void drop_graphs(BatchState *b)
{
    for (int p = 0; p < 2; p++) {
        if (b->graph[p]) cudaGraphExecDestroy(b->graph[p]);
        b->graph[p] = nullptr;
        b->graph_len[p] = 0;
    }
}

// the tiled step applies: a 2D lattice with two arrays
bool tiled(const flbm_ctx *c)
{
    return B(c)->schedule == FLBM_SCHEDULE_TILED && c->streaming == FLBM_STREAM_TWO_ARRAYS &&
           tiled_step_rows(c->lat) > 0;
}

// point every view at its slices of the shared buffers and the batch stream
void bind_views(flbm_ctx *c)
{
    BatchState *b = B(c);
    const size_t bytes = storage_bytes(c->storage);
    for (size_t r = 0; r < b->views.size(); r++) {
        flbm_ctx *v = b->views[r];
        v->storage = c->storage;
        v->streaming = c->streaming;
        v->stream = c->stream;
        v->own_stream = false;
        if (c->pop) {
            const size_t off = (size_t)2 * c->Q * (size_t)b->site_off[r] * bytes;
            v->pop = static_cast<unsigned char *>(c->pop) + off;
            v->pop_second = c->streaming == FLBM_STREAM_TWO_ARRAYS
                                ? static_cast<unsigned char *>(c->pop) + array_bytes_of(c) + off
                                : nullptr;
            v->rho = c->rho + 2 * b->site_off[r];
            v->pop_bytes = pop_bytes_of(v);
            v->rho_bytes = rho_bytes_of(v);
            v->own_buffers = false;
        }
    }
}

void sync_views(flbm_ctx *c)
{
    for (flbm_ctx *v : B(c)->views) {
        v->step = c->step;
        v->parity = c->parity;
        v->initialised = c->initialised;
    }
}

flbm_status upload_tables(flbm_ctx *c)
{
    BatchState *b = B(c);
    if (!b->d_tiles) {
        FLBM_CUDA(c, cudaMalloc((void **)&b->d_tiles, b->tiles_h.size() * sizeof(int2)), "cudaMalloc(tiles)");
        FLBM_CUDA(c, cudaMemcpy(b->d_tiles, b->tiles_h.data(), b->tiles_h.size() * sizeof(int2), cudaMemcpyHostToDevice),
                  "H2D tiles");
        // the tiles of the tiled step, where the lattice has one
        const int rows = tiled_step_rows(c->lat);
        if (rows > 0) {
            for (size_t r = 0; r < b->views.size(); r++)
                for (int y0 = 0; y0 < b->views[r]->ny; y0 += rows)
                    for (int x0 = 0; x0 < b->views[r]->nx; x0 += kTiledStepX)
                        b->tiles2_h.push_back(make_int4((int)r, x0, y0, 0));
            FLBM_CUDA(c, cudaMalloc((void **)&b->d_tiles2, b->tiles2_h.size() * sizeof(int4)), "cudaMalloc(tiles)");
            FLBM_CUDA(c, cudaMemcpy(b->d_tiles2, b->tiles2_h.data(), b->tiles2_h.size() * sizeof(int4),
                                    cudaMemcpyHostToDevice),
                      "H2D tiles");
        }
        FLBM_CUDA(c, cudaMalloc((void **)&b->d_reps, b->views.size() * sizeof(RepInfo)), "cudaMalloc(replicas)");
        FLBM_CUDA(c, cudaMalloc((void **)&b->d_step, sizeof(unsigned)), "cudaMalloc(step counter)");
        b->reps_dirty = b->step_dirty = true;
    }
    if (b->reps_dirty) {
        std::vector<RepInfo> h(b->views.size());
        bool full = true;
        for (size_t r = 0; r < h.size(); r++) {
            h[r].p = make_params(b->views[r]);
            h[r].pop_off = (unsigned long long)2 * c->Q * (unsigned long long)b->site_off[r];
            h[r].rho_off = (unsigned long long)b->site_off[r];
            exact_divider((unsigned)h[r].p.nx, h[r].mul_nx, h[r].shift_nx);
            exact_divider((unsigned)(h[r].p.nx * h[r].p.ny), h[r].mul_nxy, h[r].shift_nxy);
            full = full && !h[r].p.general_collide;
            for (int s = 0; s < 2; s++)
                for (int a = c->D + 1; a < c->Q; a++) full = full && h[r].p.cm[s][a] == 0.0f;
        }
        if (full != b->full) {
            // the captured graphs launch the collide instance of the old choice
            drop_graphs(b);
            b->full = full;
        }
        if (full) {
            // each replica's 2 (D + 1) moment planes of its N sites, in site order
            const size_t sites = (size_t)b->site_off.back() + (size_t)b->views.back()->N;
            if (!b->d_mom)
                FLBM_CUDA(c, cudaMalloc((void **)&b->d_mom, (size_t)2 * (c->D + 1) * sites * sizeof(float)),
                          "cudaMalloc(moment planes)");
            for (size_t r = 0; r < h.size(); r++) h[r].p.mom = b->d_mom + (size_t)2 * (c->D + 1) * (size_t)b->site_off[r];
        }
        // the graphs read this array on the device, so it is updated in stream order
        FLBM_CUDA(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
        FLBM_CUDA(c, cudaMemcpy(b->d_reps, h.data(), h.size() * sizeof(RepInfo), cudaMemcpyHostToDevice), "H2D replicas");
        b->reps_dirty = false;
    }
    if (b->step_dirty) {
        FLBM_CUDA(c, launch_set_u32(b->d_step, (unsigned)c->step, c->stream), "step counter launch");
        b->step_dirty = false;
    }
    return FLBM_OK;
}

flbm_status launch_steps(flbm_ctx *c, int parity, int k0, int n)
{
    BatchState *b = B(c);
    const bool two = c->streaming == FLBM_STREAM_TWO_ARRAYS, tl = tiled(c);
    for (int k = 0; k < n; k++) {
        const int par = (parity + k) & 1;
        cudaError_t e;
        if (tl)
            e = launch_batch_step_tiled(c->lat, c->storage, b->d_reps, b->d_tiles2, (int)b->tiles2_h.size(),
                                        cur_pop_at(c, par), next_pop_at(c, par), c->d_status, b->d_step,
                                        (unsigned)(k0 + k), b->full, c->stream);
        else
            e = launch_batch_step(c->lat, c->storage, two ? kStreamPush : par, b->d_reps, b->d_tiles,
                                  (int)b->tiles_h.size(), cur_pop_at(c, par), next_pop_at(c, par), c->rho,
                                  c->d_status, b->d_step, (unsigned)(k0 + k), b->full, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "batched step launch");
    }
    cudaError_t e = launch_add_u32(b->d_step, (unsigned)n, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "step counter launch");
    return FLBM_OK;
}

flbm_status ensure_graph(flbm_ctx *c, int parity)
{
    BatchState *b = B(c);
    if (b->graph[parity] && b->graph_len[parity] == b->graph_steps) return FLBM_OK;
    if (b->graph[parity]) cudaGraphExecDestroy(b->graph[parity]);
    b->graph[parity] = nullptr;
    cudaGraph_t g = nullptr;
    FLBM_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
    flbm_status st = launch_steps(c, parity, 0, b->graph_steps);
    cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (st != FLBM_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&b->graph[parity], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphInstantiate");
    b->graph_len[parity] = b->graph_steps;
    return FLBM_OK;
}

// run a single-box entry point on a view from inside the batch code
template <class F> flbm_status on_view(BatchState *b, flbm_ctx *v, F &&f)
{
    b->internal = true;
    const flbm_status st = f(v);
    b->internal = false;
    return st;
}

struct BatchCkptHeader {
    char magic[8];
    uint32_t version;
    int32_t lat, nrep, storage, parity, sdf, noise_ref, force_velocity;
    int64_t step;
    uint64_t payload_bytes, payload_hash;
};

struct BatchCkptReplica {
    int32_t nx, ny, nz, pad;
    double tau[2], kT, G, rho0[2];
    uint64_t seed;
    double lam[2][kMaxQ];
};

} // namespace

flbm_status batch_set_option(flbm_ctx *c, int key, double v)
{
    BatchState *b = B(c);
    if (key == FLBM_OPT_STORAGE && c->pop) return fail(c, FLBM_ESTATE, "the storage format is fixed once the buffers exist");
    if (key == FLBM_OPT_GHOST_NOISE) return fail(c, FLBM_EUNSUPPORTED, "the population-space noise is for single boxes");
    if (key == FLBM_OPT_STREAMING) {
        if (c->pop) return fail(c, FLBM_ESTATE, "the streaming mode is fixed once the buffers exist");
        if (v != (double)FLBM_STREAM_IN_PLACE && v != (double)FLBM_STREAM_TWO_ARRAYS)
            return fail(c, FLBM_EINVAL, "streaming must be 0 (in place) or 1 (two arrays)");
        c->streaming = (int)v;
        for (flbm_ctx *vw : b->views) vw->streaming = c->streaming;
        drop_graphs(b);
        return FLBM_OK;
    }
    if (key == FLBM_OPT_SCHEDULE) {
        if (v != (double)FLBM_SCHEDULE_TWO_KERNELS && v != (double)FLBM_SCHEDULE_TILED)
            return fail(c, FLBM_EUNSUPPORTED, "a batch runs the two-kernel (1) or the tiled (3) schedule");
        if ((int)v != b->schedule) drop_graphs(b);
        b->schedule = (int)v;
        c->schedule = (int)v;
        return FLBM_OK;
    }
    if (key == FLBM_OPT_GRAPH_STEPS) {
        if (!(v >= 0.0 && v <= 4096.0) || v != (double)(int)v)
            return fail(c, FLBM_EINVAL, "graph steps must be an integer in [0, 4096]");
        b->graph_steps = (int)v;
        drop_graphs(b);
        return FLBM_OK;
    }
    if (key == FLBM_OPT_SF_AXIS || key == FLBM_OPT_KERNEL_TIMING || key == FLBM_OPT_PIPE_LAG || key == FLBM_OPT_WAIT_LIMIT_MS || key == FLBM_OPT_TEST_STALL ||
        key == FLBM_OPT_SLABS || key == FLBM_OPT_BLOCK_X || key == FLBM_OPT_BLOCK_Y) {
        if (key == FLBM_OPT_SF_AXIS) {
            for (flbm_ctx *vw : b->views) {
                const flbm_status st = on_view(b, vw, [&](flbm_ctx *x) { return flbm_set_option(x, key, v); });
                if (st != FLBM_OK) return fail(c, st, "replica: %s", vw->err);
            }
            return FLBM_OK;
        }
        return fail(c, FLBM_EUNSUPPORTED, "option %d does not apply to a batch", key);
    }
    for (flbm_ctx *vw : b->views) {
        const flbm_status st = on_view(b, vw, [&](flbm_ctx *x) { return flbm_set_option(x, key, v); });
        if (st != FLBM_OK) return fail(c, st, "replica: %s", vw->err);
    }
    if (key == FLBM_OPT_STORAGE) c->storage = (int)v;
    if (key == FLBM_OPT_SDF) c->sdf = v != 0.0;
    if (key == FLBM_OPT_NOISE_RHO) c->noise_ref = v != 0.0;
    if (key == FLBM_OPT_FORCE_VELOCITY) c->force_velocity = v != 0.0;
    b->reps_dirty = true;
    return FLBM_OK;
}

int batch_graph_steps(const flbm_ctx *c) { return c->batch->graph_steps; }

flbm_status batch_set_stream(flbm_ctx *c, void *stream)
{
    drop_graphs(B(c));
    bind_views(c);
    (void)stream;
    return FLBM_OK;
}

flbm_status batch_attach_buffers(flbm_ctx *c, void *, size_t, void *, size_t)
{
    drop_graphs(B(c));
    bind_views(c);
    return FLBM_OK;
}

flbm_status batch_init(flbm_ctx *c, const double *rho_a, const double *rho_b)
{
    BatchState *b = B(c);
    if (!c->pop) {
        flbm_status st = ensure_stream(c);
        if (st != FLBM_OK) return st;
        c->pop_bytes = pop_bytes_of(c);
        c->rho_bytes = rho_bytes_of(c);
        cudaError_t e = cudaMalloc(&c->pop, c->pop_bytes);
        if (e != cudaSuccess) {
            c->pop = nullptr;
            return fail(c, FLBM_ENOMEM, "cudaMalloc of %zu population bytes failed", c->pop_bytes);
        }
        e = cudaMalloc((void **)&c->rho, c->rho_bytes);
        if (e != cudaSuccess) {
            cudaFree(c->pop);
            c->pop = nullptr;
            c->rho = nullptr;
            return fail(c, FLBM_ENOMEM, "cudaMalloc of %zu density bytes failed", c->rho_bytes);
        }
        c->own_buffers = true;
        if ((st = ensure_status(c)) != FLBM_OK) return st;
    }
    bind_views(c);
    for (size_t r = 0; r < b->views.size(); r++) {
        const double *ra = rho_a ? rho_a + b->site_off[r] : nullptr;
        const double *rb = rho_b ? rho_b + b->site_off[r] : nullptr;
        const flbm_status st = on_view(b, b->views[r], [&](flbm_ctx *x) { return flbm_init(x, ra, rb); });
        if (st != FLBM_OK) return fail(c, st, "replica %zu: %s", r, b->views[r]->err);
    }
    FLBM_CUDA(c, cudaMemsetAsync(c->d_status, 0, sizeof(unsigned), c->stream), "status reset");
    c->step = 0;
    c->parity = 0;
    c->faulted = c->timed_out = false;
    c->initialised = true;
    b->step_dirty = true;
    sync_views(c);
    return FLBM_OK;
}

flbm_status batch_step(flbm_ctx *c, int64_t n)
{
    BatchState *b = B(c);
    if (!c->initialised) return fail(c, FLBM_ESTATE, "flbm_step before flbm_init");
    flbm_status st = upload_tables(c);
    if (st != FLBM_OK) return st;
    while (n > 0) {
        if (b->graph_steps > 0 && n >= b->graph_steps) {
            if ((st = ensure_graph(c, c->parity)) != FLBM_OK) return st;
            FLBM_CUDA(c, cudaGraphLaunch(b->graph[c->parity], c->stream), "cudaGraphLaunch");
            c->step += b->graph_steps;
            c->parity ^= b->graph_steps & 1;
            n -= b->graph_steps;
        } else {
            const int k = (int)(n < 1024 ? n : 1024);
            if ((st = launch_steps(c, c->parity, 0, k)) != FLBM_OK) return st;
            c->step += k;
            c->parity ^= k & 1;
            n -= k;
        }
    }
    sync_views(c);
    return FLBM_OK;
}

flbm_status batch_moments(flbm_ctx *c, double *rho_a, double *rho_b, double *u, double *cons)
{
    BatchState *b = B(c);
    if (!c->initialised) return fail(c, FLBM_ESTATE, "flbm_moments before flbm_init");
    flbm_status st = sync_and_check(c);
    if (st != FLBM_OK) return st;
    double tot[5] = {0, 0, 0, 0, 0};
    for (size_t r = 0; r < b->views.size(); r++) {
        double one[5];
        const int64_t off = b->site_off[r];
        st = on_view(b, b->views[r], [&](flbm_ctx *x) {
            return flbm_moments(x, rho_a ? rho_a + off : nullptr, rho_b ? rho_b + off : nullptr,
                                u ? u + (int64_t)c->D * off : nullptr, one);
        });
        if (st != FLBM_OK) return fail(c, st, "replica %zu: %s", r, b->views[r]->err);
        for (int k = 0; k < 5; k++) tot[k] += one[k];
    }
    if (cons)
        for (int k = 0; k < 5; k++) cons[k] = tot[k];
    return FLBM_OK;
}

flbm_status batch_sf_sample(flbm_ctx *c)
{
    BatchState *b = B(c);
    if (!c->initialised) return fail(c, FLBM_ESTATE, "flbm_sf_sample before flbm_init");
    flbm_status st = sync_and_check(c);
    if (st != FLBM_OK) return st;
    for (size_t r = 0; r < b->views.size(); r++) {
        st = on_view(b, b->views[r], [&](flbm_ctx *x) { return flbm_sf_sample(x); });
        if (st != FLBM_OK) return fail(c, st, "replica %zu: %s", r, b->views[r]->err);
    }
    return FLBM_OK;
}

flbm_status batch_get_populations(flbm_ctx *c, double *f)
{
    BatchState *b = B(c);
    flbm_status st = sync_and_check(c);
    if (st != FLBM_OK) return st;
    for (size_t r = 0; r < b->views.size(); r++) {
        double *dst = f + (int64_t)2 * c->Q * b->site_off[r];
        st = on_view(b, b->views[r], [&](flbm_ctx *x) { return flbm_get_populations(x, dst); });
        if (st != FLBM_OK) return fail(c, st, "replica %zu: %s", r, b->views[r]->err);
    }
    return FLBM_OK;
}

flbm_status batch_set_populations(flbm_ctx *c, const double *f, int64_t step)
{
    BatchState *b = B(c);
    if (!c->pop) {
        flbm_status st = batch_init(c, nullptr, nullptr); // allocates and binds
        if (st != FLBM_OK) return st;
    }
    for (size_t r = 0; r < b->views.size(); r++) {
        const double *src = f + (int64_t)2 * c->Q * b->site_off[r];
        const flbm_status st = on_view(b, b->views[r], [&](flbm_ctx *x) { return flbm_set_populations(x, src, step); });
        if (st != FLBM_OK) return fail(c, st, "replica %zu: %s", r, b->views[r]->err);
    }
    FLBM_CUDA(c, cudaMemset(c->d_status, 0, sizeof(unsigned)), "status reset");
    c->step = step;
    c->parity = 0;
    c->faulted = c->timed_out = false;
    c->initialised = true;
    b->step_dirty = true;
    sync_views(c);
    return FLBM_OK;
}

flbm_status batch_checkpoint(flbm_ctx *c, void *buf, size_t *bytes)
{
    BatchState *b = B(c);
    const size_t nrep = b->views.size();
    const size_t payload = array_bytes_of(c); // the current array
    const size_t need = sizeof(BatchCkptHeader) + nrep * sizeof(BatchCkptReplica) + payload;
    if (!buf) {
        *bytes = need;
        return FLBM_OK;
    }
    if (*bytes < need) return fail(c, FLBM_EINVAL, "checkpoint buffer too small: need %zu bytes", need);
    if (!c->initialised) return fail(c, FLBM_ESTATE, "nothing to checkpoint before flbm_init");
    flbm_status st = sync_and_check(c);
    if (st != FLBM_OK) return st;
    unsigned char *dst = static_cast<unsigned char *>(buf);
    BatchCkptHeader h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, "FLBMBAT1", 8);
    h.version = 3; // 2: float storage holds deviations f_i - w_i rho0; 3: species side by side
    h.lat = c->lat;
    h.nrep = (int32_t)nrep;
    h.storage = c->storage;
    h.parity = layout_parity(c);
    h.sdf = c->sdf;
    h.noise_ref = c->noise_ref;
    h.force_velocity = c->force_velocity;
    h.step = c->step;
    h.payload_bytes = payload;
    unsigned char *reps = dst + sizeof(h);
    for (size_t r = 0; r < nrep; r++) {
        const flbm_ctx *v = b->views[r];
        BatchCkptReplica q;
        std::memset(&q, 0, sizeof(q));
        q.nx = v->nx;
        q.ny = v->ny;
        q.nz = v->nz;
        std::memcpy(q.tau, v->tau, sizeof(q.tau));
        q.kT = v->kT;
        q.G = v->G;
        std::memcpy(q.rho0, v->rho0, sizeof(q.rho0));
        q.seed = v->seed;
        std::memcpy(q.lam, v->lam, sizeof(q.lam));
        std::memcpy(reps + r * sizeof(q), &q, sizeof(q));
    }
    unsigned char *pl = reps + nrep * sizeof(BatchCkptReplica);
    FLBM_CUDA(c, cudaMemcpy(pl, cur_pop(c), payload, cudaMemcpyDeviceToHost), "D2H checkpoint");
    h.payload_hash = fnv1a(pl, payload);
    std::memcpy(dst, &h, sizeof(h));
    *bytes = need;
    return FLBM_OK;
}

flbm_status batch_restore(flbm_ctx *c, const void *buf, size_t bytes)
{
    BatchState *b = B(c);
    const size_t nrep = b->views.size();
    if (bytes < sizeof(BatchCkptHeader)) return fail(c, FLBM_EINVAL, "checkpoint image too small");
    BatchCkptHeader h;
    std::memcpy(&h, buf, sizeof(h));
    if (std::memcmp(h.magic, "FLBMBAT1", 8) != 0 || h.version != 3) return fail(c, FLBM_EINVAL, "not a batch checkpoint image");
    if (h.lat != c->lat || (size_t)h.nrep != nrep) return fail(c, FLBM_EINVAL, "checkpoint lattice or replica count differs");
    if (c->pop && h.storage != c->storage) return fail(c, FLBM_EINVAL, "checkpoint storage format differs");
    const unsigned char *reps = static_cast<const unsigned char *>(buf) + sizeof(h);
    for (size_t r = 0; r < nrep; r++) {
        BatchCkptReplica q;
        std::memcpy(&q, reps + r * sizeof(q), sizeof(q));
        const flbm_ctx *v = b->views[r];
        if (q.nx != v->nx || q.ny != v->ny || q.nz != v->nz) return fail(c, FLBM_EINVAL, "replica %zu box differs", r);
    }
    const size_t payload = (size_t)2 * c->Q * (size_t)c->N * storage_bytes(h.storage);
    if (h.payload_bytes != payload || bytes < sizeof(h) + nrep * sizeof(BatchCkptReplica) + payload)
        return fail(c, FLBM_EINVAL, "checkpoint image truncated");
    const unsigned char *pl = reps + nrep * sizeof(BatchCkptReplica);
    if (fnv1a(pl, payload) != h.payload_hash) return fail(c, FLBM_EINVAL, "checkpoint image corrupt (hash mismatch)");
    if (c->streaming == FLBM_STREAM_TWO_ARRAYS && h.parity != 0)
        return fail(c, FLBM_EINVAL, "an in-place image in the swapped layout restores into an in-place batch only");
    c->storage = h.storage;
    for (size_t r = 0; r < nrep; r++) {
        BatchCkptReplica q;
        std::memcpy(&q, reps + r * sizeof(q), sizeof(q));
        flbm_ctx *v = b->views[r];
        std::memcpy(v->tau, q.tau, sizeof(q.tau));
        v->kT = q.kT;
        v->G = q.G;
        std::memcpy(v->rho0, q.rho0, sizeof(q.rho0));
        v->seed = q.seed;
        std::memcpy(v->lam, q.lam, sizeof(q.lam));
        v->sdf = h.sdf;
        v->noise_ref = h.noise_ref;
        v->force_velocity = h.force_velocity;
        v->storage = h.storage;
    }
    c->sdf = h.sdf;
    c->noise_ref = h.noise_ref;
    c->force_velocity = h.force_velocity;
    if (!c->pop) {
        flbm_status st = batch_init(c, nullptr, nullptr);
        if (st != FLBM_OK) return st;
    }
    FLBM_CUDA(c, cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    FLBM_CUDA(c, cudaMemcpy(c->pop, pl, payload, cudaMemcpyHostToDevice), "H2D checkpoint");
    FLBM_CUDA(c, cudaMemset(c->d_status, 0, sizeof(unsigned)), "status reset");
    c->step = h.step;
    c->parity = h.parity;
    c->faulted = c->timed_out = false;
    c->initialised = true;
    b->reps_dirty = b->step_dirty = true;
    sync_views(c);
    return FLBM_OK;
}

void batch_destroy(flbm_ctx *c)
{
    BatchState *b = B(c);
    if (!b) return;
    drop_graphs(b);
    if (b->d_reps) cudaFree(b->d_reps);
    if (b->d_tiles) cudaFree(b->d_tiles);
    if (b->d_tiles2) cudaFree(b->d_tiles2);
    if (b->d_step) cudaFree(b->d_step);
    if (b->d_mom) cudaFree(b->d_mom);
    for (flbm_ctx *v : b->views) {
        v->batch = nullptr;
        v->is_view = false;
        flbm_destroy(v);
    }
    delete b;
    c->batch = nullptr;
}

bool view_call_allowed(const flbm_ctx *c)
{
    // a view may be observed but not stepped, initialised or restored, except by
    // its batch
    return !c->is_view || (c->batch && c->batch->internal);
}

} // namespace flbm

extern "C" {

flbm_status flbm_batch_create(flbm_lattice lat, int nrep, const flbm_rep_params *p, flbm_ctx **out)
{
    using namespace flbm;
    if (!out) return FLBM_EINVAL;
    *out = nullptr;
    if (nrep < 1 || !p) return FLBM_EINVAL;
    flbm_ctx *c = new (std::nothrow) flbm_ctx();
    BatchState *b = new (std::nothrow) BatchState();
    if (!c || !b) {
        delete c;
        delete b;
        return FLBM_ENOMEM;
    }
    c->batch = b;
    c->lat = lat;
    c->D = lat == FLBM_D2Q9 ? 2 : 3;
    c->Q = lat == FLBM_D2Q9 ? 9 : 19;
    int64_t total = 0;
    for (int r = 0; r < nrep; r++) {
        flbm_ctx *v = nullptr;
        const flbm_status st = flbm_create(lat, p[r].nx, p[r].ny, lat == FLBM_D2Q9 ? 1 : p[r].nz, p[r].tau_a,
                                           p[r].tau_b, p[r].kT, p[r].G, p[r].seed, &v);
        if (st != FLBM_OK || !(p[r].rho0_a > 0.0) || !(p[r].rho0_b > 0.0)) {
            if (v) flbm_destroy(v);
            flbm_destroy(c);
            return FLBM_EINVAL;
        }
        v->rho0[0] = p[r].rho0_a;
        v->rho0[1] = p[r].rho0_b;
        v->is_view = true;
        v->batch = b;
        b->views.push_back(v);
        b->site_off.push_back(total);
        for (int64_t s = 0; s < v->N; s += 128) b->tiles_h.push_back(make_int2(r, (int)s));
        total += v->N;
    }
    if (total >= (int64_t(1) << 31)) {
        flbm_destroy(c);
        return FLBM_EINVAL;
    }
    c->N = total;
    c->nx = (int)total;
    c->ny = c->nz = 1;
    *out = c;
    return FLBM_OK;
}

flbm_status flbm_batch_replica(flbm_ctx *c, int rep, flbm_ctx **view)
{
    if (!c || !view) return FLBM_EINVAL;
    *view = nullptr;
    if (!c->batch || c->is_view) return flbm::host::fail(c, FLBM_EINVAL, "not a batch context");
    if (rep < 0 || rep >= (int)c->batch->views.size()) return flbm::host::fail(c, FLBM_EINVAL, "replica %d out of range", rep);
    *view = c->batch->views[rep];
    return FLBM_OK;
}

flbm_status flbm_batch_size(const flbm_ctx *c, int *nrep, int64_t *sites)
{
    if (!c || !c->batch || c->is_view) return FLBM_EINVAL;
    if (nrep) *nrep = (int)c->batch->views.size();
    if (sites) *sites = c->N;
    return FLBM_OK;
}

} // extern "C"
