// flbm_ctx.h -- the context behind the opaque flbm_ctx handle, and the host
// helpers the C-ABI translation units share (not installed).
#pragma once
#include <cstdarg>
#include <vector>

#include "flbm_internal.h"

namespace flbm {
struct BatchState; // flbm_batch.cu
}

struct flbm_ctx {
    // problem
    int lat = 0, D = 2, Q = 9;
    int nx = 0, ny = 0, nz = 1;
    int64_t N = 0;
    double tau[2] = {1.0, 1.0}, kT = 0.0, G = 0.0;
    uint64_t seed = 0;
    // options
    double lam[2][flbm::kMaxQ] = {};
    int storage = FLBM_STORE_F32, sdf = 1, noise_ref = 0, force_velocity = 0, sf_axis = 0;
    int ghost_noise = 0; // FLBM_OPT_GHOST_NOISE
    int direct_host = 1; // FLBM_OPT_DIRECT_HOST
    int schedule = FLBM_SCHEDULE_TWO_KERNELS;
    int streaming = FLBM_STREAM_TWO_ARRAYS; // FLBM_OPT_STREAMING
    double wait_limit_ms = 2000.0;
    int pipe_lag = 0;
    int test_stall = 0;
    int test_general = 0; // FLBM_OPT_TEST_GENERAL_COLLIDE
    // CUDA graphs of graph_steps two-kernel steps, one per starting parity
    // (FLBM_OPT_GRAPH_STEPS on a single box; 0 = launch each step directly)
    int graph_steps = 0;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    unsigned *d_gstep = nullptr; // noise counter at the start of a graph replay
    float *d_mom = nullptr;      // moment planes of the full-relaxation two-array step (StepParams::mom)
    // pipelined two-array step (the fused schedule with two arrays): its ring
    // of slice slots (L2-resident scratch) and two counters per slice
    float *d_ring = nullptr;
    size_t ring_floats = 0;
    unsigned *d_ring_cnt = nullptr;
    double rho0[2] = {1.0, 1.0};
    // state
    int64_t step = 0;
    int parity = 0; // in place: 0 natural layout, 1 swapped layout (after an odd number of steps);
                    // two arrays: which of the two holds the current (natural-layout) state
    bool initialised = false;
    bool faulted = false;
    bool timed_out = false;
    // device buffers
    void *pop = nullptr;
    size_t pop_bytes = 0;
    void *pop_second = nullptr; // a batch replica view with two arrays: its slice of the second array
                                // (NULL: the second array follows the first in pop)
    float *rho = nullptr;
    size_t rho_bytes = 0;
    bool own_buffers = false;
    unsigned *d_status = nullptr;
    unsigned *d_pipe = nullptr;   // fused-step counters: next item + one per slice
    double *d_obs = nullptr;      // (2 + D) * N doubles: rho_a, rho_b, u
    double *d_partials = nullptr; // per-block totals
    size_t partials_cap = 0;
    double *d_cons = nullptr;     // 5 doubles
    double *d_sf = nullptr;       // 4 * n_axis/2 accumulators
    double *d_profile = nullptr;  // (2 + D) * n_axis
    int64_t sf_count = 0;
    // full-wavevector structure factors (flbm_sfk_*)
    float2 *d_sfk_z = nullptr;         // N complex: packed fluctuation field, transformed in place
    double *d_sfk_acc = nullptr;       // 3 N: sums of |A|^2, Re(A conj B), |B|^2
    double *d_sfk_mean = nullptr;      // the two fields' means of the current snapshot
    float2 *d_sfk_tw[3] = {nullptr, nullptr, nullptr}; // twiddles per axis
    int sfk_tw_n[3] = {0, 0, 0};
    int64_t sfk_count = 0;
    // capillary spectrum of a stripe (flbm_cap_*)
    float2 *d_cap_z = nullptr;   // N: rho_A - rho0_A (and rho_B) of the snapshot
    double *d_cap_h = nullptr;   // heights [2][ny], spectrum sums [ny/2], mean-height sums [2], bulk [2]
    double2 *d_cap_tw = nullptr; // (cos, -sin)(2 pi j / ny)
    int64_t cap_count = 0;
    int cap_xl = 0, cap_xg = 0;
    float *h_stage = nullptr;     // pinned staging, 2 * N floats
    unsigned long long *d_bad = nullptr; // first invalid initial density of each species (direct reads)
    // per-kernel event timing (FLBM_OPT_KERNEL_TIMING)
    struct TimingMark {
        size_t start, end; // ev_pool indices
        int kernel;        // 0 density (or counter reset), 1 collide (or fused step)
    };
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::vector<TimingMark> marks;
    // launch shape of the density and collide kernels
    int block_x = 128, block_y = 1;
    // overlap schedule
    int slabs = 8;
    cudaStream_t stream_d = nullptr;  // density stream, higher priority than the context's
    std::vector<cudaEvent_t> ev_dep;  // [0, K): after collide slab j; [K, 2K): after density slab j
    double kernel_ms[2] = {0.0, 0.0};
    int64_t kernel_launches[2] = {0, 0};
    // stream
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    char err[512] = {0};
    // batch of independent replicas (flbm_batch_create), or a view of one replica
    flbm::BatchState *batch = nullptr;
    bool is_view = false;
};

#define FLBM_CUDA(ctx, call, what)                                               \
    do {                                                                         \
        cudaError_t e_ = (call);                                                 \
        if (e_ != cudaSuccess) return flbm::host::cuda_fail((ctx), e_, what);   \
    } while (0)

namespace flbm {
namespace host {
flbm_status fail(flbm_ctx *c, flbm_status st, const char *fmt, ...);
flbm_status cuda_fail(flbm_ctx *c, cudaError_t e, const char *what);
StepParams make_params(const flbm_ctx *c);
flbm_status ensure_stream(flbm_ctx *c);
flbm_status ensure_status(flbm_ctx *c);
flbm_status ensure_stage(flbm_ctx *c);
flbm_status sync_and_check(flbm_ctx *c);
flbm_status ensure_obs(flbm_ctx *c);
flbm_status density_now(flbm_ctx *c, const StepParams &p);
size_t pop_bytes_of(const flbm_ctx *c);
// Where the current state is and how it is laid out: with two arrays the
// current one (natural layout, read as parity 0); in place the one array in
// the layout of its parity.  next_pop: where a two-array step writes.
size_t array_bytes_of(const flbm_ctx *c);
void *cur_pop(const flbm_ctx *c);
void *next_pop(const flbm_ctx *c);
void *cur_pop_at(const flbm_ctx *c, int parity); // the same for an explicit parity
void *next_pop_at(const flbm_ctx *c, int parity);
int layout_parity(const flbm_ctx *c);
void drop_step_graphs(flbm_ctx *c); // after any change of what a step launches
size_t rho_bytes_of(const flbm_ctx *c);
uint64_t fnv1a(const unsigned char *p, size_t n);
} // namespace host

// Float densities [2][n] (species A, then B) from the caller's double arrays
// read straight from host memory (a device that shares the host's page
// tables; NULL: uniform rho0), with the smallest index of a value that is not
// positive and finite per species atomically lowered into bad[0..1]
// (flbm_obs.cu).
cudaError_t launch_densities_from_host(const double *rho_a, const double *rho_b, double rho0_a, double rho0_b,
                                       int64_t n, float *out, unsigned long long *bad, cudaStream_t stream);

// batch entry points used by the C-ABI functions when ctx->batch is set
flbm_status batch_set_option(flbm_ctx *c, int key, double v);
flbm_status batch_set_stream(flbm_ctx *c, void *stream);
flbm_status batch_attach_buffers(flbm_ctx *c, void *pop, size_t pop_bytes, void *rho, size_t rho_bytes);
flbm_status batch_init(flbm_ctx *c, const double *rho_a, const double *rho_b);
flbm_status batch_step(flbm_ctx *c, int64_t n);
flbm_status batch_moments(flbm_ctx *c, double *rho_a, double *rho_b, double *u, double *cons);
flbm_status batch_sf_sample(flbm_ctx *c);
flbm_status batch_get_populations(flbm_ctx *c, double *f);
flbm_status batch_set_populations(flbm_ctx *c, const double *f, int64_t step);
flbm_status batch_checkpoint(flbm_ctx *c, void *buf, size_t *bytes);
flbm_status batch_restore(flbm_ctx *c, const void *buf, size_t bytes);
void batch_destroy(flbm_ctx *c);
int batch_graph_steps(const flbm_ctx *c);
void free_sfk(flbm_ctx *c); // flbm_sfk.cu
void free_cap(flbm_ctx *c); // flbm_capillary.cu
bool view_call_allowed(const flbm_ctx *c); // false for mutating calls on a replica view
inline bool is_batch(const flbm_ctx *c) { return c->batch && !c->is_view; }
} // namespace flbm
