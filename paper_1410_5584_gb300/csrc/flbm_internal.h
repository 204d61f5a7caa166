// flbm_internal.h -- shared definitions of the CUDA library (not installed).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>

#include "flbm.h"

namespace flbm {

constexpr int kMaxQ = 19;
constexpr int kSiteBlockMax = 128; // largest thread block of the density and collide kernels

// Everything one step kernel needs, passed by value (kernel parameter space).
struct StepParams {
    int nx, ny, nz;
    int N;                     // nx * ny * nz  (< 2^31)
    int y0, z0, yn, zn;        // rows [y0, y0 + yn) and planes [z0, z0 + zn) a density or collide
                               // launch covers (one slab of the overlap schedule); 0, 0, ny, nz = all
    int block_x, block_y;      // thread-block shape of the density and collide launches (x by y sites)
    float G;                   // inter-species coupling, Eq. FORCESTRUCTURE
    float lam_d;               // common momentum rate lambdabar_d of both species
    float hlam_d;              // 1 - lambdabar_d / 2  (Eq. forcerenorm)
    // Non-conserved modes a > D of species s, relaxed as in Eq. algorithm with
    // 1/N_a folded in: m*_a / N_a = cm m_a + ceq m^eq_a + cphi Phi_a + cxi sqrt(rho^s) g_a
    float cm[2][kMaxQ];        // (1 - lambdabar_a) / N_a
    float ceq[2][kMaxQ];       // lambdabar_a / N_a
    float cphi[2][kMaxQ];      // (1 - lambdabar_a / 2) / N_a
    float cxi[2][kMaxQ];       // sqrt((2 lb_a - lb_a^2) N_a kT / c_s^2) / N_a  (Eq. new-noise)
    float2 pair_eq[kMaxQ];     // (ceq[0][a], ceq[1][a]): the same constants species by species in
    float2 pair_phi[kMaxQ];    // adjacent pairs, for the collide's packed (two-species) arithmetic
    float2 pair_xi[kMaxQ];
    float noise_amp_j;         // sqrt((2 lb_d - lb_d^2) kT); times sqrt(rho rho'/rho_t); 0 = no-sdf
    float rho0[2];             // reference densities: 16-bit deviation base, noise reference
    int noise_ref;             // 1: noise amplitudes from rho0 instead of the local densities
    int force_velocity;        // 0: rho v = jbar + R_j/2 ; 1: v = vbar + a/2
    int ghost_noise;           // 1: non-conserved noise from one Gaussian per population at the
                               // density of the site it streams to (FLBM_OPT_GHOST_NOISE)
    uint32_t key0, key1;       // Philox key (seed low, seed high)
    uint32_t step;             // noise counter word for this step, or its offset from *step_dev
    const unsigned *step_dev;  // NULL, or a device word the counter is read from (CUDA-graph replays)
    int general_collide;       // test hook: 1 keeps the general collide even when every rate is 1
    float *mom;                // NULL, or 2 (D + 1) planes of N floats: m_0 .. m_D of each species,
                               // written by the density pass and read by the full-relaxation collide
                               // in place of the populations (two-array streaming)
};

// One replica of a batch: its step parameters and the offsets of its slices of
// the shared population array (elements) and density field (sites).
struct RepInfo {
    StepParams p;
    unsigned long long pop_off;
    unsigned long long rho_off;
    // site / nx and site / (nx ny) as (site * mul) >> shift, exact for sites < 2^31
    unsigned long long mul_nx, mul_nxy;
    unsigned shift_nx, shift_nxy;
};

// Multiplier and shift that divide every n < 2^31 by d exactly: with
// l = ceil(log2 d), m = floor(2^(31+l) / d) + 1 gives floor(n m / 2^(31+l))
// = floor(n / d) (Granlund and Montgomery, PLDI 1994, Thm. 4.2, N = 31).
inline void exact_divider(unsigned d, unsigned long long &mul, unsigned &shift)
{
    unsigned l = 0;
    while ((1ull << l) < d) l++;
    mul = (1ull << (31 + l)) / d + 1;
    shift = 31 + l;
}

// Device status bits (ORed by kernels, read by the host at sync points).
constexpr unsigned kStatusNonFinite = 1u;
constexpr unsigned kStatusTimeout = 2u;   // a bounded device-side wait gave up

// ---------------------------------------------------------------------------
// Population storage.  Every format stores the deviation delta_i = f_i -
// w_i rho0^s from the reference state, and kernels work on deviations: the
// small non-conserved moments stay free of cancellation, a stored value is
// rounded relative to the deviation rather than to f_i, and no base has to be
// added or subtracted on the device.
// ---------------------------------------------------------------------------
// encode() forms the stored word of a deviation, encode_w() that of the
// deviation w y, and decode() the deviation a load of a word gives; each is a
// fixed sequence of roundings without contraction, so a kernel can know
// exactly what the next step will load.  The base argument (w_i rho0^s) is
// part of the interface for formats that might need it; none does.
// load_pair / store_pair move the two species' words of one slot and site
// (adjacent, species A first: pop_index below) in one access; the _cs forms
// carry the streaming hint (evict first).
struct StoreF32 {
    using T = float;
    __device__ __forceinline__ static T encode(float dev, float) { return dev; }
    __device__ __forceinline__ static T encode_w(float w, float y, float) { return __fmul_rn(w, y); }
    __device__ __forceinline__ static float decode(T v, float) { return v; }
    __device__ __forceinline__ static float load_dev(const T *p, size_t idx, float)
    {
        return __ldg(p + idx);
    }
    __device__ __forceinline__ static void store_dev(T *p, size_t idx, float dev, float)
    {
        p[idx] = dev;
    }
    __device__ __forceinline__ static float2 load_pair(const T *p) { return __ldg(reinterpret_cast<const float2 *>(p)); }
    __device__ __forceinline__ static float2 load_pair_cs(const T *p)
    {
        return __ldcs(reinterpret_cast<const float2 *>(p));
    }
    __device__ __forceinline__ static void store_pair(T *p, T a, T b)
    {
        *reinterpret_cast<float2 *>(p) = make_float2(a, b);
    }
    __device__ __forceinline__ static void store_pair_cs(T *p, T a, T b)
    {
        __stcs(reinterpret_cast<float2 *>(p), make_float2(a, b));
    }
};

// The two 16-bit words of a pair as one 32-bit word, species A in the low half
// (the lower address).
template <class H, class R> struct Pair16 {
    __device__ __forceinline__ static unsigned pack(H a, H b)
    {
        const R ra = a, rb = b;
        return (unsigned)ra.x | ((unsigned)rb.x << 16);
    }
    __device__ __forceinline__ static void unpack(unsigned w, H &a, H &b)
    {
        R ra, rb;
        ra.x = (unsigned short)(w & 0xFFFFu);
        rb.x = (unsigned short)(w >> 16);
        a = H(ra);
        b = H(rb);
    }
};

struct StoreF16 {
    using T = __half;
    using P = Pair16<__half, __half_raw>;
    __device__ __forceinline__ static T encode(float dev, float) { return __float2half_rn(dev); }
    __device__ __forceinline__ static T encode_w(float w, float y, float) { return __float2half_rn(__fmul_rn(w, y)); }
    __device__ __forceinline__ static float decode(T v, float) { return __half2float(v); }
    __device__ __forceinline__ static float load_dev(const T *p, size_t idx, float base)
    {
        return decode(p[idx], base);
    }
    __device__ __forceinline__ static void store_dev(T *p, size_t idx, float dev, float base)
    {
        p[idx] = encode(dev, base);
    }
    __device__ __forceinline__ static float2 unpair(unsigned w)
    {
        T a, b;
        P::unpack(w, a, b);
        return make_float2(decode(a, 0.0f), decode(b, 0.0f));
    }
    __device__ __forceinline__ static float2 load_pair(const T *p) { return unpair(__ldg(reinterpret_cast<const unsigned *>(p))); }
    __device__ __forceinline__ static float2 load_pair_cs(const T *p)
    {
        return unpair(__ldcs(reinterpret_cast<const unsigned *>(p)));
    }
    __device__ __forceinline__ static void store_pair(T *p, T a, T b) { *reinterpret_cast<unsigned *>(p) = P::pack(a, b); }
    __device__ __forceinline__ static void store_pair_cs(T *p, T a, T b)
    {
        __stcs(reinterpret_cast<unsigned *>(p), P::pack(a, b));
    }
};

struct StoreBF16 {
    using T = __nv_bfloat16;
    using P = Pair16<__nv_bfloat16, __nv_bfloat16_raw>;
    __device__ __forceinline__ static T encode(float dev, float) { return __float2bfloat16_rn(dev); }
    __device__ __forceinline__ static T encode_w(float w, float y, float)
    {
        return __float2bfloat16_rn(__fmul_rn(w, y));
    }
    __device__ __forceinline__ static float decode(T v, float) { return __bfloat162float(v); }
    __device__ __forceinline__ static float load_dev(const T *p, size_t idx, float base)
    {
        return decode(p[idx], base);
    }
    __device__ __forceinline__ static void store_dev(T *p, size_t idx, float dev, float base)
    {
        p[idx] = encode(dev, base);
    }
    __device__ __forceinline__ static float2 unpair(unsigned w)
    {
        T a, b;
        P::unpack(w, a, b);
        return make_float2(decode(a, 0.0f), decode(b, 0.0f));
    }
    __device__ __forceinline__ static float2 load_pair(const T *p) { return unpair(__ldg(reinterpret_cast<const unsigned *>(p))); }
    __device__ __forceinline__ static float2 load_pair_cs(const T *p)
    {
        return unpair(__ldcs(reinterpret_cast<const unsigned *>(p)));
    }
    __device__ __forceinline__ static void store_pair(T *p, T a, T b) { *reinterpret_cast<unsigned *>(p) = P::pack(a, b); }
    __device__ __forceinline__ static void store_pair_cs(T *p, T a, T b)
    {
        __stcs(reinterpret_cast<unsigned *>(p), P::pack(a, b));
    }
};

// Population layout of a two-species array: slot j of both species at a site
// sits side by side, word (s, j, site) at index (j N + site) 2 + s, so that one
// vector access moves both species of a slot; slot j's pairs fill the j-th
// 2 N words.
__host__ __device__ __forceinline__ size_t pop_index(int s, int j, size_t site, size_t N)
{
    return ((size_t)j * N + site) * 2 + (size_t)s;
}

inline size_t storage_bytes(int storage) { return storage == FLBM_STORE_F32 ? 4 : 2; }

// ---------------------------------------------------------------------------
// Launchers (defined in the .cu files).  All are asynchronous on `stream` and
// return the launch error.
// ---------------------------------------------------------------------------

// Density pass: (rho_A, rho_B) of each site as interleaved float pairs,
// rho[2 * site + s] = rho0^s + sum_i delta_i^s(site), reading the populations
// according to the in-place streaming parity.
cudaError_t launch_density(int lat, int storage, int parity, const StepParams &p, const void *pop,
                           float *rho, cudaStream_t stream);

// Streaming mode of a collide launch: 0 / 1 = the even / odd in-place step on
// one array; kStreamPush = read one array (natural layout), write the other.
constexpr int kStreamPush = 2;

// Fused force + moment collision + noise + streaming of one step: in place in
// pop (parity 0 or 1), or from pop into pop_out (kStreamPush).
cudaError_t launch_collide(int lat, int storage, int parity, const StepParams &p, void *pop, void *pop_out,
                           const float *rho, unsigned *status, cudaStream_t stream);

// One whole step (densities and collision) as one persistent launch whose
// work items are ordered so the densities' population reads are reused from
// L2 by the collision.  counters: (number of slices) unsigned words of
// scratch, reset by the launcher.  wait_ms bounds each dependency wait; stall
// (test hook) makes every wait run out.
cudaError_t launch_step_fused(int lat, int storage, int parity, const StepParams &p, void *pop, float *rho,
                              unsigned *status, unsigned *counters, double wait_ms, int stall, int lag,
                              cudaStream_t stream);
inline int pipeline_slices(int lat, int ny, int nz) { return lat == FLBM_D2Q9 ? ny : nz; }

// One whole two-array step as one persistent launch: the densities (and, mom,
// the moments m_0 .. m_D of a full-relaxation step) of each slice go through
// a ring of slice slots that stays in L2, so that the populations cross HBM
// once each way.  pipe_geometry gives the lag, the ring's slot count (0 when
// the box has too few slices; lag_opt >= 1 overrides the lag, which any
// value >= 1 keeps correct), the ring's size in floats and the number of
// counter words (two per slice and row in 3D, per slice in 2D), which the
// launcher resets.  wait_ms bounds each dependency
// wait; stall (test hook) makes every wait run out.
cudaError_t pipe_geometry(int lat, int storage, const StepParams &p, bool mom, int lag_opt, int *lag, int *ring_slots,
                          size_t *ring_floats, size_t *counters);
cudaError_t launch_step_pipe(int lat, int storage, const StepParams &p, const void *pop, void *pop_out, float *ring,
                             unsigned *counters, int ring_slots, int lag, bool mom, unsigned *status, double wait_ms,
                             int stall, cudaStream_t stream);

// One step of every replica of a batch (density then collide over the tile
// work list: tiles[t] = (replica, first site of 128)); the noise counter of the
// step is *step_base + k.  full: every replica relaxes each non-conserved
// mode with rate 1 (the collide skips their projections).  parity 0 / 1: in
// place in pop; kStreamPush: read pop, write pop_out.
cudaError_t launch_batch_step(int lat, int storage, int parity, const RepInfo *reps, const int2 *tiles, int ntiles,
                              void *pop, void *pop_out, float *rho, unsigned *status, const unsigned *step_base,
                              unsigned k, bool full, cudaStream_t stream);

// The tiled two-array step of a 2D box: one launch; each thread block forms the
// densities of a kTileX x tiled_step_rows(lat) tile and of the one-site ring
// around it in shared memory, then collides the tile, reading pop and writing
// pop_out.  cudaErrorNotSupported for D3Q19.  The batch form steps the work
// list tiles[t] = (replica, x0, y0, unused) of every replica.
cudaError_t launch_step_tiled(int lat, int storage, const StepParams &p, const void *pop, void *pop_out,
                              unsigned *status, cudaStream_t stream);
cudaError_t launch_batch_step_tiled(int lat, int storage, const RepInfo *reps, const int4 *tiles, int ntiles,
                                    const void *pop, void *pop_out, unsigned *status, const unsigned *step_base,
                                    unsigned k, bool full, cudaStream_t stream);
constexpr int kTiledStepX = 32;   // tile width of the tiled step (sites along x)
int tiled_step_rows(int lat);     // tile height (rows), 0 when the lattice has no tiled step
// *p += v and *p = v on the device (one thread), for the batch step counter.
cudaError_t launch_add_u32(unsigned *p, unsigned v, cudaStream_t stream);
cudaError_t launch_set_u32(unsigned *p, unsigned v, cudaStream_t stream);

// Per-site observables in double: rho_a, rho_b, u (D planes), any may be NULL,
// plus per-block FP64 partial totals [nblocks][5] into `partials`; returns the
// block count in *nblocks.  Needs the density field of the current state.
cudaError_t launch_observables(int lat, int storage, int parity, const StepParams &p,
                               const void *pop, const float *rho, double *rho_a, double *rho_b,
                               double *u, double *partials, int *nblocks, cudaStream_t stream);

// Density fluctuation fields for the full-wavevector structure factor:
// z[site] = (rho_A - rho0_A, rho_B - rho0_B) in float, per-block FP64 partial
// sums [nblocks][2] into `partials`; the block count goes to *nblocks.
cudaError_t launch_sfk_fields(int lat, int storage, int parity, const StepParams &p, const void *pop, float2 *z,
                              double *partials, int *nblocks, cudaStream_t stream);

// Fixed-order sum of [nblocks][5] partials into out[5].
cudaError_t launch_sum_partials(const double *partials, int nblocks, double *out,
                                cudaStream_t stream);

// Structure-factor snapshot: profiles of (rho_a, rho_b, u_0..u_{D-1}) along
// `axis` (per-site doubles in `obs`, component-major), their DFT at
// k_m = 2 pi m / n_axis, m = 1..n_axis/2, accumulated into acc[4][n_axis/2].
cudaError_t launch_sf_accumulate(int D, int nx, int ny, int nz, int axis, const double *obs,
                                 double *profile, double *acc, cudaStream_t stream);

// Rest-state populations from a float density field (two planes of N: all of
// species A, then all of species B).
cudaError_t launch_init_rest(int lat, int storage, const StepParams &p, const float *rho_in,
                             void *pop, cudaStream_t stream);

// Natural-layout gather of selected sites: out[k][s][i] (doubles).
cudaError_t launch_gather_sites(int lat, int storage, int parity, const StepParams &p,
                                const void *pop, const int64_t *sites, int64_t nsites, double *out,
                                cudaStream_t stream);

// Read-only view of a context for the other translation units of the library.
struct CtxView {
    int lat, storage, D, Q, nx, ny, nz;
    bool batch; // a batch of replicas (one handle over many boxes), not a single box
    int64_t N;
    StepParams params; // parameters of the context's next step
};
bool ctx_view(const flbm_ctx *ctx, CtxView *out);

} // namespace flbm
