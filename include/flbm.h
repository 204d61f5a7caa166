/*
 * flbm.h -- C-ABI of the GB300 (sm_103a) library for the fluctuating two-species
 * lattice Boltzmann update of Belardinelli, Sbragaglia, Biferale, Gross and
 * Varnik, "Fluctuating multicomponent lattice Boltzmann model" (arXiv 1410.5584).
 *
 * The update is the paper's lattice algorithm (Sec. V B, Eqs. algorithm and
 * lattice finalstep), applied per site r and step n to both species:
 *   fbar_i(r + c_i, n+1) = fbar_i(r, n) + w_i sum_a T_ai R_a(r, n) / N_a,
 *   R_a = lambdabar_a (m^eq_a(rho, vbar_b + a_b/2) - mbar_a) + Phibar_a + xibar_a,
 * with the Shan-Chen inter-species force a(r) = -G sum_i w_i rho'(r + c_i) c_i
 * (Sec. VI, Eq. FORCESTRUCTURE), the D2Q9 basis of Table I, and Gaussian noise
 * with the covariances of Eq. new-noise (opposite on the two species' momenta,
 * local densities, Sec. VII).
 *
 * Conventions for every call:
 *   - Every call returns an flbm_status and never aborts or throws.  After an
 *     error, flbm_last_error() gives a one-line reason.
 *   - Lattice units: Delta t = Delta r = 1, k_B = 1, c_s^2 = 1/3.  The box is
 *     fully periodic.
 *   - Site index: site = (z * ny + y) * nx + x, x fastest.  Host arrays of one
 *     value per site are row-major [z][y][x], caller-owned, and are read or
 *     written only during the call.
 *   - Populations, where exposed, are in the natural layout
 *     [species][i][z][y][x]; species 0 = A, 1 = B; i indexes the velocity set:
 *       D2Q9 : (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1)
 *       D3Q19: (0,0,0) (1,0,0) (-1,0,0) (0,1,0) (0,-1,0) (0,0,1) (0,0,-1)
 *              (1,1,0) (-1,-1,0) (1,-1,0) (-1,1,0) (1,0,1) (-1,0,-1) (1,0,-1)
 *              (-1,0,1) (0,1,1) (0,-1,-1) (0,1,-1) (0,-1,1)
 *   - flbm_step is asynchronous on the context's stream.  Faults detected on
 *     the device (a density that is not positive and finite) are reported by
 *     the next synchronising call: flbm_sync, flbm_moments, flbm_sf_sample,
 *     flbm_structure_factor, flbm_get_populations, flbm_checkpoint.
 *   - A context is not thread-safe; distinct contexts are independent.
 */
#ifndef FLBM_H
#define FLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct flbm_ctx flbm_ctx; /* opaque; created and freed by the library */

typedef enum {
    FLBM_OK = 0,
    FLBM_EINVAL = 1,       /* an argument is out of range or inconsistent */
    FLBM_ENOMEM = 2,       /* a host or device allocation failed */
    FLBM_ECUDA = 3,        /* a CUDA runtime call failed (reason in flbm_last_error) */
    FLBM_ENONFINITE = 4,   /* a density became non-positive or non-finite on the device */
    FLBM_ETIMEOUT = 5,     /* a bounded device-side wait gave up; the state is not valid */
    FLBM_EUNSUPPORTED = 6, /* valid request that this library does not support */
    FLBM_ESTATE = 7        /* call out of order (e.g. step before init) */
} flbm_status;

typedef enum { FLBM_D2Q9 = 0, FLBM_D3Q19 = 1 } flbm_lattice;

/* Population storage formats (option FLBM_OPT_STORAGE). */
typedef enum {
    FLBM_STORE_F32 = 0,  /* stored as float deviations f_i - w_i * rho0^s; collided in float */
    FLBM_STORE_F16 = 1,  /* stored as half deviations from w_i * rho0^s; collided in float */
    FLBM_STORE_BF16 = 2  /* stored as bfloat16 deviations from w_i * rho0^s; collided in float */
} flbm_storage;

/* How flbm_step runs one update (option FLBM_OPT_SCHEDULE).  All compute the
 * same update and each is deterministic; the two-kernel and overlap schedules
 * give bitwise identical results, the fused one agrees to rounding. */
typedef enum {
    FLBM_SCHEDULE_FUSED = 0,       /* one persistent launch per step; density and collision work items
                                      ordered so the populations read for the densities are reused from
                                      L2 by the collision (one HBM pass each way).  Slower on GB300 while
                                      the collision is instruction-bound */
    FLBM_SCHEDULE_TWO_KERNELS = 1, /* a density kernel over the box, then the collide kernel */
    FLBM_SCHEDULE_OVERLAP = 2,     /* the box cut into FLBM_OPT_SLABS slabs along its last axis (z;
                                      y for D2Q9): the collide kernel runs slab by slab on the
                                      context's stream while the next step's density kernel runs, on a
                                      second stream of higher priority, on every slab whose neighbours
                                      have been collided, so the memory-bound density pass overlaps the
                                      instruction-bound collision.  Ordered by CUDA events only.  Boxes
                                      with fewer than 3 planes (rows) run the two-kernel schedule.
                                      Either streaming mode */
    FLBM_SCHEDULE_TILED = 3        /* D2Q9 with two arrays: one launch per step.  Each thread block owns
                                      a 32 x 16 tile (32 x 4 on a box of at most 512 tiles of 32 x 16,
                                      so that more blocks share it); it forms the densities of the tile and of the
                                      one-site ring around it (the force stencil, Eq. FORCESTRUCTURE)
                                      in shared memory, and at full relaxation the tile's m_0 .. m_D,
                                      then collides the tile and pushes f* into the other array.  No
                                      density field goes through HBM; bitwise the two-kernel update.
                                      D3Q19 or in place: runs the two-kernel schedule.  The one
                                      schedule besides the two-kernel one that a batch accepts */
} flbm_schedule;

/* How populations stream (option FLBM_OPT_STREAMING). */
typedef enum {
    FLBM_STREAM_IN_PLACE = 0,   /* one population array updated in place ("AA" pattern: even steps swap
                                   each site's slots, odd steps read and write the neighbours'); half the
                                   memory of two arrays */
    FLBM_STREAM_TWO_ARRAYS = 1  /* default: two population arrays; a step reads each site's populations
                                   from one (natural layout) and writes f*_i to x + c_i in the other.  On
                                   GB300 a pure copy with these reads and writes runs at the HBM copy rate,
                                   the in-place pattern at half of it or less; the collide gains a few
                                   per cent.  Runs every schedule (the fused one as a pipelined step;
                                   the tiled one on D2Q9) */
} flbm_streaming;

/* Option keys for flbm_set_option. */
enum {
    FLBM_OPT_STORAGE = 1,        /* flbm_storage; only before flbm_init / flbm_attach_buffers */
    FLBM_OPT_LAMBDA_D = 2,       /* common momentum rate lambdabar_d, 0 < value < 2 (Sec. III,
                                    Eq. diffusionrelaxation); default 1/tau if tau_A = tau_B,
                                    else 2/(tau_A + tau_B) */
    FLBM_OPT_SDF = 3,            /* 1 (default): noise on the species momenta ("sdf");
                                    0: switched off ("no-sdf" control of Sec. VI A) */
    FLBM_OPT_RHO0_A = 4,         /* reference density of A, default 1: the uniform init value and
                                    the base of the stored deviations f_i - w_i rho0 (all storage
                                    formats); fixed once the buffers exist.  Set it near the mean
                                    density: the deviations are then small, their rounding is
                                    small, and the total mass only random-walks at the rounding
                                    of one population per site and step.  Far from it (for
                                    instance rho = rho0 / 2) the deviations are as large as the
                                    populations and the walk is correspondingly wider. */
    FLBM_OPT_RHO0_B = 5,         /* same for B */
    FLBM_OPT_NOISE_RHO = 7,      /* 0 (default): local densities in the noise amplitudes
                                    (Sec. VII); 1: the reference densities rho0 (Eq. new-noise,
                                    homogeneous form) */
    FLBM_OPT_FORCE_VELOCITY = 8, /* species velocity inside Phi: 0 (default) rho v = jbar + R_j/2
                                    (Eq. alg-mom, equivalent to Eq. 2system); 1: v = vbar + a/2 */
    FLBM_OPT_SF_AXIS = 9,        /* axis of the structure-factor wavevector (0 x, 1 y, 2 z);
                                    changing it clears the accumulators; default 0 */
    FLBM_OPT_KERNEL_TIMING = 10, /* 1: flbm_step records CUDA events around each kernel on the
                                    context's stream (see flbm_kernel_times); 0 (default): off.
                                    Switching it clears the accumulated times */
    FLBM_OPT_SCHEDULE = 11,      /* flbm_schedule: how flbm_step runs one step (same results) */
    FLBM_OPT_WAIT_LIMIT_MS = 12, /* fused schedule: time after which a device-side dependency wait
                                    gives up and sets the timeout status (FLBM_ETIMEOUT at the next
                                    synchronising call); 1 .. 60000, default 2000 */
    FLBM_OPT_TEST_STALL = 13,    /* failure-detection test hook: 1 makes every dependency wait of the
                                    fused step wait for work that never comes, so it runs out after
                                    the wait limit; 0 (default) off */
    FLBM_OPT_PIPE_LAG = 14,      /* fused schedule: how many slices the density work runs ahead of the
                                    collisions; 0 (default) = two waves of work in flight and two
                                    slices, cut to what about 40 MB of slices' populations allow (the
                                    collisions re-read them from L2), never below one wave and a
                                    slice; else an integer >= 2 (results are identical) */
    FLBM_OPT_GRAPH_STEPS = 15,   /* steps per CUDA graph that flbm_step replays: batches (default 16)
                                    and single boxes (default 0: each step launched directly; the
                                    two-kernel schedule, kernel timing off).  A graph is captured per
                                    starting parity and dropped by any option or stream change.
                                    Same results; pays on small boxes whose steps are launch-bound */
    FLBM_OPT_SLABS = 16,         /* overlap schedule: number of slabs, 3 .. 256 (at most the number of
                                    planes, or rows for D2Q9); default 8 */
    FLBM_OPT_BLOCK_X = 17,       /* thread block of the density and collide kernels: sites along x,
                                    32, 64 or 128 (default; capped at nx rounded up to 32) */
    FLBM_OPT_BLOCK_Y = 18,       /* ... and rows along y, 1 (default), 2 or 4; x * y <= 128.
                                    The shape changes speed only, never results.  Set one of the
                                    two first when the other would exceed the product limit */
    FLBM_OPT_STREAMING = 19,     /* flbm_streaming; only before the buffers exist (it sets their
                                    size, see flbm_buffer_bytes).  Both modes compute bitwise the
                                    same update.  Batches and flbm_step_noalloc stream in place */
    FLBM_OPT_GHOST_NOISE = 21,   /* 1: the non-conserved modes' noise is drawn as one Gaussian per
                                    population with the variance of local equilibrium at the site
                                    the population streams to, mu w_i rho^s(r + c_i), projected on
                                    the non-conserved modes (times (2 lb_a - lb_a^2)^(1/2) as in
                                    Eq. new-noise): the off-diagonal noise between higher modes of a
                                    non-homogeneous state that the paper leaves open (Sec. V B,
                                    Sec. VII).  Equal to Eq. new-noise in distribution where the
                                    density is uniform.  0 (default): the diagonal form of Eq.
                                    new-noise.  Two-species contexts (not batches); it runs the
                                    general collide, so it is slower than the default at tau = 1,
                                    and the fused schedule with two arrays runs the two-kernel
                                    step while it is on */
    FLBM_OPT_DIRECT_HOST = 22,   /* how flbm_init and flbm_moments move fields between the caller's
                                    arrays and the device.  1 (default): where the GPU shares the
                                    host's page tables (cudaDevAttrPageableMemoryAccess, as Grace with
                                    Blackwell), kernels read the initial densities and store the
                                    moments straight from and into the caller's memory (the output
                                    arrays' pages mapped by host threads first); elsewhere as 0.
                                    0: through a pinned staging buffer (conversion on host threads;
                                    the moments in alternating chunks).  flbm_get_option reads the
                                    route in effect: 1 only where the direct route is taken */
    FLBM_OPT_TEST_GENERAL_COLLIDE = 20, /* test hook: 1 keeps the general collide kernel even when
                                    every non-conserved rate is 1, where a kernel that skips those
                                    modes' projections runs by default (the two agree to rounding;
                                    each is deterministic); 0 default */
    FLBM_OPT_LAMBDA_MODE = 1000, /* + 100 * species + a, a > D: rate lambdabar_a of one
                                    non-conserved mode, 0 < value < 2; default 1/tau_species */
    FLBM_OPT_RHO0_SPECIES = 2000 /* N-species contexts only: + s, reference density of species s
                                    (default 1): the uniform init value and the base of the
                                    stored deviations; only before flbm_minit */
};

/*
 * Create a context for an nx * ny * nz periodic box of two species (nz = 1 for
 * D2Q9).  tau_a, tau_b: relaxation times; every non-conserved mode of species s
 * relaxes with lambdabar = 1/tau_s (the lattice rate of Eq. lattice-freq), the
 * momenta with the common lambdabar_d (see FLBM_OPT_LAMBDA_D).  kT: fluctuation
 * temperature (k_B T, lattice units, >= 0).  G: inter-species coupling of
 * Eq. FORCESTRUCTURE (G > 0 repels).  seed: the 64-bit key of the
 * Philox4x32-10 noise generator.
 * Noise: the Gaussian for mode a >= 1 of species s at (site, step n) is its
 * Gaussian k = a - 1, from Philox4x32-10 with key (seed low, seed high) and
 * counter (site, n, s, k/6).  The block's words x0..x3 give six 21-bit
 * uniforms U0..U3 = x0..x3 >> 11, U4 = (x0 mod 2^11) 2^10 + (x1 mod 2^10),
 * U5 = (x2 mod 2^11) 2^10 + (x3 mod 2^10); Gaussian k is output k mod 2 of
 * Box-Muller on (U2q, U2q+1), q = (k mod 6)/2: u1 = (U2q + 1) 2^-21,
 * u2 = U2q+1 2^-21, (g0, g1) = sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2).
 * The species momenta use species 0's draws for B as well, with the opposite sign.
 * No device memory is allocated here.
 * Errors: FLBM_EINVAL if lat is unknown, nx/ny/nz < 2 (nz != 1 for D2Q9),
 * ny or nz > 65535, nx*ny*nz >= 2^31, tau <= 0.5, kT < 0, or out == NULL.
 */
flbm_status flbm_create(flbm_lattice lat, int nx, int ny, int nz, double tau_a, double tau_b,
                        double kT, double G, uint64_t seed, flbm_ctx **out);

/* Set one option (keys above).  FLBM_EINVAL for an unknown key or a value out of
 * range; FLBM_ESTATE for FLBM_OPT_STORAGE after the buffers exist. */
flbm_status flbm_set_option(flbm_ctx *ctx, int key, double value);

/* Read one option's current value into *value (FLBM_OPT_GRAPH_STEPS on batches
 * only; FLBM_OPT_LAMBDA_MODE + 100 s + a for the rate of one mode).
 * FLBM_EINVAL for an unknown key, FLBM_EUNSUPPORTED for a key the context
 * does not have. */
flbm_status flbm_get_option(const flbm_ctx *ctx, int key, double *value);

/* Run the context's work on `stream` (a cudaStream_t, NULL = the library's own
 * non-blocking stream).  The caller keeps ownership of the stream and must keep
 * it alive while the context uses it. */
flbm_status flbm_set_stream(flbm_ctx *ctx, void *stream);

/* Bytes of device memory the context needs for its populations and its density
 * field, for the current storage and streaming options: one array holds
 * 2 * Q * N populations, slot by slot, with the two species' words of a slot
 * and site side by side (species s, slot i, site x at word (i N + x) 2 + s);
 * two-array streaming needs two.  Either pointer may be
 * NULL.  Not included: at full relaxation (every non-conserved rate 1) the
 * two-kernel step also keeps 2 (D + 1) float planes
 * of moment scratch (8 (D + 1) N bytes), allocated by the library on the first
 * such step and freed with the context; the collide then reads those moments
 * instead of the populations (same results bit for bit). */
flbm_status flbm_buffer_bytes(const flbm_ctx *ctx, size_t *pop_bytes, size_t *rho_bytes);

/* Use caller-owned device buffers for the populations (pop_bytes as reported by
 * flbm_buffer_bytes, 256-byte aligned) and the density field.  The library
 * never frees them; they must outlive the context.  Without this call,
 * flbm_init allocates its own.  FLBM_ESTATE if buffers already exist. */
flbm_status flbm_attach_buffers(flbm_ctx *ctx, void *pop, size_t pop_bytes, void *rho,
                                size_t rho_bytes);

/* Rest-state initialisation f_i = w_i rho^s(r) (f^eq at zero velocity, Sec. V B).
 * rho_a, rho_b: host arrays of N doubles each, or NULL for the uniform
 * reference densities.  Resets the step counter to 0.  Allocates the buffers
 * if none are attached (FLBM_ENOMEM on failure). */
flbm_status flbm_init(flbm_ctx *ctx, const double *rho_a, const double *rho_b);

/* Advance n >= 0 steps (asynchronous).  Step n uses noise counter n.
 * FLBM_ESTATE before flbm_init; FLBM_ECUDA if a launch fails. */
flbm_status flbm_step(flbm_ctx *ctx, int64_t n);

/* Wait for the context's stream and report device-detected faults
 * (FLBM_ENONFINITE once a density was not positive and finite). */
flbm_status flbm_sync(flbm_ctx *ctx);

/* Accumulated device time of the work flbm_step launched while
 * FLBM_OPT_KERNEL_TIMING was on, in milliseconds: ms[0] the density kernel
 * (two-kernel schedule) or the counter reset (fused schedule), ms[1] the
 * collide kernel or the fused step kernel; under the overlap schedule the sums
 * of the density and of the collide slab launches (which overlap in time).
 * launches[k] is the number of steps timed.  Either array may be NULL.
 * Synchronising. */
flbm_status flbm_kernel_times(flbm_ctx *ctx, double ms[2], int64_t launches[2]);

/* Steps taken since flbm_init (or the restored checkpoint's count). */
flbm_status flbm_get_step(const flbm_ctx *ctx, int64_t *step);

/*
 * Observables of the current state (Eq. lattice-vb): per-site rho^A, rho^B and
 * the baricentric velocity u_b = (jbar^A + jbar^B + (F^A + F^B)/2) / rho_t with
 * F^s = rho^s a^s, as host arrays (rho_a, rho_b: N doubles; u: D * N doubles,
 * component-major [d][z][y][x]); cons (5 doubles) = FP64 totals
 * [sum rho^A, sum rho^B, sum (jbar_t + F_t/2)_x, _y, _z] (z entry 0 for D2Q9).
 * Any pointer may be NULL.  Synchronising.
 */
flbm_status flbm_moments(flbm_ctx *ctx, double *rho_a, double *rho_b, double *u, double *cons);

/* Add one snapshot of the axis structure factors to the FP64 accumulators:
 * for k_m = 2 pi m / n_axis, m = 1 .. n_axis/2, along the axis of
 * FLBM_OPT_SF_AXIS: |rhohat_A|^2/N, Re(rhohat_A conj rhohat_B)/N, |rhohat_B|^2/N and
 * (1/D) sum_d |uhat_d|^2/N, rhohat(k) = sum_r rho(r) e^{-i k r_axis} (Sec. VI A).
 * Synchronising. */
flbm_status flbm_sf_sample(flbm_ctx *ctx);

/* Ensemble means over the snapshots taken so far, for m = 1..nk (nk <= n_axis/2)
 * along `axis` (must equal FLBM_OPT_SF_AXIS): S_aa, S_ab, S_bb, S_uu are host
 * arrays of nk doubles (any may be NULL); *nsamples = snapshot count.
 * FLBM_ESTATE if no snapshot was taken. */
flbm_status flbm_structure_factor(flbm_ctx *ctx, int axis, int nk, double *S_aa, double *S_ab,
                                  double *S_bb, double *S_uu, int64_t *nsamples);

/* Clear the structure-factor accumulators. */
flbm_status flbm_sf_reset(flbm_ctx *ctx);

/*
 * Structure factors at every lattice wavevector (Sec. IV A: the quantities of
 * Eq. str-bin-hom off the axes too) and the structure functions of Eq.
 * structurefunctions.
 *
 * flbm_sfk_sample adds one snapshot: with delta rho^s = rho^s - <rho^s> and
 * rho_hat^s(k) = sum_r delta rho^s(r) exp(-i k.r), k_a = 2 pi m_a / n_a, it
 * accumulates |rho_hat_A|^2, Re(rho_hat_A conj rho_hat_B), |rho_hat_B|^2 in
 * FP64.  The transform runs in float on the fluctuation fields (relative
 * error ~1e-6, far below the statistical error of any estimate).  Device
 * memory: N (3 doubles + 1 complex float), allocated on the first call.
 * Axis lengths up to 4096 when a power of two, up to 3072 otherwise
 * (FLBM_EUNSUPPORTED beyond).  Asynchronous on the context's stream.
 *
 * flbm_sfk copies the ensemble means S_aa, S_ab, S_bb = <...> / N into three
 * caller-owned host arrays of N doubles each (any may be NULL), laid out
 * [m_z][m_y][m_x] like the sites (m_a >= n_a / 2 stands for the negative
 * wavevector m_a - n_a; k = 0 is 0 up to rounding).  *nsamples (may be NULL)
 * receives the snapshot count.  Synchronising; FLBM_ESTATE before a sample.
 *
 * flbm_sfk_functions forms, from the same means, the structure factors of the
 * total density rho_t = rho + rho' and the concentration C = rho / rho_t
 * linearised about (rho0_a, rho0_b):  S_tt = S_aa + 2 S_ab + S_bb,
 * S_CC = (rho0_b^2 S_aa - 2 rho0_a rho0_b S_ab + rho0_a^2 S_bb) / rho_t0^4,
 * S_tC = (rho0_b S_aa + (rho0_b - rho0_a) S_ab - rho0_a S_bb) / rho_t0^2.
 * Same layout and rules; FLBM_EINVAL for non-positive reference densities.
 *
 * flbm_sfk_reset clears the accumulators and frees their memory.
 */
flbm_status flbm_sfk_sample(flbm_ctx *ctx);
flbm_status flbm_sfk(flbm_ctx *ctx, double *S_aa, double *S_ab, double *S_bb, int64_t *nsamples);
flbm_status flbm_sfk_functions(flbm_ctx *ctx, double rho0_a, double rho0_b, double *S_tt, double *S_cc,
                               double *S_tc);
flbm_status flbm_sfk_reset(flbm_ctx *ctx);

/*
 * Capillary fluctuations of a flat interface (Sec. VI B, Eq.
 * predictionspectrum: <|h_hat(k)|^2> = kT / (gamma k^2)).  D2Q9 boxes holding a
 * stripe rich in species A that spans y and contains column x_liquid, with
 * the B-rich phase at column x_gas (FLBM_EUNSUPPORTED for D3Q19).
 *
 * flbm_cap_sample adds one snapshot.  With x_liquid = x_gas = -1 the columns
 * follow the stripe, which wanders over long runs: x_liquid is the middle of
 * the window of n_x/2 columns holding the most A (summed over y) and x_gas
 * the column half a box away, found on the device for each snapshot (the
 * mean heights then refer to each snapshot's own frame).  The bulk values rho_l, rho_g are the
 * means of rho_A over y at the two columns.  In the window of columns from
 * x_gas up to x_liquid (periodic) and in the one from x_liquid up to x_gas,
 * the liquid fraction L(y) = sum_x (rho_A - rho_g) / (rho_l - rho_g) places
 * the dividing surface of each interface, column x covering
 * [x - 1/2, x + 1/2): h1(y) = x_liquid - 1/2 - L1(y), h2(y) = x_liquid - 1/2 +
 * L2(y) (frame of x_liquid).  Each interface's mean height is removed and
 * |sum_y dh(y) exp(-i k_m y)|^2 / n_y, k_m = 2 pi m / n_y, averaged over the
 * two interfaces, is accumulated in FP64.  Asynchronous; fixed columns must
 * stay the same until flbm_cap_reset (else FLBM_EINVAL).  Device memory: N
 * complex floats and (2.5 n_y + n_x) doubles.
 *
 * flbm_cap_spectrum writes S_h[m - 1] for m = 1 .. nk (nk <= n_y / 2), the
 * means over snapshots, and h_mean[2], the mean heights of the two
 * interfaces; either may be NULL.  Synchronising; FLBM_ESTATE before a sample.
 *
 * flbm_cap_reset clears the accumulators and frees their memory.
 */
flbm_status flbm_cap_sample(flbm_ctx *ctx, int x_liquid, int x_gas);
flbm_status flbm_cap_spectrum(flbm_ctx *ctx, int nk, double *S_h, double *h_mean, int64_t *nsamples);
flbm_status flbm_cap_reset(flbm_ctx *ctx);

/* Copy the populations, natural layout [2][Q][N], to / from host doubles
 * (2 * Q * N values).  get: synchronising; set: converts to the storage format
 * and sets the step counter to `step`. */
flbm_status flbm_get_populations(flbm_ctx *ctx, double *f);
flbm_status flbm_set_populations(flbm_ctx *ctx, const double *f, int64_t step);

/* Natural-layout populations of `nsites` sites (indices in [0, N)), out = host
 * [nsites][2][Q] doubles.  For sampled checks on large boxes.  Synchronising. */
flbm_status flbm_get_site_populations(flbm_ctx *ctx, const int64_t *sites, int64_t nsites,
                                      double *out);

/* Checkpoint: the full state (parameters, options, step counter, populations)
 * as an opaque byte image.  With buf == NULL, *bytes receives the size needed;
 * otherwise *bytes must be at least that size.  Restoring into a context created
 * with the same lattice and box continues bit-identically (the noise is keyed on
 * the step).  FLBM_EINVAL on a size, lattice or box mismatch or a corrupt image. */
flbm_status flbm_checkpoint(flbm_ctx *ctx, void *buf, size_t *bytes);
flbm_status flbm_restore(flbm_ctx *ctx, const void *buf, size_t bytes);

/*
 * Step populations that the caller owns, allocating no device memory.  The
 * paper has no counterpart: this serves callers that cannot call cudaMalloc
 * (an arena or pool that owns all device memory, a real-time loop where an
 * allocation could stall or fail).  The density field and status word it
 * needs live in a fixed static device array that every GPU loading this
 * library holds until the process exits (2^21 sites: 16 MiB + 256 bytes).
 *   ctx:    supplies the lattice, box, storage format, parameters and options
 *           (from flbm_create / flbm_set_option; its own buffers and step
 *           counter are neither used nor changed).
 *   pop:    device populations in this library's in-place layout, storage
 *           format of ctx, flbm_buffer_bytes() bytes, 256-byte aligned;
 *           read and updated in place.
 *   parity: streaming parity of `pop` (0 after an even number of steps since a
 *           natural-layout state, 1 after an odd number); after n steps it is
 *           parity ^ (n & 1).
 *   step:   noise counter of the first step; n: number of steps.
 *   stream: cudaStream_t to run on (NULL = the legacy default stream).
 *   status_out: if non-NULL, receives the device status word (bit 0: a
 *           density was not positive and finite).
 * Synchronises `stream` before returning.  Every call looks up the array's
 * device address on the current device (so a device reset between calls is
 * harmless); the first call on a device may load the library's device code,
 * so make that first call before any stream capture.
 * All calls share the one array, which keeps the last call's contents: calls
 * that overlap on the GPU (other streams, other threads) race.
 * Errors: FLBM_EINVAL for bad arguments, a batch handle (from
 * flbm_batch_create: step batches with flbm_step), `pop` not 256-byte aligned
 * or a box above 2^21 sites, all found before anything is launched;
 * FLBM_ENONFINITE if the status bit is set; FLBM_ECUDA if a CUDA call fails.
 */
flbm_status flbm_step_noalloc(const flbm_ctx *ctx, void *pop, int parity, int64_t step, int64_t n,
                              void *stream, unsigned *status_out);

/*
 * Batches of independent replicas (many boxes of uneven size, parameters and
 * noise keys advanced together, as for ensembles of Sec. VI runs).  Each replica is the
 * same problem as a lone context created with its parameters -- its site index
 * and therefore its noise are replica-local -- so a replica of a batch and a
 * lone context with the same parameters and state give the same populations.
 * A step of the batch is one density launch and one collide launch over a work
 * list of 128-site tiles spanning every replica, or, under FLBM_SCHEDULE_TILED
 * (D2Q9, two arrays), one launch over a work list of 32 x 16 tiles; flbm_step
 * replays CUDA graphs of FLBM_OPT_GRAPH_STEPS steps.  Batches stream through
 * two arrays by default (FLBM_OPT_STREAMING, set before the buffers exist) and
 * accept FLBM_OPT_SCHEDULE 1 (two kernels, the default) or 3 (tiled).
 * On a batch context: flbm_set_option (applied to every replica),
 * flbm_set_stream, flbm_buffer_bytes, flbm_attach_buffers, flbm_init (host
 * densities concatenated replica by replica, or NULL), flbm_step, flbm_sync,
 * flbm_moments (fields concatenated replica by replica, u as [replica][d][site];
 * cons summed over replicas), flbm_sf_sample (every replica), flbm_sf_reset,
 * flbm_get/set_populations (concatenated [replica][species][i][site]),
 * flbm_checkpoint/restore, flbm_destroy.  Per-replica structure factors, site
 * populations and moments come from the replica views.
 */
typedef struct {
    int nx, ny, nz;             /* box of this replica (nz = 1 for D2Q9) */
    double tau_a, tau_b, kT, G; /* as in flbm_create */
    uint64_t seed;              /* Philox key of this replica */
    double rho0_a, rho0_b;      /* reference densities (uniform init, 16-bit deviation base) */
} flbm_rep_params;

/* Create a batch of nrep replicas with parameters p[0..nrep-1].  No device
 * memory is allocated here.  FLBM_EINVAL if a replica's parameters are invalid
 * (same rules as flbm_create) or the total site count reaches 2^31. */
flbm_status flbm_batch_create(flbm_lattice lat, int nrep, const flbm_rep_params *p, flbm_ctx **out);

/* Replica `rep` of a batch as a context of its own (owned by the batch, valid
 * until the batch is destroyed).  It supports the observation calls --
 * flbm_moments, flbm_sf_sample, flbm_structure_factor, flbm_sf_reset,
 * flbm_get_populations, flbm_get_site_populations, flbm_get_step,
 * flbm_set_option(FLBM_OPT_SF_AXIS) -- and answers FLBM_ESTATE to calls that
 * would change it alone (step, init, set_populations, restore, other options). */
flbm_status flbm_batch_replica(flbm_ctx *batch, int rep, flbm_ctx **view);

/* Number of replicas and total sites of a batch (either pointer may be NULL). */
flbm_status flbm_batch_size(const flbm_ctx *batch, int *nrep, int64_t *sites);

/*
 * Launch-settings autotuner (no counterpart in the paper, which gives no
 * implementation).  Times candidate settings on this context's own state and
 * keeps the fastest:
 *   single box: the two-kernel schedule and the overlap schedule with 4 or 8
 *               slabs, each with thread blocks of 128x1, 64x2 and 32x4 sites;
 *               with two arrays the fused (pipelined) schedule, and on D2Q9
 *               the tiled schedule with and without 16-step graphs;
 *   batch:      FLBM_OPT_GRAPH_STEPS of 0, 4, 16 and 64, and on D2Q9 with two
 *               arrays the same graph lengths under the tiled schedule.
 * Every candidate computes bitwise the same update, so tuning changes speed,
 * never results.  Each candidate runs 2 untimed and `steps` timed steps
 * (1 .. 100000) from the same saved state: the populations are copied aside on
 * the device (one population-array of scratch, freed before returning; a batch
 * uses a host checkpoint image), and the state, step counter and parity are
 * put back after every candidate, so the call leaves the simulation where it
 * was.  The three fastest are timed twice and the least time wins.
 * cache_path: NULL, or a JSON file of earlier choices keyed by GPU name, SM
 * count and problem (lattice, storage, box or batch size); a stored choice is
 * applied without timing, a new one is added to the file (written to a
 * temporary name, then renamed).  Read the result with flbm_get_option.
 * Synchronising.  Errors: FLBM_EINVAL for steps out of range or an unreadable
 * or unwritable cache, FLBM_ESTATE before flbm_init or on a replica view,
 * FLBM_ENOMEM without room for the scratch copy, and any error of flbm_step.
 */
flbm_status flbm_autotune(flbm_ctx *ctx, int steps, const char *cache_path);

/* One-line reason of the last error on this context ("" if none).  The string
 * is owned by the context.  Never NULL (ctx may be NULL). */
const char *flbm_last_error(const flbm_ctx *ctx);

/* Free the context and the device memory it owns (never attached buffers).
 * NULL is a no-op. */
void flbm_destroy(flbm_ctx *ctx);

/* Library version string, e.g. "flbm 0.1 sm_103a". */
const char *flbm_version(void);

/*
 * N-species mixtures (App. C-D): the update above for 2 <= N <= 4 species on
 * their own context type.  Per site r and step n, for every species sigma:
 *   - rho^sigma = sum_i fbar_i^sigma;
 *   - a^sigma(r) = -sum_{s != sigma} G_{sigma s} sum_i w_i rho^s(r + c_i) c_i
 *     (forces between different species only; G symmetric, diagonal ignored);
 *   - u = sum_sigma (jbar^sigma + rho^sigma a^sigma / 2) / rho_t;
 *   - non-conserved modes of species sigma relax with lambdabar = 1/tau_sigma,
 *     the momenta with the common rate lambdabar_d = N / sum_sigma tau_sigma;
 *   - momentum noise with covariance (2 lb_d - lb_d^2) kT (rho^sigma delta -
 *     rho^sigma rho^s / rho_t) (local densities), drawn as
 *     xi^sigma = A (eta^sigma - C^sigma sum_s eta^s), eta^s = sqrt(rho^s) g^s,
 *     C = rho / rho_t, A = sqrt((2 lb_d - lb_d^2) kT); it sums to zero over the
 *     species, so the total momentum is conserved;
 *   - the other modes' noise with the variances of Eq. new-noise per species.
 * g of mode a of species s at (site, n) is drawn as for two species (counter
 * (site, n, s, (a-1)/6), six 21-bit uniforms per block); every
 * species draws its own momentum Gaussians.  Populations are stored as float
 * in the natural layout [s][i][z][y][x] where exposed.  Conventions (errors,
 * asynchrony, site order, lattice units) are those of the two-species calls.
 */
typedef struct flbm_mctx flbm_mctx; /* opaque; created and freed by the library */

/* Create an N-species context (no device memory yet).  tau: nspecies
 * relaxation times (> 0.5); G: nspecies x nspecies row-major couplings,
 * symmetric and finite (the diagonal is ignored).  Errors: FLBM_EINVAL for
 * nspecies outside 2..4, an unknown lattice, a box outside the limits of
 * flbm_create, tau <= 0.5, kT < 0, an asymmetric or non-finite G, or NULL
 * pointers. */
flbm_status flbm_mcreate(flbm_lattice lat, int nspecies, int nx, int ny, int nz, const double *tau,
                         double kT, const double *G, uint64_t seed, flbm_mctx **out);

/* Options: FLBM_OPT_KERNEL_TIMING, FLBM_OPT_BLOCK_X, FLBM_OPT_BLOCK_Y,
 * FLBM_OPT_STREAMING (as for two species; two arrays by default, in place on
 * request, bitwise the same update), FLBM_OPT_GRAPH_STEPS (as for a single
 * two-species box, default 0) and FLBM_OPT_RHO0_SPECIES + s.
 * FLBM_EINVAL otherwise. */
flbm_status flbm_mset_option(flbm_mctx *ctx, int key, double value);

/* Read one of those options back into *value; FLBM_EINVAL for another key. */
flbm_status flbm_mget_option(const flbm_mctx *ctx, int key, double *value);

/* Run on a caller-owned cudaStream_t (NULL: a stream the context creates). */
flbm_status flbm_mset_stream(flbm_mctx *ctx, void *stream);

/* Rest state f_i = w_i rho^s: rho = host [nspecies][N] doubles (positive,
 * finite) or NULL for rho^s = the reference densities.  Allocates the
 * populations (nspecies Q N floats, twice that with two-array streaming) and
 * the density field (16 bytes a site).  Resets the step counter.
 * Synchronising. */
flbm_status flbm_minit(flbm_mctx *ctx, const double *rho);

/* Advance n >= 0 steps (asynchronous): per step a density kernel, then the
 * collide kernel.  Step n uses noise counter n.  FLBM_ESTATE before init. */
flbm_status flbm_mstep(flbm_mctx *ctx, int64_t n);

/* Wait for the stream; FLBM_ENONFINITE once a density was not positive and finite. */
flbm_status flbm_msync(flbm_mctx *ctx);

/* Device time of the density (ms[0]) and collide (ms[1]) kernels of the steps
 * taken while FLBM_OPT_KERNEL_TIMING was on; either array may be NULL.
 * Synchronising. */
flbm_status flbm_mkernel_times(flbm_mctx *ctx, double ms[2], int64_t launches[2]);

flbm_status flbm_mget_step(const flbm_mctx *ctx, int64_t *step);

/* Observables of the current state: rho = host [nspecies][N] doubles, u = host
 * [D][N] doubles (the u above), cons = nspecies + 3 FP64 totals [sum rho^0 ..
 * sum rho^{N-1}, total momentum sum (jbar_t + F_t / 2) x, y, z].  Any pointer
 * may be NULL.  Synchronising. */
flbm_status flbm_mmoments(flbm_mctx *ctx, double *rho, double *u, double *cons);

/* Populations, natural layout [nspecies][Q][N], to / from host doubles.  get:
 * synchronising; set: rounds to float, sets the step counter to `step` and
 * makes the context ready to step. */
flbm_status flbm_mget_populations(flbm_mctx *ctx, double *f);
flbm_status flbm_mset_populations(flbm_mctx *ctx, const double *f, int64_t step);

/* Natural-layout populations of `nsites` sites (indices in [0, N)), out = host
 * [nsites][nspecies][Q] doubles.  For sampled checks on large boxes.
 * Synchronising.  FLBM_EINVAL for an index out of range. */
flbm_status flbm_mget_site_populations(flbm_mctx *ctx, const int64_t *sites, int64_t nsites, double *out);

/* Axis structure factors of the N species (App. D: S_{sigma s}(k)).
 * flbm_msf_sample adds one snapshot along `axis` (0 x, 1 y, 2 z; < D) to FP64
 * accumulators: for k_m = 2 pi m / n_axis, m = 1 .. n_axis/2, and every pair
 * (sigma, s): Re(rhohat^sigma conj rhohat^s) / N, with rhohat(k) = sum_r
 * rho(r) e^{-i k r_axis} (the k = 0 mode, the conserved mass, is excluded).
 * Each axis keeps its own accumulators.  Synchronising.
 * flbm_mstructure_factor returns the means over the snapshots of `axis` for
 * m = 1 .. nk (nk <= n_axis/2) into S = host [nspecies][nspecies][nk] doubles
 * (may be NULL) and the snapshot count into *nsamples (may be NULL);
 * FLBM_ESTATE before the first snapshot of that axis.
 * flbm_msf_reset clears every axis. */
flbm_status flbm_msf_sample(flbm_mctx *ctx, int axis);
flbm_status flbm_mstructure_factor(flbm_mctx *ctx, int axis, int nk, double *S, int64_t *nsamples);
flbm_status flbm_msf_reset(flbm_mctx *ctx);

/* Checkpoint of an N-species context: parameters, step counter, streaming
 * parity and the stored populations as an opaque byte image (buf == NULL:
 * *bytes receives the size needed).  Restoring into a context created with
 * the same lattice, species count and box continues bit-identically (the
 * noise is keyed on the step).  FLBM_EINVAL on a size or shape mismatch or a
 * corrupt image; FLBM_ESTATE for a checkpoint before the state exists. */
flbm_status flbm_mcheckpoint(flbm_mctx *ctx, void *buf, size_t *bytes);
flbm_status flbm_mrestore(flbm_mctx *ctx, const void *buf, size_t bytes);

/* One-line reason of the last error ("" if none); never NULL. */
const char *flbm_mlast_error(const flbm_mctx *ctx);

/* Free the context and its device memory.  NULL is a no-op. */
void flbm_mdestroy(flbm_mctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* FLBM_H */
