// flbm_multi.cuh -- kernels of the N-species update (arXiv 1410.5584, App. C-D),
// instantiated per (lattice, species count) in the inst_multi_*.cu units.
//
// The update is the lattice algorithm of Sec. V B (Eqs. algorithm and lattice
// finalstep) for NS = 2 .. 4 species sigma, with
//   - rates lambdabar_a^sigma on the non-conserved modes of each species and one
//     common momentum rate lambdabar_d (total momentum is conserved only if the
//     momentum relaxation matrix d^{sigma s} = lambdabar_d (delta - C^s) of
//     App. C has equal rates),
//   - mean-field forces between different species only (App. D):
//     a^sigma(r) = -sum_{s != sigma} G_{sigma s} sum_i w_i rho^s(r + c_i) c_i,
//   - u = sum_sigma (jbar^sigma + rho^sigma a^sigma / 2) / rho_t,
//   - momentum noise with covariance (2 lb_d - lb_d^2) kT (rho^sigma delta -
//     rho^sigma rho^s / rho_t) (the N-species form of Eq. new-noise, local
//     densities): xi^sigma = A (eta^sigma - C^sigma sum_s eta^s), eta^s =
//     sqrt(rho^s) g^s, C = rho / rho_t, A = sqrt((2 lb_d - lb_d^2) kT), which
//     has exactly that covariance and sums to zero over the species,
//   - the other modes' noise with the per-species variances of Eq. new-noise.
// Unit Gaussian g of mode a >= 1 of species s at (site, step): Gaussian
// n = a - 1 of the species, position n mod 6 of Philox block n / 6 with
// counter (site, step, s, n / 6), as in the two-species kernels.
//
// Storage: the float deviations f_i - w_i rho0^s, with the same in-place "AA"
// streaming and plane layout [s][i][site] as the two-species kernels
// (flbm_kernels.cuh).  The density field holds one float4 per site: the
// deviations rho^s - rho0^s of up to four species.
#pragma once
#include "flbm_internal.h"
#include "flbm_kernels.cuh"
#include "flbm_lattice.cuh"
#include "flbm_noise.cuh"
#include "flbm_transform.cuh"

namespace flbm {

constexpr int kMaxSpecies = 4;

// Everything one step of an N-species box needs (kernel parameter space).
struct MStepParams {
    int nx, ny, nz, N;
    int block_x, block_y;
    float G[kMaxSpecies][kMaxSpecies]; // couplings between different species (zero diagonal)
    float lam_d, hlam_d;               // common momentum rate and 1 - lam_d / 2 (Eq. forcerenorm)
    float amp_d;                       // sqrt((2 lam_d - lam_d^2) kT)
    // non-conserved modes a > D of species s with 1/N_a folded in:
    // m*_a / N_a = cm m_a + ceq m^eq_a + cphi Phi_a + cxi sqrt(rho^s) g_a
    float cm[kMaxSpecies][kMaxQ], ceq[kMaxSpecies][kMaxQ], cphi[kMaxSpecies][kMaxQ], cxi[kMaxSpecies][kMaxQ];
    float rho0[kMaxSpecies];           // reference densities (base of the stored deviations)
    uint32_t key0, key1, step;        // step: the noise counter, or its offset from *step_dev
    const unsigned *step_dev;         // NULL, or a device word the counter is read from (graph replays)
    float *mom;                       // NULL, or NS (D + 1) planes of N floats: m_0 .. m_D of each
                                      // species, written by the density pass and read by the collide
                                      // in place of the populations (every non-conserved rate 1, two
                                      // arrays)
};

template <class T> struct MPlanes {
    T *ptr[kMaxSpecies * kMaxQ];
    template <class L> __device__ __forceinline__ T *plane(int s, int j) const { return ptr[s * L::Q + j]; }
};

// Launchers of one (lattice, species count) pair; asynchronous on `st`, return
// the launch error.
template <class L, int NS> struct MLaunch {
    // density deviations of every site (float4 per site)
    static cudaError_t density(int parity, const MStepParams &p, const float *pop, float4 *drho, cudaStream_t st);
    // force + moment collision + noise + in-place streaming of one step
    // parity 0 / 1: in place in pop; kStreamPush: read pop, write pop_out
    static cudaError_t collide(int parity, const MStepParams &p, float *pop, float *pop_out, const float4 *drho,
                               unsigned *status, cudaStream_t st);
    // per-site rho^s and u (either may be NULL) in double, per-block FP64 partial
    // totals [nblocks][NS + 3] of (rho^s, jbar_t + F_t / 2); needs drho of the state
    static cudaError_t observables(int parity, const MStepParams &p, const float *pop, const float4 *drho,
                                   double *rho, double *u, double *partials, int *nblocks, cudaStream_t st);
    // natural-layout copy [NS][Q][N] of the stored deviations
    static cudaError_t natural(int parity, const MStepParams &p, const float *pop, float *out, cudaStream_t st);
    // natural-layout populations of selected sites: out[k][s][i] (doubles)
    static cudaError_t gather(int parity, const MStepParams &p, const float *pop, const int64_t *sites, int64_t n,
                              double *out, cudaStream_t st);
    // rest state f_i = w_i rho^s (stored as w_i (rho^s - rho0^s)) from float densities [NS][N]
    static cudaError_t init_rest(const MStepParams &p, const float *rho, float *pop, cudaStream_t st);
};

// One axis structure-factor snapshot of the density deviations drho (float4 a
// site): profiles prof[s][j] = sum over the plane at coordinate j along `axis`
// (FP64, fixed order), then for k_m = 2 pi m / n, m = 1 .. n/2,
// acc[s][t][m-1] += Re(rhohat^s conj rhohat^t) / N.  prof: NS n doubles of
// scratch; acc: NS NS (n/2) doubles.
cudaError_t launch_msf_snapshot(int ns, const MStepParams &p, int axis, const float4 *drho, double *prof,
                                double *acc, cudaStream_t st);

namespace mkern {

constexpr int kObsBlock = 128;

__device__ __forceinline__ kern::Nbr make_nbr(const MStepParams &p, int x, int y, int z)
{
    kern::Nbr n;
    n.nx = p.nx;
    n.ny = p.ny;
    n.xs[0] = x == 0 ? p.nx - 1 : x - 1;
    n.xs[1] = x;
    n.xs[2] = x == p.nx - 1 ? 0 : x + 1;
    n.ys[0] = y == 0 ? p.ny - 1 : y - 1;
    n.ys[1] = y;
    n.ys[2] = y == p.ny - 1 ? 0 : y + 1;
    n.zs[0] = z == 0 ? p.nz - 1 : z - 1;
    n.zs[1] = z;
    n.zs[2] = z == p.nz - 1 ? 0 : z + 1;
    return n;
}

__device__ __forceinline__ float get4(const float4 &v, int t)
{
    return t == 0 ? v.x : (t == 1 ? v.y : (t == 2 ? v.z : v.w));
}

// Unit Gaussians of the positions of one Philox block (counter (site, step, s,
// b)) that MASK selects (bit l = position l, mode 6 b + l + 1); positions
// (0, 1), (2, 3) and (4, 5) are the cosine and sine outputs of one Box-Muller
// pair each, the third on the uniforms packed from the words' low bits.
template <int MASK>
__device__ __forceinline__ void block_gaussians(uint32_t site, uint32_t step, uint32_t s, uint32_t b, uint32_t k0,
                                                uint32_t k1, float (&g)[6])
{
    const uint4 x = philox4x32_10(make_uint4(site, step, s, b), k0, k1);
    if constexpr ((MASK & 3) != 0) box_muller(uniform_hi(x.x), uniform_hi_signed(x.y), 1.0f, g[0], g[1]);
    if constexpr ((MASK & 12) != 0) box_muller(uniform_hi(x.z), uniform_hi_signed(x.w), 1.0f, g[2], g[3]);
    if constexpr ((MASK & 48) != 0)
        box_muller(uniform_lo(x.x, x.y), uniform_lo_signed(x.z, x.w), 1.0f, g[4], g[5]);
}

// Positions of block b that hold a non-conserved mode (D < a < Q).
template <int Q, int D> __host__ __device__ constexpr int other_modes_mask(int b)
{
    int m = 0;
    for (int l = 0; l < 6; l++)
        if (6 * b + l + 1 > D && 6 * b + l + 1 < Q) m |= 1 << l;
    return m;
}

// Loads of the NS Q pre-collision deviations of a site.
template <class L, int NS, int PARITY, class P>
__device__ __forceinline__ void load_site(const P &planes, const kern::Nbr &nb, float (&d)[NS][L::Q])
{
    static_for<NS>([&](auto sc) {
        constexpr int s = decltype(sc)::value;
        static_for<L::Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            d[s][i] = __ldg(planes.template plane<L>(s, kern::read_slot<L, PARITY, i>()) +
                            kern::read_site<L, PARITY, i>(nb));
        });
    });
}

// MOM: also stores m_0 .. m_D of every species into p.mom (the moment-fed
// collide's input).
template <class L, int NS, int PARITY, bool MOM = false>
__global__ void __launch_bounds__(kSiteBlockMax) k_mdensity(const MStepParams p, const MPlanes<const float> planes,
                                                            float4 *__restrict__ drho)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= p.nx || y >= p.ny) return;
    const kern::Nbr nb = make_nbr(p, x, y, blockIdx.z);
    float d[NS][L::Q];
    load_site<L, NS, PARITY>(planes, nb, d);
    float r[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    static_for<NS>([&](auto sc) {
        constexpr int s = decltype(sc)::value;
        float m[L::Q];
        // the collide kernel computes its own densities with this same expression
        Transform<L>::forward(d[s], m);
        r[s] = m[0];
        if constexpr (MOM) {
            static_for<L::D + 1>([&](auto ac) {
                constexpr int a = decltype(ac)::value;
                p.mom[(size_t)(s * (L::D + 1) + a) * (size_t)p.N + nb.at(0, 0, 0)] = m[a];
            });
        }
    });
    drho[nb.at(0, 0, 0)] = make_float4(r[0], r[1], r[2], r[3]);
}

// Whether the collide kernel parks each site's moments in shared memory (three
// or more species: the register footprint stays that of one species at a
// time) or holds them in registers (two species, where that is faster).
template <int NS> constexpr bool kParkMoments = NS >= 3;

// Shared-memory bytes of one collide block of `threads` threads: the NS Q
// moments of each thread's site, [s][a][thread] (consecutive threads on
// consecutive banks); none when they stay in registers.
template <class L, int NS> constexpr size_t collide_smem(int threads)
{
    return kParkMoments<NS> ? (size_t)NS * L::Q * threads * 4 : 0;
}

// One step of one site: the populations of all species are loaded once and
// their moments computed; only each species' density and momentum stay in
// registers, the rest is parked (or kept in registers for two species);
// forces, the baricentric velocity and the projected momentum noise follow;
// then each species in turn is collided and streamed.  No barrier: a thread
// reads back only its own slots.
// 128 registers (16 warps an SM); three species are held to 96 (20 warps), measured
// 2 % faster at 256^3 despite a 48-byte spill, which costs four species 6 %.
// MOM (every non-conserved rate 1, so that the old non-conserved moments drop
// out of Eq. algorithm): m_0 .. m_D of every species come from the density
// pass's planes p.mom instead of the populations, which are not read.
template <class L, int NS, int PARITY, bool MOM = false>
__global__ void __launch_bounds__(kSiteBlockMax, NS == 3 ? 5 : 4)
    k_mcollide(const MStepParams p, const MPlanes<float> planes, const MPlanes<float> out,
               const float4 *__restrict__ drho, unsigned *__restrict__ status)
{
    constexpr int Q = L::Q, D = L::D;
    constexpr bool PARK = kParkMoments<NS> && !MOM;
    extern __shared__ float park[];
    const int nthr = blockDim.x * blockDim.y;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= p.nx || y >= p.ny) return;
    const kern::Nbr nb = make_nbr(p, x, y, blockIdx.z);
    const int site = nb.at(0, 0, 0);

    // 1. loads and moments of every species (Eq. modes-discrete; the density
    // with the same expression as the density kernel)
    float mc[NS][4], rs[NS];
    float mreg[PARK || MOM ? 1 : NS][Q];
    if constexpr (MOM) {
        static_for<NS>([&](auto sc) {
            constexpr int s = decltype(sc)::value;
            static_for<D + 1>([&](auto ac) {
                constexpr int a = decltype(ac)::value;
                mc[s][a] = __ldg(p.mom + (size_t)(s * (D + 1) + a) * (size_t)p.N + site);
            });
            rs[s] = p.rho0[s] + mc[s][0];
        });
    } else static_for<NS>([&](auto sc) {
        constexpr int s = decltype(sc)::value;
        float d[Q], m[Q];
        static_for<Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            d[i] = __ldg(planes.template plane<L>(s, kern::read_slot<L, PARITY, i>()) +
                         kern::read_site<L, PARITY, i>(nb));
        });
        Transform<L>::forward(d, m);
        static_for<Q>([&](auto ac) {
            constexpr int a = decltype(ac)::value;
            if constexpr (a <= D) mc[s][a] = m[a];
            if constexpr (PARK) park[(s * Q + a) * nthr + tid] = m[a];
            else mreg[PARK || MOM ? 0 : s][a] = m[a];
        });
        rs[s] = p.rho0[s] + m[0];
    });

    // 2. mean-field forces between different species (App. D, Eq. FORCESTRUCTURE
    // per pair): F[t][d] = sum_i w_i c_id rho^t(r + c_i) on the deviations (the
    // reference part sums to zero), then a^s = -sum_{t != s} G_st F[t]
    float F[NS][3];
    static_for<NS>([&](auto tc) {
        constexpr int t = decltype(tc)::value;
        F[t][0] = F[t][1] = F[t][2] = 0.0f;
    });
    static_for<Q - 1>([&](auto kc) {
        constexpr int i = decltype(kc)::value + 1;
        constexpr float wi = (float)L::wd(i);
        const float4 rn = __ldg(drho + nb.at(L::cx(i), L::cy(i), L::cz(i)));
        static_for<D>([&](auto dc) {
            constexpr int d = decltype(dc)::value;
            constexpr int cd = comp<L>(i, d);
            if constexpr (cd != 0) {
                constexpr float cw = (float)cd * wi;
                static_for<NS>([&](auto tc) {
                    constexpr int t = decltype(tc)::value;
                    F[t][d] = fmaf(cw, get4(rn, t), F[t][d]);
                });
            }
        });
    });
    float acc[NS][3];
    static_for<NS>([&](auto sc) {
        constexpr int s = decltype(sc)::value;
        acc[s][2] = 0.0f;
        static_for<D>([&](auto dc) {
            constexpr int d = decltype(dc)::value;
            float a = 0.0f;
            static_for<NS>([&](auto tc) {
                constexpr int t = decltype(tc)::value;
                if constexpr (t != s) a = fmaf(p.G[s][t], F[t][d], a);
            });
            acc[s][d] = -a;
        });
    });

    // 3. baricentric velocity with the half-force shift (Eq. lattice finalstep).
    // Here and in step 5 every rounding is explicit, so that the population-
    // reading and the moment-fed instances give the same bits.
    float rt = 0.0f;
    bool bad = false;
    static_for<NS>([&](auto sc) {
        constexpr int s = decltype(sc)::value;
        rt = __fadd_rn(rt, rs[s]);
        bad |= !(rs[s] > 0.0f);
    });
    if (bad || !isfinite(rt)) atomicOr(status, kStatusNonFinite);
    const float irt = __frcp_rn(rt);
    float u[3] = {0.0f, 0.0f, 0.0f};
    static_for<D>([&](auto dc) {
        constexpr int d = decltype(dc)::value;
        float j = 0.0f;
        static_for<NS>([&](auto sc) {
            constexpr int s = decltype(sc)::value;
            j = __fadd_rn(j, __fmaf_rn(__fmul_rn(0.5f, rs[s]), acc[s][d], mc[s][1 + d]));
        });
        u[d] = __fmul_rn(j, irt);
    });

    // 4. the momentum Gaussians of every species: modes 1 .. D, positions
    // 0 .. D-1 of Philox block 0.  Projected momentum noise.
    const uint32_t nstep = p.step_dev ? __ldg(p.step_dev) + p.step : p.step; // noise counter of this step
    float sq[NS], xi[NS][3];
    {
        float g0[NS][6];
        static_for<NS>([&](auto sc) {
            constexpr int s = decltype(sc)::value;
            block_gaussians<(1 << D) - 1>((uint32_t)site, nstep, (uint32_t)s, 0u, p.key0, p.key1, g0[s]);
            sq[s] = rs[s] * rsqrtf(rs[s]); // sqrt(rho^s); rho^s > 0 on every valid state
        });
        static_for<D>([&](auto dc) {
            constexpr int d = decltype(dc)::value;
            float sum = 0.0f;
            static_for<NS>([&](auto sc) {
                constexpr int s = decltype(sc)::value;
                sum = fmaf(sq[s], g0[s][d], sum);
            });
            const float cs = sum * irt;
            static_for<NS>([&](auto sc) {
                constexpr int s = decltype(sc)::value;
                xi[s][d] = p.amp_d * fmaf(-rs[s], cs, sq[s] * g0[s][d]);
            });
        });
    }

    // 5. each species: its moments back, momentum modes with the common rate
    // (species velocity for Phi from Eq. alg-mom), then the transport and
    // ghost modes, back-projection, mass closure on the stored values, streaming
    float X[Q];
    Closure<L>::eq(u, X);
    static_for<NS>([&](auto sc) {
        constexpr int s = decltype(sc)::value;
        float m[Q];
        static_for<Q>([&](auto ac) {
            constexpr int a = decltype(ac)::value;
            if constexpr (MOM) {
                if constexpr (a <= D) m[a] = mc[s][a];
            } else if constexpr (PARK) {
                m[a] = park[(s * Q + a) * nthr + tid];
            } else {
                m[a] = mreg[PARK || MOM ? 0 : s][a];
            }
        });
        const float irs = __frcp_rn(rs[s]);
        const float lrs = __fmul_rn(p.lam_d, rs[s]), hrs = __fmul_rn(p.hlam_d, rs[s]);
        float v[3] = {0.0f, 0.0f, 0.0f};
        static_for<D>([&](auto dc) {
            constexpr int d = decltype(dc)::value;
            constexpr int a = 1 + d;
            // R = lambdabar_d (rho^s u - j^s) + (1 - lambdabar_d / 2) rho^s a^s + xi^s
            const float R = __fmaf_rn(lrs, u[d], __fmaf_rn(-p.lam_d, m[a], __fmaf_rn(hrs, acc[s][d], xi[s][d])));
            v[d] = __fmul_rn(__fmaf_rn(0.5f, R, m[a]), irs);
            m[a] = __fadd_rn(m[a], R);
        });
        // the non-conserved modes' Gaussians (block 0 drawn again: its
        // momentum positions were used in step 4)
        float g[Q];
        static_for<kNoiseBlocks<L>>([&](auto bc) {
            constexpr int b = decltype(bc)::value;
            constexpr int mask = other_modes_mask<Q, D>(b);
            if constexpr (mask != 0) {
                float gs[6];
                block_gaussians<mask>((uint32_t)site, nstep, (uint32_t)s, (uint32_t)b, p.key0, p.key1, gs);
                static_for<6>([&](auto lc) {
                    constexpr int l = decltype(lc)::value;
                    if constexpr ((mask >> l) & 1) g[6 * b + l + 1] = gs[l];
                });
            }
        });
        float Y[Q];
        Closure<L>::force(acc[s], v, Y);
        float mu[Q], fo[Q];
        mu[0] = m[0];
        static_for<D>([&](auto dc) {
            constexpr int a = decltype(dc)::value + 1;
            constexpr float invN = (float)(1.0 / L::Nd(a));
            mu[a] = invN * m[a];
        });
        static_for<Q - D - 1>([&](auto kc) {
            constexpr int a = decltype(kc)::value + D + 1;
            // MOM: cm = 0 (rate 1), so the old moment, never formed, drops out
            float t;
            if constexpr (MOM) t = p.cxi[s][a] * (sq[s] * g[a]);
            else t = fmaf(p.cm[s][a], m[a], p.cxi[s][a] * (sq[s] * g[a]));
            if constexpr (a < Closure<L>::kGhost) t = fmaf(rs[s], fmaf(p.ceq[s][a], X[a], p.cphi[s][a] * Y[a]), t);
            mu[a] = t;
        });
        float yv[Q];
        Transform<L>::backward(mu, yv);
        // the moving deviations w_i y_i are rounded to the words stored; the rest
        // population takes m0 minus what they hold, so no mass leaks
        float word[Q];
        static_for<Q - 1>([&](auto kc) {
            constexpr int i = decltype(kc)::value + 1;
            word[i] = __fmul_rn((float)L::wd(i), yv[i]);
            fo[i] = word[i];
        });
        word[0] = Transform<L>::rest_closing_mass(fo, m[0]);
        static_for<Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            out.template plane<L>(s, kern::write_slot<L, PARITY, i>())[kern::write_site<L, PARITY, i>(nb)] = word[i];
        });
    });
}

// Observables in double from the stored floats; the forces from the float
// density deviations.  Per-block totals in a fixed-order tree.
template <class L, int NS, int PARITY>
__global__ void __launch_bounds__(kObsBlock) k_mobservables(const MStepParams p, const MPlanes<const float> planes,
                                                            const float4 *__restrict__ drho, double *rho_out,
                                                            double *u_out, double *partials)
{
    constexpr int Q = L::Q, D = L::D, NC = NS + 3;
    __shared__ double sh[NC][kObsBlock];
    const int site = blockIdx.x * kObsBlock + threadIdx.x;
    double tot[NC];
#pragma unroll
    for (int k = 0; k < NC; k++) tot[k] = 0.0;
    if (site < p.N) {
        const int x = site % p.nx, y = (site / p.nx) % p.ny, z = site / (p.nx * p.ny);
        const kern::Nbr nb = make_nbr(p, x, y, z);
        double F[NS][3] = {};
        static_for<Q - 1>([&](auto kc) {
            constexpr int i = decltype(kc)::value + 1;
            const float4 rn = drho[nb.at(L::cx(i), L::cy(i), L::cz(i))];
            static_for<NS>([&](auto tc) {
                constexpr int t = decltype(tc)::value;
                static_for<D>([&](auto dc) {
                    constexpr int d = decltype(dc)::value;
                    F[t][d] += L::wd(i) * comp<L>(i, d) * (double)get4(rn, t);
                });
            });
        });
        double rt = 0.0, j[3] = {0.0, 0.0, 0.0};
        static_for<NS>([&](auto sc) {
            constexpr int s = decltype(sc)::value;
            double r = 0.0, js[3] = {0.0, 0.0, 0.0};
            static_for<Q>([&](auto ic) {
                constexpr int i = decltype(ic)::value;
                const float base = (float)L::wd(i) * p.rho0[s];
                const double f = (double)base +
                                 (double)planes.template plane<L>(s, kern::read_slot<L, PARITY, i>())[kern::read_site<L, PARITY, i>(nb)];
                r += f;
                js[0] += L::cx(i) * f;
                js[1] += L::cy(i) * f;
                js[2] += L::cz(i) * f;
            });
            if (rho_out) rho_out[(size_t)s * p.N + site] = r;
            tot[s] = r;
            rt += r;
            static_for<D>([&](auto dc) {
                constexpr int d = decltype(dc)::value;
                double a = 0.0;
                static_for<NS>([&](auto tc) {
                    constexpr int t = decltype(tc)::value;
                    if constexpr (t != s) a -= (double)p.G[s][t] * F[t][d];
                });
                j[d] += js[d] + 0.5 * r * a;
            });
        });
        static_for<D>([&](auto dc) {
            constexpr int d = decltype(dc)::value;
            if (u_out) u_out[(size_t)d * p.N + site] = j[d] / rt;
            tot[NS + d] = j[d];
        });
    }
#pragma unroll
    for (int k = 0; k < NC; k++) sh[k][threadIdx.x] = tot[k];
    __syncthreads();
    for (int w = kObsBlock / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
#pragma unroll
            for (int k = 0; k < NC; k++) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < NC) partials[(size_t)blockIdx.x * NC + threadIdx.x] = sh[threadIdx.x][0];
}

template <class L, int NS, int PARITY>
__global__ void k_mnatural(const MStepParams p, const MPlanes<const float> planes, float *__restrict__ out)
{
    const int site = blockIdx.x * blockDim.x + threadIdx.x;
    if (site >= p.N) return;
    const int x = site % p.nx, y = (site / p.nx) % p.ny, z = site / (p.nx * p.ny);
    const kern::Nbr nb = make_nbr(p, x, y, z);
    static_for<NS>([&](auto sc) {
        constexpr int s = decltype(sc)::value;
        static_for<L::Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            out[(size_t)(s * L::Q + i) * p.N + site] =
                planes.template plane<L>(s, kern::read_slot<L, PARITY, i>())[kern::read_site<L, PARITY, i>(nb)];
        });
    });
}

template <class L, int NS, int PARITY>
__global__ void k_mgather(const MStepParams p, const MPlanes<const float> planes, const int64_t *__restrict__ sites,
                          int64_t n, double *__restrict__ out)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int site = (int)sites[k];
    const int x = site % p.nx, y = (site / p.nx) % p.ny, z = site / (p.nx * p.ny);
    const kern::Nbr nb = make_nbr(p, x, y, z);
    static_for<NS>([&](auto sc) {
        constexpr int s = decltype(sc)::value;
        static_for<L::Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            const float base = (float)L::wd(i) * p.rho0[s];
            out[(k * NS + s) * L::Q + i] =
                (double)base +
                (double)planes.template plane<L>(s, kern::read_slot<L, PARITY, i>())[kern::read_site<L, PARITY, i>(nb)];
        });
    });
}

template <class L, int NS>
__global__ void k_minit_rest(const MStepParams p, const float *__restrict__ rho, float *__restrict__ pop)
{
    const int site = blockIdx.x * blockDim.x + threadIdx.x;
    if (site >= p.N) return;
    static_for<NS>([&](auto sc) {
        constexpr int s = decltype(sc)::value;
        const float dr = __fsub_rn(rho[(size_t)s * p.N + site], p.rho0[s]);
        static_for<L::Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            pop[(size_t)(s * L::Q + i) * p.N + site] = __fmul_rn((float)L::wd(i), dr);
        });
    });
}

// prof[s][j]: sum of drho^s over the plane j of `axis`, one block per j,
// threads striding over the plane, fixed-order tree reduction.
template <int NS>
__global__ void __launch_bounds__(kObsBlock) k_mprofile(const MStepParams p, int axis, const float4 *__restrict__ drho,
                                                        double *__restrict__ prof)
{
    __shared__ double sh[NS][kObsBlock];
    const int j = blockIdx.x;
    const int n_axis = axis == 0 ? p.nx : (axis == 1 ? p.ny : p.nz);
    const int plane = p.N / n_axis;
    double acc[NS];
#pragma unroll
    for (int s = 0; s < NS; s++) acc[s] = 0.0;
    for (int k = threadIdx.x; k < plane; k += kObsBlock) {
        int site;
        if (axis == 0) site = k * p.nx + j;                                   // k = z ny + y
        else if (axis == 1) site = ((k / p.nx) * p.ny + j) * p.nx + k % p.nx; // k = z nx + x
        else site = j * p.nx * p.ny + k;                                      // k = y nx + x
        const float4 r = drho[site];
#pragma unroll
        for (int s = 0; s < NS; s++) acc[s] += (double)get4(r, s);
    }
#pragma unroll
    for (int s = 0; s < NS; s++) sh[s][threadIdx.x] = acc[s];
    __syncthreads();
    for (int w = kObsBlock / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
#pragma unroll
            for (int s = 0; s < NS; s++) sh[s][threadIdx.x] += sh[s][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < NS) prof[(size_t)threadIdx.x * n_axis + j] = sh[threadIdx.x][0];
}

// One thread per wavevector m = 1 .. n/2: the DFT of every profile at k_m
// (phase 2 pi ((m j) mod n) / n, FP64) and the products of every pair.
template <int NS>
__global__ void k_msf_accumulate(const double *__restrict__ prof, int n, double inv_sites, double *__restrict__ acc)
{
    const int nk = n / 2;
    const int m = blockIdx.x * blockDim.x + threadIdx.x + 1;
    if (m > nk) return;
    double re[NS], im[NS];
#pragma unroll
    for (int s = 0; s < NS; s++) re[s] = im[s] = 0.0;
    for (int j = 0; j < n; j++) {
        double sn, cs;
        sincospi(2.0 * (double)(((long long)m * j) % n) / (double)n, &sn, &cs);
#pragma unroll
        for (int s = 0; s < NS; s++) {
            const double v = prof[(size_t)s * n + j];
            re[s] += v * cs;
            im[s] -= v * sn;
        }
    }
#pragma unroll
    for (int s = 0; s < NS; s++)
#pragma unroll
        for (int t = 0; t < NS; t++)
            acc[((size_t)s * NS + t) * nk + (m - 1)] += (re[s] * re[t] + im[s] * im[t]) * inv_sites;
}

template <class T> MPlanes<T> mplanes(T *pop, int ns, int Q, int N)
{
    MPlanes<T> t{};
    for (int k = 0; k < ns * Q; k++) t.ptr[k] = pop + (size_t)k * (size_t)N;
    return t;
}

inline dim3 msite_block(const MStepParams &p)
{
    const int wx = ((p.nx + 31) / 32) * 32;
    return dim3(p.block_x < wx ? p.block_x : wx, p.block_y);
}
inline dim3 msite_grid(const MStepParams &p, dim3 b)
{
    return dim3((p.nx + b.x - 1) / b.x, (p.ny + b.y - 1) / b.y, p.nz);
}

} // namespace mkern

template <class L, int NS>
cudaError_t MLaunch<L, NS>::density(int parity, const MStepParams &p, const float *pop, float4 *drho, cudaStream_t st)
{
    const dim3 b = mkern::msite_block(p), g = mkern::msite_grid(p, b);
    const auto planes = mkern::mplanes(pop, NS, L::Q, p.N);
    if (p.mom && parity == 0) mkern::k_mdensity<L, NS, 0, true><<<g, b, 0, st>>>(p, planes, drho);
    else if (parity == 0) mkern::k_mdensity<L, NS, 0><<<g, b, 0, st>>>(p, planes, drho);
    else mkern::k_mdensity<L, NS, 1><<<g, b, 0, st>>>(p, planes, drho);
    return cudaGetLastError();
}

template <class L, int NS>
cudaError_t MLaunch<L, NS>::collide(int parity, const MStepParams &p, float *pop, float *pop_out, const float4 *drho,
                                    unsigned *status, cudaStream_t st)
{
    const dim3 b = mkern::msite_block(p), g = mkern::msite_grid(p, b);
    const auto planes = mkern::mplanes(pop, NS, L::Q, p.N);
    const auto out = parity == kStreamPush ? mkern::mplanes(pop_out, NS, L::Q, p.N) : planes;
    const size_t smem = mkern::collide_smem<L, NS>(b.x * b.y);
    // the moment-fed pair runs with two arrays only
    if (p.mom && parity == kStreamPush)
        mkern::k_mcollide<L, NS, kStreamPush, true><<<g, b, 0, st>>>(p, planes, out, drho, status);
    else if (parity == 0) mkern::k_mcollide<L, NS, 0><<<g, b, smem, st>>>(p, planes, out, drho, status);
    else if (parity == 1) mkern::k_mcollide<L, NS, 1><<<g, b, smem, st>>>(p, planes, out, drho, status);
    else mkern::k_mcollide<L, NS, kStreamPush><<<g, b, smem, st>>>(p, planes, out, drho, status);
    return cudaGetLastError();
}

template <class L, int NS>
cudaError_t MLaunch<L, NS>::observables(int parity, const MStepParams &p, const float *pop, const float4 *drho,
                                        double *rho, double *u, double *partials, int *nblocks, cudaStream_t st)
{
    const int nb = (p.N + mkern::kObsBlock - 1) / mkern::kObsBlock;
    *nblocks = nb;
    const auto planes = mkern::mplanes(pop, NS, L::Q, p.N);
    if (parity == 0) mkern::k_mobservables<L, NS, 0><<<nb, mkern::kObsBlock, 0, st>>>(p, planes, drho, rho, u, partials);
    else mkern::k_mobservables<L, NS, 1><<<nb, mkern::kObsBlock, 0, st>>>(p, planes, drho, rho, u, partials);
    return cudaGetLastError();
}

template <class L, int NS>
cudaError_t MLaunch<L, NS>::natural(int parity, const MStepParams &p, const float *pop, float *out, cudaStream_t st)
{
    const int nb = (p.N + 127) / 128;
    const auto planes = mkern::mplanes(pop, NS, L::Q, p.N);
    if (parity == 0) mkern::k_mnatural<L, NS, 0><<<nb, 128, 0, st>>>(p, planes, out);
    else mkern::k_mnatural<L, NS, 1><<<nb, 128, 0, st>>>(p, planes, out);
    return cudaGetLastError();
}

template <class L, int NS>
cudaError_t MLaunch<L, NS>::gather(int parity, const MStepParams &p, const float *pop, const int64_t *sites,
                                   int64_t n, double *out, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    const unsigned nb = (unsigned)((n + 127) / 128);
    const auto planes = mkern::mplanes(pop, NS, L::Q, p.N);
    if (parity == 0) mkern::k_mgather<L, NS, 0><<<nb, 128, 0, st>>>(p, planes, sites, n, out);
    else mkern::k_mgather<L, NS, 1><<<nb, 128, 0, st>>>(p, planes, sites, n, out);
    return cudaGetLastError();
}

template <class L, int NS>
cudaError_t MLaunch<L, NS>::init_rest(const MStepParams &p, const float *rho, float *pop, cudaStream_t st)
{
    mkern::k_minit_rest<L, NS><<<(p.N + 127) / 128, 128, 0, st>>>(p, rho, pop);
    return cudaGetLastError();
}

#define FLBM_MULTI_EXTERN(L)                                                                             \
    extern template struct MLaunch<L, 2>;                                                                \
    extern template struct MLaunch<L, 3>;                                                                \
    extern template struct MLaunch<L, 4>;
FLBM_MULTI_EXTERN(D2Q9)
FLBM_MULTI_EXTERN(D3Q19)
#undef FLBM_MULTI_EXTERN

} // namespace flbm
