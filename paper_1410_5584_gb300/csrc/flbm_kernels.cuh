// flbm_kernels.cuh -- kernel templates of the library, instantiated once per
// (lattice, storage) pair in the inst_*.cu translation units.
//
// The per-step update is the fluctuating two-species lattice Boltzmann
// equation of arXiv 1410.5584 (Sec. V B, Eqs. algorithm and lattice
// finalstep).  Streaming either pushes each site's post-collision f*_i to
// x + c_i in a second array (two-array mode; both arrays stay in the natural
// layout) or updates one array in place with the "AA" pattern:
//   parity 0 (natural layout, A[s][i][x] = f_i(x)):   read A[s][i][x],
//       write the post-collision f*_i(x) to A[s][opp i][x] (same site);
//   parity 1 (swapped layout, A[s][opp i][x] = f*_i(x) of the previous step):
//       read f_i(x) = A[s][opp i][x - c_i], write f*_i(x) to A[s][i][x + c_i].
// After a parity-1 step the array is back in the natural layout.  Every array
// slot is read and written by exactly one thread, so the update is race-free.
#pragma once
#include "flbm_internal.h"
#include "flbm_lattice.cuh"
#include "flbm_launch.h"
#include "flbm_noise.cuh"
#include "flbm_pair.cuh"
#include "flbm_transform.cuh"

namespace flbm {
namespace kern {

constexpr int kObsBlock = 128;


// periodic neighbour indices of one site
struct Nbr {
    int xs[3], ys[3], zs[3];
    int nx, ny;
    __device__ __forceinline__ int at(int dx, int dy, int dz) const
    {
        return (zs[dz + 1] * ny + ys[dy + 1]) * nx + xs[dx + 1];
    }
};

__device__ __forceinline__ Nbr make_nbr(const StepParams &p, int x, int y, int z)
{
    Nbr n;
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

template <class L> __device__ __forceinline__ constexpr float wf(int i) { return (float)L::wd(i); }

// Streaming modes (the PARITY template argument of the step kernels):
//   0: in place, even step: read slot i of the site, write slot opp(i) of the site;
//   1: in place, odd step:  read slot opp(i) of x - c_i, write slot i of x + c_i;
//   kPush: two arrays: read slot i of the site in one array (natural layout),
//          write slot i of x + c_i in the other (natural layout again).
constexpr int kPush = kStreamPush;

// slot and site of the population f_i(site) that the current step reads
template <class L, int PARITY, int I> __device__ __forceinline__ constexpr int read_slot()
{
    return PARITY == 1 ? L::opp(I) : I;
}
template <class L, int PARITY, int I> __device__ __forceinline__ unsigned read_site(const Nbr &nb)
{
    if constexpr (PARITY != 1) return (unsigned)nb.at(0, 0, 0);
    else return (unsigned)nb.at(-L::cx(I), -L::cy(I), -L::cz(I));
}
// slot and site where the post-collision f*_i(site) is written
template <class L, int PARITY, int I> __device__ __forceinline__ constexpr int write_slot()
{
    return PARITY == 0 ? L::opp(I) : I;
}
template <class L, int PARITY, int I> __device__ __forceinline__ unsigned write_site(const Nbr &nb)
{
    if constexpr (PARITY == 0) return (unsigned)nb.at(0, 0, 0);
    else return (unsigned)nb.at(L::cx(I), L::cy(I), L::cz(I));
}
// array index of the population f_i(site) that the current step reads
template <class L, int PARITY, int I>
__device__ __forceinline__ size_t read_index(const Nbr &nb, size_t NN, int s)
{
    return pop_index(s, read_slot<L, PARITY, I>(), read_site<L, PARITY, I>(nb), NN);
}

// Where a slot's words are (pop_index: the two species side by side): pair(j,
// site) is species A's word of slot j at site, followed by species B's;
// word(s, j, site) is species s's.  FlatPlanes computes it from the array
// start; PlaneTable carries the Q slot planes' starts in the kernel's parameter
// space, so an access is a uniform pointer plus a site offset.
template <class T> struct FlatPlanes {
    T *pop;
    size_t N;
    __device__ __forceinline__ T *pair(int j, size_t site) const { return pop + pop_index(0, j, site, N); }
    __device__ __forceinline__ T *word(int s, int j, size_t site) const { return pop + pop_index(s, j, site, N); }
};
template <class T> struct PlaneTable {
    T *ptr[kMaxQ]; // slot j's pairs
    __device__ __forceinline__ T *pair(int j, size_t site) const { return ptr[j] + 2 * site; }
    __device__ __forceinline__ T *word(int s, int j, size_t site) const { return ptr[j] + 2 * site + s; }
};

// ---------------------------------------------------------------------------
// density pass
// ---------------------------------------------------------------------------
// densities (rho_A, rho_B) of one site from its pre-collision populations
// the pre-collision deviations of both species at a site, one pair load a slot
template <class L, class S, int PARITY, class P>
__device__ __forceinline__ void load_site(const P &planes, const Nbr &nb, float (&d)[2][L::Q])
{
    static_for<L::Q>([&](auto ic) {
        constexpr int i = decltype(ic)::value;
        const float2 v = S::load_pair(planes.pair(read_slot<L, PARITY, i>(), read_site<L, PARITY, i>(nb)));
        d[0][i] = v.x;
        d[1][i] = v.y;
    });
}

template <class L, class S, int PARITY, class P>
__device__ __forceinline__ float2 site_density(const StepParams &p, const P &planes, const Nbr &nb)
{
    float r[2], d[2][L::Q];
    load_site<L, S, PARITY>(planes, nb, d);
    static_for<2>([&](auto sc) {
        constexpr int s = decltype(sc)::value;
        float m[L::Q];
        // the collide step computes its own density with this same expression
        Transform<L>::forward(d[s], m);
        r[s] = p.rho0[s] + m[0];
    });
    return make_float2(r[0], r[1]);
}

template <class L, class S, int PARITY>
__global__ void __launch_bounds__(kSiteBlockMax) k_density(const StepParams p,
                                                           const PlaneTable<const typename S::T> planes,
                                                           float2 *__restrict__ rho)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= p.nx || y >= p.yn) return;
    const Nbr nb = make_nbr(p, x, y + p.y0, blockIdx.z + p.z0);
    rho[nb.at(0, 0, 0)] = site_density<L, S, PARITY>(p, planes, nb);
}

// The density pass of a full-relaxation step (every lambdabar_a = 1): besides
// rho it stores each species' density deviation m_0 and momentum m_1..m_D, the
// only moments of the old populations that the collision then uses (Eq.
// algorithm with lambdabar_a = 1), so that the collide reads these 2 (D + 1)
// floats instead of 2 Q populations.  Same expressions as site_density and the
// collide's own transform, so the results are bitwise those of the
// population-reading collide.  Returns the densities; writes p.mom.
template <class L, class S, int PARITY, class P>
__device__ __forceinline__ float2 site_moments_to(const StepParams &p, const P &planes, const Nbr &nb,
                                                  float (&mm)[2][L::D + 1])
{
    float r[2], d[2][L::Q];
    load_site<L, S, PARITY>(planes, nb, d);
    static_for<2>([&](auto sc) {
        constexpr int s = decltype(sc)::value;
        float m[L::Q];
        Transform<L>::forward(d[s], m);
        r[s] = p.rho0[s] + m[0];
        static_for<L::D + 1>([&](auto ac) {
            constexpr int a = decltype(ac)::value;
            mm[s][a] = m[a];
        });
    });
    return make_float2(r[0], r[1]);
}

template <class L, class S, int PARITY, class P>
__device__ __forceinline__ float2 site_moments(const StepParams &p, const P &planes, const Nbr &nb)
{
    const size_t site = (size_t)nb.at(0, 0, 0);
    float mm[2][L::D + 1];
    const float2 r = site_moments_to<L, S, PARITY>(p, planes, nb, mm);
    static_for<2 * (L::D + 1)>([&](auto qc) {
        constexpr int q = decltype(qc)::value;
        p.mom[(size_t)q * (size_t)p.N + site] = mm[q / (L::D + 1)][q % (L::D + 1)];
    });
    return r;
}

template <class L, class S, int PARITY>
__global__ void __launch_bounds__(kSiteBlockMax) k_moments(const StepParams p,
                                                           const PlaneTable<const typename S::T> planes,
                                                           float2 *__restrict__ rho)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= p.nx || y >= p.yn) return;
    const Nbr nb = make_nbr(p, x, y + p.y0, blockIdx.z + p.z0);
    rho[nb.at(0, 0, 0)] = site_moments<L, S, PARITY>(p, planes, nb);
}

// ---------------------------------------------------------------------------
// fused force + moment collision + noise + streaming
// ---------------------------------------------------------------------------
// Where a collide reads the densities of its force stencil and, moment-fed,
// the moments m_0 .. m_D of its own site: the whole-box density field and
// moment planes.  COHERENT: read the density field through L2 only
// (ld.global.cg), for a field written earlier in the same launch by other
// thread blocks.
template <bool COHERENT> struct BoxSrc {
    const float2 *rho;
    const float *mom;
    size_t N, site;
    __device__ __forceinline__ float2 rho_at(const Nbr &nb, int dx, int dy, int dz) const
    {
        const float2 *rp = rho + nb.at(dx, dy, dz);
        return COHERENT ? __ldcg(rp) : __ldg(rp);
    }
    __device__ __forceinline__ float mom_at(int plane) const { return __ldg(mom + (size_t)plane * N + site); }
};

// Stored words go out with a plain store, or with the streaming hint (evict
// first: written once, not read again by this launch).
template <bool CS, class T> __device__ __forceinline__ void put_word(T *p, T v)
{
    if constexpr (CS) __stcs(p, v);
    else *p = v;
}
template <bool CS, class S> __device__ __forceinline__ void put_pair(typename S::T *p, typename S::T a, typename S::T b)
{
    if constexpr (CS) S::store_pair_cs(p, a, b);
    else S::store_pair(p, a, b);
}

// The end of a full-relaxation collision for both species at once (packed
// pairs, lane lo A, hi B): y_i = sum_a T_ai mu_a, the stored words of the
// moving populations (w_i y_i, rounded by the storage format), the rest
// population closing each species' mass on what those words hold (so the
// rounding of their stores cannot leak mass), then the stores.
template <class L, class S, int PARITY, bool STORE, bool CS, class P, class Hook2>
__device__ __forceinline__ void full_relaxation_stores(const StepParams &p, const P &out, const Nbr &nb,
                                                       const F2 (&mu2)[L::Q], Hook2 &&before_stores, bool live)
{
    constexpr int Q = L::Q;
    F2 y2[Q];
    Transform<L>::backward(mu2, y2);
    typename S::T word[2][Q];
    F2 fo2[Q];
    static_for<Q - 1>([&](auto kc) {
        constexpr int i = decltype(kc)::value + 1;
        const F2 wy = mul2(splat2((float)L::wd(i)), y2[i]); // __fmul_rn(w_i, y_i) per lane
        word[0][i] = S::encode(wy.lo(), (float)L::wd(i) * p.rho0[0]);
        word[1][i] = S::encode(wy.hi(), (float)L::wd(i) * p.rho0[1]);
        fo2[i] = F2(S::decode(word[0][i], 0.0f), S::decode(word[1][i], 0.0f));
    });
    fo2[0] = F2(0);
    const F2 rest = Transform<L>::rest_closing_mass(fo2, mu2[0]);
    word[0][0] = S::encode(rest.lo(), (float)L::wd(0) * p.rho0[0]);
    word[1][0] = S::encode(rest.hi(), (float)L::wd(0) * p.rho0[1]);
    before_stores();
    if (STORE && live) {
        static_for<Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            put_pair<CS, S>(out.pair(write_slot<L, PARITY, i>(), write_site<L, PARITY, i>(nb)), word[0][i], word[1][i]);
        });
    }
}

// Force + moment collision + noise + streaming of one site, reading the
// density stencil (and, MOM, its own moments) from `src`.  STORE = false
// computes without writing (an idle lane of a partial warp).  after_loads()
// runs once the population loads are issued; returning false abandons the
// site.  before_stores() runs once every read of the site is done, just
// before its first store.  CS: store with the streaming hint.  live = false
// does what STORE = false does, decided at run time (every lane of a warp
// then runs the same code).
template <class L, class S, int PARITY, bool STORE, bool FULL, bool MOM, bool CS, class P, class Src, class Hook,
          class Hook2>
__device__ __forceinline__ void site_collide_src(const StepParams &p, const P &planes, const P &out, const Src &src,
                                                 unsigned *__restrict__ status, const Nbr &nb, Hook &&after_loads,
                                                 Hook2 &&before_stores, bool live = true);

template <class L, class S, int PARITY, bool COHERENT_RHO, bool STORE = true, bool FULL = false, bool MOM = false,
          class P, class Hook = bool (*)()>
__device__ __forceinline__ void site_collide(const StepParams &p, const P &planes, const P &out,
                                             const float2 *__restrict__ rho, unsigned *__restrict__ status,
                                             const Nbr &nb, Hook &&after_loads)
{
    const BoxSrc<COHERENT_RHO> src{rho, p.mom, (size_t)p.N, (size_t)nb.at(0, 0, 0)};
    site_collide_src<L, S, PARITY, STORE, FULL, MOM, false>(p, planes, out, src, status, nb, after_loads, [] {});
}

template <class L, class S, int PARITY, bool STORE, bool FULL, bool MOM, bool CS, class P, class Src, class Hook,
          class Hook2>
__device__ __forceinline__ void site_collide_src(const StepParams &p, const P &planes, const P &out, const Src &src,
                                                 unsigned *__restrict__ status, const Nbr &nb, Hook &&after_loads,
                                                 Hook2 &&before_stores, bool live)
{
    constexpr int Q = L::Q, D = L::D;
    static_assert(!MOM || FULL, "the moment-fed collide needs full relaxation");
    const int site = nb.at(0, 0, 0);

    // 1. moments of both species (Eq. modes-discrete), density rho = rhobar.
    // All loads are issued first; `after_loads` runs while they are in flight.
    // MOM: the density pass stored m_0 .. m_D (k_moments), and with full
    // relaxation no other moment of the old populations enters the update.
    float m[2][Q], rs[2];
    if constexpr (MOM) {
        static_for<2>([&](auto sc) {
            constexpr int s = decltype(sc)::value;
            static_for<D + 1>([&](auto ac) {
                constexpr int a = decltype(ac)::value;
                m[s][a] = src.mom_at(s * (D + 1) + a);
            });
        });
        if (!after_loads()) return;
        rs[0] = p.rho0[0] + m[0][0];
        rs[1] = p.rho0[1] + m[1][0];
    } else {
        float d[2][Q];
        load_site<L, S, PARITY>(planes, nb, d);
        if (!after_loads()) return;
        static_for<2>([&](auto sc) {
            constexpr int s = decltype(sc)::value;
            Transform<L>::forward(d[s], m[s]);
            rs[s] = p.rho0[s] + m[s][0];
        });
    }

    // 2. Shan-Chen force from the other species' neighbour densities (Eq. FORCESTRUCTURE)
    float acc[2][3] = {{0.0f, 0.0f, 0.0f}, {0.0f, 0.0f, 0.0f}};
    if constexpr (FULL) {
        // both species at once: lane lo sums c w rho_A (species B's force),
        // lane hi c w rho_B (species A's), the same fused multiply-adds in the
        // same order as the scalar form below
        F2 ab[3] = {F2(0), F2(0), F2(0)};
        static_for<Q - 1>([&](auto kc) {
            constexpr int i = decltype(kc)::value + 1;
            constexpr float wi = (float)L::wd(i);
            const float2 rn = src.rho_at(nb, L::cx(i), L::cy(i), L::cz(i));
            const F2 r2(rn.x, rn.y);
            static_for<D>([&](auto dc) {
                constexpr int d = decltype(dc)::value;
                constexpr int cd = comp<L>(i, d);
                if constexpr (cd != 0) ab[d] = fma2(splat2((float)cd * wi), r2, ab[d]);
            });
        });
        static_for<D>([&](auto dc) {
            constexpr int d = decltype(dc)::value;
            acc[0][d] = ab[d].hi() * -p.G;
            acc[1][d] = ab[d].lo() * -p.G;
        });
    } else {
        static_for<Q - 1>([&](auto kc) {
            constexpr int i = decltype(kc)::value + 1;
            constexpr float wi = (float)L::wd(i);
            const float2 rn = src.rho_at(nb, L::cx(i), L::cy(i), L::cz(i));
            const float ra = rn.x, rb = rn.y;
            static_for<D>([&](auto dc) {
                constexpr int d = decltype(dc)::value;
                constexpr int cd = comp<L>(i, d);
                if constexpr (cd != 0) {
                    constexpr float cw = (float)cd * wi;
                    acc[0][d] = __fmaf_rn(cw, rb, acc[0][d]);
                    acc[1][d] = __fmaf_rn(cw, ra, acc[1][d]);
                }
            });
        });
        static_for<D>([&](auto dc) {
            constexpr int d = decltype(dc)::value;
            acc[0][d] *= -p.G;
            acc[1][d] *= -p.G;
        });
    }

    // 3. baricentric velocity with the half-force shift (Eq. lattice finalstep).
    // Here and in step 5 every rounding is explicit, so that each kernel that
    // inlines this function gives the same bits.
    const float rt = __fadd_rn(rs[0], rs[1]);
    const float irt = __frcp_rn(rt);
    float u[3] = {0.0f, 0.0f, 0.0f};
    static_for<D>([&](auto dc) {
        constexpr int d = decltype(dc)::value;
        const float ra = __fmaf_rn(rs[0], acc[0][d], __fmul_rn(rs[1], acc[1][d]));
        u[d] = __fmul_rn(__fmaf_rn(0.5f, ra, __fadd_rn(m[0][1 + d], m[1][1 + d])), irt);
    });
    if (STORE && live && (!(rs[0] > 0.0f) || !(rs[1] > 0.0f) || !isfinite(rt))) atomicOr(status, kStatusNonFinite);

    // 4. Gaussians scaled by the amplitudes of Eq. new-noise (local or reference
    // densities): sqrt(rho rho'/rho_t) for the shared momentum noise, sqrt(rho^s)
    // for the other modes of species s (their per-mode factors are in cxi).
    // Square roots as x rsqrt(x): the densities are positive on every valid state
    // (a non-positive one has already raised the status flag).
    // LATE (the general D3Q19 instance): only species 0's Philox block 0 (the
    // shared momentum noise, modes 1 .. 3, and modes 4 .. 6) is drawn here, and
    // each species draws the rest just before its own relaxation (step 6),
    // which keeps them out of the registers meanwhile.  Measured at 256^3 with two arrays: 1.45 -> 1.13 ms
    // for that instance, while the full-relaxation and D2Q9 instances are ~3 %
    // faster drawing everything here.
    constexpr bool LATE = L::Q == 19 && !FULL;
    const uint32_t nstep = p.step_dev ? __ldg(p.step_dev) + p.step : p.step; // noise counter of this step
    const float n0 = p.noise_ref ? p.rho0[0] : rs[0];
    const float n1 = p.noise_ref ? p.rho0[1] : rs[1];
    const float hm = n0 * n1 * __frcp_rn(n0 + n1);
    const float amp_j = p.noise_amp_j * (hm * rsqrtf(hm));
    float g0[Q], g1[Q];
    if constexpr (LATE) {
        draw_gaussians<L, 0, 0, 1>((uint32_t)site, nstep, p.key0, p.key1, amp_j, n0 * rsqrtf(n0), g0);
    } else {
        draw_gaussians<L, 0>((uint32_t)site, nstep, p.key0, p.key1, amp_j, n0 * rsqrtf(n0), g0);
        draw_gaussians<L, 1>((uint32_t)site, nstep, p.key0, p.key1, amp_j, n1 * rsqrtf(n1), g1);
    }

    float X[Q];
    Closure<L>::eq(u, X);
    if constexpr (FULL) {
        // 5'. Full relaxation: the momentum modes and the forcing moments of both
        // species in packed pairs (lane lo A, hi B), the same update as steps 5-6
        // below: R = lambdabar_d (rho u - j) + (1 - lambdabar_d/2) rho a + xi,
        // rho v = j + R/2 (or v = j/rho + a/2), j* = j + R.
        const F2 rs2(rs[0], rs[1]);
        const F2 irs2(__frcp_rn(rs[0]), __frcp_rn(rs[1]));
        const F2 lrs2 = mul2(splat2(p.lam_d), rs2), hrs2 = mul2(splat2(p.hlam_d), rs2);
        const F2 nlam = splat2(-p.lam_d), half = splat2(0.5f);
        F2 acc2[3], v2[3], mu2[Q];
        static_for<D>([&](auto dc) {
            constexpr int d = decltype(dc)::value;
            constexpr int a = 1 + d;
            constexpr float invN = (float)(1.0 / L::Nd(a));
            acc2[d] = F2(acc[0][d], acc[1][d]);
            const F2 m2(m[0][a], m[1][a]);
            const F2 R2 = fma2(lrs2, splat2(u[d]), fma2(nlam, m2, fma2(hrs2, acc2[d], F2(g0[a], -g0[a]))));
            if (p.force_velocity) v2[d] = fma2(m2, irs2, mul2(half, acc2[d]));
            else v2[d] = mul2(fma2(half, R2, m2), irs2);
            mu2[a] = mul2(splat2(invN), m2 + R2);
        });
        // 6'. mu_a = cxi g_a (+ rho (ceq X_a + cphi Y_a) on the transport modes);
        // then the back-projection, the weights and the mass balance
        F2 Y2[Q];
        ClosurePair<L>::force(acc2, v2, Y2);
        mu2[0] = F2(m[0][0], m[1][0]);
        static_for<Q - D - 1>([&](auto kc) {
            constexpr int a = decltype(kc)::value + D + 1;
            F2 t = mul2(pair2(p.pair_xi[a]), F2(g0[a], g1[a]));
            if constexpr (a < Closure<L>::kGhost)
                t = fma2(rs2, fma2(pair2(p.pair_eq[a]), splat2(X[a]), mul2(pair2(p.pair_phi[a]), Y2[a])), t);
            mu2[a] = t;
        });
        full_relaxation_stores<L, S, PARITY, STORE, CS>(p, out, nb, mu2, before_stores, live);
        return;
    }

    // 5. momentum modes: common rate, opposite noise; species velocity for Phi
    float v[2][3] = {{0.0f, 0.0f, 0.0f}, {0.0f, 0.0f, 0.0f}};
    static_for<2>([&](auto sc) {
        constexpr int s = decltype(sc)::value;
        const float irs = __frcp_rn(rs[s]);
        const float lrs = __fmul_rn(p.lam_d, rs[s]), hrs = __fmul_rn(p.hlam_d, rs[s]);
        static_for<D>([&](auto dc) {
            constexpr int d = decltype(dc)::value;
            constexpr int a = 1 + d;
            const float xi = s == 0 ? g0[a] : -g0[a];
            // the operations of the packed form of step 5', one lane at a time
            const float R = __fmaf_rn(lrs, u[d], __fmaf_rn(-p.lam_d, m[s][a], __fmaf_rn(hrs, acc[s][d], xi)));
            v[s][d] = p.force_velocity ? __fmaf_rn(m[s][a], irs, __fmul_rn(0.5f, acc[s][d]))
                                       : __fmul_rn(__fmaf_rn(0.5f, R, m[s][a]), irs);
            m[s][a] = __fadd_rn(m[s][a], R);
        });
    });

    // 6. transport and ghost modes, then back-projection and streaming.  With
    // mu_a = m*_a / N_a: m*_a = m_a + lambdabar_a (m^eq_a - m_a) + (1 - lambdabar_a/2)
    // Phi_a + xi_a, i.e. mu_a = cm m_a + rho (ceq X_a + cphi Y_a) + cxi g_a, and for
    // the ghost modes (m^eq = Phi = 0) mu_a = cm m_a + cxi g_a.  The stored
    // words of species A wait for those of B, so that each slot's pair goes
    // out in one store.
    typename S::T words[2][Q];
    static_for<2>([&](auto sc) {
        constexpr int s = decltype(sc)::value;
        typename S::T(&word)[Q] = words[s];
        float g[Q];
        if constexpr (!LATE) {
            static_for<Q>([&](auto ac) {
                constexpr int a = decltype(ac)::value;
                g[a] = s == 0 ? g0[a] : g1[a];
            });
        } else if constexpr (s == 0) {
            draw_gaussians<L, 0, 1>((uint32_t)site, nstep, p.key0, p.key1, amp_j, n0 * rsqrtf(n0), g);
            static_for<7>([&](auto ac) { // the non-momentum modes of block 0, drawn in step 4
                constexpr int a = decltype(ac)::value;
                if constexpr (a > D && a < Q) g[a] = g0[a];
            });
        } else {
            draw_gaussians<L, 1>((uint32_t)site, nstep, p.key0, p.key1, amp_j, n1 * rsqrtf(n1), g);
        }
        if (p.ghost_noise) {
            // Population-space noise: g_a = N_a^(-1/2) sum_i T_ai (w_i rho^s(r + c_i))^(1/2) eta_i,
            // which has the variance rho N_a / N_a = rho of the scaled mode draws where
            // the density is uniform, and the off-diagonal covariances of a density
            // gradient elsewhere (cxi then supplies (2 lb - lb^2) N_a mu as usual).
            float eta[Q], xs[Q], pr[Q];
            population_gaussians<Q>((uint32_t)site, nstep, 2u + (uint32_t)s, p.key0, p.key1, eta);
            static_for<Q>([&](auto ic) {
                constexpr int i = decltype(ic)::value;
                float ri = rs[s];
                if constexpr (i > 0) {
                    const float2 rn = src.rho_at(nb, L::cx(i), L::cy(i), L::cz(i));
                    ri = s == 0 ? rn.x : rn.y;
                }
                if (p.noise_ref) ri = p.rho0[s];
                xs[i] = sqrtf((float)L::wd(i) * ri) * eta[i];
            });
            Transform<L>::forward(xs, pr);
            static_for<Q - D - 1>([&](auto kc) {
                constexpr int a = decltype(kc)::value + D + 1;
                g[a] = pr[a] * __frsqrt_rn((float)L::Nd(a));
            });
        }
        float Y[Q];
        Closure<L>::force(acc[s], v[s], Y);
        float mu[Q], fo[Q];
        mu[0] = m[s][0];
        static_for<D>([&](auto dc) {
            constexpr int a = decltype(dc)::value + 1;
            constexpr float invN = (float)(1.0 / L::Nd(a));
            mu[a] = invN * m[s][a];
        });
        static_for<Q - D - 1>([&](auto kc) {
            constexpr int a = decltype(kc)::value + D + 1;
            // FULL: every cm is zero (lambdabar_a = 1), so the old moment drops out
            // exactly and its projection is never formed
            float t;
            if constexpr (FULL) t = p.cxi[s][a] * g[a];
            else t = fmaf(p.cm[s][a], m[s][a], p.cxi[s][a] * g[a]);
            if constexpr (a < Closure<L>::kGhost) t = fmaf(rs[s], fmaf(p.ceq[s][a], X[a], p.cphi[s][a] * Y[a]), t);
            mu[a] = t;
        });
        // delta*_i = w_i y_i with y_i = sum_a T_ai mu_a, the weight folded into the store
        float y[Q];
        Transform<L>::backward(mu, y);
        // Mass balance: the moving populations are encoded first and replaced by
        // the deviations their stored words will load as; the rest population
        // then takes m0 minus what they hold, so the rounding of their stores
        // cannot leak mass.
        static_for<Q - 1>([&](auto kc) {
            constexpr int i = decltype(kc)::value + 1;
            constexpr float wi = (float)L::wd(i);
            const float base = wi * p.rho0[s];
            word[i] = S::encode_w(wi, y[i], base);
            fo[i] = S::decode(word[i], base);
        });
        word[0] = S::encode(Transform<L>::rest_closing_mass(fo, m[s][0]), (float)L::wd(0) * p.rho0[s]);
    });
    before_stores();
    if (STORE && live) {
        static_for<Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            put_pair<CS, S>(out.pair(write_slot<L, PARITY, i>(), write_site<L, PARITY, i>(nb)), words[0][i], words[1][i]);
        });
    }
}

// planes: the slot planes read; out: the slot planes written (the same table
// for the in-place modes, the other array for kPush).  MOM: full relaxation
// fed by the moment planes of k_moments instead of the populations.  Register
// limits, measured: D3Q19 full relaxation 80 (six blocks an SM, 2 % faster at
// 256^3 than its own 96 despite a 24-byte spill), moment-fed 96 (five blocks,
// no spill, 2 % faster than at 80), D3Q19 general 128 (it asks for 176
// otherwise); D2Q9, whose 18 loads a site leave it short of loads in flight,
// 64 and 80 (eight and six blocks, 5-6 % faster at 2048^2, no spill).
template <class L, class S, int PARITY, bool FULL, bool MOM = false>
__global__ void __launch_bounds__(kSiteBlockMax, FULL ? (L::Q == 9 ? 8 : (MOM ? 5 : 6)) : (L::Q == 9 ? 6 : 4)) k_collide(const StepParams p, const PlaneTable<typename S::T> planes,
                                                           const PlaneTable<typename S::T> out,
                                                           const float2 *__restrict__ rho,
                                                           unsigned *__restrict__ status)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= p.nx || y >= p.yn) return;
    const Nbr nb = make_nbr(p, x, y + p.y0, blockIdx.z + p.z0);
    site_collide<L, S, PARITY, false, true, FULL, MOM>(p, planes, out, rho, status, nb, [] { return true; });
}

// True when every non-conserved mode relaxes fully (lambdabar_a = 1, so cm = 0
// exactly for both species): the collide can skip those modes' projections.
template <class L> inline bool full_relaxation(const StepParams &p)
{
    if (p.general_collide) return false;
    for (int s = 0; s < 2; s++)
        for (int a = L::D + 1; a < L::Q; a++)
            if (p.cm[s][a] != 0.0f) return false;
    return true;
}

// ---------------------------------------------------------------------------
// One whole step in one persistent launch.  The lattice is cut into slices
// along its outermost axis (z in 3D, y in 2D) and each slice into warp tiles of
// 32 sites along x (T tiles per slice).  Two kinds of work:
//   D(k, t): densities of tile t of slice k;  C(j, t): collide tile t of slice j,
//   which needs the densities of slices j-1, j, j+1.
// Work items, in order:
//   prologue: D(k, t) for k in {S-1, 0, 1, ..., L}   ((L+2) T items)
//   main    : item (j, t) = D(j+L+1, t) (when j+L+1 <= S-2) then C(j, t)   (S T items)
// so the densities run L slices ahead of the collisions.  L is the smallest lag
// that keeps the density work of a slice ahead of the window of items in flight
// (one per warp of the grid); the populations a D item pulls from HBM are then
// re-read from L2 by the C item of the same slice L+1 slices later, so each
// population crosses HBM once each way per step.
// Warp w takes items w, w + W, w + 2W, ...  (W warps, all resident: cooperative
// launch).  A C part checks per-slice counters of finished D tiles; an item only
// waits on items of smaller index, which resident warps already own, so the
// waits always end (and are bounded in time anyway: a timeout sets a status bit
// and the warp returns).  In-place streaming stays race-free: the slots a site's
// C part reads and writes are touched by no other C part, and a D part reads
// them only before the C part of that site runs.
// ---------------------------------------------------------------------------
struct PipeArgs {
    unsigned *done;   // finished D tiles per slice (zero at launch)
    int slices, tiles_per_slice, tiles_per_row, lag;
    int prologue, total;
    unsigned target;            // D tiles a slice needs before its neighbours' C parts may run
    unsigned long long wait_ns; // give-up time of one dependency wait
};

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned load_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned load_relaxed(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void fence_acq_rel() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

__device__ __forceinline__ void red_add_relaxed(unsigned *p, unsigned v)
{
    asm volatile("red.relaxed.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// item -> (D slice or -1, C slice or -1, tile)
__device__ __forceinline__ void decode_item(const PipeArgs &a, int item, int &dslice, int &cslice, int &tile)
{
    const int S = a.slices, T = a.tiles_per_slice;
    if (a.lag < 0) { // few slices: all densities, then all collisions
        const int q = item / T;
        tile = item - q * T;
        dslice = q < S ? q : -1;
        cslice = q < S ? -1 : q - S;
        return;
    }
    if (item < a.prologue) {
        const int q = item / T;
        tile = item - q * T;
        dslice = q == 0 ? S - 1 : q - 1;
        cslice = -1;
        return;
    }
    const int r = item - a.prologue;
    const int j = r / T;
    tile = r - j * T;
    cslice = j;
    dslice = j + a.lag + 1 <= S - 2 ? j + a.lag + 1 : -1;
}

template <class L, class S, int PARITY>
__global__ void __launch_bounds__(128) k_step_fused(const StepParams p, typename S::T *__restrict__ pop,
                                                    float2 *__restrict__ rho, unsigned *__restrict__ status,
                                                    const PipeArgs a)
{
    const FlatPlanes<typename S::T> planes{pop, (size_t)p.N};
    const int lane = threadIdx.x & 31;
    const int W = (int)((gridDim.x * blockDim.x) >> 5);
    for (int item = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); item < a.total; item += W) {
        int dslice, cslice, tile;
        decode_item(a, item, dslice, cslice, tile);
        // dependency counters of the C part, read early (relaxed); the fence
        // issued after the population loads gives them acquire semantics
        unsigned c0 = 0, c1 = 0, c2 = 0;
        int nb3[3] = {0, 0, 0};
        if (cslice >= 0) {
            const int Sl = a.slices;
            nb3[0] = cslice == 0 ? Sl - 1 : cslice - 1;
            nb3[1] = cslice;
            nb3[2] = cslice == Sl - 1 ? 0 : cslice + 1;
            if (lane == 0) {
                c0 = load_relaxed(a.done + nb3[0]);
                c1 = load_relaxed(a.done + nb3[1]);
                c2 = load_relaxed(a.done + nb3[2]);
            }
        }
        // ---- D part
        if (dslice >= 0) {
            int y, z;
            if (L::D == 3) {
                z = dslice;
                y = tile / a.tiles_per_row;
            } else {
                z = 0;
                y = dslice;
            }
            const int x = (tile - (L::D == 3 ? y * a.tiles_per_row : 0)) * 32 + lane;
            if (x < p.nx) {
                const Nbr nb = make_nbr(p, x, y, z);
                rho[nb.at(0, 0, 0)] = site_density<L, S, PARITY>(p, planes, nb);
            }
            __syncwarp();
            if (cslice < 0 && lane == 0) { // no C part to carry the signal: publish now
                fence_acq_rel();
                red_add_relaxed(a.done + dslice, 1u);
            }
        }
        // ---- C part
        if (cslice >= 0) {
            int y, z;
            if (L::D == 3) {
                z = cslice;
                y = tile / a.tiles_per_row;
            } else {
                z = 0;
                y = cslice;
            }
            const int x0 = (tile - (L::D == 3 ? y * a.tiles_per_row : 0)) * 32;
            const bool active = x0 + lane < p.nx;
            const int x = active ? x0 + lane : p.nx - 1; // idle lanes compute a real site without storing
            const Nbr nb = make_nbr(p, x, y, z);
            auto after_loads = [&]() -> bool {
                int ok = 1;
                if (lane == 0) {
                    // release this item's densities; acquire the counters read above
                    fence_acq_rel();
                    if (dslice >= 0) red_add_relaxed(a.done + dslice, 1u);
                    if (c0 < a.target || c1 < a.target || c2 < a.target) {
                        const unsigned long long t0 = global_ns();
                        for (int k = 0; k < 3 && ok; k++)
                            while (load_acquire(a.done + nb3[k]) < a.target) {
                                if (global_ns() - t0 > a.wait_ns) {
                                    ok = 0;
                                    break;
                                }
                                __nanosleep(64);
                            }
                        if (!ok) atomicOr(status, kStatusTimeout);
                    }
                }
                return __shfl_sync(0xffffffffu, ok, 0) != 0;
            };
            bool alive = true;
            if (active) {
                site_collide<L, S, PARITY, true, true>(p, planes, planes, rho, status, nb,
                                                       [&] { return alive = after_loads(); });
            } else {
                site_collide<L, S, PARITY, true, false>(p, planes, planes, rho, status, nb,
                                                        [&] { return alive = after_loads(); });
            }
            if (!__shfl_sync(0xffffffffu, alive ? 1 : 0, 0)) return; // a wait gave up: the host sees the status bit
        }
    }
}

// ---------------------------------------------------------------------------
// Pipelined step with two arrays: one persistent launch per step in which the
// density pass of the force stencil reads each population once from HBM and
// the collide writes each once, with nothing else of the step going to HBM.
// The box is cut into slices along its outermost axis (z in 3D, y in 2D) and
// each slice into warp tiles of 32 sites along x (T per slice).  Work items,
// in order:
//   prologue: D(k, t) for k = S-1, 0, 1, ..., L                 ((L+2) T items)
//   main    : item (j, t) = D(j+L+1, t) if j+L+1 <= S-2, then C(j, t)  (S T items)
// D(k, t) reads the populations of tile t of slice k (natural layout) and
// stores the densities, and with MOM the moments m_0 .. m_D of both species,
// into a ring of slice slots that stays in L2; C(j, t) collides tile t of slice
// j from those slots (own moments, the density stencil of slices j-1 .. j+1)
// and pushes f* into the other array.  Without MOM (some rate below 1) the
// collide reads its own populations again, from L2 when the lag is short.
// Slices 0 and S-1 keep slots 0 and 1 for the whole step (the periodic wrap
// needs them at both ends); slice k of 1 .. S-2 uses slot 2 + (k-1) mod R.
// Dependencies, counted per row of a slice: C(j) needs the D tiles of the
// neighbouring rows of slices j-1, j, j+1; D(k) reuses the slot of slice k-R
// and waits until the C tiles that read it (slices k-R-1 .. k-R+1) are done.
// Items are drawn dynamically from interleaved work lanes (see kPipeLanes),
// in increasing order within each lane.  Every wait is on an item of smaller
// index; the smallest item that waits can only wait on a smaller one that
// is being processed or is the next of its lane, whose resident warps
// (cooperative launch) all hold smaller items still, so every wait ends; each
// is also bounded in time (the warp sets a status bit and returns).  The
// per-site arithmetic is that of the two-kernel step, so the update is the
// same.
// ---------------------------------------------------------------------------
struct PipeRing {
    float2 *rho;       // slots x sp: (rho_A, rho_B) of the slice's sites
    float *mom;        // slots x 2 (D + 1) planes x sp (MOM only)
    unsigned *dcount;  // finished D tiles per unit (zero at launch)
    unsigned *ccount;  // finished C tiles per unit (zero at launch)
    int R;             // ring slots of slices 1 .. S-2
    int sp;            // sites per slice
    int slices, rows, tiles_per_slice, tiles_per_row, lag, prologue, total; // tiles: kPipeTiles warp tiles each
    unsigned long long mul_T, mul_row, mul_R; // exact dividers by tiles_per_slice, tiles_per_row, R
    unsigned shift_T, shift_row, shift_R;
    unsigned target;            // tiles a unit needs before its readers run (tiles_per_row; one more tests timeouts)
    unsigned long long wait_ns; // give-up time of one dependency wait
    unsigned *next;             // kPipeLanes work counters, kPipeStride words apart (zero at launch)
};

// Items are handed out dynamically, in order within each of kPipeLanes
// interleaved lanes (lane c: items c, c + kPipeLanes, ...); warp w draws from
// lane w mod kPipeLanes, so warps that run slower take fewer items instead of
// holding back the ones that depend on theirs, and the lanes' counters sit on
// separate cache lines.
constexpr int kPipeLanes = 32;
constexpr int kPipeStride = 32;
// An item covers kPipeTiles consecutive warp tiles of a row.  Two tiles
// spread the decoding, polls and publication over 64 sites (1,829 -> 1,666
// warp-instructions per 32 sites) but serialise two rounds of loads in the
// density part at the 96-register cap, and measured slower (1.43 -> 1.63 ms a
// step at 256^3), so an item is one tile.
constexpr int kPipeTiles = 1;

__device__ __forceinline__ int pipe_slot(const PipeRing &a, int k)
{
    if (k == 0) return 0;
    if (k == a.slices - 1) return 1;
    const unsigned q = (unsigned)(k - 1), d = (unsigned)(((unsigned long long)q * a.mul_R) >> a.shift_R);
    return 2 + (int)(q - d * (unsigned)a.R);
}

__device__ __forceinline__ unsigned exact_div(unsigned n, unsigned long long mul, unsigned shift)
{
    return (unsigned)(((unsigned long long)n * mul) >> shift);
}

// item -> (D slice or -1, C slice or -1, tile)
__device__ __forceinline__ void pipe_decode(const PipeRing &a, int item, int &dslice, int &cslice, unsigned &tile)
{
    const int Sl = a.slices;
    if (item < a.prologue) {
        const unsigned q = exact_div((unsigned)item, a.mul_T, a.shift_T);
        tile = (unsigned)item - q * (unsigned)a.tiles_per_slice;
        dslice = q == 0 ? Sl - 1 : (int)q - 1;
        cslice = -1;
    } else {
        const unsigned r = (unsigned)(item - a.prologue);
        const unsigned j = exact_div(r, a.mul_T, a.shift_T);
        tile = r - j * (unsigned)a.tiles_per_slice;
        cslice = (int)j;
        dslice = (int)j + a.lag + 1 <= Sl - 2 ? (int)j + a.lag + 1 : -1;
    }
}

// Counters are kept per unit: one row of tiles of a slice in 3D (slice k,
// row y: unit k ny + y), one slice in 2D.  The units a tile of slice k, row y
// depends on are those of slices k-1 .. k+1 and, in 3D, rows y-1 .. y+1
// (periodic); lane q < 9 (3D) or < 3 (2D) watches unit q with acquire loads,
// and the warp's later reads are ordered after them by the warp-wide vote.
// On timeout: status bit, false for every lane.
template <int D>
__device__ __forceinline__ bool pipe_wait(const PipeRing &a, const unsigned *cnt, int k, int y, unsigned *status)
{
    const int lane = threadIdx.x & 31;
    int ok = 1;
    if (lane < (D == 3 ? 9 : 3)) {
        const int dk = (D == 3 ? lane / 3 : lane) - 1, dy = D == 3 ? lane % 3 - 1 : 0;
        const int kk = k + dk < 0 ? a.slices - 1 : (k + dk >= a.slices ? 0 : k + dk);
        const int yy = y + dy < 0 ? a.rows - 1 : (y + dy >= a.rows ? 0 : y + dy);
        const unsigned *c = cnt + (size_t)kk * a.rows + yy;
        if (load_acquire(c) < a.target) {
            const unsigned long long t0 = global_ns();
            unsigned nap = 32;
            while (load_acquire(c) < a.target) {
                if (global_ns() - t0 > a.wait_ns) {
                    ok = 0;
                    break;
                }
                __nanosleep(nap); // back off: a spinning warp takes issue slots from the working ones
                nap = nap < 1024 ? 2 * nap : nap;
            }
        }
    }
    ok = __all_sync(0xffffffffu, ok);
    if (!ok) {
        if (lane == 0) atomicOr(status, kStatusTimeout);
        return false;
    }
    return true;
}

// Every lane's earlier memory accesses are ordered before the counts (one
// per unit given, -1: none), which lane 0 adds.
__device__ __forceinline__ void pipe_publish(unsigned *c0, long long u0, unsigned *c1, long long u1)
{
    fence_acq_rel();
    __syncwarp();
    if ((threadIdx.x & 31) == 0) {
        if (u0 >= 0) red_add_relaxed(c0 + u0, 1u);
        if (u1 >= 0) red_add_relaxed(c1 + u1, 1u);
    }
}

// The collide's view of the ring: density stencil from the slots of slices
// j-1, j, j+1 (3D: by dz; 2D: by dy), own moments from slice j's slot.
template <int D> struct RingSrc {
    const float2 *rho[3];
    const float *mom;
    int sp, insite;
    __device__ __forceinline__ float2 rho_at(const Nbr &nb, int dx, int dy, int dz) const
    {
        if constexpr (D == 3) return __ldcg(rho[dz + 1] + nb.ys[dy + 1] * nb.nx + nb.xs[dx + 1]);
        else return __ldcg(rho[dy + 1] + nb.xs[dx + 1]);
    }
    __device__ __forceinline__ float mom_at(int plane) const { return __ldcg(mom + (size_t)plane * sp + insite); }
};

template <class L, class S, bool MOM>
__global__ void __launch_bounds__(128, L::Q == 9 ? (MOM ? 8 : 6) : (MOM ? 5 : 4))
    k_step_pipe(const StepParams p, const PlaneTable<typename S::T> in, const PlaneTable<typename S::T> out,
                const PipeRing a, unsigned *__restrict__ status)
{
    constexpr int D = L::D, NM = 2 * (D + 1);
    const int lane = threadIdx.x & 31;
    const int Sl = a.slices;
    // the work lane of this warp and its first two items; a third is always
    // requested one item ahead, so the counter's latency is hidden
    const int wid = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int wl = wid % kPipeLanes;
    unsigned *ctr = a.next + wl * kPipeStride;
    auto draw = [&]() -> int {
        unsigned k = 0;
        if (lane == 0) k = atomicAdd(ctr, 1u);
        return wl + kPipeLanes * (int)__shfl_sync(0xffffffffu, k, 0);
    };
    int item = draw();
    int nitem = draw();
    int dslice = -1, cslice = -1;
    unsigned tile = 0;
    if (item < a.total) pipe_decode(a, item, dslice, cslice, tile);
    while (item < a.total) {
        unsigned kreq = 0; // request for the item after next; read at the end of this one
        if (lane == 0) kreq = atomicAdd(ctr, 1u);
        const unsigned row = exact_div(tile, a.mul_row, a.shift_row); // y of the tile (3D; 0 in 2D)
        const int x0 = (int)(tile - row * (unsigned)a.tiles_per_row) * (32 * kPipeTiles) + lane;
        // the next item of this warp (an L2 prefetch of its density tiles here
        // measured 4 % slower once the species' words sat side by side)
        int ndslice = -1, ncslice = -1;
        unsigned ntile = 0;
        if (nitem < a.total) pipe_decode(a, nitem, ndslice, ncslice, ntile);
        // unit counters of this item
        const int yrow = D == 3 ? (int)row : 0;
        const long long dunit = dslice >= 0 ? (long long)dslice * a.rows + yrow : -1;
        const long long cunit = cslice >= 0 ? (long long)cslice * a.rows + yrow : -1;
        // ---- D part: densities (and moments) of the tiles of slice dslice
        if (dslice >= 0) {
            // the slice that held this ring slot before (slices 0 and S-1 keep
            // slots of their own)
            const int prev = dslice - a.R;
            if (dslice <= Sl - 2 && prev >= 1 && !pipe_wait<D>(a, a.ccount, prev, yrow, status)) return;
            const int slot = pipe_slot(a, dslice);
            static_for<kPipeTiles>([&](auto uc) {
                constexpr int u = decltype(uc)::value;
                const int x = x0 + 32 * u;
                if (x < p.nx) {
                    const int insite = D == 3 ? (int)row * p.nx + x : x;
                    const int site = D == 3 ? dslice * a.sp + insite : dslice * p.nx + x;
                    float r[2], mm[2][D + 1], d[2][L::Q];
                    static_for<L::Q>([&](auto ic) {
                        constexpr int i = decltype(ic)::value;
                        const float2 v = S::load_pair_cs(in.pair(i, site));
                        d[0][i] = v.x;
                        d[1][i] = v.y;
                    });
                    static_for<2>([&](auto sc) {
                        constexpr int s = decltype(sc)::value;
                        float m[L::Q];
                        // the same expressions as the density pass of the two-kernel step
                        Transform<L>::forward(d[s], m);
                        r[s] = p.rho0[s] + m[0];
                        static_for<D + 1>([&](auto ac) {
                            constexpr int q = decltype(ac)::value;
                            mm[s][q] = m[q];
                        });
                    });
                    a.rho[(size_t)slot * a.sp + insite] = make_float2(r[0], r[1]);
                    if constexpr (MOM) {
                        static_for<NM>([&](auto qc) {
                            constexpr int q = decltype(qc)::value;
                            a.mom[((size_t)slot * NM + q) * a.sp + insite] = mm[q / (D + 1)][q % (D + 1)];
                        });
                    }
                }
            });
            if (cslice < 0) pipe_publish(a.dcount, dunit, a.ccount, -1);
        }
        // ---- C part: collide the tiles of slice cslice.  The counts of this
        // item (its D tiles, and its C tiles for the slots' next users) are
        // published once every ring read is done, before the last tile's
        // population stores, so that the fence does not wait for those.
        if (cslice >= 0) {
            const int jm = cslice == 0 ? Sl - 1 : cslice - 1, jp = cslice == Sl - 1 ? 0 : cslice + 1;
            if (!pipe_wait<D>(a, a.dcount, cslice, yrow, status)) return;
            RingSrc<D> src;
            const int sc = pipe_slot(a, cslice);
            src.rho[0] = a.rho + (size_t)pipe_slot(a, jm) * a.sp;
            src.rho[1] = a.rho + (size_t)sc * a.sp;
            src.rho[2] = a.rho + (size_t)pipe_slot(a, jp) * a.sp;
            src.mom = a.mom + (size_t)sc * NM * a.sp;
            src.sp = a.sp;
            const int y = D == 3 ? (int)row : cslice, z = D == 3 ? cslice : 0;
            static_for<kPipeTiles>([&](auto uc) {
                constexpr int u = decltype(uc)::value;
                const int x = x0 + 32 * u;
                const bool active = x < p.nx;
                const int xc = active ? x : p.nx - 1; // idle lanes compute a real site without storing
                const Nbr nb = make_nbr(p, xc, y, z);
                src.insite = D == 3 ? (int)row * p.nx + xc : xc;
                if constexpr (u == kPipeTiles - 1) {
                    auto publish = [&] { pipe_publish(a.dcount, dunit, a.ccount, cunit); };
                    site_collide_src<L, S, kPush, true, MOM, MOM, true>(p, in, out, src, status, nb,
                                                                       [] { return true; }, publish, active);
                } else {
                    site_collide_src<L, S, kPush, true, MOM, MOM, true>(p, in, out, src, status, nb,
                                                                       [] { return true; }, [] {}, active);
                }
            });
        }
        dslice = ndslice;
        cslice = ncslice;
        tile = ntile;
        item = nitem;
        nitem = wl + kPipeLanes * (int)__shfl_sync(0xffffffffu, kreq, 0);
    }
}

// ---------------------------------------------------------------------------
// Batched step: many independent boxes of uneven size in one launch.  The
// work list holds one entry per 128 consecutive sites of a replica; a block
// stages its replica's parameters in shared memory and runs the same per-site
// code as the single-box kernels on that replica's slice of the shared buffers.
// The step's noise counter is read from device memory (base + k), so a CUDA
// graph of several steps can be replayed without changing its parameters.
// ---------------------------------------------------------------------------
// A replica's step parameters, offsets and exact dividers, staged in shared memory.
struct StagedRep {
    StepParams sp;
    unsigned long long pop_off, rho_off, mul_nx, mul_nxy;
    unsigned shift_nx, shift_nxy;
    // (x, y, z) of a replica-local site without integer division
    __device__ __forceinline__ void coords(int site, int &x, int &y, int &z) const
    {
        const unsigned row = (unsigned)(((unsigned long long)(unsigned)site * mul_nx) >> shift_nx);
        const unsigned plane = (unsigned)(((unsigned long long)(unsigned)site * mul_nxy) >> shift_nxy);
        x = site - (int)row * sp.nx;
        y = (int)row - (int)plane * sp.ny;
        z = (int)plane;
    }
};

__device__ __forceinline__ void stage_params(const RepInfo *__restrict__ reps, int r, StagedRep &st,
                                             const unsigned *__restrict__ step_base, unsigned k)
{
    constexpr int words = (int)(sizeof(StepParams) / sizeof(unsigned));
    static_assert(sizeof(StepParams) % sizeof(unsigned) == 0, "StepParams must be a whole number of words");
    const unsigned *src = reinterpret_cast<const unsigned *>(&reps[r].p);
    unsigned *dst = reinterpret_cast<unsigned *>(&st.sp);
    for (int w = threadIdx.x; w < words; w += blockDim.x) dst[w] = __ldg(src + w);
    if (threadIdx.x == 0) {
        st.pop_off = reps[r].pop_off;
        st.rho_off = reps[r].rho_off;
        st.mul_nx = reps[r].mul_nx;
        st.mul_nxy = reps[r].mul_nxy;
        st.shift_nx = reps[r].shift_nx;
        st.shift_nxy = reps[r].shift_nxy;
    }
    __syncthreads();
    if (threadIdx.x == 0) st.sp.step = *step_base + k;
    __syncthreads();
}

// MOM: the replicas relax fully and their StepParams::mom point at their
// moment planes (the moment-fed collide, as for a single box)
template <class L, class S, int PARITY, bool MOM = false>
__global__ void __launch_bounds__(128) k_density_batch(const RepInfo *__restrict__ reps, const int2 *__restrict__ tiles,
                                                       typename S::T *__restrict__ pop, float2 *__restrict__ rho,
                                                       const unsigned *__restrict__ step_base, unsigned k)
{
    __shared__ StagedRep st;
    const int2 t = tiles[blockIdx.x];
    stage_params(reps, t.x, st, step_base, k);
    const int site = t.y + (int)threadIdx.x;
    if (site >= st.sp.N) return;
    int x, y, z;
    st.coords(site, x, y, z);
    const Nbr nb = make_nbr(st.sp, x, y, z);
    const FlatPlanes<const typename S::T> fp{pop + st.pop_off, (size_t)st.sp.N};
    if constexpr (MOM) rho[st.rho_off + site] = site_moments<L, S, PARITY>(st.sp, fp, nb);
    else rho[st.rho_off + site] = site_density<L, S, PARITY>(st.sp, fp, nb);
}

// PARITY kPush: read pop, write pop_out (two arrays); otherwise in place in pop.
template <class L, class S, int PARITY, bool FULL, bool MOM = false>
__global__ void __launch_bounds__(128) k_collide_batch(const RepInfo *__restrict__ reps, const int2 *__restrict__ tiles,
                                                       typename S::T *__restrict__ pop, typename S::T *__restrict__ pop_out,
                                                       const float2 *__restrict__ rho, unsigned *__restrict__ status,
                                                       const unsigned *__restrict__ step_base, unsigned k)
{
    __shared__ StagedRep st;
    const int2 t = tiles[blockIdx.x];
    stage_params(reps, t.x, st, step_base, k);
    const int site = t.y + (int)threadIdx.x;
    if (site >= st.sp.N) return;
    int x, y, z;
    st.coords(site, x, y, z);
    const Nbr nb = make_nbr(st.sp, x, y, z);
    const FlatPlanes<typename S::T> fp{pop + st.pop_off, (size_t)st.sp.N};
    const FlatPlanes<typename S::T> fo{(PARITY == kPush ? pop_out : pop) + st.pop_off, (size_t)st.sp.N};
    site_collide<L, S, PARITY, false, true, FULL, MOM>(st.sp, fp, fo, rho + st.rho_off, status, nb, [] { return true; });
}

// ---------------------------------------------------------------------------
// Tiled two-array step (2D): one launch per step, no density field in HBM.
// A thread block owns a tile of kTileX x TileGeom::Y sites.  It forms the
// densities of the tile and of the one-site ring around it (periodic) into
// shared memory, and, at full relaxation, each tile site's m_0 .. m_D; after
// one barrier it collides the tile from there and pushes f* into the other
// array.  The ring's densities are formed again by the neighbouring blocks
// (about 20 % more density work at 32 x 16), but the populations cross HBM
// once each way (the ring's reads hit L2) and the densities never leave the
// SM.  The per-site expressions are those of the two-kernel step, so the
// update is bitwise the same.  Reads only `in`, writes only `out`: no two
// blocks touch the same word of either.
// ---------------------------------------------------------------------------
constexpr int kTileX = kTiledStepX;
// NT threads (NT / 32 rows of lanes), R rows per thread
template <int NT, int R> struct TileGeom {
    static constexpr int Y = (NT / kTileX) * R;     // rows of the tile
    static constexpr int W = kTileX + 2, H = Y + 2; // with the ring
    static constexpr int RING = 2 * W + 2 * Y;      // ring sites
    static constexpr int MOMS = Y * kTileX;         // floats of one moment plane
};
// blocks an SM is asked to hold (register budget): 1024 threads at full
// relaxation, 768 otherwise
template <int NT, bool FULL> constexpr int tile_min_blocks() { return (FULL ? 1024 : 768) / NT > 0 ? (FULL ? 1024 : 768) / NT : 1; }

// periodic coordinate g in [-n, 2n + kTileX) brought into [0, n)
__device__ __forceinline__ int wrap_coord(int g, int n)
{
    while (g >= n) g -= n;
    while (g < 0) g += n;
    return g;
}

// The collide's view of a tile: the density stencil and, MOM, the site's own
// moments from shared memory.
template <class G> struct TileSrc {
    const float2 *rho; // (H x W) densities, ring included
    const float *mom;  // 2 (D + 1) planes of Y x kTileX
    int c, m;          // this site's cell in rho and in each moment plane
    __device__ __forceinline__ float2 rho_at(const Nbr &, int dx, int dy, int) const { return rho[c + dy * G::W + dx]; }
    __device__ __forceinline__ float mom_at(int plane) const { return mom[plane * G::MOMS + m]; }
};

// One tile: densities (and moments) into shared memory, a barrier, then the
// collisions.
template <class L, class S, bool FULL, bool MOM, int NT, int R, class P>
__device__ __forceinline__ void tile_step(const StepParams &p, const P &in, const P &out, unsigned *__restrict__ status,
                                          int x0, int y0, float2 *srho, float *smom)
{
    static_assert(L::D == 2, "the tiled step is two-dimensional");
    using G = TileGeom<NT, R>;
    constexpr int NM = 2 * (L::D + 1), LR = NT / kTileX;
    const int tid = (int)threadIdx.x, tx = tid % kTileX, ty = tid / kTileX;
    // densities (and moments) of the tile's own sites
#pragma unroll
    for (int r = 0; r < R; r++) {
        const int ly = ty + LR * r;
        const Nbr nb = make_nbr(p, wrap_coord(x0 + tx, p.nx), wrap_coord(y0 + ly, p.ny), 0);
        float2 rr;
        if constexpr (MOM) {
            float mm[2][L::D + 1];
            rr = site_moments_to<L, S, 0>(p, in, nb, mm);
            static_for<NM>([&](auto qc) {
                constexpr int q = decltype(qc)::value;
                smom[q * G::MOMS + ly * kTileX + tx] = mm[q / (L::D + 1)][q % (L::D + 1)];
            });
        } else {
            rr = site_density<L, S, 0>(p, in, nb);
        }
        srho[(ly + 1) * G::W + tx + 1] = rr;
    }
    // densities of the ring: the rows above and below (corners included), then
    // the columns left and right
    for (int h = tid; h < G::RING; h += NT) {
        int sx, sy;
        if (h < 2 * G::W) {
            sx = h % G::W - 1;
            sy = h < G::W ? -1 : G::Y;
        } else {
            sx = h < 2 * G::W + G::Y ? -1 : kTileX;
            sy = (h - 2 * G::W) % G::Y;
        }
        const Nbr nb = make_nbr(p, wrap_coord(x0 + sx, p.nx), wrap_coord(y0 + sy, p.ny), 0);
        srho[(sy + 1) * G::W + sx + 1] = site_density<L, S, 0>(p, in, nb);
    }
    __syncthreads();
#pragma unroll 1
    for (int r = 0; r < R; r++) {
        const int ly = ty + LR * r;
        const int x = x0 + tx, y = y0 + ly;
        const bool active = x < p.nx && y < p.ny;
        // idle lanes of a ragged tile compute a real site without storing
        const Nbr nb = make_nbr(p, wrap_coord(x, p.nx), wrap_coord(y, p.ny), 0);
        const TileSrc<G> src{srho, smom, (ly + 1) * G::W + tx + 1, ly * kTileX + tx};
        site_collide_src<L, S, kPush, true, FULL, MOM, false>(p, in, out, src, status, nb, [] { return true; },
                                                              [] {}, active);
    }
}

// One tile a block (a grid of persistent blocks walking the tiles, with or
// without an L2 prefetch of each next tile, measured slower).
template <class L, class S, bool FULL, bool MOM, int NT, int R>
__global__ void __launch_bounds__(NT, (tile_min_blocks<NT, FULL>()))
    k_step_tiled(const StepParams p, const PlaneTable<typename S::T> in, const PlaneTable<typename S::T> out,
                 unsigned *__restrict__ status)
{
    using G = TileGeom<NT, R>;
    __shared__ float2 srho[G::H * G::W];
    __shared__ float smom[MOM ? 2 * (L::D + 1) * G::MOMS : 1];
    tile_step<L, S, FULL, MOM, NT, R>(p, in, out, status, (int)blockIdx.x * kTileX, (int)blockIdx.y * G::Y, srho,
                                      smom);
}

// The tiled step of a batch: block b steps tile tiles[b] = (replica, x0, y0)
// with that replica's staged parameters, on its slices of the two arrays.
template <class L, class S, bool FULL, bool MOM, int NT, int R>
__global__ void __launch_bounds__(NT, (tile_min_blocks<NT, FULL>()))
    k_step_tiled_batch(const RepInfo *__restrict__ reps, const int4 *__restrict__ tiles,
                       const typename S::T *__restrict__ pop, typename S::T *__restrict__ pop_out,
                       unsigned *__restrict__ status, const unsigned *__restrict__ step_base, unsigned k)
{
    using G = TileGeom<NT, R>;
    __shared__ StagedRep st;
    __shared__ float2 srho[G::H * G::W];
    __shared__ float smom[MOM ? 2 * (L::D + 1) * G::MOMS : 1];
    const int4 t = tiles[blockIdx.x];
    stage_params(reps, t.x, st, step_base, k);
    // the input is only read; FlatPlanes<T> of a const pointer would give the
    // two tables different types
    const FlatPlanes<typename S::T> in{const_cast<typename S::T *>(pop) + st.pop_off, (size_t)st.sp.N};
    const FlatPlanes<typename S::T> out{pop_out + st.pop_off, (size_t)st.sp.N};
    tile_step<L, S, FULL, MOM, NT, R>(st.sp, in, out, status, t.y, t.z, srho, smom);
}

// ---------------------------------------------------------------------------
// rest-state initialisation and site gather
// ---------------------------------------------------------------------------
template <class L, class S>
__global__ void k_init_rest(const StepParams p, const float *__restrict__ rho_in, typename S::T *__restrict__ pop)
{
    const size_t NN = (size_t)p.N;
    for (size_t site = blockIdx.x * (size_t)blockDim.x + threadIdx.x; site < NN; site += (size_t)gridDim.x * blockDim.x) {
        const float ra = rho_in[site], rb = rho_in[NN + site];
        static_for<L::Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            constexpr float wi = (float)L::wd(i);
            S::store_pair(pop + pop_index(0, i, site, NN), S::encode(wi * (ra - p.rho0[0]), wi * p.rho0[0]),
                          S::encode(wi * (rb - p.rho0[1]), wi * p.rho0[1]));
        });
    }
}

template <class L, class S, int PARITY>
__global__ void k_gather_sites(const StepParams p, const typename S::T *__restrict__ pop,
                               const int64_t *__restrict__ sites, int64_t nsites, double *__restrict__ out)
{
    const size_t NN = (size_t)p.N;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nsites; k += (int64_t)gridDim.x * blockDim.x) {
        const int site = (int)sites[k];
        const int x = site % p.nx, y = (site / p.nx) % p.ny, z = site / (p.nx * p.ny);
        const Nbr nb = make_nbr(p, x, y, z);
        static_for<2>([&](auto sc) {
            constexpr int s = decltype(sc)::value;
            static_for<L::Q>([&](auto ic) {
                constexpr int i = decltype(ic)::value;
                constexpr float wi = (float)L::wd(i);
                const float base = wi * p.rho0[s];
                const float dev = S::load_dev(pop, read_index<L, PARITY, i>(nb, NN, s), base);
                out[(k * 2 + s) * L::Q + i] = (double)base + (double)dev;
            });
        });
    }
}


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

// Density fluctuation fields for the full-wavevector structure factor:
// z(site) = (sum_i delta_i^A, sum_i delta_i^B), each species' density minus its
// reference rho0, summed in float as in the step kernels, plus per-block FP64
// partial sums (fixed order) from which the means follow.
template <class L, class S, int PARITY>
__global__ void __launch_bounds__(kObsBlock) k_sfk_fields(const StepParams p,
                                                          const PlaneTable<const typename S::T> planes,
                                                          float2 *__restrict__ z, double *__restrict__ partials)
{
    __shared__ double sh[kObsBlock][2];
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    double tot[2] = {0.0, 0.0};
    if (x < p.nx) {
        const Nbr nb = make_nbr(p, x, blockIdx.y, blockIdx.z);
        float sum[2] = {0.0f, 0.0f};
        static_for<L::Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            const float2 v = S::load_pair(planes.pair(read_slot<L, PARITY, i>(), read_site<L, PARITY, i>(nb)));
            sum[0] += v.x;
            sum[1] += v.y;
        });
        z[nb.at(0, 0, 0)] = make_float2(sum[0], sum[1]);
        tot[0] = sum[0];
        tot[1] = sum[1];
    }
    block_sum<2, kObsBlock>(tot, sh);
    if (threadIdx.x == 0) {
        const size_t b = blockIdx.x + (size_t)gridDim.x * (blockIdx.y + (size_t)gridDim.y * blockIdx.z);
        partials[2 * b] = tot[0];
        partials[2 * b + 1] = tot[1];
    }
}

template <class L, class S, int PARITY>
__global__ void __launch_bounds__(kObsBlock) k_observables(const StepParams p, const typename S::T *__restrict__ pop,
                                                           const float2 *__restrict__ rho, double *__restrict__ rho_a,
                                                           double *__restrict__ rho_b, double *__restrict__ u,
                                                           double *__restrict__ partials)
{
    constexpr int Q = L::Q, D = L::D;
    __shared__ double sh[kObsBlock][5];
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, z = blockIdx.z;
    double tot[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (x < p.nx) {
        const int xs[3] = {x == 0 ? p.nx - 1 : x - 1, x, x == p.nx - 1 ? 0 : x + 1};
        const int ys[3] = {y == 0 ? p.ny - 1 : y - 1, y, y == p.ny - 1 ? 0 : y + 1};
        const int zs[3] = {z == 0 ? p.nz - 1 : z - 1, z, z == p.nz - 1 ? 0 : z + 1};
        auto at = [&](int dx, int dy, int dz) { return (zs[dz + 1] * p.ny + ys[dy + 1]) * p.nx + xs[dx + 1]; };
        const size_t NN = (size_t)p.N;
        const int site = at(0, 0, 0);
        // per-site sums in float, as in the step kernels: the deviations are
        // small, so their float sums are accurate to ~1e-7 of themselves, and
        // rho = rho0 + sum is formed in double (the totals keep FP64
        // precision; this GPU's FP64 rate is a small fraction of its FP32 rate)
        float sum[2] = {0.0f, 0.0f}, j[2][3] = {{0.0f, 0.0f, 0.0f}, {0.0f, 0.0f, 0.0f}};
        float a[2][3] = {{0.0f, 0.0f, 0.0f}, {0.0f, 0.0f, 0.0f}};
        static_for<Q>([&](auto ic) {
            constexpr int i = decltype(ic)::value;
            const size_t idx = PARITY == 0 ? pop_index(0, i, site, NN)
                                           : pop_index(0, L::opp(i), at(-L::cx(i), -L::cy(i), -L::cz(i)), NN);
            const float2 v = S::load_pair(pop + idx);
            static_for<2>([&](auto sc) {
                constexpr int s = decltype(sc)::value;
                const float dv = s == 0 ? v.x : v.y;
                sum[s] += dv;
                static_for<3>([&](auto dc) {
                    constexpr int d = decltype(dc)::value;
                    constexpr int cd = comp<L>(i, d);
                    if constexpr (cd != 0) j[s][d] += (float)cd * dv;
                });
            });
        });
        // force with the density field (the same values the step kernel uses)
        static_for<Q - 1>([&](auto kc) {
            constexpr int i = decltype(kc)::value + 1;
            const float2 rn = rho[at(L::cx(i), L::cy(i), L::cz(i))];
            static_for<3>([&](auto dc) {
                constexpr int d = decltype(dc)::value;
                constexpr int cd = comp<L>(i, d);
                if constexpr (cd != 0) {
                    constexpr float cw = (float)(L::wd(i) * cd);
                    a[0][d] += cw * rn.y;
                    a[1][d] += cw * rn.x;
                }
            });
        });
        const float ra0 = rho[site].x, rb0 = rho[site].y;
        const double r0 = (double)p.rho0[0] + (double)sum[0], r1 = (double)p.rho0[1] + (double)sum[1];
        const float rt = (float)(r0 + r1);
        if (rho_a) rho_a[site] = r0;
        if (rho_b) rho_b[site] = r1;
        tot[0] = r0;
        tot[1] = r1;
#pragma unroll
        for (int d = 0; d < D; d++) {
            const float Ft = -p.G * (ra0 * a[0][d] + rb0 * a[1][d]);
            const float jt = j[0][d] + j[1][d] + 0.5f * Ft;
            if (u) u[(size_t)d * NN + site] = (double)(jt / rt);
            tot[2 + d] = (double)jt;
        }
    }
    block_sum<5, kObsBlock>(tot, sh);
    if (threadIdx.x == 0) {
        const size_t b = blockIdx.x + (size_t)gridDim.x * (blockIdx.y + (size_t)gridDim.y * blockIdx.z);
#pragma unroll
        for (int k = 0; k < 5; k++) partials[b * 5 + k] = tot[k];
    }
}


// thread block of the density and collide launches: block_x sites along x (at
// most nx rounded up to a warp) by block_y rows
inline dim3 site_block(const StepParams &p)
{
    const int wx = ((p.nx + 31) / 32) * 32;
    return dim3(p.block_x < wx ? p.block_x : wx, p.block_y);
}
inline dim3 site_grid(const StepParams &p, dim3 blk)
{
    return dim3((p.nx + blk.x - 1) / blk.x, (p.yn + blk.y - 1) / blk.y, p.zn);
}

} // namespace kern

namespace kern {
template <class T> PlaneTable<T> plane_table(T *pop, int Q, int N)
{
    PlaneTable<T> t{};
    for (int k = 0; k < Q; k++) t.ptr[k] = pop + (size_t)2 * k * (size_t)N;
    return t;
}
} // namespace kern

template <class L, class S>
cudaError_t Launch<L, S>::density(int parity, const StepParams &p, const void *pop, float *rho, cudaStream_t st)
{
    const dim3 b = kern::site_block(p), g = kern::site_grid(p, b);
    const auto planes = kern::plane_table(static_cast<const typename S::T *>(pop), L::Q, p.N);
    auto *r2 = reinterpret_cast<float2 *>(rho);
    if (p.mom && parity == 0) kern::k_moments<L, S, 0><<<g, b, 0, st>>>(p, planes, r2);
    else if (p.mom) kern::k_moments<L, S, 1><<<g, b, 0, st>>>(p, planes, r2);
    else if (parity == 0) kern::k_density<L, S, 0><<<g, b, 0, st>>>(p, planes, r2);
    else kern::k_density<L, S, 1><<<g, b, 0, st>>>(p, planes, r2);
    return cudaGetLastError();
}

template <class L, class S>
cudaError_t Launch<L, S>::collide(int parity, const StepParams &p, void *pop, void *pop_out, const float *rho,
                                  unsigned *status, cudaStream_t st)
{
    const dim3 b = kern::site_block(p), g = kern::site_grid(p, b);
    const auto planes = kern::plane_table(static_cast<typename S::T *>(pop), L::Q, p.N);
    const auto out = parity == kern::kPush ? kern::plane_table(static_cast<typename S::T *>(pop_out), L::Q, p.N) : planes;
    auto *r2 = reinterpret_cast<const float2 *>(rho);
    const bool full = kern::full_relaxation<L>(p);
    if (parity == 0) {
        if (full && p.mom) kern::k_collide<L, S, 0, true, true><<<g, b, 0, st>>>(p, planes, out, r2, status);
        else if (full) kern::k_collide<L, S, 0, true><<<g, b, 0, st>>>(p, planes, out, r2, status);
        else kern::k_collide<L, S, 0, false><<<g, b, 0, st>>>(p, planes, out, r2, status);
    } else if (parity == 1) {
        if (full && p.mom) kern::k_collide<L, S, 1, true, true><<<g, b, 0, st>>>(p, planes, out, r2, status);
        else if (full) kern::k_collide<L, S, 1, true><<<g, b, 0, st>>>(p, planes, out, r2, status);
        else kern::k_collide<L, S, 1, false><<<g, b, 0, st>>>(p, planes, out, r2, status);
    } else {
        if (full && p.mom) kern::k_collide<L, S, kern::kPush, true, true><<<g, b, 0, st>>>(p, planes, out, r2, status);
        else if (full) kern::k_collide<L, S, kern::kPush, true><<<g, b, 0, st>>>(p, planes, out, r2, status);
        else kern::k_collide<L, S, kern::kPush, false><<<g, b, 0, st>>>(p, planes, out, r2, status);
    }
    return cudaGetLastError();
}

template <class L, class S>
cudaError_t Launch<L, S>::step_fused(int parity, const StepParams &p, void *pop, float *rho, unsigned *status,
                                     unsigned *counters, double wait_ms, int stall, int lag_opt, cudaStream_t st)
{
    // one resident wave of persistent blocks (queried once per parity instance)
    static int blocks[2] = {0, 0};
    if (!blocks[parity]) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = parity == 0 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern::k_step_fused<L, S, 0>, 128, 0)
                            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern::k_step_fused<L, S, 1>, 128, 0);
        if (e != cudaSuccess) return e;
        blocks[parity] = sms * (per_sm > 0 ? per_sm : 1);
    }
    kern::PipeArgs a;
    a.done = counters;
    a.tiles_per_row = (p.nx + 31) / 32;
    a.slices = L::D == 3 ? p.nz : p.ny;
    a.tiles_per_slice = L::D == 3 ? p.ny * a.tiles_per_row : a.tiles_per_row;
    const int nT = a.tiles_per_slice, nS = a.slices;
    // smallest lag whose density lead exceeds the warps in flight, unless set
    const int warps = blocks[parity] * 4;
    int lag = 2;
    while (lag * nT < warps) lag++;
    if (lag_opt >= 2) lag = lag_opt;
    if (nS >= lag + 3) {
        a.lag = lag;
        a.prologue = (lag + 2) * nT;
    } else {
        a.lag = -1;
        a.prologue = 0;
    }
    a.total = a.lag < 0 ? 2 * nS * nT : a.prologue + nS * nT;
    a.target = (unsigned)nT + (stall ? 1u : 0u);
    a.wait_ns = (unsigned long long)(wait_ms * 1e6);
    const int need_warps = a.total;
    int grid = blocks[parity];
    if (grid * 4 > need_warps) grid = (need_warps + 3) / 4;
    cudaError_t e = cudaMemsetAsync(counters, 0, sizeof(unsigned) * nS, st);
    if (e != cudaSuccess) return e;
    auto *ptr = static_cast<typename S::T *>(pop);
    auto *r2 = reinterpret_cast<float2 *>(rho);
    StepParams pc = p;
    void *args[] = {(void *)&pc, (void *)&ptr, (void *)&r2, (void *)&status, (void *)&a};
    const void *fn = parity == 0 ? (const void *)kern::k_step_fused<L, S, 0> : (const void *)kern::k_step_fused<L, S, 1>;
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(128), args, 0, st);
}

// Resident blocks of the pipelined step on the current device (queried once
// per instance).
template <class L, class S> static cudaError_t pipe_blocks(bool mom, int *out)
{
    static int blocks[2] = {0, 0};
    int &b = blocks[mom ? 1 : 0];
    if (!b) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = mom ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern::k_step_pipe<L, S, true>, 128, 0)
                    : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern::k_step_pipe<L, S, false>, 128, 0);
        if (e != cudaSuccess) return e;
        b = sms * (per_sm > 0 ? per_sm : 1);
    }
    *out = b;
    return cudaSuccess;
}

template <class L, class S>
cudaError_t Launch<L, S>::pipe_geometry(const StepParams &p, bool mom, int lag_opt, int *lag, int *ring_slots,
                                        size_t *ring_floats, size_t *counters)
{
    int blocks = 0;
    const cudaError_t e = pipe_blocks<L, S>(mom, &blocks);
    if (e != cudaSuccess) return e;
    const int S_ = L::D == 3 ? p.nz : p.ny;
    const int tpr = (p.nx + 32 * kern::kPipeTiles - 1) / (32 * kern::kPipeTiles); // items per row
    const int T = L::D == 3 ? p.ny * tpr : tpr;
    const int sp = L::D == 3 ? p.nx * p.ny : p.nx;
    // slices of items in flight (one item per warp, W warps: a wave of W items
    // spans `inflight` slices).  By default the density work runs two waves
    // and two slices ahead of the collisions, but no further than the
    // populations of about 40 MB of slices (a third of the 129 MB L2; the
    // collisions re-read them from there) allow, and never less than a wave
    // and a slice; a slot is reused two waves and two slices after its last
    // readers were due.  Measured, ms a
    // step at full relaxation (two kernels / pipeline):
    //   128^3 (a wave = 6 slices of 2.5 MB): lag 14, 29 slots: 0.158 / 0.159
    //   192^3 (3 slices of 5.6 MB): lag 6, 14 slots: 0.535 / 0.501
    //   256^3 (2 slices of 10 MB): lag 3, 9 slots: 1.162 / 1.183
    // while lag 6 with 13 slots took 1.201 at 256^3, lag 7 with 21 slots 0.219
    // at 128^3 and 4 slots of margin (lag 6, 10 slots) 1.338 at 256^3.  Any
    // lag >= 1 with a ring of lag + 3 slots or more is correct (shorter ones
    // wait more); an explicitly given lag gets lag + 6 slots.
    const int inflight = (int)(((long long)blocks * 4 + T - 1) / T);
    const double slice_bytes = (double)sp * L::Q * 2 * sizeof(typename S::T);
    const int l_fit = (int)(40e6 / slice_bytes) - 1;
    const int l = lag_opt >= 1 ? lag_opt : std::max(inflight + 1, std::min(2 * inflight + 2, l_fit));
    const int R = lag_opt >= 1 ? l + 6 : l + 2 * inflight + 2;
    *lag = l;
    *ring_slots = S_ >= 2 * (l + 2) + R ? R : 0; // 0: too few slices for the pipeline
    *counters = 2 * (size_t)S_ * (L::D == 3 ? p.ny : 1) + (size_t)kern::kPipeLanes * kern::kPipeStride;
    *ring_floats = ((size_t)R + 2) * sp * (2 + (mom ? 2 * (L::D + 1) : 0));
    return cudaSuccess;
}

template <class L, class S>
cudaError_t Launch<L, S>::step_pipe(const StepParams &p, const void *pop, void *pop_out, float *ring, unsigned *counters,
                                    int ring_slots, int lag, bool mom, unsigned *status, double wait_ms, int stall,
                                    cudaStream_t st)
{
    const int S_ = L::D == 3 ? p.nz : p.ny;
    const int tpr = (p.nx + 32 * kern::kPipeTiles - 1) / (32 * kern::kPipeTiles); // items per row
    const int T = L::D == 3 ? p.ny * tpr : tpr;
    const int sp = L::D == 3 ? p.nx * p.ny : p.nx;
    int blocks = 0;
    cudaError_t e = pipe_blocks<L, S>(mom, &blocks);
    if (e != cudaSuccess) return e;
    kern::PipeRing a;
    a.R = ring_slots;
    a.sp = sp;
    a.slices = S_;
    a.rows = L::D == 3 ? p.ny : 1;
    a.tiles_per_slice = T;
    a.tiles_per_row = tpr;
    a.lag = lag;
    a.prologue = (lag + 2) * T;
    a.total = a.prologue + S_ * T;
    exact_divider((unsigned)T, a.mul_T, a.shift_T);
    exact_divider((unsigned)tpr, a.mul_row, a.shift_row);
    exact_divider((unsigned)ring_slots, a.mul_R, a.shift_R);
    a.target = (unsigned)tpr + (stall ? 1u : 0u);
    a.wait_ns = (unsigned long long)(wait_ms * 1e6);
    const size_t slots = (size_t)ring_slots + 2;
    a.rho = reinterpret_cast<float2 *>(ring);
    a.mom = ring + slots * sp * 2;
    const size_t units = (size_t)S_ * a.rows;
    a.dcount = counters;
    a.ccount = counters + units;
    a.next = counters + 2 * units;
    e = cudaMemsetAsync(counters, 0, sizeof(unsigned) * (2 * units + (size_t)kern::kPipeLanes * kern::kPipeStride), st);
    if (e != cudaSuccess) return e;
    int grid = blocks;
    if ((long long)grid * 4 > a.total) grid = (a.total + 3) / 4;
    if (grid * 4 < kern::kPipeLanes) grid = kern::kPipeLanes / 4; // every work lane needs a warp
    const auto in = kern::plane_table(static_cast<typename S::T *>(const_cast<void *>(pop)), L::Q, p.N);
    const auto out = kern::plane_table(static_cast<typename S::T *>(pop_out), L::Q, p.N);
    StepParams pc = p;
    unsigned *stat = status;
    void *args[] = {(void *)&pc, (void *)&in, (void *)&out, (void *)&a, (void *)&stat};
    const void *fn = mom ? (const void *)kern::k_step_pipe<L, S, true> : (const void *)kern::k_step_pipe<L, S, false>;
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(128), args, 0, st);
}

template <class L, class S>
cudaError_t Launch<L, S>::batch_step(int parity, const RepInfo *reps, const int2 *tiles, int ntiles, void *pop,
                                     void *pop_out, float *rho, unsigned *status, const unsigned *step_base, unsigned k,
                                     bool full, cudaStream_t st)
{
    auto *ptr = static_cast<typename S::T *>(pop);
    auto *po = static_cast<typename S::T *>(pop_out);
    auto *r2 = reinterpret_cast<float2 *>(rho);
    // full: every replica relaxes fully and its StepParams::mom points at its
    // moment planes, so the moment-fed pair of kernels runs.  Two arrays
    // (kPush): the density pass reads pop in the natural layout.
    auto pair = [&](auto dpar, auto cpar) {
        constexpr int DP = decltype(dpar)::value, CP = decltype(cpar)::value;
        if (full) {
            kern::k_density_batch<L, S, DP, true><<<ntiles, 128, 0, st>>>(reps, tiles, ptr, r2, step_base, k);
            kern::k_collide_batch<L, S, CP, true, true><<<ntiles, 128, 0, st>>>(reps, tiles, ptr, po, r2, status,
                                                                                 step_base, k);
        } else {
            kern::k_density_batch<L, S, DP><<<ntiles, 128, 0, st>>>(reps, tiles, ptr, r2, step_base, k);
            kern::k_collide_batch<L, S, CP, false><<<ntiles, 128, 0, st>>>(reps, tiles, ptr, po, r2, status,
                                                                            step_base, k);
        }
    };
    if (parity == 0) pair(std::integral_constant<int, 0>{}, std::integral_constant<int, 0>{});
    else if (parity == 1) pair(std::integral_constant<int, 1>{}, std::integral_constant<int, 1>{});
    else pair(std::integral_constant<int, 0>{}, std::integral_constant<int, kern::kPush>{});
    return cudaGetLastError();
}

// threads and rows per thread of the tiled step's blocks: 32 x 16 tiles (measured against
// 32 x 32 of 256 or 512 threads and 32 x 8 or 32 x 16 of two rows a thread)
constexpr int kTileThreads = 128, kTileRowsPerThread = 4;

// rows a thread of a single box's tiled step: 4 (32 x 16 tiles), or 1 (32 x 4
// tiles, four times the blocks) on a box of at most 512 such tiles, which
// would not fill half the GPU.  Measured (us a step, tau = 1 / 0.8/1.0, rows
// a thread 4 / 1): 256^2 8.7 / 5.0 and 9.2 / 5.3; 512^2 13.4 / 10.9 and
// 14.7 / 12.9; 2048^2 141 / 138 and 155 / 166; 4096^2 514 / 536 and 590 /
// 646 (two rows a thread was best only at tau = 0.8/1.0 on 384^2 and 768^2,
// by 2-3 %).
inline int tiled_rows_per_thread(int nx, int ny)
{
    const long long tiles = (long long)((nx + kern::kTileX - 1) / kern::kTileX) * ((ny + 15) / 16);
    return tiles <= 512 ? 1 : kTileRowsPerThread;
}

template <class L, class S>
cudaError_t Launch<L, S>::step_tiled(const StepParams &p, const void *pop, void *pop_out, unsigned *status,
                                     cudaStream_t st)
{
    if constexpr (L::D != 2) {
        return cudaErrorNotSupported;
    } else {
        constexpr int NT = kTileThreads;
        const auto in = kern::plane_table(const_cast<typename S::T *>(static_cast<const typename S::T *>(pop)), L::Q, p.N);
        const auto out = kern::plane_table(static_cast<typename S::T *>(pop_out), L::Q, p.N);
        const bool full = kern::full_relaxation<L>(p);
        auto launch = [&](auto rc) {
            constexpr int R = decltype(rc)::value;
            using G = kern::TileGeom<NT, R>;
            const dim3 g((p.nx + kern::kTileX - 1) / kern::kTileX, (p.ny + G::Y - 1) / G::Y);
            if (full) kern::k_step_tiled<L, S, true, true, NT, R><<<g, NT, 0, st>>>(p, in, out, status);
            else kern::k_step_tiled<L, S, false, false, NT, R><<<g, NT, 0, st>>>(p, in, out, status);
        };
        if (tiled_rows_per_thread(p.nx, p.ny) == 1) launch(std::integral_constant<int, 1>{});
        else launch(std::integral_constant<int, kTileRowsPerThread>{});
        return cudaGetLastError();
    }
}

template <class L, class S>
cudaError_t Launch<L, S>::batch_step_tiled(const RepInfo *reps, const int4 *tiles, int ntiles, const void *pop,
                                           void *pop_out, unsigned *status, const unsigned *step_base, unsigned k,
                                           bool full, cudaStream_t st)
{
    if constexpr (L::D != 2) {
        return cudaErrorNotSupported;
    } else {
        constexpr int NT = kTileThreads, R = kTileRowsPerThread;
        auto *in = static_cast<const typename S::T *>(pop);
        auto *out = static_cast<typename S::T *>(pop_out);
        if (full)
            kern::k_step_tiled_batch<L, S, true, true, NT, R><<<ntiles, NT, 0, st>>>(reps, tiles, in, out, status,
                                                                                  step_base, k);
        else
            kern::k_step_tiled_batch<L, S, false, false, NT, R><<<ntiles, NT, 0, st>>>(reps, tiles, in, out, status,
                                                                                    step_base, k);
        return cudaGetLastError();
    }
}

// rows of the tiles of the tiled step (the host cuts boxes into kTileX x rows)
template <class L, class S> int Launch<L, S>::tile_rows() { return kern::TileGeom<kTileThreads, kTileRowsPerThread>::Y; }

template <class L, class S>
cudaError_t Launch<L, S>::init_rest(const StepParams &p, const float *rho_in, void *pop, cudaStream_t st)
{
    kern::k_init_rest<L, S><<<1024, 256, 0, st>>>(p, rho_in, static_cast<typename S::T *>(pop));
    return cudaGetLastError();
}

template <class L, class S>
cudaError_t Launch<L, S>::gather(int parity, const StepParams &p, const void *pop, const int64_t *sites, int64_t n,
                                 double *out, cudaStream_t st)
{
    auto *ptr = static_cast<const typename S::T *>(pop);
    const int blocks = (int)((n + 127) / 128);
    if (parity == 0) kern::k_gather_sites<L, S, 0><<<blocks, 128, 0, st>>>(p, ptr, sites, n, out);
    else kern::k_gather_sites<L, S, 1><<<blocks, 128, 0, st>>>(p, ptr, sites, n, out);
    return cudaGetLastError();
}

template <class L, class S>
cudaError_t Launch<L, S>::sfk_fields(int parity, const StepParams &p, const void *pop, float2 *z, double *partials,
                                     int *nblocks, cudaStream_t st)
{
    const dim3 b(kern::kObsBlock), g((p.nx + kern::kObsBlock - 1) / kern::kObsBlock, p.ny, p.nz);
    *nblocks = (int)(g.x * g.y * g.z);
    const auto planes = kern::plane_table(static_cast<const typename S::T *>(pop), L::Q, p.N);
    if (parity == 0) kern::k_sfk_fields<L, S, 0><<<g, b, 0, st>>>(p, planes, z, partials);
    else kern::k_sfk_fields<L, S, 1><<<g, b, 0, st>>>(p, planes, z, partials);
    return cudaGetLastError();
}

template <class L, class S>
cudaError_t Launch<L, S>::observables(int parity, const StepParams &p, const void *pop, const float *rho, double *ra,
                                      double *rb, double *u, double *partials, int *nblocks, cudaStream_t st)
{
    const dim3 b(kern::kObsBlock), g((p.nx + kern::kObsBlock - 1) / kern::kObsBlock, p.ny, p.nz);
    *nblocks = (int)(g.x * g.y * g.z);
    auto *ptr = static_cast<const typename S::T *>(pop);
    auto *r2 = reinterpret_cast<const float2 *>(rho);
    if (parity == 0) kern::k_observables<L, S, 0><<<g, b, 0, st>>>(p, ptr, r2, ra, rb, u, partials);
    else kern::k_observables<L, S, 1><<<g, b, 0, st>>>(p, ptr, r2, ra, rb, u, partials);
    return cudaGetLastError();
}

} // namespace flbm
