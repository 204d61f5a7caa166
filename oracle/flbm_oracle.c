/*
 * flbm_oracle.c -- plain FP64 CPU oracle for the fluctuating two-species lattice
 * Boltzmann update of Belardinelli, Sbragaglia, Biferale, Gross and Varnik,
 * "Fluctuating multicomponent lattice Boltzmann model" (arXiv 1410.5584).
 *
 * TEST INFRASTRUCTURE ONLY.  This program is the yardstick the CUDA library is
 * checked against.  Only the test suite, the package smoke check and the CPU
 * baseline leg of bench.py may load or run it; the product path never does.
 * It shares no code, header, table or constant with the CUDA library: every
 * table below is built here from the paper's definitions.
 *
 * What it computes, in the paper's order (Sec. V, "Fluctuating lattice
 * Boltzmann equation", Eqs. (algorithm) and (lattice finalstep)), per site r
 * and step n, for both species sigma in {A, B} (primes = the other species):
 *   1. rho = sum_i fbar_i                                 (Sec. V B, after Eq. finalstep;
 *                                                          R_0 = 0 gives rho = rhobar, Sec. V A)
 *   2. a(r) = -G sum_i w_i rho'(r + c_i) c_i               (Sec. VI, Eq. FORCESTRUCTURE)
 *   3. mbar_a = sum_i T_ai fbar_i                           (Eq. modes-discrete, Table I)
 *   4. u = vbar_b + a_b / 2, vbar_b = (jbar + jbar')/rho_t,
 *      a_b = (rho a + rho' a')/rho_t                       (Eq. finalstep and the line after it)
 *   5. Gaussian noise xibar_a with the variances of Eq. (new-noise), local
 *      densities (Sec. VII: actual local densities are used in practice),
 *      xibar'_alpha = -xibar_alpha on the momentum modes (Sec. IV A)
 *   6. R_a = lambdabar_a (m^eq_a(rho, u) - mbar_a) + (1 - lambdabar_a/2) Phi_a + xibar_a
 *      (Eq. finalstep with Eq. forcerenorm); R_0 = 0 (Sec. V A)
 *      m^eq_a = sum_i T_ai f^eq_i, f^eq = 2nd-order Hermite expansion (Eq. hermite-feq)
 *      Phi_a  = sum_i T_ai Phi_i,  Phi  = 2nd-order Hermite expansion (Eq. hermite-for)
 *      with the species velocity from m = mbar + R/2 (Eq. alg-mom, equivalent to Eq. 2system)
 *   7. fbar_i(r + c_i, n+1) = fbar_i(r, n) + w_i sum_a T_ai R_a / N_a   (Eq. algorithm)
 * Streaming is plain two-array push streaming on a fully periodic box.
 *
 * Readings where the paper is silent:
 *   - lambdabar = 1/tau per species for every non-conserved mode; the common
 *     momentum rate lambdabar_d = 2/(tau_A + tau_B) (Sec. III, Eq. diffusionrelaxation
 *     requires one common rate), overridable.
 *   - noise generator: Philox4x32-10 (Salmon et al., SC'11) keyed by the seed;
 *     the Gaussian of mode a >= 1 is Gaussian n = a - 1 of its species, from
 *     counter (site, step, species, n / 6), whose four words are cut into six
 *     21-bit uniforms and three Box-Muller pairs (the paper only says
 *     "Box-Muller", Sec. VI A); see orc_gaussian.
 *   - D3Q19 basis: not in the paper; rows given in d3q19_tables() below.
 *
 * The orcm_* functions at the end hold the N-species update of App. C-D (more
 * than two species, forces between different species only, projected momentum
 * noise); their readings are listed beside them.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXQ 19

/* option keys: same numbers as the public C-ABI's option keys */
#define ORC_OPT_LAMBDA_D 2
#define ORC_OPT_SDF 3
#define ORC_OPT_RHO0_A 4
#define ORC_OPT_RHO0_B 5
#define ORC_OPT_NOISE_RHO 7
#define ORC_OPT_FORCE_VELOCITY 8
#define ORC_OPT_GHOST_NOISE 21
#define ORC_OPT_LAMBDA_MODE 1000 /* + 100*species + a */

typedef struct {
    int D, Q;
    int c[ORC_MAXQ][3];
    double w[ORC_MAXQ];
    double T[ORC_MAXQ][ORC_MAXQ]; /* T[a][i] */
    double N[ORC_MAXQ];
    int opp[ORC_MAXQ];
} orc_lattice;

typedef struct {
    int lat;
    orc_lattice L;
    int nx, ny, nz;
    long N;
    double tau[2], kT, G;
    uint64_t seed;
    double lam[2][ORC_MAXQ]; /* lambdabar per species and mode */
    int sdf;
    int noise_ref;          /* 0: local densities in the noise, 1: reference rho0 */
    int force_velocity;     /* 0: rho v = jbar + R_j/2 ; 1: v = vbar + a/2 */
    int ghost_noise;        /* 1: non-conserved noise from population-space draws at the
                               destination densities (see collide_site) */
    double rho0[2];
    double *f[2];   /* f[s][i*N + site] */
    double *fn[2];  /* push-streaming target */
    double *rho[2]; /* density field of the current step */
    long step;
    int threads; /* OpenMP threads for the site loops (1 = serial) */
    /* noise site numbering: by default the site's own index; for a block cut
     * out of a larger box, the index the site has in that box */
    int rng_global;
    long gnx, gny, gnz, ox, oy, oz;
    /* structure-factor accumulators, index m-1 for k_m = 2 pi m / n_axis */
    int sf_axis, sf_nk;
    double *sf_aa, *sf_ab, *sf_bb, *sf_uu;
    long sf_n;
} orc_t;

/* ------------------------------------------------------------------------ */
/* Lattices                                                                  */
/* ------------------------------------------------------------------------ */

/* D2Q9 with the basis of Table I (Sec. VI).  Weights 4/9, 1/9, 1/36 are the
 * Gauss-Hermite weights that satisfy the isotropy relations Eq. (w-rel) with
 * c_T^2 = 1/3 (Sec. V B). */
static void d2q9_tables(orc_lattice *L)
{
    static const int cv[9][2] = {{0, 0}, {1, 0}, {0, 1}, {-1, 0}, {0, -1},
                                 {1, 1}, {-1, 1}, {-1, -1}, {1, -1}};
    /* squared norms N_a exactly as printed in Table I */
    static const double Nt[9] = {1.0, 1.0 / 3.0, 1.0 / 3.0, 4.0, 4.0 / 9.0,
                                 1.0 / 9.0, 2.0 / 3.0, 2.0 / 3.0, 16.0};
    memset(L, 0, sizeof(*L));
    L->D = 2;
    L->Q = 9;
    for (int i = 0; i < 9; i++) {
        int cx = cv[i][0], cy = cv[i][1];
        double c2 = cx * cx + cy * cy;
        L->c[i][0] = cx;
        L->c[i][1] = cy;
        L->c[i][2] = 0;
        L->w[i] = (c2 == 0) ? 4.0 / 9.0 : (c2 == 1 ? 1.0 / 9.0 : 1.0 / 36.0);
        /* rows of Table I */
        L->T[0][i] = 1.0;
        L->T[1][i] = cx;
        L->T[2][i] = cy;
        L->T[3][i] = 3.0 * c2 - 2.0;
        L->T[4][i] = 2.0 * cx * cx - c2;
        L->T[5][i] = (double)cx * cy;
        L->T[6][i] = (3.0 * c2 - 4.0) * cx;
        L->T[7][i] = (3.0 * c2 - 4.0) * cy;
        L->T[8][i] = 9.0 * c2 * c2 - 15.0 * c2 + 2.0;
    }
    for (int a = 0; a < 9; a++) L->N[a] = Nt[a];
}

/* D3Q19: not in the paper.  Reading: standard D3Q19 velocities and weights
 * (1/3, 1/18, 1/36), first 10 rows the Hermite modes of order <= 2 (as in
 * Eq. setofT), then an orthogonal completion by ghost modes. */
static void d3q19_tables(orc_lattice *L)
{
    static const int cv[19][3] = {
        {0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},   {0, -1, 0},
        {0, 0, 1},  {0, 0, -1}, {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
        {-1, 1, 0}, {1, 0, 1},  {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
        {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
    memset(L, 0, sizeof(*L));
    L->D = 3;
    L->Q = 19;
    for (int i = 0; i < 19; i++) {
        double x = cv[i][0], y = cv[i][1], z = cv[i][2];
        double c2 = x * x + y * y + z * z;
        for (int d = 0; d < 3; d++) L->c[i][d] = cv[i][d];
        L->w[i] = (c2 == 0) ? 1.0 / 3.0 : (c2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
        L->T[0][i] = 1.0;
        L->T[1][i] = x;
        L->T[2][i] = y;
        L->T[3][i] = z;
        L->T[4][i] = c2 - 1.0;
        L->T[5][i] = 2.0 * x * x - y * y - z * z;
        L->T[6][i] = y * y - z * z;
        L->T[7][i] = x * y;
        L->T[8][i] = y * z;
        L->T[9][i] = x * z;
        L->T[10][i] = (3.0 * c2 - 5.0) * x;
        L->T[11][i] = (3.0 * c2 - 5.0) * y;
        L->T[12][i] = (3.0 * c2 - 5.0) * z;
        L->T[13][i] = x * (y * y - z * z);
        L->T[14][i] = y * (z * z - x * x);
        L->T[15][i] = z * (x * x - y * y);
        L->T[16][i] = 3.0 * c2 * c2 - 6.0 * c2 + 1.0;
        L->T[17][i] = (2.0 * c2 - 3.0) * (2.0 * x * x - y * y - z * z);
        L->T[18][i] = (2.0 * c2 - 3.0) * (y * y - z * z);
    }
    /* squared norms N_a = sum_i w_i T_ai^2 (Eq. V-orthog-compl-discrete) */
    for (int a = 0; a < 19; a++) {
        double s = 0.0;
        for (int i = 0; i < 19; i++) s += L->w[i] * L->T[a][i] * L->T[a][i];
        L->N[a] = s;
    }
}

static int build_lattice(int lat, orc_lattice *L)
{
    if (lat == 0)
        d2q9_tables(L);
    else if (lat == 1)
        d3q19_tables(L);
    else
        return -1;
    for (int i = 0; i < L->Q; i++) {
        L->opp[i] = -1;
        for (int j = 0; j < L->Q; j++)
            if (L->c[j][0] == -L->c[i][0] && L->c[j][1] == -L->c[i][1] &&
                L->c[j][2] == -L->c[i][2])
                L->opp[i] = j;
    }
    return 0;
}


/* ------------------------------------------------------------------------ */
/* Noise: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers:  */
/* as easy as 1, 2, 3", SC'11) and the Box-Muller transform.                 */
/* ------------------------------------------------------------------------ */

static void mulhilo32(uint32_t a, uint32_t b, uint32_t *hi, uint32_t *lo)
{
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    *lo = (uint32_t)p;
}

/* Philox4x32 with R = 10 rounds.  One round maps (x0,x1,x2,x3) with key
 * (k0,k1) to (hi(M1*x2) ^ x1 ^ k0, lo(M1*x2), hi(M0*x0) ^ x3 ^ k1, lo(M0*x0));
 * the key is bumped by the Weyl constants between rounds. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; r++) {
        if (r > 0) {
            k0 += W0;
            k1 += W1;
        }
        uint32_t hi0, lo0, hi1, lo1;
        mulhilo32(M0, x0, &hi0, &lo0);
        mulhilo32(M1, x2, &hi1, &lo1);
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0;
        x1 = y1;
        x2 = y2;
        x3 = y3;
    }
    out[0] = x0;
    out[1] = x1;
    out[2] = x2;
    out[3] = x3;
}

/* Box-Muller on two 21-bit uniforms U1, U2 in [0, 2^21): u1 = (U1 + 1) 2^-21
 * in (0, 1], u2 = U2 2^-21 in [0, 1); g0 = sqrt(-2 ln u1) cos(2 pi u2),
 * g1 = sqrt(-2 ln u1) sin(2 pi u2). */
static void box_muller(uint32_t U1, uint32_t U2, double *g0, double *g1)
{
    const double two_m21 = 1.0 / 2097152.0;
    double u1 = ((double)U1 + 1.0) * two_m21;
    double u2 = (double)U2 * two_m21;
    double r = sqrt(-2.0 * log(u1));
    double th = 2.0 * M_PI * u2;
    *g0 = r * cos(th);
    *g1 = r * sin(th);
}

/* The standard Gaussian used for mode a >= 1 of species s at (site, step).
 * Mode a is Gaussian n = a - 1 of the species.  Philox counter
 * (site, step, s, n / 6) gives four words x0 .. x3, cut into six 21-bit
 * uniforms: U_k = x_k >> 11 for k = 0 .. 3, and from the low bits
 * U4 = (x0 mod 2^11) 2^10 + (x1 mod 2^10), U5 = (x2 mod 2^11) 2^10 + (x3 mod 2^10).
 * Gaussian n is the cosine (n even) or sine (n odd) output of Box-Muller on
 * the pair (U_2q, U_2q+1), q = (n mod 6) / 2.  Mode 0 (the conserved density)
 * has no Gaussian: NAN. */
double orc_gaussian(uint64_t seed, uint32_t site, uint32_t step, uint32_t species, uint32_t a)
{
    if (a == 0u) return NAN;
    const uint32_t n = a - 1u;
    uint32_t ctr[4] = {site, step, species, n / 6u};
    uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
    uint32_t x[4];
    orc_philox4x32_10(ctr, key, x);
    uint32_t U[6];
    for (int k = 0; k < 4; k++) U[k] = x[k] >> 11;
    U[4] = ((x[0] & 0x7FFu) << 10) | (x[1] & 0x3FFu);
    U[5] = ((x[2] & 0x7FFu) << 10) | (x[3] & 0x3FFu);
    const uint32_t q = (n % 6u) / 2u;
    double g0, g1;
    box_muller(U[2 * q], U[2 * q + 1], &g0, &g1);
    return (n % 2u == 0u) ? g0 : g1;
}

/* ------------------------------------------------------------------------ */
/* Equilibrium and forcing moments by projection (Eqs. hermite-feq, hermite-for) */
/* ------------------------------------------------------------------------ */

/* f^eq_i(rho, u) truncated at second order in u (Eq. hermite-feq on the
 * lattice, c_T^2 = 1/3):  w_i rho [1 + c.u/c_T^2 + (c c - c_T^2 I):u u/(2 c_T^4)]. */
static void feq_pop(const orc_lattice *L, double rho, const double u[3], double out[ORC_MAXQ])
{
    const double cs2 = 1.0 / 3.0;
    for (int i = 0; i < L->Q; i++) {
        double cu = 0.0, uu = 0.0;
        for (int d = 0; d < 3; d++) {
            cu += L->c[i][d] * u[d];
            uu += u[d] * u[d];
        }
        out[i] = L->w[i] * rho * (1.0 + cu / cs2 + (cu * cu - cs2 * uu) / (2.0 * cs2 * cs2));
    }
}

/* Phi_i(rho, a, v) truncated at second order (Eq. hermite-for):
 * w_i rho [c.a/c_T^2 + (c c - c_T^2 I):(a v)/c_T^4]. */
static void phi_pop(const orc_lattice *L, double rho, const double acc[3], const double v[3],
                    double out[ORC_MAXQ])
{
    const double cs2 = 1.0 / 3.0;
    for (int i = 0; i < L->Q; i++) {
        double ca = 0.0, cv = 0.0, av = 0.0;
        for (int d = 0; d < 3; d++) {
            ca += L->c[i][d] * acc[d];
            cv += L->c[i][d] * v[d];
            av += acc[d] * v[d];
        }
        out[i] = L->w[i] * rho * (ca / cs2 + (ca * cv - cs2 * av) / (cs2 * cs2));
    }
}

static void project(const orc_lattice *L, const double pop[ORC_MAXQ], double mom[ORC_MAXQ])
{
    for (int a = 0; a < L->Q; a++) {
        double s = 0.0;
        for (int i = 0; i < L->Q; i++) s += L->T[a][i] * pop[i];
        mom[a] = s;
    }
}

/* m^eq_a(rho, u) = sum_i T_ai f^eq_i(rho, u)  (Table I caption) */
int orc_meq(int lat, double rho, const double *u, double *out)
{
    orc_lattice L;
    if (build_lattice(lat, &L)) return -1;
    double uu[3] = {u[0], u[1], L.D == 3 ? u[2] : 0.0};
    double p[ORC_MAXQ];
    feq_pop(&L, rho, uu, p);
    project(&L, p, out);
    return 0;
}

/* Phi_a(rho, a, v) = sum_i T_ai Phi_i(rho, a, v) */
int orc_phi(int lat, double rho, const double *acc, const double *v, double *out)
{
    orc_lattice L;
    if (build_lattice(lat, &L)) return -1;
    double aa[3] = {acc[0], acc[1], L.D == 3 ? acc[2] : 0.0};
    double vv[3] = {v[0], v[1], L.D == 3 ? v[2] : 0.0};
    double p[ORC_MAXQ];
    phi_pop(&L, rho, aa, vv, p);
    project(&L, p, out);
    return 0;
}

/* Export of the lattice tables for the basis pins. */
int orc_tables(int lat, int *D, int *Q, int *c, double *w, double *T, double *N)
{
    orc_lattice L;
    if (build_lattice(lat, &L)) return -1;
    *D = L.D;
    *Q = L.Q;
    for (int i = 0; i < L.Q; i++) {
        for (int d = 0; d < 3; d++) c[i * 3 + d] = L.c[i][d];
        w[i] = L.w[i];
    }
    for (int a = 0; a < L.Q; a++) {
        N[a] = L.N[a];
        for (int i = 0; i < L.Q; i++) T[a * L.Q + i] = L.T[a][i];
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* State                                                                     */
/* ------------------------------------------------------------------------ */

static void set_default_rates(orc_t *o)
{
    for (int s = 0; s < 2; s++)
        for (int a = 0; a < o->L.Q; a++) o->lam[s][a] = (a == 0) ? 0.0 : 1.0 / o->tau[s];
    double lam_d = (o->tau[0] == o->tau[1]) ? 1.0 / o->tau[0] : 2.0 / (o->tau[0] + o->tau[1]);
    for (int s = 0; s < 2; s++)
        for (int a = 1; a <= o->L.D; a++) o->lam[s][a] = lam_d;
}

orc_t *orc_create(int lat, int nx, int ny, int nz, double tau_a, double tau_b, double kT,
                  double G, uint64_t seed)
{
    orc_t *o = (orc_t *)calloc(1, sizeof(orc_t));
    if (!o) return NULL;
    if (build_lattice(lat, &o->L)) {
        free(o);
        return NULL;
    }
    if (lat == 0) nz = 1;
    o->lat = lat;
    o->nx = nx;
    o->ny = ny;
    o->nz = nz;
    o->N = (long)nx * ny * nz;
    o->tau[0] = tau_a;
    o->tau[1] = tau_b;
    o->kT = kT;
    o->G = G;
    o->seed = seed;
    o->sdf = 1;
    o->threads = 1;
    o->rho0[0] = o->rho0[1] = 1.0;
    set_default_rates(o);
    for (int s = 0; s < 2; s++) {
        o->f[s] = (double *)calloc((size_t)o->L.Q * o->N, sizeof(double));
        o->fn[s] = (double *)calloc((size_t)o->L.Q * o->N, sizeof(double));
        o->rho[s] = (double *)calloc((size_t)o->N, sizeof(double));
        if (!o->f[s] || !o->fn[s] || !o->rho[s]) return NULL;
    }
    return o;
}

static void sf_free(orc_t *o)
{
    free(o->sf_aa);
    free(o->sf_ab);
    free(o->sf_bb);
    free(o->sf_uu);
    o->sf_aa = o->sf_ab = o->sf_bb = o->sf_uu = NULL;
    o->sf_n = 0;
}

void orc_destroy(orc_t *o)
{
    if (!o) return;
    for (int s = 0; s < 2; s++) {
        free(o->f[s]);
        free(o->fn[s]);
        free(o->rho[s]);
    }
    sf_free(o);
    free(o);
}

int orc_set_option(orc_t *o, int key, double value)
{
    if (key == ORC_OPT_LAMBDA_D) {
        for (int s = 0; s < 2; s++)
            for (int a = 1; a <= o->L.D; a++) o->lam[s][a] = value;
    } else if (key == ORC_OPT_SDF) {
        o->sdf = value != 0.0;
    } else if (key == ORC_OPT_RHO0_A) {
        o->rho0[0] = value;
    } else if (key == ORC_OPT_RHO0_B) {
        o->rho0[1] = value;
    } else if (key == ORC_OPT_NOISE_RHO) {
        o->noise_ref = value != 0.0;
    } else if (key == ORC_OPT_FORCE_VELOCITY) {
        o->force_velocity = value != 0.0;
    } else if (key == ORC_OPT_GHOST_NOISE) {
        o->ghost_noise = value != 0.0;
    } else if (key >= ORC_OPT_LAMBDA_MODE && key < ORC_OPT_LAMBDA_MODE + 200) {
        int s = (key - ORC_OPT_LAMBDA_MODE) / 100, a = (key - ORC_OPT_LAMBDA_MODE) % 100;
        if (a <= o->L.D || a >= o->L.Q) return 1;
        o->lam[s][a] = value;
    } else {
        return 1;
    }
    return 0;
}

/* Rest-state populations f_i = w_i rho(r) (f^eq at u = 0, Sec. V B). */
int orc_init(orc_t *o, const double *rho_a, const double *rho_b)
{
    const double *in[2] = {rho_a, rho_b};
    for (int s = 0; s < 2; s++)
        for (long site = 0; site < o->N; site++) {
            double r = in[s] ? in[s][site] : o->rho0[s];
            for (int i = 0; i < o->L.Q; i++) o->f[s][i * o->N + site] = o->L.w[i] * r;
        }
    o->step = 0;
    return 0;
}

void orc_set_f(orc_t *o, const double *f, long step)
{
    for (int s = 0; s < 2; s++)
        memcpy(o->f[s], f + (size_t)s * o->L.Q * o->N, sizeof(double) * o->L.Q * o->N);
    o->step = step;
}

void orc_get_f(const orc_t *o, double *f)
{
    for (int s = 0; s < 2; s++)
        memcpy(f + (size_t)s * o->L.Q * o->N, o->f[s], sizeof(double) * o->L.Q * o->N);
}

long orc_get_step(const orc_t *o) { return o->step; }

void orc_set_threads(orc_t *o, int n) { o->threads = n > 0 ? n : 1; }

/* Treat this box as the block of a periodic gnx * gny * gnz box whose local
 * site (0,0,0) sits at (ox, oy, oz): the noise of a site is then drawn with
 * its index in the large box, so a block's update can be checked against a
 * run on the large box. */
void orc_set_rng_origin(orc_t *o, long gnx, long gny, long gnz, long ox, long oy, long oz)
{
    o->rng_global = 1;
    o->gnx = gnx;
    o->gny = gny;
    o->gnz = gnz;
    o->ox = ox;
    o->oy = oy;
    o->oz = oz;
}

static uint32_t rng_site(const orc_t *o, long site)
{
    if (!o->rng_global) return (uint32_t)site;
    long x = site % o->nx, y = (site / o->nx) % o->ny, z = site / ((long)o->nx * o->ny);
    long gx = (x + o->ox) % o->gnx, gy = (y + o->oy) % o->gny, gz = (z + o->oz) % o->gnz;
    return (uint32_t)((gz * o->gny + gy) * o->gnx + gx);
}

/* site index r + c (periodic) */
static long neighbour(const orc_t *o, long site, const int c[3])
{
    long x = site % o->nx;
    long y = (site / o->nx) % o->ny;
    long z = site / ((long)o->nx * o->ny);
    x = (x + c[0] + o->nx) % o->nx;
    y = (y + c[1] + o->ny) % o->ny;
    z = (z + c[2] + o->nz) % o->nz;
    return (z * o->ny + y) * o->nx + x;
}

static void density_pass(orc_t *o)
{
    for (int s = 0; s < 2; s++)
#pragma omp parallel for num_threads(o->threads) schedule(static)
        for (long site = 0; site < o->N; site++) {
            double r = 0.0;
            for (int i = 0; i < o->L.Q; i++) r += o->f[s][i * o->N + site];
            o->rho[s][site] = r;
        }
}

/* a^s(r) = -G sum_i w_i rho^{s'}(r + c_i) c_i   (Eq. FORCESTRUCTURE) */
static void acceleration(const orc_t *o, long site, int s, double acc[3])
{
    const double *rp = o->rho[1 - s];
    acc[0] = acc[1] = acc[2] = 0.0;
    for (int i = 0; i < o->L.Q; i++) {
        double r = rp[neighbour(o, site, o->L.c[i])];
        for (int d = 0; d < 3; d++) acc[d] += -o->G * o->L.w[i] * r * o->L.c[i][d];
    }
}

/* Collision at one site: fills R[s][a] for both species.  Returns nonzero if a
 * density is not positive and finite. */
static int collide_site(const orc_t *o, long site, double R[2][ORC_MAXQ])
{
    const orc_lattice *L = &o->L;
    const int D = L->D, Q = L->Q;
    double rho[2], m[2][ORC_MAXQ], acc[2][3];
    for (int s = 0; s < 2; s++) {
        double pop[ORC_MAXQ];
        for (int i = 0; i < Q; i++) pop[i] = o->f[s][i * o->N + site];
        project(L, pop, m[s]);
        rho[s] = o->rho[s][site];
        if (!(rho[s] > 0.0) || !isfinite(rho[s])) return 1;
        acceleration(o, site, s, acc[s]);
    }
    /* baricentric velocity with the half-force shift (Eq. finalstep) */
    double rho_t = rho[0] + rho[1];
    double u[3] = {0.0, 0.0, 0.0};
    for (int d = 0; d < D; d++) {
        double vb = (m[0][1 + d] + m[1][1 + d]) / rho_t;
        double ab = (rho[0] * acc[0][d] + rho[1] * acc[1][d]) / rho_t;
        u[d] = vb + 0.5 * ab;
    }
    /* noise amplitudes, Eq. (new-noise) with Delta t = 1 */
    double nr[2];
    for (int s = 0; s < 2; s++) nr[s] = o->noise_ref ? o->rho0[s] : rho[s];
    const double mu = 3.0 * o->kT; /* k_B T / c_T^2 */
    double xi[2][ORC_MAXQ];
    for (int s = 0; s < 2; s++)
        for (int a = 0; a < Q; a++) xi[s][a] = 0.0;
    {
        double lam_d = o->lam[0][1];
        double var_j = (2.0 * lam_d - lam_d * lam_d) * o->kT * nr[0] * nr[1] / (nr[0] + nr[1]);
        double sj = o->sdf ? sqrt(var_j) : 0.0;
        for (int d = 0; d < D; d++) {
            double g = orc_gaussian(o->seed, rng_site(o, site), (uint32_t)o->step, 0u, (uint32_t)(1 + d));
            xi[0][1 + d] = sj * g;
            xi[1][1 + d] = -xi[0][1 + d];
        }
    }
    if (!o->ghost_noise) {
        for (int s = 0; s < 2; s++)
            for (int a = D + 1; a < Q; a++) {
                double lam = o->lam[s][a];
                double var = (2.0 * lam - lam * lam) * L->N[a] * mu * nr[s];
                double g = orc_gaussian(o->seed, rng_site(o, site), (uint32_t)o->step, (uint32_t)s, (uint32_t)a);
                xi[s][a] = sqrt(var) * g;
            }
    } else {
        /* Off-diagonal noise of the non-conserved modes (the correction the
         * paper describes after Eq. finalstep, Sec. V B, and leaves open in
         * Sec. VII; reading in the design notes): population i of species s
         * leaves r for r + c_i, where local equilibrium gives it the variance
         * mu w_i rho^s(r + c_i).  One Gaussian eta_i per population, scaled so,
         * projected on the non-conserved rows, with the factor
         * (2 lambdabar_a - lambdabar_a^2)^(1/2) of Eq. new-noise:
         *   xi_a = sqrt(2 lb_a - lb_a^2) sum_i T_ai sqrt(mu w_i rho^s(r + c_i)) eta_i,
         * covariance (for equal rates) (2 lb - lb^2) mu sum_i T_ai T_bi w_i rho^s(r + c_i),
         * which is Eq. new-noise (diagonal, N_a mu rho) wherever rho^s is
         * uniform.  eta_i is Gaussian number i of species slot s + 2 (the
         * slots of the mode draws are 0 and 1). */
        for (int s = 0; s < 2; s++) {
            double x[ORC_MAXQ];
            for (int i = 0; i < Q; i++) {
                const double ri = o->noise_ref ? o->rho0[s] : o->rho[s][neighbour(o, site, L->c[i])];
                if (!(ri > 0.0) || !isfinite(ri)) return 1;
                const double eta = orc_gaussian(o->seed, rng_site(o, site), (uint32_t)o->step, (uint32_t)(s + 2),
                                                (uint32_t)(i + 1));
                x[i] = sqrt(mu * L->w[i] * ri) * eta;
            }
            for (int a = D + 1; a < Q; a++) {
                double lam = o->lam[s][a], t = 0.0;
                for (int i = 0; i < Q; i++) t += L->T[a][i] * x[i];
                xi[s][a] = sqrt(2.0 * lam - lam * lam) * t;
            }
        }
    }
    /* momentum modes: R_alpha (Eq. finalstep, m^eq_alpha = rho u_alpha, Phi_alpha = rho a_alpha) */
    double meq[2][ORC_MAXQ], phi[2][ORC_MAXQ], v[2][3];
    for (int s = 0; s < 2; s++) {
        double pfeq[ORC_MAXQ];
        feq_pop(L, rho[s], u, pfeq);
        project(L, pfeq, meq[s]);
        /* The momentum projection of Phi is rho a whatever v is (the second-order
         * term of Eq. hermite-for is even in c), so v = 0 may be used here,
         * before v is known. */
        double zero[3] = {0.0, 0.0, 0.0};
        double pphi[ORC_MAXQ];
        phi_pop(L, rho[s], acc[s], zero, pphi);
        project(L, pphi, phi[s]);
        R[s][0] = 0.0;
        for (int d = 0; d < D; d++) {
            int a = 1 + d;
            double lam = o->lam[s][a];
            R[s][a] = lam * (meq[s][a] - m[s][a]) + (1.0 - 0.5 * lam) * phi[s][a] + xi[s][a];
        }
        /* species velocity for the second-order forcing moments */
        v[s][0] = v[s][1] = v[s][2] = 0.0;
        for (int d = 0; d < D; d++) {
            if (o->force_velocity == 0)
                v[s][d] = (m[s][1 + d] + 0.5 * R[s][1 + d]) / rho[s]; /* m = mbar + R/2, Eq. alg-mom */
            else
                v[s][d] = m[s][1 + d] / rho[s] + 0.5 * acc[s][d];
        }
    }
    /* transport and ghost modes (Eq. finalstep with Eq. forcerenorm) */
    for (int s = 0; s < 2; s++) {
        double pphi[ORC_MAXQ], mphi[ORC_MAXQ];
        phi_pop(L, rho[s], acc[s], v[s], pphi);
        project(L, pphi, mphi);
        for (int a = D + 1; a < Q; a++) {
            double lam = o->lam[s][a];
            R[s][a] = lam * (meq[s][a] - m[s][a]) + (1.0 - 0.5 * lam) * mphi[a] + xi[s][a];
        }
    }
    return 0;
}

/* n steps of Eq. (algorithm).  Returns 0, or 4 if a density became
 * non-positive or non-finite (the state is then left at the failing step). */
int orc_step(orc_t *o, long n)
{
    const orc_lattice *L = &o->L;
    for (long t = 0; t < n; t++) {
        density_pass(o);
        int bad = 0;
        /* sites are independent: each writes only its own Q destinations */
#pragma omp parallel for num_threads(o->threads) schedule(static) reduction(|| : bad)
        for (long site = 0; site < o->N; site++) {
            double R[2][ORC_MAXQ];
            if (collide_site(o, site, R)) {
                bad = 1;
                continue;
            }
            for (int s = 0; s < 2; s++)
                for (int i = 0; i < L->Q; i++) {
                    double dr = 0.0;
                    for (int a = 0; a < L->Q; a++) dr += L->T[a][i] * R[s][a] / L->N[a];
                    long dst = neighbour(o, site, L->c[i]);
                    o->fn[s][i * o->N + dst] = o->f[s][i * o->N + site] + L->w[i] * dr;
                }
        }
        if (bad) return 4;
        for (int s = 0; s < 2; s++) {
            double *t2 = o->f[s];
            o->f[s] = o->fn[s];
            o->fn[s] = t2;
        }
        o->step++;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Observables                                                               */
/* ------------------------------------------------------------------------ */

/* rho^A, rho^B, u_b = (jbar + jbar' + (F + F')/2)/rho_t with F = rho a
 * (Eq. lattice-vb), and the conserved totals
 * cons = [sum rho^A, sum rho^B, sum (jbar_t + F_t/2)_x, _y, _z]. */
int orc_moments(orc_t *o, double *rho_a, double *rho_b, double *u, double *cons)
{
    const orc_lattice *L = &o->L;
    density_pass(o);
    double tot[5] = {0, 0, 0, 0, 0};
    for (long site = 0; site < o->N; site++) {
        double rho[2], j[2][3] = {{0}}, acc[2][3];
        for (int s = 0; s < 2; s++) {
            rho[s] = o->rho[s][site];
            for (int i = 0; i < L->Q; i++)
                for (int d = 0; d < 3; d++) j[s][d] += L->c[i][d] * o->f[s][i * o->N + site];
            acceleration(o, site, s, acc[s]);
        }
        double rho_t = rho[0] + rho[1];
        if (rho_a) rho_a[site] = rho[0];
        if (rho_b) rho_b[site] = rho[1];
        tot[0] += rho[0];
        tot[1] += rho[1];
        for (int d = 0; d < L->D; d++) {
            double jt = j[0][d] + j[1][d] + 0.5 * (rho[0] * acc[0][d] + rho[1] * acc[1][d]);
            if (u) u[(long)d * o->N + site] = jt / rho_t;
            tot[2 + d] += jt;
        }
    }
    if (cons)
        for (int k = 0; k < 5; k++) cons[k] = tot[k];
    return 0;
}

/* One structure-factor snapshot along a lattice axis (0 = x, 1 = y, 2 = z):
 * S(k_m) += |sum_r drho(r) e^{-i k_m r_axis}|^2 / N for k_m = 2 pi m / n_axis,
 * m = 1..nk, i.e. the wavevector lies along the axis (Sec. VI A); the profile
 * along the axis is summed over the other coordinates first. */
int orc_sf_sample(orc_t *o, int axis, int nk)
{
    const int D = o->L.D;
    int n_axis = axis == 0 ? o->nx : (axis == 1 ? o->ny : o->nz);
    if (axis < 0 || axis >= D || nk < 1 || nk > n_axis / 2) return 1;
    if (!o->sf_aa || o->sf_axis != axis || o->sf_nk != nk) {
        sf_free(o);
        o->sf_axis = axis;
        o->sf_nk = nk;
        o->sf_aa = (double *)calloc(nk, sizeof(double));
        o->sf_ab = (double *)calloc(nk, sizeof(double));
        o->sf_bb = (double *)calloc(nk, sizeof(double));
        o->sf_uu = (double *)calloc(nk, sizeof(double));
    }
    double *ra = (double *)malloc(sizeof(double) * o->N);
    double *rb = (double *)malloc(sizeof(double) * o->N);
    double *u = (double *)malloc(sizeof(double) * o->N * D);
    double *pa = (double *)calloc(n_axis, sizeof(double));
    double *pb = (double *)calloc(n_axis, sizeof(double));
    double *pu = (double *)calloc((size_t)n_axis * D, sizeof(double));
    orc_moments(o, ra, rb, u, NULL);
    for (long site = 0; site < o->N; site++) {
        long x = site % o->nx, y = (site / o->nx) % o->ny, z = site / ((long)o->nx * o->ny);
        long p = axis == 0 ? x : (axis == 1 ? y : z);
        pa[p] += ra[site];
        pb[p] += rb[site];
        for (int d = 0; d < D; d++) pu[d * n_axis + p] += u[(long)d * o->N + site];
    }
    for (int m = 1; m <= nk; m++) {
        double k = 2.0 * M_PI * m / n_axis;
        double are = 0, aim = 0, bre = 0, bim = 0, uu = 0;
        for (int p = 0; p < n_axis; p++) {
            are += pa[p] * cos(k * p);
            aim -= pa[p] * sin(k * p);
            bre += pb[p] * cos(k * p);
            bim -= pb[p] * sin(k * p);
        }
        for (int d = 0; d < D; d++) {
            double ure = 0, uim = 0;
            for (int p = 0; p < n_axis; p++) {
                ure += pu[d * n_axis + p] * cos(k * p);
                uim -= pu[d * n_axis + p] * sin(k * p);
            }
            uu += (ure * ure + uim * uim) / D;
        }
        o->sf_aa[m - 1] += (are * are + aim * aim) / o->N;
        o->sf_bb[m - 1] += (bre * bre + bim * bim) / o->N;
        o->sf_ab[m - 1] += (are * bre + aim * bim) / o->N;
        o->sf_uu[m - 1] += uu / o->N;
    }
    o->sf_n++;
    free(ra);
    free(rb);
    free(u);
    free(pa);
    free(pb);
    free(pu);
    return 0;
}

/* Ensemble means of the accumulated snapshots; resets nothing. */
int orc_structure_factor(const orc_t *o, double *s_aa, double *s_ab, double *s_bb, double *s_uu,
                         long *nsamples)
{
    *nsamples = o->sf_n;
    if (o->sf_n == 0) return 1;
    for (int m = 0; m < o->sf_nk; m++) {
        s_aa[m] = o->sf_aa[m] / o->sf_n;
        s_ab[m] = o->sf_ab[m] / o->sf_n;
        s_bb[m] = o->sf_bb[m] / o->sf_n;
        s_uu[m] = o->sf_uu[m] / o->sf_n;
    }
    return 0;
}

void orc_sf_reset(orc_t *o) { sf_free(o); }

/* ======================================================================== */
/* N species (App. C-D: the multicomponent generalisation), N = 2 .. 8       */
/* ======================================================================== */
/*
 * The update of Sec. V for N species sigma, each with its own rate
 * lambdabar_sigma = 1/tau_sigma for every non-conserved mode, a common
 * momentum rate lambdabar_d (total momentum conservation needs one; by default
 * N / sum_sigma tau_sigma, i.e. 2/(tau_A + tau_B) for two species) and
 * mean-field forces between different species only (App. D: the species are
 * not self-interacting; G symmetric, G_ss = 0):
 *   a^s(r) = -sum_{s' != s} G_{s s'} sum_i w_i rho^{s'}(r + c_i) c_i
 *   u = sum_s (jbar^s + rho^s a^s / 2) / rho_t
 * Noise (App. D, homogeneous form with the local densities): the momentum
 * noises have the covariance (2 lb_d - lb_d^2) k_B T (rho^s delta_{s s'} -
 * rho^s rho^{s'} / rho_t); drawn as xi^s = A (eta^s - C^s sum_{s'} eta^{s'}) with
 * eta^s = sqrt(rho^s) g^s, C^s = rho^s / rho_t, A = sqrt((2 lb_d - lb_d^2) k_B T),
 * which has exactly that covariance and zero total.  The other modes have the
 * variances of Eq. new-noise per species, independent.  g^s of mode a comes
 * from orc_gaussian(seed, site, step, s, a) for every mode a >= 1.
 */
#define ORCM_MAXS 8

typedef struct {
    int lat;
    orc_lattice L;
    int ns, nx, ny, nz;
    long N;
    double tau[ORCM_MAXS], kT, G[ORCM_MAXS][ORCM_MAXS], lam_d;
    uint64_t seed;
    double *f[ORCM_MAXS], *fn[ORCM_MAXS], *rho[ORCM_MAXS];
    long step;
    int rng_global;           /* noise drawn with site indices of a larger box */
    long gnx, gny, gnz, ox, oy, oz;
} orcm_t;

void orcm_destroy(orcm_t *o);

orcm_t *orcm_create(int lat, int ns, int nx, int ny, int nz, const double *tau, double kT, const double *G,
                    uint64_t seed)
{
    if (ns < 2 || ns > ORCM_MAXS) return NULL;
    orcm_t *o = (orcm_t *)calloc(1, sizeof(orcm_t));
    if (!o) return NULL;
    if (build_lattice(lat, &o->L)) {
        free(o);
        return NULL;
    }
    o->lat = lat;
    o->ns = ns;
    o->nx = nx;
    o->ny = ny;
    o->nz = o->L.D == 2 ? 1 : nz;
    o->N = (long)o->nx * o->ny * o->nz;
    o->kT = kT;
    o->seed = seed;
    double tsum = 0.0;
    for (int s = 0; s < ns; s++) {
        o->tau[s] = tau[s];
        tsum += tau[s];
        for (int t = 0; t < ns; t++) o->G[s][t] = s == t ? 0.0 : G[s * ns + t];
    }
    o->lam_d = ns / tsum;
    for (int s = 0; s < ns; s++) {
        o->f[s] = (double *)calloc((size_t)o->L.Q * o->N, sizeof(double));
        o->fn[s] = (double *)calloc((size_t)o->L.Q * o->N, sizeof(double));
        o->rho[s] = (double *)calloc((size_t)o->N, sizeof(double));
        if (!o->f[s] || !o->fn[s] || !o->rho[s]) {
            orcm_destroy(o); /* frees what was allocated (the rest is NULL) */
            return NULL;
        }
    }
    return o;
}

void orcm_destroy(orcm_t *o)
{
    if (!o) return;
    for (int s = 0; s < o->ns; s++) {
        free(o->f[s]);
        free(o->fn[s]);
        free(o->rho[s]);
    }
    free(o);
}

/* rest state f_i = w_i rho^s (rho: ns planes of N, or NULL for rho = 1) */
void orcm_init(orcm_t *o, const double *rho)
{
    for (int s = 0; s < o->ns; s++)
        for (int i = 0; i < o->L.Q; i++)
            for (long site = 0; site < o->N; site++)
                o->f[s][i * o->N + site] = o->L.w[i] * (rho ? rho[s * o->N + site] : 1.0);
    o->step = 0;
}

void orcm_set_f(orcm_t *o, const double *f, long step)
{
    for (int s = 0; s < o->ns; s++) memcpy(o->f[s], f + (size_t)s * o->L.Q * o->N, sizeof(double) * o->L.Q * o->N);
    o->step = step;
}

void orcm_get_f(const orcm_t *o, double *f)
{
    for (int s = 0; s < o->ns; s++) memcpy(f + (size_t)s * o->L.Q * o->N, o->f[s], sizeof(double) * o->L.Q * o->N);
}

/* Treat this box as the block of a periodic gnx * gny * gnz box whose local
 * site (0,0,0) sits at (ox, oy, oz) (as orc_set_rng_origin). */
void orcm_set_rng_origin(orcm_t *o, long gnx, long gny, long gnz, long ox, long oy, long oz)
{
    o->rng_global = 1;
    o->gnx = gnx;
    o->gny = gny;
    o->gnz = gnz;
    o->ox = ox;
    o->oy = oy;
    o->oz = oz;
}

static uint32_t rng_site_m(const orcm_t *o, long site)
{
    if (!o->rng_global) return (uint32_t)site;
    long x = site % o->nx, y = (site / o->nx) % o->ny, z = site / ((long)o->nx * o->ny);
    long gx = (x + o->ox) % o->gnx, gy = (y + o->oy) % o->gny, gz = (z + o->oz) % o->gnz;
    return (uint32_t)((gz * o->gny + gy) * o->gnx + gx);
}

static long neighbour_m(const orcm_t *o, long site, const int c[3])
{
    long x = site % o->nx, y = (site / o->nx) % o->ny, z = site / ((long)o->nx * o->ny);
    x = (x + c[0] + o->nx) % o->nx;
    y = (y + c[1] + o->ny) % o->ny;
    z = (z + c[2] + o->nz) % o->nz;
    return (z * o->ny + y) * o->nx + x;
}

static void density_pass_m(orcm_t *o)
{
    for (int s = 0; s < o->ns; s++)
        for (long site = 0; site < o->N; site++) {
            double r = 0.0;
            for (int i = 0; i < o->L.Q; i++) r += o->f[s][i * o->N + site];
            o->rho[s][site] = r;
        }
}

/* a^s(r) = -sum_{s'} G_{s s'} sum_i w_i rho^{s'}(r + c_i) c_i */
static void acceleration_m(const orcm_t *o, long site, int s, double acc[3])
{
    acc[0] = acc[1] = acc[2] = 0.0;
    for (int t = 0; t < o->ns; t++) {
        if (o->G[s][t] == 0.0) continue;
        for (int i = 0; i < o->L.Q; i++) {
            double r = o->rho[t][neighbour_m(o, site, o->L.c[i])];
            for (int d = 0; d < 3; d++) acc[d] += -o->G[s][t] * o->L.w[i] * r * o->L.c[i][d];
        }
    }
}

/* R[s][a] for every species at one site; nonzero if a density is not positive */
static int collide_site_m(const orcm_t *o, long site, double R[ORCM_MAXS][ORC_MAXQ])
{
    const orc_lattice *L = &o->L;
    const int D = L->D, Q = L->Q, ns = o->ns;
    double rho[ORCM_MAXS], m[ORCM_MAXS][ORC_MAXQ], acc[ORCM_MAXS][3];
    double rho_t = 0.0;
    for (int s = 0; s < ns; s++) {
        double pop[ORC_MAXQ];
        for (int i = 0; i < Q; i++) pop[i] = o->f[s][i * o->N + site];
        project(L, pop, m[s]);
        rho[s] = o->rho[s][site];
        if (!(rho[s] > 0.0) || !isfinite(rho[s])) return 1;
        acceleration_m(o, site, s, acc[s]);
        rho_t += rho[s];
    }
    double u[3] = {0.0, 0.0, 0.0};
    for (int d = 0; d < D; d++) {
        double jt = 0.0;
        for (int s = 0; s < ns; s++) jt += m[s][1 + d] + 0.5 * rho[s] * acc[s][d];
        u[d] = jt / rho_t;
    }
    const double mu = 3.0 * o->kT;
    const double lam_d = o->lam_d;
    const double amp_d = sqrt((2.0 * lam_d - lam_d * lam_d) * o->kT);
    double xi[ORCM_MAXS][ORC_MAXQ];
    for (int d = 0; d < D; d++) {
        double eta[ORCM_MAXS], sum = 0.0;
        for (int s = 0; s < ns; s++) {
            eta[s] = sqrt(rho[s]) * orc_gaussian(o->seed, rng_site_m(o, site), (uint32_t)o->step, (uint32_t)s, (uint32_t)(1 + d));
            sum += eta[s];
        }
        for (int s = 0; s < ns; s++) xi[s][1 + d] = amp_d * (eta[s] - rho[s] / rho_t * sum);
    }
    for (int s = 0; s < ns; s++) {
        const double lam = 1.0 / o->tau[s];
        for (int a = D + 1; a < Q; a++) {
            double var = (2.0 * lam - lam * lam) * L->N[a] * mu * rho[s];
            xi[s][a] = sqrt(var) * orc_gaussian(o->seed, rng_site_m(o, site), (uint32_t)o->step, (uint32_t)s, (uint32_t)a);
        }
    }
    for (int s = 0; s < ns; s++) {
        double pfeq[ORC_MAXQ], meq[ORC_MAXQ], pphi[ORC_MAXQ], phi0[ORC_MAXQ], mphi[ORC_MAXQ], v[3] = {0, 0, 0};
        const double zero[3] = {0.0, 0.0, 0.0};
        feq_pop(L, rho[s], u, pfeq);
        project(L, pfeq, meq);
        phi_pop(L, rho[s], acc[s], zero, pphi); /* momentum rows: rho a whatever v is */
        project(L, pphi, phi0);
        R[s][0] = 0.0;
        for (int d = 0; d < D; d++) {
            int a = 1 + d;
            R[s][a] = lam_d * (meq[a] - m[s][a]) + (1.0 - 0.5 * lam_d) * phi0[a] + xi[s][a];
            v[d] = (m[s][a] + 0.5 * R[s][a]) / rho[s]; /* m = mbar + R/2, Eq. alg-mom */
        }
        phi_pop(L, rho[s], acc[s], v, pphi);
        project(L, pphi, mphi);
        const double lam = 1.0 / o->tau[s];
        for (int a = D + 1; a < Q; a++) R[s][a] = lam * (meq[a] - m[s][a]) + (1.0 - 0.5 * lam) * mphi[a] + xi[s][a];
    }
    return 0;
}

int orcm_step(orcm_t *o, long n)
{
    const orc_lattice *L = &o->L;
    for (long t = 0; t < n; t++) {
        density_pass_m(o);
        for (long site = 0; site < o->N; site++) {
            double R[ORCM_MAXS][ORC_MAXQ];
            if (collide_site_m(o, site, R)) return 4;
            for (int s = 0; s < o->ns; s++)
                for (int i = 0; i < L->Q; i++) {
                    double dr = 0.0;
                    for (int a = 0; a < L->Q; a++) dr += L->T[a][i] * R[s][a] / L->N[a];
                    o->fn[s][i * o->N + neighbour_m(o, site, L->c[i])] = o->f[s][i * o->N + site] + L->w[i] * dr;
                }
        }
        for (int s = 0; s < o->ns; s++) {
            double *t2 = o->f[s];
            o->f[s] = o->fn[s];
            o->fn[s] = t2;
        }
        o->step++;
    }
    return 0;
}

/* rho (ns planes), u = sum_s (jbar^s + rho^s a^s / 2) / rho_t (D planes), and
 * cons = [sum rho^0 .. sum rho^{ns-1}, total momentum with the half force x3] */
int orcm_moments(orcm_t *o, double *rho, double *u, double *cons)
{
    const orc_lattice *L = &o->L;
    const int ns = o->ns;
    density_pass_m(o);
    double tot[ORCM_MAXS + 3] = {0};
    for (long site = 0; site < o->N; site++) {
        double rt = 0.0, jt[3] = {0, 0, 0};
        for (int s = 0; s < ns; s++) {
            double r = o->rho[s][site], acc[3];
            acceleration_m(o, site, s, acc);
            if (rho) rho[s * o->N + site] = r;
            tot[s] += r;
            rt += r;
            for (int d = 0; d < 3; d++) {
                double j = 0.0;
                for (int i = 0; i < L->Q; i++) j += L->c[i][d] * o->f[s][i * o->N + site];
                jt[d] += j + 0.5 * r * acc[d];
            }
        }
        for (int d = 0; d < L->D; d++) {
            if (u) u[(long)d * o->N + site] = jt[d] / rt;
            tot[ns + d] += jt[d];
        }
    }
    if (cons)
        for (int k = 0; k < ns + 3; k++) cons[k] = tot[k];
    return 0;
}
