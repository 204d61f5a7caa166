// flbm_lattice.cuh -- velocity sets, moment bases and closed-form equilibrium and
// forcing moments of the two lattices (compile-time constants).
//
// D2Q9: the basis of Table I (arXiv 1410.5584, Sec. VI), c_s^2 = 1/3.
// D3Q19: not in the paper.  Standard D3Q19 velocities and weights; rows 0-9 are
// the Hermite modes of order <= 2 (Eq. setofT: 1, c, c c - c_s^2 I in the
// bulk/shear combinations below), rows 10-18 an orthogonal ghost completion.
//
// Everything here is constexpr so that, inside fully unrolled loops, the
// 0/+-1/+-2 structure of T folds into straight-line adds.
#pragma once
#include <utility>

#include "flbm_pair.cuh"

namespace flbm {

// Compile-time loop: f(std::integral_constant<int, I>{}) for I = 0 .. N-1, so
// that every table lookup inside f is a constant expression (if constexpr).
template <class F, int... I>
__host__ __device__ __forceinline__ void static_for_impl(F &&f, std::integer_sequence<int, I...>)
{
    (f(std::integral_constant<int, I>{}), ...);
}
template <int N, class F> __host__ __device__ __forceinline__ void static_for(F &&f)
{
    static_for_impl(f, std::make_integer_sequence<int, N>{});
}

struct D2Q9 {
    static constexpr int D = 2;
    static constexpr int Q = 9;
    // velocity order: (0,0) (1,0) (0,1) (-1,0) (0,-1) (1,1) (-1,1) (-1,-1) (1,-1)
    __host__ __device__ static constexpr int cx(int i)
    {
        return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
    }
    __host__ __device__ static constexpr int cy(int i)
    {
        return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
    }
    __host__ __device__ static constexpr int cz(int) { return 0; }
    // opposite pairs: 1-3, 2-4, 5-7, 6-8
    __host__ __device__ static constexpr int opp(int i)
    {
        return i == 0 ? 0 : (i <= 4 ? (i <= 2 ? i + 2 : i - 2) : (i <= 6 ? i + 2 : i - 2));
    }
    // Gauss-Hermite weights: 4/9 rest, 1/9 axis, 1/36 diagonal
    __host__ __device__ static constexpr double wd(int i)
    {
        return i == 0 ? 4.0 / 9.0 : (i <= 4 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
    // rows of Table I, integer valued
    __host__ __device__ static constexpr int T(int a, int i)
    {
        const int x = cx(i), y = cy(i), c2 = x * x + y * y;
        return a == 0 ? 1
             : a == 1 ? x
             : a == 2 ? y
             : a == 3 ? 3 * c2 - 2
             : a == 4 ? 2 * x * x - c2
             : a == 5 ? x * y
             : a == 6 ? (3 * c2 - 4) * x
             : a == 7 ? (3 * c2 - 4) * y
             :          9 * c2 * c2 - 15 * c2 + 2;
    }
    // squared norms of Table I
    __host__ __device__ static constexpr double Nd(int a)
    {
        return a == 0 ? 1.0
             : a <= 2 ? 1.0 / 3.0
             : a == 3 ? 4.0
             : a == 4 ? 4.0 / 9.0
             : a == 5 ? 1.0 / 9.0
             : a <= 7 ? 2.0 / 3.0
             :          16.0;
    }
};

struct D3Q19 {
    static constexpr int D = 3;
    static constexpr int Q = 19;
    // velocity order: rest; +-x, +-y, +-z; then the 12 edges in opposite pairs
    __host__ __device__ static constexpr int cx(int i)
    {
        return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
             : ((i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0);
    }
    __host__ __device__ static constexpr int cy(int i)
    {
        return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
             : ((i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0);
    }
    __host__ __device__ static constexpr int cz(int i)
    {
        return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1
             : ((i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0);
    }
    // opposite directions are stored in adjacent pairs (1,2), (3,4), ..., (17,18)
    __host__ __device__ static constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
    __host__ __device__ static constexpr double wd(int i)
    {
        return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
    __host__ __device__ static constexpr int T(int a, int i)
    {
        const int x = cx(i), y = cy(i), z = cz(i);
        const int c2 = x * x + y * y + z * z;
        return a == 0  ? 1
             : a == 1  ? x
             : a == 2  ? y
             : a == 3  ? z
             : a == 4  ? c2 - 1
             : a == 5  ? 2 * x * x - y * y - z * z
             : a == 6  ? y * y - z * z
             : a == 7  ? x * y
             : a == 8  ? y * z
             : a == 9  ? x * z
             : a == 10 ? (3 * c2 - 5) * x
             : a == 11 ? (3 * c2 - 5) * y
             : a == 12 ? (3 * c2 - 5) * z
             : a == 13 ? x * (y * y - z * z)
             : a == 14 ? y * (z * z - x * x)
             : a == 15 ? z * (x * x - y * y)
             : a == 16 ? 3 * c2 * c2 - 6 * c2 + 1
             : a == 17 ? (2 * c2 - 3) * (2 * x * x - y * y - z * z)
             :           (2 * c2 - 3) * (y * y - z * z);
    }
    // squared norms N_a (equal to sum_i w_i T_ai^2, checked below)
    __host__ __device__ static constexpr double Nd(int a)
    {
        return a == 0 ? 1.0
             : a <= 3 ? 1.0 / 3.0
             : a == 4 ? 2.0 / 3.0
             : a == 5 ? 4.0 / 3.0
             : a == 6 ? 4.0 / 9.0
             : a <= 9 ? 1.0 / 9.0
             : a <= 12 ? 2.0 / 3.0
             : a <= 15 ? 2.0 / 9.0
             : a == 16 ? 2.0
             : a == 17 ? 4.0 / 3.0
             :           4.0 / 9.0;
    }
};

// component d of velocity i
template <class L> __host__ __device__ constexpr int comp(int i, int d)
{
    return d == 0 ? L::cx(i) : (d == 1 ? L::cy(i) : L::cz(i));
}

// Compile-time check of a basis: orthogonality sum_i w_i T_ai T_bi = N_a delta_ab
// (Eq. V-orthog-compl-discrete) up to rounding of the weights.
template <class L> constexpr bool basis_is_orthogonal()
{
    for (int a = 0; a < L::Q; a++)
        for (int b = 0; b < L::Q; b++) {
            double s = 0.0;
            for (int i = 0; i < L::Q; i++) s += L::wd(i) * L::T(a, i) * L::T(b, i);
            const double want = a == b ? L::Nd(a) : 0.0;
            if (s - want > 1e-12 || want - s > 1e-12) return false;
        }
    return true;
}
static_assert(basis_is_orthogonal<D2Q9>(), "D2Q9 basis is not orthogonal with the Table I norms");
static_assert(basis_is_orthogonal<D3Q19>(), "D3Q19 basis is not orthogonal with its norms");

// Closed-form equilibrium and forcing moments of the non-conserved transport
// modes a = D+1 .. kGhost-1.  The second-order Hermite equilibrium gives
// m^eq_a = rho X_a(u) (the Table I column for D2Q9; for D3Q19 the rows
// |u|^2, 2ux^2 - uy^2 - uz^2, uy^2 - uz^2, u_a u_b), X depending on the
// baricentric velocity alone and so common to both species.  The forcing
// moments of Eq. hermite-for truncated at second order, Phi_ab = rho (a_a v_b +
// v_a a_b), projected on the same rows give Phi_a = rho Y_a(a, v).  The ghost
// modes a >= kGhost have m^eq = Phi = 0; the momentum rows are handled apart.
template <class L> struct Closure;

template <> struct Closure<D2Q9> {
    static constexpr int kGhost = 6;
    __device__ __forceinline__ static void eq(const float *u, float *X)
    {
        const float uxx = u[0] * u[0], uyy = u[1] * u[1];
        X[3] = 3.0f * (uxx + uyy);
        X[4] = uxx - uyy;
        X[5] = u[0] * u[1];
    }
    __device__ __forceinline__ static void force(const float *a, const float *v, float *Y)
    {
        const float axvx = a[0] * v[0], ayvy = a[1] * v[1];
        Y[3] = 6.0f * (axvx + ayvy);
        Y[4] = 2.0f * (axvx - ayvy);
        Y[5] = a[0] * v[1] + a[1] * v[0];
    }
};

template <> struct Closure<D3Q19> {
    static constexpr int kGhost = 10;
    __device__ __forceinline__ static void eq(const float *u, float *X)
    {
        const float uxx = u[0] * u[0], uyy = u[1] * u[1], uzz = u[2] * u[2];
        X[4] = uxx + uyy + uzz;
        X[5] = 2.0f * uxx - uyy - uzz;
        X[6] = uyy - uzz;
        X[7] = u[0] * u[1];
        X[8] = u[1] * u[2];
        X[9] = u[0] * u[2];
    }
    __device__ __forceinline__ static void force(const float *a, const float *v, float *Y)
    {
        const float pxx = 2.0f * a[0] * v[0], pyy = 2.0f * a[1] * v[1], pzz = 2.0f * a[2] * v[2];
        Y[4] = pxx + pyy + pzz;
        Y[5] = 2.0f * pxx - pyy - pzz;
        Y[6] = pyy - pzz;
        Y[7] = a[0] * v[1] + a[1] * v[0];
        Y[8] = a[1] * v[2] + a[2] * v[1];
        Y[9] = a[0] * v[2] + a[2] * v[0];
    }
};

// The forcing moments of Closure<L>::force for both species at once (packed
// pairs, lane lo species A, hi species B; flbm_pair.cuh supplies F2).
template <class L> struct ClosurePair;

template <> struct ClosurePair<D2Q9> {
    template <class F>
    __device__ __forceinline__ static void force(const F *a, const F *v, F *Y)
    {
        const F axvx = mul2(a[0], v[0]), ayvy = mul2(a[1], v[1]);
        Y[3] = mul2(splat2(6.0f), axvx + ayvy);
        Y[4] = mul2(splat2(2.0f), axvx - ayvy);
        Y[5] = fma2(a[0], v[1], mul2(a[1], v[0]));
    }
};

template <> struct ClosurePair<D3Q19> {
    template <class F>
    __device__ __forceinline__ static void force(const F *a, const F *v, F *Y)
    {
        const F two = splat2(2.0f);
        const F pxx = mul2(mul2(two, a[0]), v[0]), pyy = mul2(mul2(two, a[1]), v[1]), pzz = mul2(mul2(two, a[2]), v[2]);
        const F pyz = pyy + pzz;
        Y[4] = pxx + pyz;
        Y[5] = mul2(two, pxx) - pyz;
        Y[6] = pyy - pzz;
        Y[7] = fma2(a[0], v[1], mul2(a[1], v[0]));
        Y[8] = fma2(a[1], v[2], mul2(a[2], v[1]));
        Y[9] = fma2(a[0], v[2], mul2(a[2], v[0]));
    }
};

} // namespace flbm
