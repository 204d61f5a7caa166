// flbm_transform.cuh -- moment transforms m_a = sum_i T_ai f_i and
// y_i = sum_a T_ai mu_a (mu_a = m_a / N_a, so that f_i = w_i y_i, Eq.
// modes-discrete) factored over opposite-velocity pairs.  The weights w_i are
// left to the caller, which folds them into the store.
//
// Rows of T are either even or odd in c, so with S_p = f_i + f_opp(i) and
// D_p = f_i - f_opp(i) the even moments need only the pair sums and the odd
// moments only the pair differences; shared partial sums cut the work to
// roughly a third of the dense 0/+-1/+-2 products.  A compile-time check below
// proves both factored transforms equal the generic T-matrix forms on every
// basis vector (exact small-integer arithmetic).
#pragma once
#include "flbm_lattice.cuh"

namespace flbm {

template <class L> struct Transform;

// D2Q9, Table I rows.  Pairs (first, opposite): P1 (1,3) c=(1,0); P2 (2,4) c=(0,1);
// P3 (5,7) c=(1,1); P4 (6,8) c=(-1,1).
template <> struct Transform<D2Q9> {
    template <class R>
    __host__ __device__ __forceinline__ static constexpr void forward(const R (&f)[9], R (&m)[9])
    {
        const R S1 = f[1] + f[3], D1 = f[1] - f[3];
        const R S2 = f[2] + f[4], D2 = f[2] - f[4];
        const R S3 = f[5] + f[7], D3 = f[5] - f[7];
        const R S4 = f[6] + f[8], D4 = f[6] - f[8];
        const R A = S1 + S2, E = S3 + S4;
        m[0] = f[0] + A + E;                       // 1
        m[1] = D1 + (D3 - D4);                     // c_x
        m[2] = D2 + (D3 + D4);                     // c_y
        m[3] = (R)-2 * f[0] + A + (R)4 * E;        // 3|c|^2 - 2
        m[4] = S1 - S2;                            // c_x^2 - c_y^2
        m[5] = S3 - S4;                            // c_x c_y
        m[6] = (R)-1 * D1 + (R)2 * (D3 - D4);      // (3|c|^2 - 4) c_x
        m[7] = (R)-1 * D2 + (R)2 * (D3 + D4);      // (3|c|^2 - 4) c_y
        m[8] = (R)2 * f[0] + (R)-4 * A + (R)8 * E; // 9|c|^4 - 15|c|^2 + 2
    }
    // y_i = sum_a T_ai mu_a
    template <class R>
    __host__ __device__ __forceinline__ static constexpr void backward(const R (&u)[9], R (&f)[9])
    {
        // even parts per pair class
        const R ax = u[0] + u[3] + (R)-4 * u[8];   // axis: T0=1, T3=1, T8=-4
        const R dg = u[0] + (R)4 * u[3] + (R)8 * u[8];
        const R E1 = ax + u[4], E2 = ax - u[4];
        const R E3 = dg + u[5], E4 = dg - u[5];
        // odd parts
        const R O1 = u[1] - u[6], O2 = u[2] - u[7];
        const R px = u[1] + (R)2 * u[6], py = u[2] + (R)2 * u[7];
        const R O3 = px + py, O4 = py - px;
        f[0] = u[0] + (R)-2 * u[3] + (R)2 * u[8];
        f[1] = E1 + O1;
        f[3] = E1 - O1;
        f[2] = E2 + O2;
        f[4] = E2 - O2;
        f[5] = E3 + O3;
        f[7] = E3 - O3;
        f[6] = E4 + O4;
        f[8] = E4 - O4;
    }
    // Rest population that makes the density expression of forward() return m0:
    // the float weights do not sum to 1 exactly, so w_i m0 spread over the
    // directions would leak mass at a rate proportional to rho - rho0.
    template <class R> __host__ __device__ __forceinline__ static constexpr R rest_closing_mass(const R (&f)[9], R m0)
    {
        const R A = (f[1] + f[3]) + (f[2] + f[4]);
        const R E = (f[5] + f[7]) + (f[6] + f[8]);
        return (m0 - E) - A;
    }
};

// D3Q19 with the basis of flbm_lattice.cuh.  Pairs: P1 (1,2) x; P2 (3,4) y;
// P3 (5,6) z; P4 (7,8) (1,1,0); P5 (9,10) (1,-1,0); P6 (11,12) (1,0,1);
// P7 (13,14) (1,0,-1); P8 (15,16) (0,1,1); P9 (17,18) (0,1,-1).
template <> struct Transform<D3Q19> {
    template <class R>
    __host__ __device__ __forceinline__ static constexpr void forward(const R (&f)[19], R (&m)[19])
    {
        const R S1 = f[1] + f[2], D1 = f[1] - f[2];
        const R S2 = f[3] + f[4], D2 = f[3] - f[4];
        const R S3 = f[5] + f[6], D3 = f[5] - f[6];
        const R S4 = f[7] + f[8], D4 = f[7] - f[8];
        const R S5 = f[9] + f[10], D5 = f[9] - f[10];
        const R S6 = f[11] + f[12], D6 = f[11] - f[12];
        const R S7 = f[13] + f[14], D7 = f[13] - f[14];
        const R S8 = f[15] + f[16], D8 = f[15] - f[16];
        const R S9 = f[17] + f[18], D9 = f[17] - f[18];
        // even rows
        const R A = (S1 + S2) + S3;
        const R s45 = S4 + S5, s67 = S6 + S7, s89 = S8 + S9;
        const R E = (s45 + s67) + s89;
        m[0] = f[0] + A + E;
        m[4] = E - f[0];
        m[16] = f[0] + (R)-2 * A + E;
        const R B = (s45 + s67) + (R)-2 * s89;
        m[5] = (R)2 * S1 - (S2 + S3) + B;
        m[17] = (R)-2 * S1 + (S2 + S3) + B;
        const R C = s45 - s67;
        m[6] = (S2 - S3) + C;
        m[18] = (S3 - S2) + C;
        m[7] = S4 - S5;
        m[8] = S8 - S9;
        m[9] = S6 - S7;
        // odd rows
        const R X = (D4 + D5) + (D6 + D7);
        const R Y = (D4 - D5) + (D8 + D9);
        const R Z = (D6 - D7) + (D8 - D9);
        m[1] = D1 + X;
        m[2] = D2 + Y;
        m[3] = D3 + Z;
        m[10] = (R)-2 * D1 + X;
        m[11] = (R)-2 * D2 + Y;
        m[12] = (R)-2 * D3 + Z;
        m[13] = (D4 + D5) - (D6 + D7);
        m[14] = (D5 - D4) + (D8 + D9);
        m[15] = (D6 - D7) - (D8 - D9);
    }
    template <class R>
    __host__ __device__ __forceinline__ static constexpr void backward(const R (&u)[19], R (&f)[19])
    {
        // even parts: axis pairs
        const R L = u[0] + (R)-2 * u[16];
        const R h = u[5] - u[17], g = u[6] - u[18];
        const R E1 = L + (R)2 * h;
        const R E2 = L - h + g;
        const R E3 = L - h - g;
        // even parts: edge pairs
        const R K = u[0] + u[4] + u[16];
        const R H = u[5] + u[17], G6 = u[6] + u[18];
        const R KH = K + H, KH2 = K + (R)-2 * H;
        const R E4 = KH + G6 + u[7], E5 = KH + G6 - u[7];
        const R E6 = KH - G6 + u[9], E7 = KH - G6 - u[9];
        const R E8 = KH2 + u[8], E9 = KH2 - u[8];
        // odd parts
        const R O1 = u[1] + (R)-2 * u[10];
        const R O2 = u[2] + (R)-2 * u[11];
        const R O3 = u[3] + (R)-2 * u[12];
        const R Xe = u[1] + u[10], Ye = u[2] + u[11], Ze = u[3] + u[12];
        const R O4 = Xe + Ye + (u[13] - u[14]);
        const R O5 = Xe - Ye + (u[13] + u[14]);
        const R O6 = Xe + Ze + (u[15] - u[13]);
        const R O7 = Xe - Ze - (u[13] + u[15]);
        const R O8 = Ye + Ze + (u[14] - u[15]);
        const R O9 = Ye - Ze + (u[14] + u[15]);
        f[0] = u[0] - u[4] + u[16];
        f[1] = E1 + O1;
        f[2] = E1 - O1;
        f[3] = E2 + O2;
        f[4] = E2 - O2;
        f[5] = E3 + O3;
        f[6] = E3 - O3;
        f[7] = E4 + O4;
        f[8] = E4 - O4;
        f[9] = E5 + O5;
        f[10] = E5 - O5;
        f[11] = E6 + O6;
        f[12] = E6 - O6;
        f[13] = E7 + O7;
        f[14] = E7 - O7;
        f[15] = E8 + O8;
        f[16] = E8 - O8;
        f[17] = E9 + O9;
        f[18] = E9 - O9;
    }
    // Rest population that makes the density expression of forward() return m0
    // (see the D2Q9 version).
    template <class R> __host__ __device__ __forceinline__ static constexpr R rest_closing_mass(const R (&f)[19], R m0)
    {
        const R A = ((f[1] + f[2]) + (f[3] + f[4])) + (f[5] + f[6]);
        const R E = (((f[7] + f[8]) + (f[9] + f[10])) + ((f[11] + f[12]) + (f[13] + f[14]))) +
                    ((f[15] + f[16]) + (f[17] + f[18]));
        return (m0 - E) - A;
    }
};

// Compile-time proof: on every unit vector the factored forward transform
// returns the column T_.i and the factored backward transform the row T_a.
// (all values are small integers, exact in double).
template <class L> constexpr bool factored_transforms_match()
{
    constexpr int Q = L::Q;
    for (int k = 0; k < Q; k++) {
        double e[Q] = {}, out[Q] = {};
        e[k] = 1.0;
        Transform<L>::forward(e, out);
        for (int a = 0; a < Q; a++)
            if (out[a] != (double)L::T(a, k)) return false;
        Transform<L>::backward(e, out);
        for (int i = 0; i < Q; i++)
            if (out[i] != (double)L::T(k, i)) return false;
    }
    return true;
}
static_assert(factored_transforms_match<D2Q9>(), "D2Q9 factored transforms differ from Table I");
static_assert(factored_transforms_match<D3Q19>(), "D3Q19 factored transforms differ from the basis");

} // namespace flbm
