// general_basis.cuh -- B-spline basis weights of any odd degree on uniform and on
// non-uniform periodic grids (Appendix, the B-spline recurrence), for the general
// evaluation kernel and the host-side construction of the non-uniform interpolation systems.
//
// The recurrence b_j^k = w_j^k b_j^{k-1} + (1 - w_{j+1}^k) b_{j+1}^{k-1},
// w_j^k(x) = (x - x_j)/(x_{j+k} - x_j), b_j^0 = C on [x_j, x_{j+1}), gives on the knot
// interval [x_i, x_{i+1}) the k + 1 nonzero functions b_{i-k}^k .. b_i^k.  The basis of grid
// point m is b_j^k with j = m - (k+1)/2 (odd k), so on interval i the stencil is the grid
// points i - (k-1)/2 .. i + (k+1)/2, weight index r = m - i + (k-1)/2.
#pragma once

#include <cmath>

namespace qmcspl {

constexpr int kMaxDegree = 7;

// C_n = 1 / B_n(0) (the centred basis peaks at one; 3/2 for the cubic as in the paper)
__host__ __device__ inline double degree_constant(int n)
{
    switch (n) {
    case 1: return 1.0;
    case 3: return 1.5;
    case 5: return 20.0 / 11.0;
    default: return 315.0 / 151.0;   // n = 7
    }
}

// Uniform knots (unit spacing), local coordinate t in [0, 1) of the interval.  With the
// partition-of-unity levels P_d[r] = b_{i-d+r}^d (C = 1):
//   P_d[r] = ((t + d - r) P_{d-1}[r-1] + (r + 1 - t) P_{d-1}[r]) / d,
//   d/du P_n[r] = P_{n-1}[r-1] - P_{n-1}[r],   d2/du2 P_n[r] = D_{n-1}[r-1] - D_{n-1}[r]
// with D_{n-1}[r] = P_{n-2}[r-1] - P_{n-2}[r] (entries outside 0..d are zero); in general the
// m-th derivative is the m-th backward difference of P_{n-m}, so the third is
//   d3/du3 P_n[r] = P_{n-3}[r-3] - 3 P_{n-3}[r-2] + 3 P_{n-3}[r-1] - P_{n-3}[r].
// The weights are C_n P_n; derivatives are with respect to u = N s (grid units).  d2w and
// d3w may be null.
template <typename A, int DEG>
__host__ __device__ inline void uniform_weights(A t, A C, A* w, A* dw, A* d2w, A* d3w = nullptr)
{
    A lev[3][DEG + 1];   // P_{DEG-2}, P_{DEG-1}, P_{DEG-3} (zero padded)
    A P[DEG + 1];
#pragma unroll
    for (int r = 0; r <= DEG; ++r) P[r] = A(0);
    P[0] = A(1);
#pragma unroll
    for (int l = 0; l < 3; ++l)
#pragma unroll
        for (int r = 0; r <= DEG; ++r) lev[l][r] = A(0);
    if (DEG - 2 == 0) lev[0][0] = A(1);
    if (DEG - 3 == 0) lev[2][0] = A(1);
#pragma unroll
    for (int d = 1; d <= DEG; ++d) {
        A Q[DEG + 1];
#pragma unroll
        for (int r = 0; r <= DEG; ++r) {
            if (r > d) {
                Q[r] = A(0);
                continue;
            }
            const A left = r > 0 ? P[r - 1] : A(0);
            const A right = r < d ? P[r] : A(0);
            Q[r] = ((t + A(d - r)) * left + (A(r + 1) - t) * right) / A(d);
        }
#pragma unroll
        for (int r = 0; r <= DEG; ++r) P[r] = Q[r];
        if (d == DEG - 2)
#pragma unroll
            for (int r = 0; r <= DEG; ++r) lev[0][r] = P[r];
        if (d == DEG - 1)
#pragma unroll
            for (int r = 0; r <= DEG; ++r) lev[1][r] = P[r];
        if (d == DEG - 3)
#pragma unroll
            for (int r = 0; r <= DEG; ++r) lev[2][r] = P[r];
    }
    if (DEG == 1) {   // P_0 = [1] is the degree-0 level
        lev[1][0] = A(1);
    }
#pragma unroll
    for (int r = 0; r <= DEG; ++r) {
        w[r] = C * P[r];
        const A a = r > 0 ? lev[1][r - 1] : A(0);
        const A b = r < DEG ? lev[1][r] : A(0);
        dw[r] = C * (a - b);
        if (d2w) {
            // D_{n-1}[q] = P_{n-2}[q-1] - P_{n-2}[q], q = 0..n-1
            auto D = [&](int q) -> A {
                if (q < 0 || q > DEG - 1 || DEG < 2) return A(0);
                const A x = q > 0 ? lev[0][q - 1] : A(0);
                const A y = q < DEG - 1 ? lev[0][q] : A(0);
                return x - y;
            };
            d2w[r] = C * (D(r - 1) - D(r));
        }
        if (d3w) {
            auto P3 = [&](int q) -> A {   // P_{DEG-3}[q], zero outside 0..DEG-3
                return (DEG >= 3 && q >= 0 && q <= DEG - 3) ? lev[2][q] : A(0);
            };
            d3w[r] = C * (P3(r - 3) - A(3) * P3(r - 2) + A(3) * P3(r - 1) - P3(r));
        }
    }
}

// x_j of the periodic extension of knots[0..n-1] in [0, 1)
__host__ __device__ inline double periodic_knot(const double* knots, int n, int j)
{
    int q = j / n, r = j - q * n;
    if (r < 0) {
        r += n;
        q -= 1;
    }
    return knots[r] + (double)q;
}

// Largest i with knots[i] <= f (f in [0, 1)); points below knots[0] belong to the last
// interval of the previous period: i = n - 1 and f becomes f + 1.  Bisection, at most
// log2(n) + 1 steps.
__host__ __device__ inline int knot_interval(const double* knots, int n, double& f)
{
    if (!(f >= knots[0])) {
        f += 1.0;
        return n - 1;
    }
    int lo = 0, hi = n - 1;   // knots[lo] <= f
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (knots[mid] <= f) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Cubic weights on the non-uniform interval [x_i, x_{i+1}) at x (same period as the knots),
// for the grid points i-1 .. i+2, and their first and second derivatives with respect to
// the reduced coordinate.  De Boor's triangular evaluation of the recurrence.
template <typename A>
__host__ __device__ inline void nonuniform_cubic_weights(const double* knots, int n, int i, double x, A C,
                                                         A* w, A* dw, A* d2w)
{
    double left[4], right[4];
    for (int j = 1; j <= 3; ++j) {
        left[j] = x - periodic_knot(knots, n, i + 1 - j);
        right[j] = periodic_knot(knots, n, i + j) - x;
    }
    double N1[2], N2[3], N3[4];
    double Nl[4] = {1.0, 0.0, 0.0, 0.0};
    for (int j = 1; j <= 3; ++j) {
        double saved = 0.0;
        for (int r = 0; r < j; ++r) {
            const double temp = Nl[r] / (right[r + 1] + left[j - r]);
            Nl[r] = saved + right[r + 1] * temp;
            saved = left[j - r] * temp;
        }
        Nl[j] = saved;
        if (j == 1) { N1[0] = Nl[0]; N1[1] = Nl[1]; }
        if (j == 2) { N2[0] = Nl[0]; N2[1] = Nl[1]; N2[2] = Nl[2]; }
    }
    for (int r = 0; r < 4; ++r) N3[r] = Nl[r];
    // N_d[q] is the degree-d function starting at knot i - d + q
    auto kn = [&](int j) { return periodic_knot(knots, n, j); };
    auto b1 = [&](int k) -> double {   // degree-1 function starting at knot k
        const int q = k - (i - 1);
        return (q >= 0 && q <= 1) ? N1[q] : 0.0;
    };
    auto b2 = [&](int k) -> double {
        const int q = k - (i - 2);
        return (q >= 0 && q <= 2) ? N2[q] : 0.0;
    };
    auto db2 = [&](int k) -> double {
        return 2.0 * (b1(k) / (kn(k + 2) - kn(k)) - b1(k + 1) / (kn(k + 3) - kn(k + 1)));
    };
    for (int r = 0; r < 4; ++r) {
        const int k = i - 3 + r;          // start knot of the function of grid point i-1+r
        w[r] = C * (A)N3[r];
        const double ak = 3.0 / (kn(k + 3) - kn(k)), bk = 3.0 / (kn(k + 4) - kn(k + 1));
        dw[r] = C * (A)(ak * b2(k) - bk * b2(k + 1));
        if (d2w) d2w[r] = C * (A)(ak * db2(k) - bk * db2(k + 1));
    }
}

// Weights of odd degree DEG on the non-uniform interval [x_i, x_{i+1}): the DEG + 1 nonzero
// functions b_{i-DEG}^DEG .. b_i^DEG (grid points i - (DEG-1)/2 .. i + (DEG+1)/2) at
// x = x_i + dx, with their first and second derivatives with respect to the reduced
// coordinate; de Boor's triangular evaluation of the recurrence, and
//   d/dx b_j^k = k (b_j^{k-1} / (x_{j+k} - x_j) - b_{j+1}^{k-1} / (x_{j+k+1} - x_{j+1})).
// Everything comes from dx and the periodic knot spacings hs[j] = x_{j+1} - x_j (j mod n), in
// the arithmetic type S of the spacings: every knot difference the recurrence needs is a sum
// of consecutive spacings, so no absolute coordinate (and no FP64 for FP32 tables) is involved.
template <typename S, typename A, int DEG>
__host__ __device__ inline void nonuniform_weights_local(const S* hs, int n, int i, S dx, A C, A* w, A* dw,
                                                         A* d2w, A* d3w = nullptr)
{
    auto h = [&](int j) -> S {
        j %= n;
        return hs[j < 0 ? j + n : j];
    };
    // kd(a, b) = x_a - x_b for b <= a <= b + DEG + 1
    auto kd = [&](int a, int b) -> S {
        S s = S(0);
        for (int j = b; j < a; ++j) s += h(j);
        return s;
    };
    S left[DEG + 1], right[DEG + 1];
    left[1] = dx;
    right[1] = h(i) - dx;
    for (int j = 2; j <= DEG; ++j) {
        left[j] = left[j - 1] + h(i - j + 1);
        right[j] = right[j - 1] + h(i + j - 1);
    }
    // Nl[q]: the level-j function starting at knot i - j + q; levels DEG - 1, DEG - 2 and
    // DEG - 3 kept
    S Nl[DEG + 1], N1[DEG + 1], N2[DEG + 1], N3[DEG + 1];
    for (int q = 0; q <= DEG; ++q) Nl[q] = N1[q] = N2[q] = N3[q] = S(0);
    Nl[0] = S(1);
    if (DEG == 1) N1[0] = S(1);
    if (DEG == 2) N2[0] = S(1);
    if (DEG == 3) N3[0] = S(1);
    for (int j = 1; j <= DEG; ++j) {
        S saved = S(0);
        for (int r = 0; r < j; ++r) {
            const S temp = Nl[r] / (right[r + 1] + left[j - r]);
            Nl[r] = saved + right[r + 1] * temp;
            saved = left[j - r] * temp;
        }
        Nl[j] = saved;
        if (j == DEG - 1)
            for (int q = 0; q <= j; ++q) N1[q] = Nl[q];
        if (j == DEG - 2)
            for (int q = 0; q <= j; ++q) N2[q] = Nl[q];
        if (j == DEG - 3)
            for (int q = 0; q <= j; ++q) N3[q] = Nl[q];
    }
    auto b1 = [&](int k) -> S {   // level DEG - 1, starting at knot k
        const int q = k - (i - (DEG - 1));
        return (q >= 0 && q <= DEG - 1) ? N1[q] : S(0);
    };
    auto b2 = [&](int k) -> S {   // level DEG - 2
        const int q = k - (i - (DEG - 2));
        return (DEG >= 2 && q >= 0 && q <= DEG - 2) ? N2[q] : S(0);
    };
    auto db1 = [&](int k) -> S {
        return S(DEG - 1) * (b2(k) / kd(k + DEG - 1, k) - b2(k + 1) / kd(k + DEG, k + 1));
    };
    auto b3 = [&](int k) -> S {   // level DEG - 3
        const int q = k - (i - (DEG - 3));
        return (DEG >= 3 && q >= 0 && q <= DEG - 3) ? N3[q] : S(0);
    };
    auto db2 = [&](int k) -> S {   // derivative of the level DEG - 2 function starting at knot k
        return DEG >= 3 ? S(DEG - 2) * (b3(k) / kd(k + DEG - 2, k) - b3(k + 1) / kd(k + DEG - 1, k + 1)) : S(0);
    };
    auto d2b1 = [&](int k) -> S {  // second derivative of the level DEG - 1 function
        return S(DEG - 1) * (db2(k) / kd(k + DEG - 1, k) - db2(k + 1) / kd(k + DEG, k + 1));
    };
    for (int r = 0; r <= DEG; ++r) {
        const int k = i - DEG + r;   // start knot of the function of grid point i - (DEG-1)/2 + r
        w[r] = C * (A)Nl[r];
        const S ak = S(DEG) / kd(k + DEG, k), bk = S(DEG) / kd(k + DEG + 1, k + 1);
        dw[r] = C * (A)(ak * b1(k) - bk * b1(k + 1));
        if (d2w) d2w[r] = DEG >= 2 ? C * (A)(ak * db1(k) - bk * db1(k + 1)) : A(0);
        if (d3w) d3w[r] = DEG >= 3 ? C * (A)(ak * d2b1(k) - bk * d2b1(k + 1)) : A(0);
    }
}

}  // namespace qmcspl
