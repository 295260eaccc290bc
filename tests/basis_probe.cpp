// basis_probe.cpp -- host build of the library's general B-spline basis (general_basis.cuh)
// for tests/test_basis_host.py: prints, per degree, the largest mismatch of each derivative
// order against central differences of the order below, on uniform and on graded knots, and
// between the uniform and the non-uniform routine on evenly spaced knots.
#define __host__
#define __device__
#include <cmath>
#include <cstdio>

#include "general_basis.cuh"

using qmcspl::nonuniform_weights_local;
using qmcspl::uniform_weights;

template <int DEG>
static void probe(const double* hs, int n)
{
    const int W = DEG + 1;
    const double C = qmcspl::degree_constant(DEG);
    const double h = 1e-5;
    double e_uni[3] = {0, 0, 0}, e_non[3] = {0, 0, 0}, e_same = 0, scale[4] = {0, 0, 0, 0};
    for (int s = 1; s < 20; ++s) {
        const double t = s / 20.0;
        double w[4][W], wp[4][W], wm[4][W];
        // uniform knots, derivatives in grid units
        uniform_weights<double, DEG>(t, C, w[0], w[1], w[2], w[3]);
        uniform_weights<double, DEG>(t + h, C, wp[0], wp[1], wp[2], wp[3]);
        uniform_weights<double, DEG>(t - h, C, wm[0], wm[1], wm[2], wm[3]);
        for (int d = 1; d < 4; ++d)
            for (int r = 0; r < W; ++r) {
                const double fd = (wp[d - 1][r] - wm[d - 1][r]) / (2 * h);
                e_uni[d - 1] = std::fmax(e_uni[d - 1], std::fabs(fd - w[d][r]));
            }
        for (int d = 0; d < 4; ++d)
            for (int r = 0; r < W; ++r) scale[d] = std::fmax(scale[d], std::fabs(w[d][r]));
        // the non-uniform routine on evenly spaced knots: derivatives in s = u / n
        double even[64];
        for (int j = 0; j < n; ++j) even[j] = 1.0 / n;
        double v[4][W];
        nonuniform_weights_local<double, double, DEG>(even, n, 3, t / n, C, v[0], v[1], v[2], v[3]);
        double f = 1.0;
        for (int d = 0; d < 4; ++d, f *= n)
            for (int r = 0; r < W; ++r) e_same = std::fmax(e_same, std::fabs(v[d][r] - f * w[d][r]) / f);
        // graded knots: interval 3, offset t of its width
        const double dx = t * hs[3], hx = h * hs[3];
        nonuniform_weights_local<double, double, DEG>(hs, n, 3, dx, C, w[0], w[1], w[2], w[3]);
        nonuniform_weights_local<double, double, DEG>(hs, n, 3, dx + hx, C, wp[0], wp[1], wp[2], wp[3]);
        nonuniform_weights_local<double, double, DEG>(hs, n, 3, dx - hx, C, wm[0], wm[1], wm[2], wm[3]);
        for (int d = 1; d < 4; ++d)
            for (int r = 0; r < W; ++r) {
                const double fd = (wp[d - 1][r] - wm[d - 1][r]) / (2 * hx);
                const double ref = std::fmax(1.0, std::fabs(w[d][r]));
                e_non[d - 1] = std::fmax(e_non[d - 1], std::fabs(fd - w[d][r]) / ref);
            }
    }
    std::printf("%d %.3e %.3e %.3e %.3e %.3e %.3e %.3e %.3e\n", DEG, e_uni[0] / std::fmax(scale[1], 1e-300),
                e_uni[1] / std::fmax(scale[2], 1e-300), DEG >= 3 ? e_uni[2] / scale[3] : 0.0, e_non[0], e_non[1],
                e_non[2], e_same, scale[3]);
}

int main()
{
    // graded spacings of a 16-point axis (sum 1), varying by a factor of about 3
    const int n = 16;
    double hs[n], sum = 0.0;
    for (int j = 0; j < n; ++j) {
        hs[j] = 1.0 + 0.5 * std::sin(2.0 * M_PI * (j + 0.3) / n);
        sum += hs[j];
    }
    for (int j = 0; j < n; ++j) hs[j] /= sum;
    probe<1>(hs, n);
    probe<3>(hs, n);
    probe<5>(hs, n);
    probe<7>(hs, n);
    return 0;
}
