/*
 * qmcspl_oracle.c -- plain, slow, FP64 CPU oracle for planewave-orbital splines.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The product (CUDA) path
 * never links, loads or calls it, and it shares no code with the product path.
 *
 * Everything here follows Parker, Umrigar, Alfe, Hennig, Wilkins,
 * "Comparison of polynomial approximations to speed up planewave-based quantum
 * Monte Carlo calculations" (arXiv:1309.6250):
 *
 *   - Eq. (pw_orbital)             phi_PW(r) = sum_G c_G exp(i G.r)
 *   - Eq. (reducedcoordinate)      crystal -> grid-interval -> reduced coordinate
 *   - Sec. II "Coordinates"        chain rule to Cartesian gradient / Laplacian
 *   - Eq. (b-splinebasis)          cubic B-spline basis b_{-1..2}(t), C = 3/2
 *   - Eq. (b-splineapproximation)  phi = sum_{l,m,n=-1..2} b_l b_m b_n beta_{lmn}
 *   - Eq. (lagrangebasis)          cubic Lagrange basis l_{-1..2}(t)
 *   - Eq. (lagrangeinterpolation3) phi = sum l_i l_j l_k phi_PW(i,j,k)
 *   - Eq. (pp-splinebasis)         s_0^1, s_1^1, s_0^2, s_1^2
 *   - Eq. (pp-splineinterpolation3) 8 coefficients sigma^{kappa mu nu} per point
 *
 * Conventions (the readings the code depends on):
 *   - lattice[9] is row-major with the lattice vectors a_i as COLUMNS, r = a s.
 *   - Grid point l of axis i sits at crystal coordinate s_i = l / N_i.
 *   - Tables are canonical: T[((x*Ny + y)*Nz + z)*n_orb + o], no padding or ghosts.
 *   - The Laplacian chain rule uses N_i N_j (a^-1 a^-T)_ij; the printed N_i^2 is the
 *     same thing for N_1 = N_2 = N_3.
 *   - Positions may be anywhere; they are wrapped into the cell.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (no FMA contraction, so the
 * result is the same on x86-64 and AArch64 hosts).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads the OpenMP loops below use (timing only; results do not depend on it). */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

#define TWO_PI 6.283185307179586476925286766559

/* ------------------------------------------------------------------ */
/* 3x3 helpers                                                          */
/* ------------------------------------------------------------------ */

/* Inverse of a row-major 3x3 matrix by cofactors.  Returns 0 if singular. */
static int inv3(const double m[9], double out[9])
{
    double c00 = m[4] * m[8] - m[5] * m[7];
    double c01 = m[5] * m[6] - m[3] * m[8];
    double c02 = m[3] * m[7] - m[4] * m[6];
    double det = m[0] * c00 + m[1] * c01 + m[2] * c02;
    if (det == 0.0) return 0;
    double id = 1.0 / det;
    out[0] = c00 * id;
    out[1] = (m[2] * m[7] - m[1] * m[8]) * id;
    out[2] = (m[1] * m[5] - m[2] * m[4]) * id;
    out[3] = c01 * id;
    out[4] = (m[0] * m[8] - m[2] * m[6]) * id;
    out[5] = (m[2] * m[3] - m[0] * m[5]) * id;
    out[6] = c02 * id;
    out[7] = (m[1] * m[6] - m[0] * m[7]) * id;
    out[8] = (m[0] * m[4] - m[1] * m[3]) * id;
    return 1;
}

/* ------------------------------------------------------------------ */
/* Eq. (reducedcoordinate): s = a^-1 r, keep the fraction, scale by N,  */
/* split into the grid index below the point and the reduced t in [0,1) */
/* ------------------------------------------------------------------ */
static void reduced_coordinate(const double ainv[9], const int dims[3], const double r[3],
                               int i0[3], double t[3])
{
    for (int i = 0; i < 3; ++i) {
        double s = ainv[3 * i + 0] * r[0] + ainv[3 * i + 1] * r[1] + ainv[3 * i + 2] * r[2];
        double f = s - floor(s);             /* crystal coordinate inside the cell */
        double u = (double)dims[i] * f;      /* units of the grid interval */
        double fl = floor(u);
        t[i] = u - fl;                       /* reduced coordinate in [0,1) */
        int k = (int)fl;
        /* f can round up to exactly 1.0 for a tiny negative s; wrap the index. */
        if (k >= dims[i]) k -= dims[i];
        if (k < 0) k += dims[i];
        i0[i] = k;
    }
}

static inline int wrap(int i, int n)
{
    i %= n;
    return i < 0 ? i + n : i;
}

/* ------------------------------------------------------------------ */
/* Eq. (b-splinebasis): cubic B-spline with C = 3/2, j = -1..2 stored   */
/* at index j+1; `d` selects the derivative order 0..3 with respect to t */
/* ------------------------------------------------------------------ */
void orc_bspline_basis(double t, int d, double w[4])
{
    double t2 = t * t, t3 = t2 * t;
    switch (d) {
    case 0:
        w[0] = -0.25 * t3 + 0.75 * t2 - 0.75 * t + 0.25;
        w[1] = 0.75 * t3 - 1.5 * t2 + 1.0;
        w[2] = -0.75 * t3 + 0.75 * t2 + 0.75 * t + 0.25;
        w[3] = 0.25 * t3;
        break;
    case 1:
        w[0] = -0.75 * t2 + 1.5 * t - 0.75;
        w[1] = 2.25 * t2 - 3.0 * t;
        w[2] = -2.25 * t2 + 1.5 * t + 0.75;
        w[3] = 0.75 * t2;
        break;
    case 2:
        w[0] = -1.5 * t + 1.5;
        w[1] = 4.5 * t - 3.0;
        w[2] = -4.5 * t + 1.5;
        w[3] = 1.5 * t;
        break;
    default:
        w[0] = -1.5;
        w[1] = 4.5;
        w[2] = -4.5;
        w[3] = 1.5;
        break;
    }
}

/* Eq. (lagrangebasis): cubic Lagrange basis, j = -1..2 at index j+1. */
void orc_lagrange_basis(double t, int d, double w[4])
{
    double t2 = t * t, t3 = t2 * t;
    switch (d) {
    case 0:
        w[0] = -t3 / 6.0 + 0.5 * t2 - t / 3.0;
        w[1] = 0.5 * t3 - t2 - 0.5 * t + 1.0;
        w[2] = -0.5 * t3 + 0.5 * t2 + t;
        w[3] = t3 / 6.0 - t / 6.0;
        break;
    case 1:
        w[0] = -0.5 * t2 + t - 1.0 / 3.0;
        w[1] = 1.5 * t2 - 2.0 * t - 0.5;
        w[2] = -1.5 * t2 + t + 1.0;
        w[3] = 0.5 * t2 - 1.0 / 6.0;
        break;
    case 2:
        w[0] = -t + 1.0;
        w[1] = 3.0 * t - 2.0;
        w[2] = -3.0 * t + 1.0;
        w[3] = t;
        break;
    default:
        w[0] = -1.0;
        w[1] = 3.0;
        w[2] = -3.0;
        w[3] = 1.0;
        break;
    }
}

/* Eq. (pp-splinebasis): w[0]=s_0^1, w[1]=s_1^1, w[2]=s_0^2, w[3]=s_1^2 (derivative d). */
void orc_pp_basis(double t, int d, double w[4])
{
    double t2 = t * t, t3 = t2 * t;
    switch (d) {
    case 0:
        w[0] = -t + 1.0;
        w[1] = t;
        w[2] = -t3 / 6.0 + 0.5 * t2 - t / 3.0;
        w[3] = t3 / 6.0 - t / 6.0;
        break;
    case 1:
        w[0] = -1.0;
        w[1] = 1.0;
        w[2] = -0.5 * t2 + t - 1.0 / 3.0;
        w[3] = 0.5 * t2 - 1.0 / 6.0;
        break;
    case 2:
        w[0] = 0.0;
        w[1] = 0.0;
        w[2] = -t + 1.0;
        w[3] = t;
        break;
    default:
        w[0] = 0.0;
        w[1] = 0.0;
        w[2] = -1.0;
        w[3] = 1.0;
        break;
    }
}

/* ------------------------------------------------------------------ */
/* Tensor-product derivative of a tricubic stencil sum:                 */
/*   D(dx,dy,dz) = sum_{l,m,n=-1..2} b^(dx)_l(tx) b^(dy)_m(ty) b^(dz)_n(tz) T[i0+l, j0+m, k0+n] */
/* for one orbital.  `basis` selects Eq. (b-splinebasis) or (lagrangebasis). */
/* ------------------------------------------------------------------ */
typedef void (*basis_fn)(double, int, double[4]);

static double stencil_derivative(basis_fn basis, const double* T, const int dims[3], int n_orb,
                                 int o, const int i0[3], const double t[3],
                                 int dx, int dy, int dz)
{
    double wx[4], wy[4], wz[4];
    basis(t[0], dx, wx);
    basis(t[1], dy, wy);
    basis(t[2], dz, wz);
    double acc = 0.0;
    for (int l = -1; l <= 2; ++l) {
        int x = wrap(i0[0] + l, dims[0]);
        for (int m = -1; m <= 2; ++m) {
            int y = wrap(i0[1] + m, dims[1]);
            for (int n = -1; n <= 2; ++n) {
                int z = wrap(i0[2] + n, dims[2]);
                long g = ((long)x * dims[1] + y) * dims[2] + z;
                acc += wx[l + 1] * wy[m + 1] * wz[n + 1] * T[g * n_orb + o];
            }
        }
    }
    return acc;
}

/* Chain-rule matrices of Sec. II "Coordinates":
 *   Mg[alpha][i] = N_i (a^-1)_{i alpha}               (Cartesian grad = Mg . grad_t)
 *   Ml[i][j]     = N_i N_j (a^-1 a^-T)_{ij}           (Laplacian = sum Ml_ij H_ij)   */
static void chain_matrices(const double ainv[9], const int dims[3], double Mg[9], double Ml[9])
{
    for (int a = 0; a < 3; ++a)
        for (int i = 0; i < 3; ++i) Mg[3 * a + i] = dims[i] * ainv[3 * i + a];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int a = 0; a < 3; ++a) s += ainv[3 * i + a] * ainv[3 * j + a];
            Ml[3 * i + j] = (double)dims[i] * dims[j] * s;
        }
}

/* Derivative orders of the reduced Hessian in the order xx, yy, zz, xy, xz, yz. */
static const int HORD[6][3] = {{2, 0, 0}, {0, 2, 0}, {0, 0, 2}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1}};
static const int HI[6] = {0, 1, 2, 0, 0, 1};
static const int HJ[6] = {0, 1, 2, 1, 2, 2};

/* Laplacian from a reduced Hessian h[6] (xx,yy,zz,xy,xz,yz). */
static double lap_from_hessian(const double Ml[9], const double h[6])
{
    double s = 0.0;
    for (int k = 0; k < 6; ++k) {
        double f = (HI[k] == HJ[k]) ? 1.0 : 2.0;
        s += f * Ml[3 * HI[k] + HJ[k]] * h[k];
    }
    return s;
}

/* ------------------------------------------------------------------ */
/* Tricubic B-spline evaluation, Eq. (b-splineapproximation).           */
/* val [P][O], grad [P][3][O] Cartesian, lap [P][O].                    */
/* beta_lap != NULL: lap is the value of the separate Laplacian spline  */
/* (Sec. III A, Sec. III C); otherwise lap comes from the spline's own  */
/* Hessian through the chain rule.                                      */
/* Returns 0 on success, 1 for a singular lattice.                      */
/* ------------------------------------------------------------------ */
int orc_bspline_eval(const double* beta, const double* beta_lap, const int dims[3], int n_orb,
                     const double lattice[9], long n_pos, const double* pos,
                     double* val, double* grad, double* lap)
{
    double ainv[9], Mg[9], Ml[9];
    if (!inv3(lattice, ainv)) return 1;
    chain_matrices(ainv, dims, Mg, Ml);
#pragma omp parallel for schedule(static)
    for (long p = 0; p < n_pos; ++p) {
        int i0[3];
        double t[3];
        reduced_coordinate(ainv, dims, pos + 3 * p, i0, t);
        for (int o = 0; o < n_orb; ++o) {
            double v = stencil_derivative(orc_bspline_basis, beta, dims, n_orb, o, i0, t, 0, 0, 0);
            double g[3];
            g[0] = stencil_derivative(orc_bspline_basis, beta, dims, n_orb, o, i0, t, 1, 0, 0);
            g[1] = stencil_derivative(orc_bspline_basis, beta, dims, n_orb, o, i0, t, 0, 1, 0);
            g[2] = stencil_derivative(orc_bspline_basis, beta, dims, n_orb, o, i0, t, 0, 0, 1);
            val[p * n_orb + o] = v;
            for (int a = 0; a < 3; ++a)
                grad[(p * 3 + a) * n_orb + o] = Mg[3 * a] * g[0] + Mg[3 * a + 1] * g[1] + Mg[3 * a + 2] * g[2];
            if (beta_lap) {
                lap[p * n_orb + o] =
                    stencil_derivative(orc_bspline_basis, beta_lap, dims, n_orb, o, i0, t, 0, 0, 0);
            } else {
                double h[6];
                for (int k = 0; k < 6; ++k)
                    h[k] = stencil_derivative(orc_bspline_basis, beta, dims, n_orb, o, i0, t,
                                              HORD[k][0], HORD[k][1], HORD[k][2]);
                lap[p * n_orb + o] = lap_from_hessian(Ml, h);
            }
        }
    }
    return 0;
}

/* Reduced-coordinate derivatives of a B-spline table at given positions,
 * D[P][O] for one derivative order (dx,dy,dz).  Used by the tests to check
 * continuity and the chain rule independently of evaluation. */
int orc_bspline_reduced_derivative(const double* beta, const int dims[3], int n_orb,
                                   const double lattice[9], long n_pos, const double* pos,
                                   int dx, int dy, int dz, double* out)
{
    double ainv[9];
    if (!inv3(lattice, ainv)) return 1;
#pragma omp parallel for schedule(static)
    for (long p = 0; p < n_pos; ++p) {
        int i0[3];
        double t[3];
        reduced_coordinate(ainv, dims, pos + 3 * p, i0, t);
        for (int o = 0; o < n_orb; ++o)
            out[p * n_orb + o] =
                stencil_derivative(orc_bspline_basis, beta, dims, n_orb, o, i0, t, dx, dy, dz);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Lagrange evaluation, Eq. (lagrangeinterpolation3), with the five     */
/* separate tables of Sec. III C: tabs = [5][Nx][Ny][Nz][O] holding the */
/* grid values of phi, d_x phi, d_y phi, d_z phi and lap phi.           */
/* The interpolated derivative tables give the Cartesian gradient and   */
/* Laplacian directly.                                                  */
/* ------------------------------------------------------------------ */
int orc_lagrange_eval(const double* tabs, const int dims[3], int n_orb, const double lattice[9],
                      long n_pos, const double* pos, double* val, double* grad, double* lap)
{
    double ainv[9];
    if (!inv3(lattice, ainv)) return 1;
    long tsz = (long)dims[0] * dims[1] * dims[2] * n_orb;
#pragma omp parallel for schedule(static)
    for (long p = 0; p < n_pos; ++p) {
        int i0[3];
        double t[3];
        reduced_coordinate(ainv, dims, pos + 3 * p, i0, t);
        for (int o = 0; o < n_orb; ++o) {
            val[p * n_orb + o] =
                stencil_derivative(orc_lagrange_basis, tabs, dims, n_orb, o, i0, t, 0, 0, 0);
            for (int a = 0; a < 3; ++a)
                grad[(p * 3 + a) * n_orb + o] = stencil_derivative(
                    orc_lagrange_basis, tabs + (1 + a) * tsz, dims, n_orb, o, i0, t, 0, 0, 0);
            lap[p * n_orb + o] =
                stencil_derivative(orc_lagrange_basis, tabs + 4 * tsz, dims, n_orb, o, i0, t, 0, 0, 0);
        }
    }
    return 0;
}

/* Reduced derivative of the Lagrange interpolant of one table (negative control
 * for continuity: Appendix A says this basis has no continuous derivative). */
int orc_lagrange_reduced_derivative(const double* tab, const int dims[3], int n_orb,
                                    const double lattice[9], long n_pos, const double* pos,
                                    int dx, int dy, int dz, double* out)
{
    double ainv[9];
    if (!inv3(lattice, ainv)) return 1;
    for (long p = 0; p < n_pos; ++p) {
        int i0[3];
        double t[3];
        reduced_coordinate(ainv, dims, pos + 3 * p, i0, t);
        for (int o = 0; o < n_orb; ++o)
            out[p * n_orb + o] =
                stencil_derivative(orc_lagrange_basis, tab, dims, n_orb, o, i0, t, dx, dy, dz);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* pp-spline evaluation, Eq. (pp-splineinterpolation3).                 */
/* sig = [8][Nx][Ny][Nz][O]; table e = 4(kappa-1) + 2(mu-1) + (nu-1)    */
/* holds sigma^{kappa mu nu} of Eq. (pp-splinecoefficients3).           */
/* Derivatives with respect to t are those of the basis polynomials;    */
/* the chain rule then gives Cartesian gradient and Laplacian.          */
/* ------------------------------------------------------------------ */
static double pp_derivative(const double* sig, const int dims[3], int n_orb, int o,
                            const int i0[3], const double t[3], int dx, int dy, int dz)
{
    long tsz = (long)dims[0] * dims[1] * dims[2] * n_orb;
    double sx[4], sy[4], sz[4];
    orc_pp_basis(t[0], dx, sx);
    orc_pp_basis(t[1], dy, sy);
    orc_pp_basis(t[2], dz, sz);
    double acc = 0.0;
    for (int kappa = 1; kappa <= 2; ++kappa)
        for (int mu = 1; mu <= 2; ++mu)
            for (int nu = 1; nu <= 2; ++nu) {
                const double* s = sig + (long)(4 * (kappa - 1) + 2 * (mu - 1) + (nu - 1)) * tsz;
                for (int i = 0; i <= 1; ++i) {
                    int x = wrap(i0[0] + i, dims[0]);
                    double wx = sx[2 * (kappa - 1) + i];
                    for (int j = 0; j <= 1; ++j) {
                        int y = wrap(i0[1] + j, dims[1]);
                        double wy = sy[2 * (mu - 1) + j];
                        for (int k = 0; k <= 1; ++k) {
                            int z = wrap(i0[2] + k, dims[2]);
                            double wz = sz[2 * (nu - 1) + k];
                            long g = ((long)x * dims[1] + y) * dims[2] + z;
                            acc += wx * wy * wz * s[g * n_orb + o];
                        }
                    }
                }
            }
    return acc;
}

int orc_pp_eval(const double* sig, const int dims[3], int n_orb, const double lattice[9],
                long n_pos, const double* pos, double* val, double* grad, double* lap)
{
    double ainv[9], Mg[9], Ml[9];
    if (!inv3(lattice, ainv)) return 1;
    chain_matrices(ainv, dims, Mg, Ml);
#pragma omp parallel for schedule(static)
    for (long p = 0; p < n_pos; ++p) {
        int i0[3];
        double t[3];
        reduced_coordinate(ainv, dims, pos + 3 * p, i0, t);
        for (int o = 0; o < n_orb; ++o) {
            double g[3], h[6];
            val[p * n_orb + o] = pp_derivative(sig, dims, n_orb, o, i0, t, 0, 0, 0);
            g[0] = pp_derivative(sig, dims, n_orb, o, i0, t, 1, 0, 0);
            g[1] = pp_derivative(sig, dims, n_orb, o, i0, t, 0, 1, 0);
            g[2] = pp_derivative(sig, dims, n_orb, o, i0, t, 0, 0, 1);
            for (int a = 0; a < 3; ++a)
                grad[(p * 3 + a) * n_orb + o] = Mg[3 * a] * g[0] + Mg[3 * a + 1] * g[1] + Mg[3 * a + 2] * g[2];
            for (int k = 0; k < 6; ++k)
                h[k] = pp_derivative(sig, dims, n_orb, o, i0, t, HORD[k][0], HORD[k][1], HORD[k][2]);
            lap[p * n_orb + o] = lap_from_hessian(Ml, h);
        }
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Direct planewave sums, Eq. (pw_orbital), and their derivatives:      */
/*   grad phi = sum i G c_G e^{iG.r},  lap phi = -sum |G|^2 c_G e^{iG.r} */
/* with G = 2 pi a^-T n and G.r = 2 pi n.(a^-1 r).                      */
/* coef = [O][n_pw][2] (re, im).  The imaginary part of the value sum   */
/* must vanish for a Gamma-point orbital; its largest magnitude is      */
/* returned in *max_imag.                                               */
/* ------------------------------------------------------------------ */
int orc_pw_eval(int n_pw, const int* miller, int n_orb, const double* coef,
                const double lattice[9], long n_pos, const double* pos,
                double* val, double* grad, double* lap, double* max_imag)
{
    double ainv[9];
    if (!inv3(lattice, ainv)) return 1;
    double* G = (double*)malloc(sizeof(double) * 3 * (size_t)(n_pw > 0 ? n_pw : 1));
    if (!G) return 2;
    for (int k = 0; k < n_pw; ++k)
        for (int a = 0; a < 3; ++a) {
            double s = 0.0;
            for (int i = 0; i < 3; ++i) s += ainv[3 * i + a] * miller[3 * k + i];
            G[3 * k + a] = TWO_PI * s;
        }
    double worst = 0.0;
#pragma omp parallel for schedule(static) reduction(max : worst)
    for (long p = 0; p < n_pos; ++p) {
        const double* r = pos + 3 * p;
        double s[3];
        for (int i = 0; i < 3; ++i)
            s[i] = ainv[3 * i + 0] * r[0] + ainv[3 * i + 1] * r[1] + ainv[3 * i + 2] * r[2];
        for (int o = 0; o < n_orb; ++o) {
            double vre = 0.0, vim = 0.0, gx = 0.0, gy = 0.0, gz = 0.0, lp = 0.0;
            for (int k = 0; k < n_pw; ++k) {
                double ph = TWO_PI * (miller[3 * k] * s[0] + miller[3 * k + 1] * s[1] +
                                      miller[3 * k + 2] * s[2]);
                double cr = coef[((long)o * n_pw + k) * 2], ci = coef[((long)o * n_pw + k) * 2 + 1];
                double cs = cos(ph), sn = sin(ph);
                double re = cr * cs - ci * sn; /* Re(c e^{i ph}) */
                double im = cr * sn + ci * cs; /* Im(c e^{i ph}) */
                double g2 = G[3 * k] * G[3 * k] + G[3 * k + 1] * G[3 * k + 1] + G[3 * k + 2] * G[3 * k + 2];
                vre += re;
                vim += im;
                /* Re(i G c e^{i ph}) = -G Im(c e^{i ph}) */
                gx -= G[3 * k] * im;
                gy -= G[3 * k + 1] * im;
                gz -= G[3 * k + 2] * im;
                lp -= g2 * re;
            }
            val[p * n_orb + o] = vre;
            grad[(p * 3 + 0) * n_orb + o] = gx;
            grad[(p * 3 + 1) * n_orb + o] = gy;
            grad[(p * 3 + 2) * n_orb + o] = gz;
            lap[p * n_orb + o] = lp;
            if (fabs(vim) > worst) worst = fabs(vim);
        }
    }
    free(G);
    if (max_imag) *max_imag = worst;
    return 0;
}

/* ------------------------------------------------------------------ */
/* Adjoint of the tricubic B-spline evaluation (the backward pass).     */
/* Given upstream weights gv [P][O], gg [P][3][O], gl [P][O] for the    */
/* outputs of orc_bspline_eval, accumulate                              */
/*   dbeta[g][o]     += d(sum w.out)/d beta[g][o]                        */
/*   dbeta_lap[g][o] += d(sum w.out)/d beta_lap[g][o]  (if beta_lap)     */
/* and write dpos[P][3] = d(sum w.out)/d r.                             */
/* The loss is linear in beta, so this is the exact transpose of the    */
/* evaluation; the position derivative needs one more derivative order. */
/* ------------------------------------------------------------------ */
int orc_bspline_adjoint(const double* beta, const double* beta_lap, const int dims[3], int n_orb,
                        const double lattice[9], long n_pos, const double* pos,
                        const double* gv, const double* gg, const double* gl,
                        double* dbeta, double* dbeta_lap, double* dpos)
{
    double ainv[9], Mg[9], Ml[9];
    if (!inv3(lattice, ainv)) return 1;
    chain_matrices(ainv, dims, Mg, Ml);
    /* Coefficient adjoint: serial over positions (scatter into shared rows). */
    for (long p = 0; p < n_pos; ++p) {
        int i0[3];
        double t[3];
        reduced_coordinate(ainv, dims, pos + 3 * p, i0, t);
        double w[4][3][4]; /* w[d][axis][j]: basis derivative d of each axis */
        for (int d = 0; d < 4; ++d)
            for (int a = 0; a < 3; ++a) orc_bspline_basis(t[a], d, w[d][a]);
        for (int l = -1; l <= 2; ++l)
            for (int m = -1; m <= 2; ++m)
                for (int n = -1; n <= 2; ++n) {
                    long g = ((long)wrap(i0[0] + l, dims[0]) * dims[1] + wrap(i0[1] + m, dims[1])) * dims[2] +
                             wrap(i0[2] + n, dims[2]);
                    /* derivative of the basis product with respect to reduced coordinates */
                    double B = w[0][0][l + 1] * w[0][1][m + 1] * w[0][2][n + 1];
                    double dB[3] = {w[1][0][l + 1] * w[0][1][m + 1] * w[0][2][n + 1],
                                    w[0][0][l + 1] * w[1][1][m + 1] * w[0][2][n + 1],
                                    w[0][0][l + 1] * w[0][1][m + 1] * w[1][2][n + 1]};
                    double hB[6];
                    for (int k = 0; k < 6; ++k)
                        hB[k] = w[HORD[k][0]][0][l + 1] * w[HORD[k][1]][1][m + 1] * w[HORD[k][2]][2][n + 1];
                    double lapB = lap_from_hessian(Ml, hB);
                    for (int o = 0; o < n_orb; ++o) {
                        double acc = gv[p * n_orb + o] * B;
                        for (int a = 0; a < 3; ++a) {
                            double dBa = Mg[3 * a] * dB[0] + Mg[3 * a + 1] * dB[1] + Mg[3 * a + 2] * dB[2];
                            acc += gg[(p * 3 + a) * n_orb + o] * dBa;
                        }
                        if (beta_lap) {
                            dbeta_lap[g * n_orb + o] += gl[p * n_orb + o] * B;
                        } else {
                            acc += gl[p * n_orb + o] * lapB;
                        }
                        dbeta[g * n_orb + o] += acc;
                    }
                }
    }
    /* Position adjoint. */
#pragma omp parallel for schedule(static)
    for (long p = 0; p < n_pos; ++p) {
        int i0[3];
        double t[3];
        reduced_coordinate(ainv, dims, pos + 3 * p, i0, t);
        double acc[3] = {0.0, 0.0, 0.0};
        for (int o = 0; o < n_orb; ++o) {
            double d1[3], d2[3][3], d3l[3];
            d1[0] = stencil_derivative(orc_bspline_basis, beta, dims, n_orb, o, i0, t, 1, 0, 0);
            d1[1] = stencil_derivative(orc_bspline_basis, beta, dims, n_orb, o, i0, t, 0, 1, 0);
            d1[2] = stencil_derivative(orc_bspline_basis, beta, dims, n_orb, o, i0, t, 0, 0, 1);
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    int ord[3] = {0, 0, 0};
                    ord[i] += 1;
                    ord[j] += 1;
                    d2[i][j] = stencil_derivative(orc_bspline_basis, beta, dims, n_orb, o, i0, t,
                                                  ord[0], ord[1], ord[2]);
                }
            /* reduced gradient of the Laplacian output */
            for (int k = 0; k < 3; ++k) {
                if (beta_lap) {
                    int ord[3] = {0, 0, 0};
                    ord[k] = 1;
                    d3l[k] = stencil_derivative(orc_bspline_basis, beta_lap, dims, n_orb, o, i0, t,
                                                ord[0], ord[1], ord[2]);
                } else {
                    double s = 0.0;
                    for (int i = 0; i < 3; ++i)
                        for (int j = 0; j < 3; ++j) {
                            int ord[3] = {0, 0, 0};
                            ord[k] += 1;
                            ord[i] += 1;
                            ord[j] += 1;
                            s += Ml[3 * i + j] * stencil_derivative(orc_bspline_basis, beta, dims, n_orb,
                                                                    o, i0, t, ord[0], ord[1], ord[2]);
                        }
                    d3l[k] = s;
                }
            }
            /* Cartesian: grad = Mg d1, Hessian = Mg d2 Mg^T, grad lap = Mg d3l */
            double gcart[3], H[3][3], glap[3];
            for (int a = 0; a < 3; ++a) {
                gcart[a] = 0.0;
                glap[a] = 0.0;
                for (int i = 0; i < 3; ++i) {
                    gcart[a] += Mg[3 * a + i] * d1[i];
                    glap[a] += Mg[3 * a + i] * d3l[i];
                }
            }
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    double s = 0.0;
                    for (int i = 0; i < 3; ++i)
                        for (int j = 0; j < 3; ++j) s += Mg[3 * a + i] * d2[i][j] * Mg[3 * b + j];
                    H[a][b] = s;
                }
            double wv = gv[p * n_orb + o], wl = gl[p * n_orb + o];
            for (int a = 0; a < 3; ++a) {
                double s = wv * gcart[a] + wl * glap[a];
                for (int b = 0; b < 3; ++b) s += H[a][b] * gg[(p * 3 + b) * n_orb + o];
                acc[a] += s;
            }
        }
        for (int a = 0; a < 3; ++a) dpos[3 * p + a] = acc[a];
    }
    return 0;
}
