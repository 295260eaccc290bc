// construct.cu -- coefficient-table construction (FP64) for every method.
//
// Every table of the paper is a real-space sum over the planewave set,
//     T(x_l) = sum_G w(G) c_G exp(i G.x_l),       x_l = grid point l (s = l / N),
// with a per-planewave multiplier w(G) = (basis factor) x (derivative factor):
//   basis   smoothing B-spline   1/gamma_G                     Eq. (b-splinecoefficients)
//           interpolating        1/prod_m (1 + cos(th_m)/2)    the periodic [1/4 1 1/4]
//                                                              system of "Interpolating
//                                                              B-spline coefficients",
//                                                              diagonalised
//           grid values          1                             Lagrange tables (App. A)
//           pp-spline sigma      prod over the axes labelled 2 of the periodic
//                                [4 1 .. 1] second-derivative system, diagonalised:
//                                6 (cos th - 1) / (2 + cos th) Eq. (pp-splinecoefficients3)
//   deriv   value 1; d_a phi i G_a; lap phi -|G|^2 (the separate gradient and Laplacian
//           approximations of Sec. III C: B-splines optionally, Lagrange always)
//   odd degree n (uniform grid): interpolating 1 / prod_m S_n(th_m), S_n(th) = sum_j C_n B_n(j)
//           e^{i j th}, the symbol of the periodic interpolation system of the degree-n basis;
//           smoothing 1 / prod_m C_n sinc^{n+1}(th_m / 2), the Fourier transform of the
//           degree-n basis (the paper's gamma_G for n = 3)
// with th_m = 2 pi n_m / N_m.  The cyclic systems of uniform grids are circulant, so dividing
// the folded spectrum by their eigenvalues is their exact solution.
//
// Non-uniform grids (Sec. II "Grid": interpolating splines need no even spacing): the
// planewave sum is evaluated at the per-axis grid points by the same separable passes with
// the true frequencies (the band must fit the grid, 2 n_max + 1 <= N, so folded indices
// map back to frequencies), then the periodic interpolation system of the non-uniform basis
// is solved along each axis: cyclic tridiagonal for the cubic (Thomas + Sherman-Morrison),
// the identity for degree 1, and for degrees 5 and 7 the FP64 inverse of the banded cyclic
// collocation matrix applied to every grid line.
//
// Bloch orbitals (Sec. II, phi = u exp(i k.r)): the same sums give the complex periodic
// part u (and, for the derivative tables, the periodic parts of grad phi and lap phi,
// whose multipliers use k + G: i (k+G)_a, -|k+G|^2); the layout step then stores Re and
// Im of each orbital as two adjacent real functions.
//
// Steps (all FP64, all in this file's kernels):
//   1. scatter_kernel: fold c_G w(G) onto the N1 x N2 x N3 frequency grid
//      F[k1][k2][k3][o] (aliases add up, as in the sum above);
//   2. dft_pass_kernel x 3: separable inverse DFT along z, y, x, skipping frequency
//      lines outside the planewave band and summing only over in-band frequencies;
//   3. layout_kernel: real part -> stored dtype, orbital-innermost rows, ghost planes.
// Orbitals are processed in chunks so the complex grids stay below a fixed budget.
#include <cmath>
#include <cstring>
#include <type_traits>
#include <utility>
#include <vector>

#include "general_basis.cuh"
#include "qmcspl_internal.cuh"

namespace qmcspl {
namespace {

constexpr int kDftInner = 16;          // inner elements per DFT block (threads x)
constexpr int kDftRows = 16;           // output rows in flight per DFT block (threads y)
constexpr size_t kGridBudget = size_t(2) << 30;   // bytes per complex work grid

struct ScatterArgs {
    const int* miller;        // [n_pw][3]
    const double2* coef;      // [n_orb][n_pw]
    int n_pw;
    int o0, oc;               // orbital chunk
    int dims[3];
    double bmat[9];           // G_a = sum_i bmat[3a+i] n_i
    double kc[3];             // Cartesian k added to G in the derivative multipliers (0: Gamma)
    double sym[4];            // kBasisInterpN: C_n B_n(j), j = 0..3
    int degree;               // kBasisSmoothN: the odd degree n
    double cdeg;              // kBasisSmoothN: C_n
    int basis, deriv;         // BuildBasis, BuildDeriv
    int pp_axes;              // bit 2: x, bit 1: y, bit 0: z carry label 2
    double2* F;               // [N1][N2][N3][oc]
};

__device__ __forceinline__ int fold(int n, int N)
{
    int k = n % N;
    return k < 0 ? k + N : k;
}

// One axis of gamma_G: 3(3 - 4 cos th + cos 2th)/th^4 = 24 sin^4(th/2)/th^4, 3/2 at 0.
__device__ __forceinline__ double gamma_axis(int n, int N)
{
    if (n == 0) return 1.5;
    const double th = 6.283185307179586476925286766559 * (double)n / (double)N;
    const double s = sinpi((double)n / (double)N);          // sin(th / 2)
    const double s2 = s * s, th2 = th * th;
    return 24.0 * s2 * s2 / (th2 * th2);
}

// Eigenvalue of the periodic interpolation matrix rows [1/4, 1, 1/4].
__device__ __forceinline__ double interp_axis(int k, int N)
{
    return 1.0 + 0.5 * cospi(2.0 * (double)k / (double)N);
}

// Eigenvalue ratio of the pp system: rhs 6(f[i-1] - 2 f[i] + f[i+1]) over rows
// [1, 4, 1]: 12 (cos th - 1)/(4 + 2 cos th) = -12 sin^2(th/2)/(2 + cos th).
__device__ __forceinline__ double pp_axis(int k, int N)
{
    const double s = sinpi((double)k / (double)N);
    return -12.0 * s * s / (2.0 + cospi(2.0 * (double)k / (double)N));
}

__global__ void scatter_kernel(const ScatterArgs a)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = (long long)a.oc * a.n_pw;
    if (idx >= total) return;
    const int oc = (int)(idx / a.n_pw);
    const int g = (int)(idx - (long long)oc * a.n_pw);
    const int n0 = a.miller[3 * g], n1 = a.miller[3 * g + 1], n2 = a.miller[3 * g + 2];
    const int k0 = fold(n0, a.dims[0]), k1 = fold(n1, a.dims[1]), k2 = fold(n2, a.dims[2]);
    const double2 c = a.coef[(long long)(a.o0 + oc) * a.n_pw + g];
    const double G0 = a.bmat[0] * n0 + a.bmat[1] * n1 + a.bmat[2] * n2 + a.kc[0];
    const double G1 = a.bmat[3] * n0 + a.bmat[4] * n1 + a.bmat[5] * n2 + a.kc[1];
    const double G2 = a.bmat[6] * n0 + a.bmat[7] * n1 + a.bmat[8] * n2 + a.kc[2];
    const double g2 = G0 * G0 + G1 * G1 + G2 * G2;
    double b = 1.0;              // basis factor (real)
    switch (a.basis) {
    case kBasisSmooth:
        b = 1.0 / (gamma_axis(n0, a.dims[0]) * gamma_axis(n1, a.dims[1]) * gamma_axis(n2, a.dims[2]));
        break;
    case kBasisInterp:
        b = 1.0 / (interp_axis(k0, a.dims[0]) * interp_axis(k1, a.dims[1]) * interp_axis(k2, a.dims[2]));
        break;
    case kBasisInterpN: {
        const int kk[3] = {k0, k1, k2};
        for (int ax = 0; ax < 3; ++ax) {
            double sv = a.sym[0];
            for (int j = 1; j < 4; ++j) sv += 2.0 * a.sym[j] * cospi(2.0 * (double)(j * kk[ax]) / (double)a.dims[ax]);
            b /= sv;
        }
        break;
    }
    case kBasisSmoothN: {
        // gamma per axis: C_n (sin(th/2) / (th/2))^{n+1}, C_n at th = 0
        const int nn[3] = {n0, n1, n2};
        for (int ax = 0; ax < 3; ++ax) {
            double g = a.cdeg;
            if (nn[ax] != 0) {
                const double h = 3.141592653589793238462643383279502884 * (double)nn[ax] / (double)a.dims[ax];
                const double sc = sinpi((double)nn[ax] / (double)a.dims[ax]) / h;
                double pw = 1.0;
                for (int e = 0; e <= a.degree; ++e) pw *= sc;
                g *= pw;
            }
            b /= g;
        }
        break;
    }
    case kBasisPP:
        if (a.pp_axes & 4) b *= pp_axis(k0, a.dims[0]);
        if (a.pp_axes & 2) b *= pp_axis(k1, a.dims[1]);
        if (a.pp_axes & 1) b *= pp_axis(k2, a.dims[2]);
        break;
    default: break;
    }
    double wr = b, wi = 0.0;     // complex multiplier w(G) = basis x derivative factor
    switch (a.deriv) {
    case kDerivX: wr = 0.0; wi = b * G0; break;
    case kDerivY: wr = 0.0; wi = b * G1; break;
    case kDerivZ: wr = 0.0; wi = b * G2; break;
    case kDerivLap: wr = -g2 * b; break;
    default: break;
    }
    const double vr = c.x * wr - c.y * wi;
    const double vi = c.x * wi + c.y * wr;
    double2* dst = a.F + ((((long long)k0 * a.dims[1] + k1) * a.dims[2] + k2) * a.oc + oc);
    atomicAdd(&dst->x, vr);
    atomicAdd(&dst->y, vi);
}

struct DftArgs {
    const double2* in;
    double2* out;
    long long outer;          // array viewed as [outer][N][inner]
    long long inner;
    int N;
    int kmax;                 // nonzero input rows: k <= kmax or k >= N - kmax; -1 = all
    int skip_mode;            // 0: every line; 1: outer = k1; 2: outer = k1 * D2 + k2
    int D1, kmax1, D2, kmax2; // band of the outer index (skip_mode 1, 2)
    const double* pts;        // non-uniform output points s_l in [0, 1) (null: s_l = l / N)
};

__device__ __forceinline__ bool in_band(int k, int kmax, int N)
{
    return kmax < 0 || k <= kmax || k >= N - kmax;
}

// out[o][l][i] = sum_k in[o][k][i] exp(+2 pi i k l / N), k over the input band.
__global__ void __launch_bounds__(kDftInner * kDftRows) dft_pass_kernel(const DftArgs a)
{
    extern __shared__ double2 smem[];
    const long long tiles_inner = (a.inner + kDftInner - 1) / kDftInner;
    const long long b = blockIdx.x;
    const long long outer = b / tiles_inner;
    const long long i = (b - outer * tiles_inner) * kDftInner + (threadIdx.x % kDftInner);
    const int ty = threadIdx.x / kDftInner;
    const int N = a.N;
    const bool nonuni = a.pts != nullptr;

    bool zero = false;
    if (a.skip_mode == 1) {
        zero = !in_band((int)outer, a.kmax1, a.D1);
    } else if (a.skip_mode == 2) {
        const int q1 = (int)(outer / a.D2), q2 = (int)(outer % a.D2);
        zero = !(in_band(q1, a.kmax1, a.D1) && in_band(q2, a.kmax2, a.D2));
    }
    if (zero) {   // every input row of this line is zero
        if (i < a.inner)
            for (int l = ty; l < N; l += kDftRows)
                a.out[((long long)outer * N + l) * a.inner + i] = make_double2(0.0, 0.0);
        return;
    }
    // non-uniform points need the true frequency of every row: never the folded "full" view
    const int full = (a.kmax < 0 || (!nonuni && 2 * a.kmax + 1 >= N));
    const int nlo = full ? N : a.kmax + 1;           // rows k = 0 .. nlo-1
    const int nhi = full ? 0 : a.kmax;               // rows k = N-kmax .. N-1
    const int nb = nlo + nhi;
    double2* rows = smem;                            // [nb][kDftInner]
    double2* tw = smem + (size_t)nb * kDftInner;     // [N]
    for (int m = threadIdx.x; m < N; m += blockDim.x) {
        double s, c;
        sincospi(2.0 * (double)m / (double)N, &s, &c);
        tw[m] = make_double2(c, s);
    }
    for (int j = ty; j < nb; j += kDftRows) {
        const int k = j < nlo ? j : N - nhi + (j - nlo);
        rows[j * kDftInner + (threadIdx.x % kDftInner)] =
            (i < a.inner) ? a.in[((long long)outer * N + k) * a.inner + i] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    if (i >= a.inner) return;
    const int tx = threadIdx.x % kDftInner;
    if (nonuni) {
        // out[l] = sum_k in[k] exp(2 pi i f(k) s_l), f(k) = k (low rows) or k - N (high rows);
        // the factors follow by repeated multiplication with exp(2 pi i s_l)
        for (int l = ty; l < N; l += kDftRows) {
            const double sl = a.pts[l];
            double sb, cb;
            sincospi(2.0 * sl, &sb, &cb);
            double re = 0.0, im = 0.0;
            double wr = 1.0, wi = 0.0;
            for (int j = 0; j < nlo; ++j) {
                const double2 v = rows[j * kDftInner + tx];
                re = fma(v.x, wr, fma(-v.y, wi, re));
                im = fma(v.x, wi, fma(v.y, wr, im));
                const double t = wr * cb - wi * sb;
                wi = wr * sb + wi * cb;
                wr = t;
            }
            if (nhi) {
                sincospi(-2.0 * (double)nhi * sl, &wi, &wr);
                for (int j = nlo; j < nb; ++j) {
                    const double2 v = rows[j * kDftInner + tx];
                    re = fma(v.x, wr, fma(-v.y, wi, re));
                    im = fma(v.x, wi, fma(v.y, wr, im));
                    const double t = wr * cb - wi * sb;
                    wi = wr * sb + wi * cb;
                    wr = t;
                }
            }
            a.out[((long long)outer * N + l) * a.inner + i] = make_double2(re, im);
        }
        return;
    }
    for (int l = ty; l < N; l += kDftRows) {
        double re = 0.0, im = 0.0;
        int idx = 0;                                  // (k l) mod N for k = 0, 1, ...
        for (int j = 0; j < nlo; ++j) {
            const double2 v = rows[j * kDftInner + tx];
            const double2 w = tw[idx];
            re = fma(v.x, w.x, fma(-v.y, w.y, re));
            im = fma(v.x, w.y, fma(v.y, w.x, im));
            idx += l;
            if (idx >= N) idx -= N;
        }
        if (nhi) {
            idx = (int)(((long long)(N - nhi) * l) % N);
            for (int j = nlo; j < nb; ++j) {
                const double2 v = rows[j * kDftInner + tx];
                const double2 w = tw[idx];
                re = fma(v.x, w.x, fma(-v.y, w.y, re));
                im = fma(v.x, w.y, fma(v.y, w.x, im));
                idx += l;
                if (idx >= N) idx -= N;
            }
        }
        a.out[((long long)outer * N + l) * a.inner + i] = make_double2(re, im);
    }
}

template <typename T> __device__ __forceinline__ T from_double(double v);
template <> __device__ __forceinline__ double from_double<double>(double v) { return v; }
template <> __device__ __forceinline__ float from_double<float>(double v) { return __double2float_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 from_double<__nv_bfloat16>(double v)
{
    return __double2bfloat16(v);
}

struct LayoutArgs {
    const double2* F;         // [N1][N2][N3][oc]
    void* tab;                // this table
    int N1, N2, N3;
    int oc, o0;
    int o_p;
    int rows_z;
    int entries, entry;
    int zshift;               // 1: zz = z + 1 (B-spline / Lagrange); 0: zz = z (pp)
    int cplx;                 // 1: Bloch, functions 2o and 2o + 1 are Re and Im of orbital o
};

// Real orbitals:  table[x][y][zz][entry][o0 + o] = Re F[x][y][(zz - zshift) mod N3][o]
// Bloch orbitals: table[...][2 (o0 + o) + part] = (Re, Im) F[...][o], part = 0, 1.
// Thread f covers function f of the chunk (oc << cplx functions).
template <typename T>
__global__ void layout_kernel(const LayoutArgs a)
{
    const int nf = a.oc << a.cplx;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = (long long)a.N1 * a.N2 * a.rows_z * nf;
    if (idx >= total) return;
    const int f = (int)(idx % nf);
    const int o = f >> a.cplx;
    long long r = idx / nf;
    const int zz = (int)(r % a.rows_z);
    r /= a.rows_z;
    const int y = (int)(r % a.N2);
    const int x = (int)(r / a.N2);
    int z = zz - a.zshift;
    z = z < 0 ? z + a.N3 : (z >= a.N3 ? z - a.N3 : z);
    const double2 F = a.F[(((long long)x * a.N2 + y) * a.N3 + z) * a.oc + o];
    const double v = (f & a.cplx) ? F.y : F.x;
    T* t = static_cast<T*>(a.tab);
    t[((((long long)x * a.N2 + y) * a.rows_z + zz) * a.entries + a.entry) * a.o_p + (a.o0 << a.cplx) + f] =
        from_double<T>(v);
}

// Double-float tables: orbital o of a row lives in the 16-byte chunk o/2 as
// (hi0, hi1, lo0, lo1), hi = v rounded to float, lo = (v - hi) rounded to float.
__global__ void layout_df_kernel(const LayoutArgs a)
{
    const int nf = a.oc << a.cplx;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = (long long)a.N1 * a.N2 * a.rows_z * nf;
    if (idx >= total) return;
    const int f = (int)(idx % nf);
    const int o = f >> a.cplx;
    long long r = idx / nf;
    const int zz = (int)(r % a.rows_z);
    r /= a.rows_z;
    const int y = (int)(r % a.N2);
    const int x = (int)(r / a.N2);
    int z = zz - a.zshift;
    z = z < 0 ? z + a.N3 : (z >= a.N3 ? z - a.N3 : z);
    const double2 F = a.F[(((long long)x * a.N2 + y) * a.N3 + z) * a.oc + o];
    const double v = (f & a.cplx) ? F.y : F.x;
    const float hi = __double2float_rn(v);
    const float lo = __double2float_rn(v - (double)hi);
    const long long row = (((long long)x * a.N2 + y) * a.rows_z + zz) * a.o_p;   // in 8-byte elements
    const int oo = (a.o0 << a.cplx) + f;
    float* dst = static_cast<float*>(a.tab) + 2 * (row + (oo & ~1)) + (oo & 1);
    dst[0] = hi;
    dst[2] = lo;
}

// A table given by the caller in canonical layout src[x][y][z][f] (f < nf stored functions per
// row, as qmcspl_get_table returns it) written in the stored layout with the same conversion and
// ghost planes as layout_kernel / layout_df_kernel; the padding entries of each row are left as
// they are (zero since construction).
struct PairTable {};            // double-float storage: (hi, lo) float pairs, as layout_df_kernel

struct SetTableArgs {
    const void* src;
    int src_double;           // 1: src is double, 0: float
    void* tab;
    int N1, N2, N3;
    int nf, o_p;
    int rows_z;
    int entries, entry;
    int zshift;
};

template <typename T>
__global__ void set_table_kernel(const SetTableArgs a)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = (long long)a.N1 * a.N2 * a.rows_z * a.nf;
    if (idx >= total) return;
    const int f = (int)(idx % a.nf);
    long long r = idx / a.nf;
    const int zz = (int)(r % a.rows_z);
    r /= a.rows_z;
    const int y = (int)(r % a.N2);
    const int x = (int)(r / a.N2);
    int z = zz - a.zshift;
    z = z < 0 ? z + a.N3 : (z >= a.N3 ? z - a.N3 : z);
    const long long s = (((long long)x * a.N2 + y) * a.N3 + z) * a.nf + f;
    const double v = a.src_double ? static_cast<const double*>(a.src)[s] : (double)static_cast<const float*>(a.src)[s];
    const long long row = (((long long)x * a.N2 + y) * a.rows_z + zz) * a.entries + a.entry;
    if constexpr (std::is_same<T, PairTable>::value) {
        const float hi = __double2float_rn(v);
        const float lo = __double2float_rn(v - (double)hi);
        float* dst = static_cast<float*>(a.tab) + 2 * (row * a.o_p + (f & ~1)) + (f & 1);
        dst[0] = hi;
        dst[2] = lo;
    } else {
        static_cast<T*>(a.tab)[row * a.o_p + f] = from_double<T>(v);
    }
}

int launch_layout(const Handle* h, const double2* F, int tab, int entry, int o0, int oc,
                  cudaStream_t st)
{
    LayoutArgs a;
    a.F = F;
    a.tab = const_cast<Handle*>(h)->table(tab);
    a.N1 = h->dims[0];
    a.N2 = h->dims[1];
    a.N3 = h->dims[2];
    a.oc = oc;
    a.o0 = o0;
    a.o_p = h->n_orb_p;
    a.rows_z = h->rows_z;
    a.entries = h->entries;
    a.entry = entry;
    a.zshift = h->zshift;
    a.cplx = h->bloch ? 1 : 0;
    const long long total = (long long)a.N1 * a.N2 * a.rows_z * (a.oc << a.cplx);
    const unsigned blocks = (unsigned)((total + 255) / 256);
    switch (h->storage) {
    case QMCSPL_DF64: layout_df_kernel<<<blocks, 256, 0, st>>>(a); break;
    case QMCSPL_F64: layout_kernel<double><<<blocks, 256, 0, st>>>(a); break;
    case QMCSPL_F32: layout_kernel<float><<<blocks, 256, 0, st>>>(a); break;
    default: layout_kernel<__nv_bfloat16><<<blocks, 256, 0, st>>>(a); break;
    }
    return cuda_error(cudaGetLastError(), "layout_kernel launch");
}

int launch_dft(const DftArgs& a, cudaStream_t st)
{
    const int full = (a.kmax < 0 || (!a.pts && 2 * a.kmax + 1 >= a.N));
    const int nb = full ? a.N : 2 * a.kmax + 1;
    const size_t smem = ((size_t)nb * kDftInner + a.N) * sizeof(double2);
    const long long tiles_inner = (a.inner + kDftInner - 1) / kDftInner;
    const long long blocks = a.outer * tiles_inner;
    if (blocks <= 0) return QMCSPL_OK;
    if (blocks > 0x7fffffffLL) return set_error(QMCSPL_ERR_UNSUPPORTED, "DFT grid too large");
    cudaError_t e = cudaFuncSetAttribute(dft_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute(dft_pass_kernel)");
    dft_pass_kernel<<<(unsigned)blocks, kDftInner * kDftRows, smem, st>>>(a);
    return cuda_error(cudaGetLastError(), "dft_pass_kernel launch");
}

struct TableJob {
    int tab, entry, basis, deriv, pp_axes;
};

// Cyclic tridiagonal interpolation system of one non-uniform axis, row i:
//   a_i beta_{i-1} + b_i beta_i + c_i beta_{i+1} = f_i   (indices mod N),
// a, b, c the cubic basis of grid points i-1, i, i+1 at grid point i.  Sherman-Morrison:
// A = T + u v^T with gamma = -b_0, T's corners removed and diagonal b_0 - gamma,
// b_{N-1} - a_0 c_{N-1} / gamma; u = (gamma, 0.., c_{N-1}), v = (1, 0.., a_0 / gamma);
// x = y - (v.y) / (1 + v.q) q with T y = f, T q = u.  The Thomas factors of T and q do not
// depend on the right-hand side, so they are computed once here:
//   coef[0][i] = a_i, coef[1][i] = c'_i, coef[2][i] = 1 / m_i, coef[3][i] = q_i.
struct AxisSystem {
    std::vector<double> coef;   // 4 N
    double v_last = 0.0;        // a_0 / gamma
    double inv_denom = 0.0;     // 1 / (1 + v.q)
};

AxisSystem axis_system(const double* knots, int n, double C)
{
    std::vector<double> a(n), b(n), c(n);
    for (int i = 0; i < n; ++i) {
        double w[4], dw[4];
        nonuniform_cubic_weights<double>(knots, n, i, periodic_knot(knots, n, i), C, w, dw, nullptr);
        a[i] = w[0];
        b[i] = w[1];
        c[i] = w[2];
    }
    const double gamma = -b[0];
    std::vector<double> bd(b);
    bd[0] = b[0] - gamma;
    bd[n - 1] = b[n - 1] - a[0] * c[n - 1] / gamma;
    AxisSystem s;
    s.coef.assign(4 * (size_t)n, 0.0);
    double* A = s.coef.data();
    double* CP = A + n;
    double* IM = A + 2 * n;
    double* Q = A + 3 * n;
    for (int i = 0; i < n; ++i) A[i] = a[i];
    IM[0] = 1.0 / bd[0];
    CP[0] = c[0] * IM[0];
    for (int i = 1; i < n; ++i) {
        IM[i] = 1.0 / (bd[i] - a[i] * CP[i - 1]);
        CP[i] = (i < n - 1) ? c[i] * IM[i] : 0.0;
    }
    std::vector<double> u(n, 0.0);
    u[0] = gamma;
    u[n - 1] = c[n - 1];
    Q[0] = u[0] * IM[0];
    for (int i = 1; i < n; ++i) Q[i] = (u[i] - a[i] * Q[i - 1]) * IM[i];
    for (int i = n - 2; i >= 0; --i) Q[i] -= CP[i] * Q[i + 1];
    s.v_last = a[0] / gamma;
    s.inv_denom = 1.0 / (1.0 + Q[0] + s.v_last * Q[n - 1]);
    return s;
}

struct SolveArgs {
    double2* F;               // array viewed as [outer][N][inner], solved in place along N
    long long outer, inner;
    int N;
    const double* coef;       // AxisSystem::coef on the device
    double v_last, inv_denom;
};

__global__ void cyclic_solve_kernel(const SolveArgs s)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= s.outer * s.inner) return;
    const long long o = idx / s.inner, in = idx - o * s.inner;
    double2* x = s.F + o * s.N * s.inner + in;
    const long long st = s.inner;
    const int N = s.N;
    const double* A = s.coef;
    const double* CP = A + N;
    const double* IM = A + 2 * N;
    const double* Q = A + 3 * N;
    double2 prev = x[0];
    prev.x *= IM[0];
    prev.y *= IM[0];
    x[0] = prev;
    for (int l = 1; l < N; ++l) {   // forward sweep
        double2 cur = x[l * st];
        cur.x = (cur.x - A[l] * prev.x) * IM[l];
        cur.y = (cur.y - A[l] * prev.y) * IM[l];
        x[l * st] = cur;
        prev = cur;
    }
    double2 next = prev;             // back substitution
    for (int l = N - 2; l >= 0; --l) {
        double2 y = x[l * st];
        y.x -= CP[l] * next.x;
        y.y -= CP[l] * next.y;
        x[l * st] = y;
        next = y;
    }
    const double2 y0 = x[0], yn = x[(N - 1) * st];
    const double cr = (y0.x + s.v_last * yn.x) * s.inv_denom;
    const double ci = (y0.y + s.v_last * yn.y) * s.inv_denom;
    for (int l = 0; l < N; ++l) {
        double2 v = x[l * st];
        v.x -= cr * Q[l];
        v.y -= ci * Q[l];
        x[l * st] = v;
    }
}

int launch_solve(double2* F, long long outer, int N, long long inner, const double* coef, const AxisSystem& sys,
                 cudaStream_t st)
{
    SolveArgs s;
    s.F = F;
    s.outer = outer;
    s.inner = inner;
    s.N = N;
    s.coef = coef;
    s.v_last = sys.v_last;
    s.inv_denom = sys.inv_denom;
    const long long n = outer * inner;
    cyclic_solve_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(s);
    return cuda_error(cudaGetLastError(), "cyclic_solve_kernel launch");
}

// Degree-n interpolation on a non-uniform periodic axis (n = 5, 7): the collocation matrix
// M[i][m] = sum over periodic images of the basis of grid point m at grid point x_i is cyclic
// with bandwidth n; it is inverted once on the host (Gauss-Jordan elimination with partial
// pivoting, FP64; N <= 512) and the inverse applied to every grid line on the device.
template <int DEG>
void collocation_row(const std::vector<double>& hs, int n, int i, double C, double* w)
{
    double dw[DEG + 1];
    nonuniform_weights_local<double, double, DEG>(hs.data(), n, i, 0.0, C, w, dw, nullptr);
}

bool collocation_inverse(const double* knots, int n, int degree, std::vector<double>& inv)
{
    std::vector<double> hs(n);
    for (int i = 0; i < n; ++i) hs[i] = (i + 1 < n ? knots[i + 1] : knots[0] + 1.0) - knots[i];
    const double C = degree_constant(degree);
    const int H = (degree - 1) / 2;
    std::vector<double> M((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) {
        double w[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        if (degree == 5) collocation_row<5>(hs, n, i, C, w);
        else collocation_row<7>(hs, n, i, C, w);
        for (int r = 0; r <= degree; ++r) {
            int m = (i - H + r) % n;
            if (m < 0) m += n;
            M[(size_t)i * n + m] += w[r];
        }
    }
    inv.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1.0;
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(M[(size_t)r * n + c]) > std::fabs(M[(size_t)piv * n + c])) piv = r;
        if (!(std::fabs(M[(size_t)piv * n + c]) > 0.0)) return false;
        if (piv != c)
            for (int k = 0; k < n; ++k) {
                std::swap(M[(size_t)c * n + k], M[(size_t)piv * n + k]);
                std::swap(inv[(size_t)c * n + k], inv[(size_t)piv * n + k]);
            }
        const double d = 1.0 / M[(size_t)c * n + c];
        for (int k = 0; k < n; ++k) {
            M[(size_t)c * n + k] *= d;
            inv[(size_t)c * n + k] *= d;
        }
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            const double f = M[(size_t)r * n + c];
            if (f == 0.0) continue;
            for (int k = 0; k < n; ++k) {
                M[(size_t)r * n + k] -= f * M[(size_t)c * n + k];
                inv[(size_t)r * n + k] -= f * inv[(size_t)c * n + k];
            }
        }
    }
    return true;
}

struct DenseArgs {
    const double2* in;        // [outer][N][inner]
    double2* out;             // the same shape
    long long outer, inner;
    int N;
    const double* minv;       // N x N, row-major
};

// out[o][i][k] = sum_m minv[i][m] in[o][m][k], one thread per output element
__global__ void dense_axis_kernel(const DenseArgs a)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long line = (long long)a.N * a.inner;
    if (idx >= a.outer * line) return;
    const long long o = idx / line, rem = idx - o * line;
    const int i = (int)(rem / a.inner);
    const long long k = rem - (long long)i * a.inner;
    const double* row = a.minv + (size_t)i * a.N;
    const double2* x = a.in + o * line + k;
    double re = 0.0, im = 0.0;
    for (int m = 0; m < a.N; ++m) {
        const double c = __ldg(row + m);
        const double2 v = x[(long long)m * a.inner];
        re = fma(c, v.x, re);
        im = fma(c, v.y, im);
    }
    a.out[idx] = make_double2(re, im);
}

int launch_dense(const double2* in, double2* out, long long outer, int N, long long inner, const double* minv,
                 cudaStream_t st)
{
    DenseArgs a;
    a.in = in;
    a.out = out;
    a.outer = outer;
    a.inner = inner;
    a.N = N;
    a.minv = minv;
    const long long n = outer * N * inner;
    dense_axis_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a);
    return cuda_error(cudaGetLastError(), "dense_axis_kernel launch");
}

// C_n B_n(j), j = 0..3: the symbol coefficients of the degree-n interpolation system
void degree_symbol(int n, double sym[4])
{
    static const double B[4][4] = {{1.0, 0.0, 0.0, 0.0},
                                   {2.0 / 3.0, 1.0 / 6.0, 0.0, 0.0},
                                   {11.0 / 20.0, 13.0 / 60.0, 1.0 / 120.0, 0.0},
                                   {151.0 / 315.0, 397.0 / 1680.0, 1.0 / 42.0, 1.0 / 5040.0}};
    const int r = (n - 1) / 2;
    for (int j = 0; j < 4; ++j) sym[j] = degree_constant(n) * B[r][j];
}

}  // namespace

int launch_set_table(Handle* h, int table, const void* src, int src_double, cudaStream_t st)
{
    SetTableArgs a;
    const bool pp = h->method == QMCSPL_PPSPLINE;
    a.src = src;
    a.src_double = src_double;
    a.tab = h->table(pp ? 0 : table);
    a.N1 = h->dims[0];
    a.N2 = h->dims[1];
    a.N3 = h->dims[2];
    a.nf = h->n_orb;
    a.o_p = h->n_orb_p;
    a.rows_z = h->rows_z;
    a.entries = h->entries;
    a.entry = pp ? table : 0;
    a.zshift = h->zshift;
    const long long total = (long long)a.N1 * a.N2 * a.rows_z * a.nf;
    const unsigned blocks = (unsigned)((total + 255) / 256);
    switch (h->storage) {
    case QMCSPL_DF64: set_table_kernel<PairTable><<<blocks, 256, 0, st>>>(a); break;
    case QMCSPL_F64: set_table_kernel<double><<<blocks, 256, 0, st>>>(a); break;
    case QMCSPL_F32: set_table_kernel<float><<<blocks, 256, 0, st>>>(a); break;
    default: set_table_kernel<__nv_bfloat16><<<blocks, 256, 0, st>>>(a); break;
    }
    return cuda_error(cudaGetLastError(), "set_table_kernel launch");
}

int build_tables(Handle* h, int n_pw, const int* miller_host, const double* coef_host,
                 cudaStream_t st)
{
    const int N1 = h->dims[0], N2 = h->dims[1], N3 = h->dims[2];
    int kmax[3] = {0, 0, 0};
    for (int g = 0; g < n_pw; ++g)
        for (int a = 0; a < 3; ++a) {
            int v = miller_host[3 * g + a];
            v = v < 0 ? -v : v;
            if (v > kmax[a]) kmax[a] = v;
        }
    if (h->nonuniform)
        for (int a = 0; a < 3; ++a)
            if (2 * kmax[a] + 1 > h->dims[a])
                return set_error(QMCSPL_ERR_ARG, "a non-uniform grid needs N >= 2 n_max + 1 points per axis "
                                                 "(the planewave band must fit the grid)");
    for (int a = 0; a < 3; ++a)
        if (2 * kmax[a] + 1 >= h->dims[a] && !(h->nonuniform && 2 * kmax[a] + 1 == h->dims[a]))
            kmax[a] = -1;   // band covers the whole axis

    std::vector<TableJob> jobs;
    int basis = h->method == QMCSPL_BSPLINE_SMOOTH   ? kBasisSmooth
                : h->method == QMCSPL_BSPLINE_INTERP ? kBasisInterp
                : h->method == QMCSPL_LAGRANGE       ? kBasisGrid
                                                     : kBasisPP;
    if (h->nonuniform) basis = kBasisGrid;                 // grid values, then the axis solves
    else if (h->degree != 3) basis = h->method == QMCSPL_BSPLINE_SMOOTH ? kBasisSmoothN : kBasisInterpN;
    double sym[4] = {0.0, 0.0, 0.0, 0.0};
    if (basis == kBasisInterpN) degree_symbol(h->degree, sym);
    // non-uniform grids: cubic, the cyclic tridiagonal systems; degree 5 and 7, dense inverses;
    // degree 1 interpolates with the identity (the coefficients are the grid values)
    const bool tridiag = h->nonuniform && h->degree == 3;
    const bool dense = h->nonuniform && h->degree >= 5;
    AxisSystem sys[3];
    std::vector<double> minv[3];
    if (tridiag)
        for (int a = 0; a < 3; ++a) sys[a] = axis_system(h->knots[a], h->dims[a], degree_constant(3));
    if (dense)
        for (int a = 0; a < 3; ++a)
            if (!collocation_inverse(h->knots[a], h->dims[a], h->degree, minv[a]))
                return set_error(QMCSPL_ERR_ARG, "the interpolation system of a non-uniform axis is singular");
    if (h->method == QMCSPL_PPSPLINE) {
        // entry e = 4(kappa-1) + 2(mu-1) + (nu-1); label 2 <=> bit set
        for (int e = 0; e < 8; ++e) jobs.push_back({0, e, kBasisPP, kDerivValue, e});
    } else if (h->n_tables == 5) {   // phi, d_x phi, d_y phi, d_z phi, lap phi
        for (int d = 0; d < 5; ++d) jobs.push_back({d, 0, basis, d, 0});
    } else {
        jobs.push_back({0, 0, basis, kDerivValue, 0});
        if (h->separate_lap) jobs.push_back({1, 0, basis, kDerivLap, 0});
    }

    const size_t per_orb = (size_t)N1 * N2 * N3 * sizeof(double2);
    int oc_max = (int)(kGridBudget / per_orb);
    if (oc_max < 1) oc_max = 1;
    const int n_band = h->n_orb >> h->bloch;   // coefficient rows (complex orbitals when Bloch)
    if (oc_max > n_band) oc_max = n_band;

    int* d_miller = nullptr;
    double2* d_coef = nullptr;
    double2* F[2] = {nullptr, nullptr};
    double* d_sys = nullptr;   // non-uniform: 3 axis systems of 4 N doubles, or 3 inverses of N^2
    int rc = QMCSPL_OK;
    cudaError_t e;
    do {
        if (dense) {
            const size_t nd = (size_t)N1 * N1 + (size_t)N2 * N2 + (size_t)N3 * N3;
            e = dev_malloc_async((void**)&d_sys, sizeof(double) * nd, st);
            if (e != cudaSuccess) { rc = cuda_error(e, "cudaMallocAsync(axis inverses)"); break; }
            size_t off = 0;
            for (int a = 0; a < 3; ++a) {
                e = cudaMemcpyAsync(d_sys + off, minv[a].data(), sizeof(double) * minv[a].size(),
                                    cudaMemcpyHostToDevice, st);
                if (e != cudaSuccess) break;
                off += minv[a].size();
            }
            if (e != cudaSuccess) { rc = cuda_error(e, "upload axis inverses"); break; }
        }
        if (tridiag) {
            const size_t nd = 4 * (size_t)(N1 + N2 + N3);
            e = dev_malloc_async((void**)&d_sys, sizeof(double) * nd, st);
            if (e != cudaSuccess) { rc = cuda_error(e, "cudaMallocAsync(axis systems)"); break; }
            size_t off = 0;
            for (int a = 0; a < 3; ++a) {
                e = cudaMemcpyAsync(d_sys + off, sys[a].coef.data(), sizeof(double) * sys[a].coef.size(),
                                    cudaMemcpyHostToDevice, st);
                if (e != cudaSuccess) break;
                off += sys[a].coef.size();
            }
            if (e != cudaSuccess) { rc = cuda_error(e, "upload axis systems"); break; }
        }
        e = dev_malloc_async((void**)&d_miller, sizeof(int) * 3 * (size_t)n_pw, st);
        if (e != cudaSuccess) { rc = cuda_error(e, "cudaMallocAsync(miller)"); break; }
        e = dev_malloc_async((void**)&d_coef, sizeof(double2) * (size_t)n_pw * n_band, st);
        if (e != cudaSuccess) { rc = cuda_error(e, "cudaMallocAsync(coef)"); break; }
        e = dev_malloc_async((void**)&F[0], per_orb * oc_max, st);
        if (e != cudaSuccess) { rc = cuda_error(e, "cudaMallocAsync(grid)"); break; }
        e = dev_malloc_async((void**)&F[1], per_orb * oc_max, st);
        if (e != cudaSuccess) { rc = cuda_error(e, "cudaMallocAsync(grid)"); break; }
        e = cudaMemcpyAsync(d_miller, miller_host, sizeof(int) * 3 * (size_t)n_pw,
                            cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) { rc = cuda_error(e, "upload miller"); break; }
        e = cudaMemcpyAsync(d_coef, coef_host, sizeof(double2) * (size_t)n_pw * n_band,
                            cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) { rc = cuda_error(e, "upload coefficients"); break; }

        double bmat[9];
        for (int a = 0; a < 3; ++a)
            for (int i = 0; i < 3; ++i) bmat[3 * a + i] = 2.0 * M_PI * h->ainv[3 * i + a];

        for (int o0 = 0; o0 < n_band && rc == QMCSPL_OK; o0 += oc_max) {
            const int oc = (n_band - o0 < oc_max) ? n_band - o0 : oc_max;
            for (const TableJob& job : jobs) {
                e = cudaMemsetAsync(F[0], 0, per_orb * oc, st);
                if (e != cudaSuccess) { rc = cuda_error(e, "cudaMemsetAsync(grid)"); break; }
                ScatterArgs s;
                s.miller = d_miller;
                s.coef = d_coef;
                s.n_pw = n_pw;
                s.o0 = o0;
                s.oc = oc;
                for (int a = 0; a < 3; ++a) s.dims[a] = h->dims[a];
                std::memcpy(s.bmat, bmat, sizeof(bmat));
                for (int a = 0; a < 3; ++a) s.kc[a] = h->kcart[a];
                for (int j = 0; j < 4; ++j) s.sym[j] = sym[j];
                s.degree = h->degree;
                s.cdeg = degree_constant(h->degree);
                s.basis = job.basis;
                s.deriv = job.deriv;
                s.pp_axes = job.pp_axes;
                s.F = F[0];
                const long long tot = (long long)oc * n_pw;
                scatter_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(s);
                if ((rc = cuda_error(cudaGetLastError(), "scatter_kernel launch")) != QMCSPL_OK) break;

                DftArgs d;
                // z: [N1*N2][N3][oc], lines outside the (k1, k2) band are zero
                d.in = F[0]; d.out = F[1];
                d.outer = (long long)N1 * N2; d.N = N3; d.inner = oc; d.kmax = kmax[2];
                d.skip_mode = 2; d.D1 = N1; d.kmax1 = kmax[0]; d.D2 = N2; d.kmax2 = kmax[1];
                d.pts = h->nonuniform ? h->d_knots + 2 * kMaxDim : nullptr;
                if ((rc = launch_dft(d, st)) != QMCSPL_OK) break;
                // y: [N1][N2][N3*oc], lines outside the k1 band are zero
                d.in = F[1]; d.out = F[0];
                d.outer = N1; d.N = N2; d.inner = (long long)N3 * oc; d.kmax = kmax[1];
                d.skip_mode = 1; d.D1 = N1; d.kmax1 = kmax[0]; d.D2 = 1; d.kmax2 = -1;
                d.pts = h->nonuniform ? h->d_knots + kMaxDim : nullptr;
                if ((rc = launch_dft(d, st)) != QMCSPL_OK) break;
                // x: [1][N1][N2*N3*oc]
                d.in = F[0]; d.out = F[1];
                d.outer = 1; d.N = N1; d.inner = (long long)N2 * N3 * oc; d.kmax = kmax[0];
                d.skip_mode = 0;
                d.pts = h->nonuniform ? h->d_knots : nullptr;
                if ((rc = launch_dft(d, st)) != QMCSPL_OK) break;
                double2* res = F[1];
                if (tridiag) {   // interpolation systems along x, y, z (any order)
                    const double* c0 = d_sys;
                    const double* c1 = c0 + 4 * (size_t)N1;
                    const double* c2 = c1 + 4 * (size_t)N2;
                    if ((rc = launch_solve(F[1], 1, N1, (long long)N2 * N3 * oc, c0, sys[0], st)) != QMCSPL_OK) break;
                    if ((rc = launch_solve(F[1], N1, N2, (long long)N3 * oc, c1, sys[1], st)) != QMCSPL_OK) break;
                    if ((rc = launch_solve(F[1], (long long)N1 * N2, N3, oc, c2, sys[2], st)) != QMCSPL_OK) break;
                } else if (dense) {   // x: F1 -> F0, y: F0 -> F1, z: F1 -> F0
                    const double* m0 = d_sys;
                    const double* m1 = m0 + (size_t)N1 * N1;
                    const double* m2 = m1 + (size_t)N2 * N2;
                    if ((rc = launch_dense(F[1], F[0], 1, N1, (long long)N2 * N3 * oc, m0, st)) != QMCSPL_OK) break;
                    if ((rc = launch_dense(F[0], F[1], N1, N2, (long long)N3 * oc, m1, st)) != QMCSPL_OK) break;
                    if ((rc = launch_dense(F[1], F[0], (long long)N1 * N2, N3, oc, m2, st)) != QMCSPL_OK) break;
                    res = F[0];
                }
                if ((rc = launch_layout(h, res, job.tab, job.entry, o0, oc, st)) != QMCSPL_OK) break;
            }
        }
    } while (0);
    if (d_sys) cudaFreeAsync(d_sys, st);
    if (F[0]) cudaFreeAsync(F[0], st);
    if (F[1]) cudaFreeAsync(F[1], st);
    if (d_coef) cudaFreeAsync(d_coef, st);
    if (d_miller) cudaFreeAsync(d_miller, st);
    e = cudaStreamSynchronize(st);
    if (rc == QMCSPL_OK && e != cudaSuccess) rc = cuda_error(e, "table construction");
    return rc;
}

}  // namespace qmcspl
