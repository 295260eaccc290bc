// eval_variants.cu -- five-table and pp-spline evaluation.
//
// Five tables (Sec. III C, separate approximations of the gradient and the Laplacian):
// tables of phi, d_x phi, d_y phi, d_z phi and lap phi, interpolated with one set of
// weights w_i(tx) w_j(ty) w_k(tz), so the gradient and Laplacian come out Cartesian with
// no chain rule.  Two bases use it:
//   Lagrange (Appendix A, Eq. lagrangeinterpolation3, basis Eq. lagrangebasis): the
//   tables are grid values; Lagrange always uses the separate approximations;
//   B-splines with separate gradient tables (opts.separate_grad): the tables are
//   smoothing or interpolating B-spline coefficients, weights Eq. (b-splinebasis).
//
// pp-spline (Appendix B, Eq. pp-splineinterpolation3 with the basis of
// Eq. pp-splinebasis): eight coefficients sigma^{kappa mu nu} per grid point stored
// together, a 2 x 2 x 2 corner stencil; gradient and Laplacian are derivatives of the
// basis polynomials followed by the chain rule of Sec. II.
//
// Work mapping, loads and stores as in eval_bspline.cu: a group of L lanes per
// position, one 16-byte chunk of each row per lane, one block per SM.  Float and bfloat16
// tables sum on packed FP32 pairs with the rows of the next load units in flight; double
// tables take a scalar path, double-float tables (B-splines) double-float arithmetic.  Bloch
// orbitals (Sec. II) take the same epilogue as the B-splines (bloch_apply).
#include <type_traits>

#include "eval_common.cuh"

namespace qmcspl {
namespace {

template <typename A>
__device__ __forceinline__ void lagrange_weights(A t, A* w)
{
    // Eq. (lagrangebasis), stencil offsets -1..2
    const A tm1 = t - A(1), tm2 = t - A(2), tp1 = t + A(1);
    w[0] = A(-1.0 / 6.0) * t * tm1 * tm2;
    w[1] = A(0.5) * tp1 * tm1 * tm2;
    w[2] = A(-0.5) * tp1 * t * tm2;
    w[3] = A(1.0 / 6.0) * tp1 * t * tm1;
}

// Value weights of the five-table bases at offsets -1..2.
enum FiveTableBasis : int { kFiveLagrange = 0, kFiveBSpline = 1 };

template <int BASIS, typename A>
__device__ __forceinline__ void value_weights(A t, A* w)
{
    if constexpr (BASIS == kFiveLagrange) {
        lagrange_weights<A>(t, w);
    } else {   // Eq. (b-splinebasis)
        const A s = A(1) - t;
        const A t2 = t * t;
        w[0] = A(0.25) * s * s * s;
        w[1] = (A(0.75) * t - A(1.5)) * t2 + A(1);
        w[2] = ((A(-0.75) * t + A(0.75)) * t + A(0.75)) * t + A(0.25);
        w[3] = A(0.25) * t2 * t;
    }
}

// Scalar path (double tables): one warp task = the groups [w0, w0 + groups per warp).
template <typename T, int BASIS>
__device__ __forceinline__ void five_table_task(const EvalArgs& p, long long w0, int lane)
{
    using A = typename Traits<T>::A;
    constexpr int E = Traits<T>::E;
    const int L = 1 << p.lanes_log2;
    const int sub = lane & (L - 1);
    const int gbase = lane & ~(L - 1);
    const long long total = p.n_pos * p.tiles;
    const size_t rowb = (size_t)p.row_stride * sizeof(T);
    const size_t colb = (size_t)p.col_stride * sizeof(T);

    const long long gid = w0 + (lane >> p.lanes_log2);
    const bool active = gid < total;
    const long long q = active ? gid / p.tiles : 0;
    const int tile = active ? (int)(gid - q * p.tiles) : 0;
    const long long ip = active ? order_index(p, q) : q;
    int ix, iy, iz;
    A tx, ty, tz;
    bool ok;
    coords_double(p, ip, L, sub, gbase, ix, iy, iz, tx, ty, tz, ok);
    if (!active) return;
    if (!ok && sub == 0 && tile == 0) atomicOr(p.err, 1);
    A lx[4], ly[4], lz[4];
    value_weights<BASIS, A>(tx, lx);
    value_weights<BASIS, A>(ty, ly);
    value_weights<BASIS, A>(tz, lz);
    const int chunk = tile * L + sub;
    const size_t off = (size_t)chunk * 16 + (size_t)iz * rowb;
    A acc[5][E];
#pragma unroll
    for (int k = 0; k < 5; ++k)
#pragma unroll
        for (int e = 0; e < E; ++e) acc[k][e] = A(0);
#pragma unroll
    for (int l = 0; l < 4; ++l) {
        const int x = wrap1(ix + l - 1, p.nx);
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int y = wrap1(iy + m - 1, p.ny);
            const size_t col = (size_t)(x * p.ny + y) * colb + off;
            const A wxy = lx[l] * ly[m];
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                const char* base = static_cast<const char*>(p.tab[k]) + col;
                uint4 raw[4];
#pragma unroll
                for (int n = 0; n < 4; ++n) raw[n] = ldg_table(p, base + n * rowb);
                A a[E];
#pragma unroll
                for (int e = 0; e < E; ++e) a[e] = A(0);
#pragma unroll
                for (int n = 0; n < 4; ++n) {
                    A c[E];
                    unpack<T>(raw[n], c);
#pragma unroll
                    for (int e = 0; e < E; ++e) a[e] = fma(lz[n], c[e], a[e]);
                }
#pragma unroll
                for (int e = 0; e < E; ++e) acc[k][e] = fma(wxy, a[e], acc[k][e]);
            }
        }
    }
    const int o0 = chunk * E;
    if (o0 >= p.n_orb) return;
    const bool vec = p.vec_out != 0;
    // Bloch: the gradient and Laplacian tables hold the periodic parts of grad phi, lap phi
    if (p.phase) bloch_apply<A, E>(p, ip, acc[0], acc + 1, acc[4], false, false);
    if (p.val) store_run<A, E>(static_cast<A*>(p.val) + ip * p.n_orb + o0, acc[0], o0, p.n_orb, vec);
    if (p.grad)
#pragma unroll
        for (int a = 0; a < 3; ++a)
            store_run<A, E>(static_cast<A*>(p.grad) + (ip * 3 + a) * p.n_orb + o0, acc[1 + a], o0, p.n_orb, vec);
    if (p.lap) store_run<A, E>(static_cast<A*>(p.lap) + ip * p.n_orb + o0, acc[4], o0, p.n_orb, vec);
}

// float and bfloat16 tables: packed FP32 pairs (fma.rn.f32x2), and the 80 loads units of a
// position (16 columns x 5 tables, four z rows each) walked through a ring of three, so two
// units' rows are in flight while one is contracted.  Same products and sums, in the same
// order, as the scalar path.
template <typename T, int BASIS>
__device__ __forceinline__ void five_table_task_x2(const EvalArgs& p, long long w0, int lane)
{
    constexpr int E = Traits<T>::E;
    constexpr int NP = Pairs<T>::N;
    constexpr int kUnits = 16 * 5;
    constexpr int kRing = 3;
    const int L = 1 << p.lanes_log2;
    const int sub = lane & (L - 1);
    const int gbase = lane & ~(L - 1);
    const long long total = p.n_pos * p.tiles;
    const size_t rowb = (size_t)p.row_stride * sizeof(T);
    const size_t colb = (size_t)p.col_stride * sizeof(T);

    const long long gid = w0 + (lane >> p.lanes_log2);
    const bool active = gid < total;
    const long long q = active ? gid / p.tiles : 0;
    const int tile = active ? (int)(gid - q * p.tiles) : 0;
    const long long ip = active ? order_index(p, q) : q;
    int ix, iy, iz;
    float tx, ty, tz;
    bool ok;
    coords_float(p, ip, L, sub, gbase, ix, iy, iz, tx, ty, tz, ok);
    if (!active) return;
    if (!ok && sub == 0 && tile == 0) atomicOr(p.err, 1);
    float lx[4], ly[4], lz[4];
    value_weights<BASIS, float>(tx, lx);
    value_weights<BASIS, float>(ty, ly);
    value_weights<BASIS, float>(tz, lz);
    f32x2 lz2[4];
#pragma unroll
    for (int n = 0; n < 4; ++n) lz2[n] = pack2(lz[n], lz[n]);
    int xs[4], ys[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        xs[j] = wrap1(ix + j - 1, p.nx);
        ys[j] = wrap1(iy + j - 1, p.ny);
    }
    const int chunk = tile * L + sub;
    const size_t off = (size_t)chunk * 16 + (size_t)iz * rowb;
    auto load_unit = [&](int u, uint4* dst) {
        const int c = u / 5, k = u - 5 * (u / 5);
        const char* base = static_cast<const char*>(p.tab[k]) + (size_t)(xs[c >> 2] * p.ny + ys[c & 3]) * colb + off;
#pragma unroll
        for (int n = 0; n < 4; ++n) dst[n] = ldg_table(p, base + n * rowb);
    };
    f32x2 ACC[5][NP];
#pragma unroll
    for (int k = 0; k < 5; ++k)
#pragma unroll
        for (int j = 0; j < NP; ++j) ACC[k][j] = 0ull;
    uint4 ring[kRing][4];
    load_unit(0, ring[0]);
    load_unit(1, ring[1]);
#pragma unroll
    for (int u = 0; u < kUnits; ++u) {
        if (u + 2 < kUnits) load_unit(u + 2, ring[(u + 2) % kRing]);
        const int c = u / 5, k = u - 5 * (u / 5);
        f32x2 a[NP];
#pragma unroll
        for (int j = 0; j < NP; ++j) a[j] = 0ull;
#pragma unroll
        for (int n = 0; n < 4; ++n) {
            f32x2 cv[NP];
            Pairs<T>::get(ring[u % kRing][n], cv);
#pragma unroll
            for (int j = 0; j < NP; ++j) a[j] = ffma2(lz2[n], cv[j], a[j]);
        }
        const float wxy = lx[c >> 2] * ly[c & 3];
        const f32x2 W = pack2(wxy, wxy);
#pragma unroll
        for (int j = 0; j < NP; ++j) ACC[k][j] = ffma2(W, a[j], ACC[k][j]);
    }
    const int o0 = chunk * E;
    if (o0 >= p.n_orb) return;
    const bool vec = p.vec_out != 0;
    float acc[5][E];
#pragma unroll
    for (int k = 0; k < 5; ++k)
#pragma unroll
        for (int j = 0; j < NP; ++j) unpack2(ACC[k][j], acc[k][2 * j], acc[k][2 * j + 1]);
    if (p.phase) bloch_apply<float, E>(p, ip, acc[0], acc + 1, acc[4], false, false);
    if (p.val) store_run<float, E>(static_cast<float*>(p.val) + ip * p.n_orb + o0, acc[0], o0, p.n_orb, vec);
    if (p.grad)
#pragma unroll
        for (int a = 0; a < 3; ++a)
            store_run<float, E>(static_cast<float*>(p.grad) + (ip * 3 + a) * p.n_orb + o0, acc[1 + a], o0,
                                p.n_orb, vec);
    if (p.lap) store_run<float, E>(static_cast<float*>(p.lap) + ip * p.n_orb + o0, acc[4], o0, p.n_orb, vec);
}

// Double-float tables (B-splines with separate gradient tables): every weight, product and sum
// a double-float pair on the FP32 pipe (df_fma2, two orbitals per packed operation), as the
// double-float B-spline kernel; the outputs are converted to double for the epilogue.
template <int BASIS>
__device__ __forceinline__ void five_table_task_df(const EvalArgs& p, long long w0, int lane)
{
    const int L = 1 << p.lanes_log2;
    const int sub = lane & (L - 1);
    const int gbase = lane & ~(L - 1);
    const long long total = p.n_pos * p.tiles;
    const size_t rowb = (size_t)p.row_stride * 8;
    const size_t colb = (size_t)p.col_stride * 8;

    const long long gid = w0 + (lane >> p.lanes_log2);
    const bool active = gid < total;
    const long long q = active ? gid / p.tiles : 0;
    const int tile = active ? (int)(gid - q * p.tiles) : 0;
    const long long ip = active ? order_index(p, q) : q;
    int ix, iy, iz;
    dfloat t[3];
    bool ok;
    if (p.rec) {   // kind-3 record: cell and double-float t
        const float4* qr = static_cast<const float4*>(p.rec) + 2 * ip;
        const float4 a = __ldg(qr), b = __ldg(qr + 1);
        unpack_cell(__float_as_int(a.x), ix, iy, iz, ok);
        t[0] = {a.y, a.z};
        t[1] = {a.w, b.x};
        t[2] = {b.y, b.z};
    } else {
        const double r[3] = {p.pos[3 * ip], p.pos[3 * ip + 1], p.pos[3 * ip + 2]};
        double dx, dy, dz;
        reduced_coordinates(p, r, L, sub, gbase, ix, iy, iz, dx, dy, dz, ok);
        t[0] = df_from_double(dx);
        t[1] = df_from_double(dy);
        t[2] = df_from_double(dz);
    }
    if (!active) return;
    if (!ok && sub == 0 && tile == 0) atomicOr(p.err, 1);
    static_assert(BASIS == kFiveBSpline, "double-float five-table handles are B-splines");
    dfloat lw[3][4], scratch[4];
#pragma unroll
    for (int a = 0; a < 3; ++a) bspline_weights_df(t[a], lw[a], scratch, nullptr);
    int xs[4], ys[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        xs[j] = wrap1(ix + j - 1, p.nx);
        ys[j] = wrap1(iy + j - 1, p.ny);
    }
    const int chunk = tile * L + sub;
    const size_t off = (size_t)chunk * 16 + (size_t)iz * rowb;
    f32x2 Ah[5], Al[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) Ah[k] = Al[k] = 0ull;
#pragma unroll 1
    for (int c = 0; c < 16; ++c) {
        const int l = c >> 2, m = c & 3;
        const size_t col = (size_t)(xs[l] * p.ny + ys[m]) * colb + off;
        const dfloat wxy = df_mul(lw[0][l], lw[1][m]);
        const f32x2 xh = pack2(wxy.h, wxy.h), xl = pack2(wxy.l, wxy.l), nxh = pack2(-wxy.h, -wxy.h);
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const char* base = static_cast<const char*>(p.tab[k]) + col;
            uint4 raw[4];
#pragma unroll
            for (int n = 0; n < 4; ++n) raw[n] = ldg_table(p, base + n * rowb);
            f32x2 Sh = 0ull, Sl = 0ull;
#pragma unroll
            for (int n = 0; n < 4; ++n) {
                const f32x2 Bh = pack2u(raw[n].x, raw[n].y), Bl = pack2u(raw[n].z, raw[n].w);
                const dfloat z = lw[2][n];
                df_fma2(Sh, Sl, pack2(z.h, z.h), pack2(z.l, z.l), pack2(-z.h, -z.h), Bh, Bl);
            }
            df_fma2(Ah[k], Al[k], xh, xl, nxh, Sh, Sl);
        }
    }
    constexpr int E = 2;
    const int o0 = chunk * E;
    if (o0 >= p.n_orb) return;
    const bool vec = p.vec_out != 0;
    double acc[5][E];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        float h0, h1, l0, l1;
        unpack2(Ah[k], h0, h1);
        unpack2(Al[k], l0, l1);
        acc[k][0] = df_to_double(h0, l0);
        acc[k][1] = df_to_double(h1, l1);
    }
    // Bloch: the gradient and Laplacian tables hold the periodic parts of grad phi, lap phi
    if (p.phase) bloch_apply<double, E>(p, ip, acc[0], acc + 1, acc[4], false, false);
    if (p.val) store_run<double, E>(static_cast<double*>(p.val) + ip * p.n_orb + o0, acc[0], o0, p.n_orb, vec);
    if (p.grad)
#pragma unroll
        for (int a = 0; a < 3; ++a)
            store_run<double, E>(static_cast<double*>(p.grad) + (ip * 3 + a) * p.n_orb + o0, acc[1 + a], o0,
                                 p.n_orb, vec);
    if (p.lap) store_run<double, E>(static_cast<double*>(p.lap) + ip * p.n_orb + o0, acc[4], o0, p.n_orb, vec);
}

#ifndef QMCSPL_FIVE_THREADS
#define QMCSPL_FIVE_THREADS 512
#endif
// Five-table and pp kernels: one block of QMCSPL_FIVE_THREADS per SM, as the B-spline kernel: the warps of an SM evaluate consecutive
// (cell-ordered, neighbouring) positions, whose stencil rows then hit in that SM's L1.
template <typename T, int BASIS, int THREADS>
__global__ void __launch_bounds__(THREADS, 1) five_table_vgl_kernel(const EvalArgs p)
{
    constexpr int WPB = THREADS / 32;
    const int lane = threadIdx.x & 31;
    const int gpw = 32 >> p.lanes_log2;
    const long long total = p.n_pos * p.tiles;
    const long long warp = (long long)blockIdx.x * WPB + (threadIdx.x >> 5);
    const long long wstride = (long long)gridDim.x * WPB;
    for (long long w0 = warp * gpw; w0 < total; w0 += wstride * gpw) {
        if constexpr (std::is_same<T, DF64Tag>::value) five_table_task_df<BASIS>(p, w0, lane);
        else if constexpr (sizeof(T) == 8) five_table_task<T, BASIS>(p, w0, lane);
        else five_table_task_x2<T, BASIS>(p, w0, lane);
    }
}

// Eq. (pp-splinebasis): w[k][i] = s_i^{k+1}(t) and derivatives (d = 0, 1, 2).
template <typename A>
__device__ __forceinline__ void pp_weights(A t, A w[2][2], A dw[2][2], A d2w[2][2])
{
    const A t2 = t * t;
    w[0][0] = A(1) - t;
    w[0][1] = t;
    w[1][0] = ((A(-1.0 / 6.0) * t + A(0.5)) * t - A(1.0 / 3.0)) * t;
    w[1][1] = (A(1.0 / 6.0) * t2 - A(1.0 / 6.0)) * t;
    dw[0][0] = A(-1);
    dw[0][1] = A(1);
    dw[1][0] = A(-0.5) * t2 + t - A(1.0 / 3.0);
    dw[1][1] = A(0.5) * t2 - A(1.0 / 6.0);
    d2w[0][0] = A(0);
    d2w[0][1] = A(0);
    d2w[1][0] = A(1) - t;
    d2w[1][1] = t;
}

// Scalar path (double tables): one warp task = the groups [w0, w0 + groups per warp).
template <typename T>
__device__ __forceinline__ void pp_task(const EvalArgs& p, long long w0, int lane)
{
    using A = typename Traits<T>::A;
    constexpr int E = Traits<T>::E;
    const int L = 1 << p.lanes_log2;
    const int sub = lane & (L - 1);
    const int gbase = lane & ~(L - 1);
    const long long total = p.n_pos * p.tiles;
    const size_t rowb = (size_t)p.row_stride * sizeof(T);     // one z row: 8 entries x O_p
    const size_t entb = rowb / 8;                              // one entry: O_p
    const size_t colb = (size_t)p.col_stride * sizeof(T);

    {
        const long long gid = w0 + (lane >> p.lanes_log2);
        const bool active = gid < total;
        const long long q = active ? gid / p.tiles : 0;
        const int tile = active ? (int)(gid - q * p.tiles) : 0;
        const long long ip = active ? order_index(p, q) : q;
        int ix, iy, iz;
        A tx, ty, tz;
        bool ok;
        if constexpr (sizeof(A) == 8) coords_double(p, ip, L, sub, gbase, ix, iy, iz, tx, ty, tz, ok);
        else coords_float(p, ip, L, sub, gbase, ix, iy, iz, tx, ty, tz, ok);
        if (!active) return;
        if (!ok && sub == 0 && tile == 0) atomicOr(p.err, 1);
        A wx[2][2], dwx[2][2], d2wx[2][2], wy[2][2], dwy[2][2], d2wy[2][2], wz[2][2], dwz[2][2], d2wz[2][2];
        pp_weights<A>((A)tx, wx, dwx, d2wx);
        pp_weights<A>((A)ty, wy, dwy, d2wy);
        pp_weights<A>((A)tz, wz, dwz, d2wz);
        const A* mlv = nullptr;
        if constexpr (sizeof(A) == 8) mlv = p.ml; else mlv = p.mlf;
        const A ml0 = mlv[0], ml1 = mlv[1], ml2 = mlv[2];
        const A ml3 = mlv[3], ml4 = mlv[4], ml5 = mlv[5];
        const int chunk = tile * L + sub;
        const size_t off = (size_t)chunk * 16 + (size_t)iz * rowb;
        A v[E], gx[E], gy[E], gz[E], lp[E];
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = gx[e] = gy[e] = gz[e] = lp[e] = A(0);
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int x = ix + i < p.nx ? ix + i : 0;
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int y = iy + j < p.ny ? iy + j : 0;
                const char* col = static_cast<const char*>(p.tab[0]) + (size_t)(x * p.ny + y) * colb + off;
#pragma unroll
                for (int km = 0; km < 4; ++km) {          // (kappa, mu) labels of x and y
                    const int kap = km >> 1, mu = km & 1;
                    A a0[E], a1[E], a2[E];
#pragma unroll
                    for (int e = 0; e < E; ++e) a0[e] = a1[e] = a2[e] = A(0);
#pragma unroll
                    for (int k = 0; k < 2; ++k)
#pragma unroll
                        for (int nu = 0; nu < 2; ++nu) {
                            A c[E];
                            unpack<T>(ldg_table(p, col + k * rowb + (size_t)(4 * kap + 2 * mu + nu) * entb), c);
#pragma unroll
                            for (int e = 0; e < E; ++e) {
                                a0[e] = fma(wz[nu][k], c[e], a0[e]);
                                a1[e] = fma(dwz[nu][k], c[e], a1[e]);
                                a2[e] = fma(d2wz[nu][k], c[e], a2[e]);
                            }
                        }
                    const A w00 = wx[kap][i] * wy[mu][j];
                    const A w10 = dwx[kap][i] * wy[mu][j];
                    const A w01 = wx[kap][i] * dwy[mu][j];
                    const A c0 = ml0 * (d2wx[kap][i] * wy[mu][j]) + ml1 * (wx[kap][i] * d2wy[mu][j]) +
                                 ml3 * (dwx[kap][i] * dwy[mu][j]);
                    const A c1 = ml4 * w10 + ml5 * w01;
                    const A c2 = ml2 * w00;
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        v[e] = fma(w00, a0[e], v[e]);
                        gx[e] = fma(w10, a0[e], gx[e]);
                        gy[e] = fma(w01, a0[e], gy[e]);
                        gz[e] = fma(w00, a1[e], gz[e]);
                        lp[e] = fma(c0, a0[e], fma(c1, a1[e], fma(c2, a2[e], lp[e])));
                    }
                }
            }
        }
        const int o0 = chunk * E;
        if (o0 >= p.n_orb) return;
        const bool vec = p.vec_out != 0;
        A cg[3][E];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const A* mgv = nullptr;
            if constexpr (sizeof(A) == 8) mgv = p.mg; else mgv = p.mgf;
            const A m0 = mgv[3 * a], m1 = mgv[3 * a + 1], m2 = mgv[3 * a + 2];
#pragma unroll
            for (int e = 0; e < E; ++e) cg[a][e] = fma(m0, gx[e], fma(m1, gy[e], m2 * gz[e]));
        }
        if (p.phase) bloch_apply<A, E>(p, ip, v, cg, lp, true, true);
        if (p.val) store_run<A, E>(static_cast<A*>(p.val) + ip * p.n_orb + o0, v, o0, p.n_orb, vec);
        if (p.grad) {
            A* g = static_cast<A*>(p.grad) + ip * 3 * p.n_orb + o0;
#pragma unroll
            for (int a = 0; a < 3; ++a) store_run<A, E>(g + (size_t)a * p.n_orb, cg[a], o0, p.n_orb, vec);
        }
        if (p.lap) store_run<A, E>(static_cast<A*>(p.lap) + ip * p.n_orb + o0, lp, o0, p.n_orb, vec);
    }
}

// float and bfloat16 tables: packed FP32 pairs, the 16 load units of a position (2 x 2
// corner columns x 4 (kappa, mu) labels, four rows each: 2 z corners x 2 nu labels) through a
// ring of three.  Same products and sums, in the same order, as the scalar path.
template <typename T>
__device__ __forceinline__ void pp_task_x2(const EvalArgs& p, long long w0, int lane)
{
    constexpr int E = Traits<T>::E;
    constexpr int NP = Pairs<T>::N;
    constexpr int kUnits = 16;
    constexpr int kRing = 3;
    const int L = 1 << p.lanes_log2;
    const int sub = lane & (L - 1);
    const int gbase = lane & ~(L - 1);
    const long long total = p.n_pos * p.tiles;
    const size_t rowb = (size_t)p.row_stride * sizeof(T);     // one z row: 8 entries x O_p
    const size_t entb = rowb / 8;                              // one entry: O_p
    const size_t colb = (size_t)p.col_stride * sizeof(T);

    const long long gid = w0 + (lane >> p.lanes_log2);
    const bool active = gid < total;
    const long long q = active ? gid / p.tiles : 0;
    const int tile = active ? (int)(gid - q * p.tiles) : 0;
    const long long ip = active ? order_index(p, q) : q;
    int ix, iy, iz;
    float tx, ty, tz;
    bool ok;
    coords_float(p, ip, L, sub, gbase, ix, iy, iz, tx, ty, tz, ok);
    if (!active) return;
    if (!ok && sub == 0 && tile == 0) atomicOr(p.err, 1);
    float wx[2][2], dwx[2][2], d2wx[2][2], wy[2][2], dwy[2][2], d2wy[2][2], wz[2][2], dwz[2][2], d2wz[2][2];
    pp_weights<float>(tx, wx, dwx, d2wx);
    pp_weights<float>(ty, wy, dwy, d2wy);
    pp_weights<float>(tz, wz, dwz, d2wz);
    f32x2 wz2[2][2], dwz2[2][2], d2wz2[2][2];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            wz2[a][b] = pack2(wz[a][b], wz[a][b]);
            dwz2[a][b] = pack2(dwz[a][b], dwz[a][b]);
            d2wz2[a][b] = pack2(d2wz[a][b], d2wz[a][b]);
        }
    const float ml0 = p.mlf[0], ml1 = p.mlf[1], ml2 = p.mlf[2];
    const float ml3 = p.mlf[3], ml4 = p.mlf[4], ml5 = p.mlf[5];
    const int chunk = tile * L + sub;
    const size_t off = (size_t)chunk * 16 + (size_t)iz * rowb;
    const int xs[2] = {ix, ix + 1 < p.nx ? ix + 1 : 0};
    const int ys[2] = {iy, iy + 1 < p.ny ? iy + 1 : 0};
    // unit u: column (i, j) = (u >> 3, (u >> 2) & 1), label km = u & 3; its rows
    // n = 0..3 are (z corner k, label nu) = (n >> 1, n & 1), entry 4 kappa + 2 mu + nu = 2 km + nu
    auto load_unit = [&](int u, uint4* dst) {
        const int i = u >> 3, j = (u >> 2) & 1, km = u & 3;
        const char* col = static_cast<const char*>(p.tab[0]) + (size_t)(xs[i] * p.ny + ys[j]) * colb + off +
                          (size_t)(2 * km) * entb;
#pragma unroll
        for (int n = 0; n < 4; ++n) dst[n] = ldg_table(p, col + (n >> 1) * rowb + (size_t)(n & 1) * entb);
    };
    f32x2 V[NP], GX[NP], GY[NP], GZ[NP], LP[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) V[j] = GX[j] = GY[j] = GZ[j] = LP[j] = 0ull;
    uint4 ring[kRing][4];
    load_unit(0, ring[0]);
    load_unit(1, ring[1]);
#pragma unroll
    for (int u = 0; u < kUnits; ++u) {
        if (u + 2 < kUnits) load_unit(u + 2, ring[(u + 2) % kRing]);
        const int i = u >> 3, j = (u >> 2) & 1, km = u & 3;
        const int kap = km >> 1, mu = km & 1;
        f32x2 a0[NP], a1[NP], a2[NP];
#pragma unroll
        for (int e = 0; e < NP; ++e) a0[e] = a1[e] = a2[e] = 0ull;
#pragma unroll
        for (int n = 0; n < 4; ++n) {
            const int k = n >> 1, nu = n & 1;
            f32x2 cv[NP];
            Pairs<T>::get(ring[u % kRing][n], cv);
#pragma unroll
            for (int e = 0; e < NP; ++e) {
                a0[e] = ffma2(wz2[nu][k], cv[e], a0[e]);
                a1[e] = ffma2(dwz2[nu][k], cv[e], a1[e]);
                a2[e] = ffma2(d2wz2[nu][k], cv[e], a2[e]);
            }
        }
        const float w00 = wx[kap][i] * wy[mu][j];
        const float w10 = dwx[kap][i] * wy[mu][j];
        const float w01 = wx[kap][i] * dwy[mu][j];
        const float c0 = ml0 * (d2wx[kap][i] * wy[mu][j]) + ml1 * (wx[kap][i] * d2wy[mu][j]) +
                         ml3 * (dwx[kap][i] * dwy[mu][j]);
        const float c1 = ml4 * w10 + ml5 * w01;
        const float c2 = ml2 * w00;
        const f32x2 W00 = pack2(w00, w00), W10 = pack2(w10, w10), W01 = pack2(w01, w01);
        const f32x2 C0 = pack2(c0, c0), C1 = pack2(c1, c1), C2 = pack2(c2, c2);
#pragma unroll
        for (int e = 0; e < NP; ++e) {
            V[e] = ffma2(W00, a0[e], V[e]);
            GX[e] = ffma2(W10, a0[e], GX[e]);
            GY[e] = ffma2(W01, a0[e], GY[e]);
            GZ[e] = ffma2(W00, a1[e], GZ[e]);
            LP[e] = ffma2(C0, a0[e], ffma2(C1, a1[e], ffma2(C2, a2[e], LP[e])));
        }
    }
    const int o0 = chunk * E;
    if (o0 >= p.n_orb) return;
    const bool vec = p.vec_out != 0;
    float v[E], gx[E], gy[E], gz[E], lp[E];
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        unpack2(V[j], v[2 * j], v[2 * j + 1]);
        unpack2(GX[j], gx[2 * j], gx[2 * j + 1]);
        unpack2(GY[j], gy[2 * j], gy[2 * j + 1]);
        unpack2(GZ[j], gz[2 * j], gz[2 * j + 1]);
        unpack2(LP[j], lp[2 * j], lp[2 * j + 1]);
    }
    float cg[3][E];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float m0 = p.mgf[3 * a], m1 = p.mgf[3 * a + 1], m2 = p.mgf[3 * a + 2];
#pragma unroll
        for (int e = 0; e < E; ++e) cg[a][e] = fmaf(m0, gx[e], fmaf(m1, gy[e], m2 * gz[e]));
    }
    if (p.phase) bloch_apply<float, E>(p, ip, v, cg, lp, true, true);
    if (p.val) store_run<float, E>(static_cast<float*>(p.val) + ip * p.n_orb + o0, v, o0, p.n_orb, vec);
    if (p.grad) {
        float* g = static_cast<float*>(p.grad) + ip * 3 * p.n_orb + o0;
#pragma unroll
        for (int a = 0; a < 3; ++a) store_run<float, E>(g + (size_t)a * p.n_orb, cg[a], o0, p.n_orb, vec);
    }
    if (p.lap) store_run<float, E>(static_cast<float*>(p.lap) + ip * p.n_orb + o0, lp, o0, p.n_orb, vec);
}

template <typename T, int THREADS>
__global__ void __launch_bounds__(THREADS, 1) pp_vgl_kernel(const EvalArgs p)
{
    constexpr int WPB = THREADS / 32;
    const int lane = threadIdx.x & 31;
    const int gpw = 32 >> p.lanes_log2;
    const long long total = p.n_pos * p.tiles;
    const long long warp = (long long)blockIdx.x * WPB + (threadIdx.x >> 5);
    const long long wstride = (long long)gridDim.x * WPB;
    for (long long w0 = warp * gpw; w0 < total; w0 += wstride * gpw) {
        if constexpr (sizeof(T) == 8) pp_task<T>(p, w0, lane);
        else pp_task_x2<T>(p, w0, lane);
    }
}

template <typename K>
int launch_one_block_per_sm(K kernel, int threads, const EvalArgs& a, cudaStream_t st, const char* name)
{
    const int gpw = 32 >> a.lanes_log2;
    const long long warps = (a.n_pos * a.tiles + gpw - 1) / gpw;
    long long blocks = (warps + threads / 32 - 1) / (threads / 32);
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0);
    if (e != cudaSuccess) return cuda_error(e, "occupancy query");
    if (per_sm < 1) per_sm = 1;
    const long long cap = (long long)sm_count() * per_sm;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    kernel<<<(unsigned)blocks, threads, 0, st>>>(a);
    return cuda_error(cudaGetLastError(), name);
}

template <typename T, int BASIS>
int launch_five(const EvalArgs& a, cudaStream_t st)
{
    return launch_one_block_per_sm(five_table_vgl_kernel<T, BASIS, QMCSPL_FIVE_THREADS>, QMCSPL_FIVE_THREADS, a, st,
                                   "five_table_vgl_kernel launch");
}

template <typename T>
int launch_pp(const EvalArgs& a, cudaStream_t st)
{
    return launch_one_block_per_sm(pp_vgl_kernel<T, QMCSPL_FIVE_THREADS>, QMCSPL_FIVE_THREADS, a, st,
                                   "pp_vgl_kernel launch");
}

EvalArgs make_args(const Handle* h, const double* pos, const Prepared& pr, long long n_pos, void* val,
                   void* grad, void* lap)
{
    EvalArgs a;
    fill_eval_args(h, &a);
    a.pos = pos;
    a.rec = pr.rec;
    a.perm = pr.perm;
    a.phase = pr.phase;
    a.n_pos = n_pos;
    a.val = val;
    a.grad = grad;
    a.lap = lap;
    const size_t ob = (h->storage == QMCSPL_F64 || h->storage == QMCSPL_DF64) ? 8 : 4;
    const uintptr_t al = (uintptr_t)val | (uintptr_t)grad | (uintptr_t)lap;
    a.vec_out = ((h->n_orb * ob) % 16 == 0) && (al % 16 == 0);
    return a;
}

}  // namespace

int launch_five_table_vgl(const Handle* h, const double* pos, const Prepared& pr, long long n_pos, void* val,
                          void* grad, void* lap, cudaStream_t st)
{
    const EvalArgs a = make_args(h, pos, pr, n_pos, val, grad, lap);
    const bool lag = h->method == QMCSPL_LAGRANGE;
    switch (h->storage) {
    case QMCSPL_F64: return lag ? launch_five<double, kFiveLagrange>(a, st) : launch_five<double, kFiveBSpline>(a, st);
    case QMCSPL_F32: return lag ? launch_five<float, kFiveLagrange>(a, st) : launch_five<float, kFiveBSpline>(a, st);
    case QMCSPL_DF64: return launch_five<DF64Tag, kFiveBSpline>(a, st);   // B-splines only (qmcspl_create)
    default:
        return lag ? launch_five<__nv_bfloat16, kFiveLagrange>(a, st) : launch_five<__nv_bfloat16, kFiveBSpline>(a, st);
    }
}

int launch_pp_vgl(const Handle* h, const double* pos, const Prepared& pr, long long n_pos, void* val,
                  void* grad, void* lap, cudaStream_t st)
{
    const EvalArgs a = make_args(h, pos, pr, n_pos, val, grad, lap);
    switch (h->storage) {
    case QMCSPL_F64: return launch_pp<double>(a, st);
    case QMCSPL_F32: return launch_pp<float>(a, st);
    default: return launch_pp<__nv_bfloat16>(a, st);
    }
}

}  // namespace qmcspl
