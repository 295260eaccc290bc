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
// position, one 16-byte chunk of each row per lane.  Bloch orbitals (Sec. II) take the
// same epilogue as the B-splines (bloch_apply).
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

template <typename T, int BASIS>
__global__ void __launch_bounds__(kEvalThreads, 2) five_table_vgl_kernel(const EvalArgs p)
{
    using A = typename Traits<T>::A;
    constexpr int E = Traits<T>::E;
    const int lane = threadIdx.x & 31;
    const int L = 1 << p.lanes_log2;
    const int sub = lane & (L - 1);
    const int gbase = lane & ~(L - 1);
    const int gpw = 32 >> p.lanes_log2;
    const long long total = p.n_pos * p.tiles;
    const long long warp = (long long)blockIdx.x * (kEvalThreads / 32) + (threadIdx.x >> 5);
    const long long wstride = (long long)gridDim.x * (kEvalThreads / 32);
    const size_t rowb = (size_t)p.row_stride * sizeof(T);
    const size_t colb = (size_t)p.col_stride * sizeof(T);

    for (long long w0 = warp * gpw; w0 < total; w0 += wstride * gpw) {
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
        if (!active) continue;
        if (!ok && sub == 0 && tile == 0) atomicOr(p.err, 1);
        A lx[4], ly[4], lz[4];
        value_weights<BASIS, A>((A)tx, lx);
        value_weights<BASIS, A>((A)ty, ly);
        value_weights<BASIS, A>((A)tz, lz);
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
        if (o0 >= p.n_orb) continue;
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

template <typename T>
__global__ void __launch_bounds__(kEvalThreads, 2) pp_vgl_kernel(const EvalArgs p)
{
    using A = typename Traits<T>::A;
    constexpr int E = Traits<T>::E;
    const int lane = threadIdx.x & 31;
    const int L = 1 << p.lanes_log2;
    const int sub = lane & (L - 1);
    const int gbase = lane & ~(L - 1);
    const int gpw = 32 >> p.lanes_log2;
    const long long total = p.n_pos * p.tiles;
    const long long warp = (long long)blockIdx.x * (kEvalThreads / 32) + (threadIdx.x >> 5);
    const long long wstride = (long long)gridDim.x * (kEvalThreads / 32);
    const size_t rowb = (size_t)p.row_stride * sizeof(T);     // one z row: 8 entries x O_p
    const size_t entb = rowb / 8;                              // one entry: O_p
    const size_t colb = (size_t)p.col_stride * sizeof(T);

    for (long long w0 = warp * gpw; w0 < total; w0 += wstride * gpw) {
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
        if (!active) continue;
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
        if (o0 >= p.n_orb) continue;
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

template <template <typename> class K, typename T>
int launch_variant(void (*kernel)(EvalArgs), const EvalArgs& a, cudaStream_t st, const char* name)
{
    const int gpw = 32 >> a.lanes_log2;
    const long long groups = a.n_pos * a.tiles;
    const long long warps = (groups + gpw - 1) / gpw;
    long long blocks = (warps + kEvalThreads / 32 - 1) / (kEvalThreads / 32);
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kEvalThreads, 0);
    if (e != cudaSuccess) return cuda_error(e, "occupancy query");
    if (per_sm < 1) per_sm = 1;
    const long long cap = (long long)sm_count() * per_sm;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    kernel<<<(unsigned)blocks, kEvalThreads, 0, st>>>(a);
    return cuda_error(cudaGetLastError(), name);
}

template <typename T> struct FiveK {};
template <typename T> struct PPK {};

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
    const size_t ob = (h->storage == QMCSPL_F64) ? 8 : 4;
    const uintptr_t al = (uintptr_t)val | (uintptr_t)grad | (uintptr_t)lap;
    a.vec_out = ((h->n_orb * ob) % 16 == 0) && (al % 16 == 0);
    return a;
}

}  // namespace

int launch_five_table_vgl(const Handle* h, const double* pos, const Prepared& pr, long long n_pos, void* val,
                          void* grad, void* lap, cudaStream_t st)
{
    const EvalArgs a = make_args(h, pos, pr, n_pos, val, grad, lap);
    const char* name = "five_table_vgl_kernel";
    if (h->method == QMCSPL_LAGRANGE) {
        switch (h->storage) {
        case QMCSPL_F64: return launch_variant<FiveK, double>(five_table_vgl_kernel<double, kFiveLagrange>, a, st, name);
        case QMCSPL_F32: return launch_variant<FiveK, float>(five_table_vgl_kernel<float, kFiveLagrange>, a, st, name);
        default:
            return launch_variant<FiveK, __nv_bfloat16>(five_table_vgl_kernel<__nv_bfloat16, kFiveLagrange>, a, st,
                                                        name);
        }
    }
    switch (h->storage) {
    case QMCSPL_F64: return launch_variant<FiveK, double>(five_table_vgl_kernel<double, kFiveBSpline>, a, st, name);
    case QMCSPL_F32: return launch_variant<FiveK, float>(five_table_vgl_kernel<float, kFiveBSpline>, a, st, name);
    default:
        return launch_variant<FiveK, __nv_bfloat16>(five_table_vgl_kernel<__nv_bfloat16, kFiveBSpline>, a, st, name);
    }
}

int launch_pp_vgl(const Handle* h, const double* pos, const Prepared& pr, long long n_pos, void* val,
                  void* grad, void* lap, cudaStream_t st)
{
    const EvalArgs a = make_args(h, pos, pr, n_pos, val, grad, lap);
    switch (h->storage) {
    case QMCSPL_F64: return launch_variant<PPK, double>(pp_vgl_kernel<double>, a, st, "pp_vgl_kernel");
    case QMCSPL_F32: return launch_variant<PPK, float>(pp_vgl_kernel<float>, a, st, "pp_vgl_kernel");
    default: return launch_variant<PPK, __nv_bfloat16>(pp_vgl_kernel<__nv_bfloat16>, a, st, "pp_vgl_kernel");
    }
}

}  // namespace qmcspl
