// eval_general.cuh -- B-splines of odd degree n = 1, 3, 5, 7 on uniform grids and
// interpolating ones of the same degrees on non-uniform periodic grids (Sec. II "Common
// features": any order; "Grid": interpolating splines need no even spacing; Appendix, the
// B-spline recurrence).
//
//   phi(r) = sum_{l,m,k = 0..n} w_l(x) w_m(y) w_k(z) beta[ix+l-(n-1)/2][iy+m-(n-1)/2][iz+k-(n-1)/2]
//
// with the weights of general_basis.cuh.  Uniform grids: cell index and local coordinate
// from u = N s, derivatives with respect to u, chain rule with N_i as for the cubic.
// Non-uniform grids: the cell is found by bisection in the axis' grid points, derivatives
// are with respect to s, so the chain rule uses a^-1 alone (the handle's metric says so).
// Tables keep the cubic layout with (n - 1)/2 ghost planes below z = 0 and (n + 1)/2 above,
// so a stencil column is n + 1 contiguous rows.
//
// One group of L lanes per position and one 16-byte chunk per lane, as in eval_bspline.cu;
// scalar arithmetic (this path is not the tuned cubic one).  With per-position records
// (order.cu) the cell and local coordinate come precomputed and the weights are built in
// the table's arithmetic type; without them every lane reduces its position in FP64.
#pragma once

#include "eval_common.cuh"
#include "general_basis.cuh"

namespace qmcspl {
namespace {

__device__ __forceinline__ int wrapn(int x, int n)
{
    x %= n;
    return x < 0 ? x + n : x;
}

// Knot spacings of the three axes in the arithmetic type A: the device grid-point buffer
// holds [3][kMaxDim] points, then [3][kMaxDim] double spacings, then [3][kMaxDim] float ones.
template <typename A>
__device__ __forceinline__ const A* spacings(const EvalArgs& p)
{
    const double* base = p.knots[0] + 3 * kMaxDim;
    if constexpr (sizeof(A) == 8) return base;
    else return reinterpret_cast<const float*>(base + 3 * kMaxDim);
}

// Cell index and local coordinate of the fractional coordinate f in [0, 1) on one axis:
// uniform grids u = N f, cell floor(u), t = u - floor(u); graded grids the interval of the
// grid points and the offset from its left point (both in FP64, then rounded to A).
template <typename A, bool NONUNI>
__device__ __forceinline__ void locate(const EvalArgs& p, int axis, double f, int n, int& i0, A& loc)
{
    if constexpr (NONUNI) {
        const double* kn = p.knots[axis];
        double x = f;
        i0 = knot_interval(kn, n, x);
        loc = (A)(x - kn[i0]);
    } else {
        const double u = (double)n * f;
        const double fl = floor(u);
        int k = (int)fl;
        if (k >= n) k -= n;
        i0 = k;
        loc = (A)(u - fl);
    }
}

// Weights of one axis from its cell and local coordinate.
template <typename A, int DEG, bool NONUNI>
__device__ __forceinline__ void axis_weights(const EvalArgs& p, int axis, int i0, A loc, A* w, A* dw, A* d2w)
{
    if constexpr (NONUNI) {
        const int n = axis == 0 ? p.nx : (axis == 1 ? p.ny : p.nz);
        nonuniform_weights_local<A, A, DEG>(spacings<A>(p) + axis * kMaxDim, n, i0, loc, (A)p.cdeg, w, dw, d2w);
    } else {
        uniform_weights<A, DEG>(loc, (A)p.cdeg, w, dw, d2w);
    }
}

// Two blocks per SM (at most 128 registers) for the stencils of degree 3 and up: their weight
// arrays would otherwise take up to 255 registers and leave 8 warps per SM (degree 7: 0.184 ->
// 0.160 ms, graded cubic 0.062 -> 0.056 ms on the Si-like 16-orbital step; three blocks spill
// too much).
template <typename T, int DEG, bool NONUNI, bool LAPTAB>
__global__ void __launch_bounds__(kEvalThreads, DEG == 1 ? 1 : 2) general_vgl_kernel(const EvalArgs p)
{
    using A = typename Traits<T>::A;
    constexpr int E = Traits<T>::E;
    constexpr int W = DEG + 1;
    constexpr int H = (DEG - 1) / 2;   // stencil points below the cell
    const int lane = threadIdx.x & 31;
    const int L = 1 << p.lanes_log2;
    const int sub = lane & (L - 1);
    const int gpw = 32 >> p.lanes_log2;
    const long long total = p.n_pos * p.tiles;
    const long long warp = (long long)blockIdx.x * (kEvalThreads / 32) + (threadIdx.x >> 5);
    const long long wstride = (long long)gridDim.x * (kEvalThreads / 32);
    const size_t rowb = (size_t)p.row_stride * sizeof(T);
    const size_t colb = (size_t)p.col_stride * sizeof(T);
    const A* mgv;
    const A* mlv;
    if constexpr (sizeof(A) == 8) { mgv = p.mg; mlv = p.ml; } else { mgv = p.mgf; mlv = p.mlf; }

    for (long long w0 = warp * gpw; w0 < total; w0 += wstride * gpw) {
        const long long gid = w0 + (lane >> p.lanes_log2);
        if (gid >= total) continue;
        const long long q = gid / p.tiles;
        const int tile = (int)(gid - q * p.tiles);
        const long long ip = order_index(p, q);
        // cell and local coordinate per axis (t on uniform grids, the offset from the
        // interval's left grid point on graded ones): from the per-position record, or
        // reduced here in FP64; the weights are then built once, from these alone
        int ci[3];
        A loc[3];
        bool ok = true;
        if (p.rec) {
            int cell;
            if constexpr (sizeof(A) == 8) {
                const double2* qr = static_cast<const double2*>(p.rec) + 2 * ip;
                const double2 a0 = __ldg(qr), a1 = __ldg(qr + 1);
                loc[0] = a0.x;
                loc[1] = a0.y;
                loc[2] = a1.x;
                cell = __double2loint(a1.y);
            } else {
                const float4 qr = __ldg(static_cast<const float4*>(p.rec) + ip);
                cell = __float_as_int(qr.x);
                loc[0] = qr.y;
                loc[1] = qr.z;
                loc[2] = qr.w;
            }
            unpack_cell(cell, ci[0], ci[1], ci[2], ok);
        } else {
            const double r[3] = {p.pos[3 * ip], p.pos[3 * ip + 1], p.pos[3 * ip + 2]};
            const int dims[3] = {p.nx, p.ny, p.nz};
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const double s = crystal(p.ainv[3 * a], p.ainv[3 * a + 1], p.ainv[3 * a + 2], r);
                double f = s - floor(s);
                const bool o = isfinite(f);
                ok = ok && o;
                if (!o) f = 0.0;
                locate<A, NONUNI>(p, a, f, dims[a], ci[a], loc[a]);
                if (!o) loc[a] = A(__longlong_as_double(0x7ff8000000000000LL));
            }
        }
        if (!ok && sub == 0 && tile == 0) atomicOr(p.err, 1);
        const int ix = ci[0], iy = ci[1], iz = ci[2];
        A wx[W], dwx[W], d2wx[W], wy[W], dwy[W], d2wy[W], wz[W], dwz[W], d2wz[W];
        axis_weights<A, DEG, NONUNI>(p, 0, ix, loc[0], wx, dwx, LAPTAB ? nullptr : d2wx);
        axis_weights<A, DEG, NONUNI>(p, 1, iy, loc[1], wy, dwy, LAPTAB ? nullptr : d2wy);
        axis_weights<A, DEG, NONUNI>(p, 2, iz, loc[2], wz, dwz, LAPTAB ? nullptr : d2wz);
        if (!ok) {   // NaN outputs for a non-finite position
            const A nan = A(__longlong_as_double(0x7ff8000000000000LL));
#pragma unroll
            for (int j = 0; j < W; ++j) wx[j] = nan;
        }
        int xs[W], ys[W];
#pragma unroll
        for (int j = 0; j < W; ++j) {
            xs[j] = wrapn(ix + j - H, p.nx);
            ys[j] = wrapn(iy + j - H, p.ny);
        }
        const int chunk = tile * L + sub;
        // rows zz = z + H: the W rows of the stencil start at zz = iz
        const size_t off = (size_t)chunk * 16 + (size_t)iz * rowb;
        A v[E], gx[E], gy[E], gz[E], lp[E];
        if constexpr (sizeof(A) == 4) {
            // float and bfloat16 tables: the same sums on packed FP32 pairs (fma.rn.f32x2, two
            // orbitals per instruction, the same rounding per element as the scalar path)
            constexpr int NP = Pairs<T>::N;
            f32x2 V[NP], GX[NP], GY[NP], GZ[NP], LP[NP];
#pragma unroll
            for (int j = 0; j < NP; ++j) V[j] = GX[j] = GY[j] = GZ[j] = LP[j] = 0ull;
            f32x2 wz2[W], dwz2[W], d2wz2[W];
#pragma unroll
            for (int k = 0; k < W; ++k) {
                wz2[k] = pack2(wz[k], wz[k]);
                dwz2[k] = pack2(dwz[k], dwz[k]);
                if (!LAPTAB) d2wz2[k] = pack2(d2wz[k], d2wz[k]);
            }
#pragma unroll
            for (int l = 0; l < W; ++l) {
#pragma unroll
                for (int m = 0; m < W; ++m) {
                    const size_t col = (size_t)(xs[l] * p.ny + ys[m]) * colb + off;
                    const char* c0 = static_cast<const char*>(p.tab[0]) + col;
                    f32x2 A0[NP], A1[NP], A2[NP], AL[NP];
#pragma unroll
                    for (int j = 0; j < NP; ++j) A0[j] = A1[j] = A2[j] = AL[j] = 0ull;
#pragma unroll
                    for (int k = 0; k < W; ++k) {
                        f32x2 cv[NP];
                        Pairs<T>::get(ldg_table(p, c0 + k * rowb), cv);
#pragma unroll
                        for (int j = 0; j < NP; ++j) {
                            A0[j] = ffma2(wz2[k], cv[j], A0[j]);
                            A1[j] = ffma2(dwz2[k], cv[j], A1[j]);
                            if (!LAPTAB) A2[j] = ffma2(d2wz2[k], cv[j], A2[j]);
                        }
                        if (LAPTAB) {
                            Pairs<T>::get(ldg_table(p, static_cast<const char*>(p.tab[1]) + col + k * rowb), cv);
#pragma unroll
                            for (int j = 0; j < NP; ++j) AL[j] = ffma2(wz2[k], cv[j], AL[j]);
                        }
                    }
                    const A w00 = wx[l] * wy[m], w10 = dwx[l] * wy[m], w01 = wx[l] * dwy[m];
                    const f32x2 W00 = pack2(w00, w00), W10 = pack2(w10, w10), W01 = pack2(w01, w01);
#pragma unroll
                    for (int j = 0; j < NP; ++j) {
                        V[j] = ffma2(W00, A0[j], V[j]);
                        GX[j] = ffma2(W10, A0[j], GX[j]);
                        GY[j] = ffma2(W01, A0[j], GY[j]);
                        GZ[j] = ffma2(W00, A1[j], GZ[j]);
                    }
                    if (LAPTAB) {
#pragma unroll
                        for (int j = 0; j < NP; ++j) LP[j] = ffma2(W00, AL[j], LP[j]);
                    } else {
                        const A c0w = mlv[0] * (d2wx[l] * wy[m]) + mlv[1] * (wx[l] * d2wy[m]) + mlv[3] * (dwx[l] * dwy[m]);
                        const A c1w = mlv[4] * w10 + mlv[5] * w01;
                        const A c2w = mlv[2] * w00;
                        const f32x2 C0 = pack2(c0w, c0w), C1 = pack2(c1w, c1w), C2 = pack2(c2w, c2w);
#pragma unroll
                        for (int j = 0; j < NP; ++j) LP[j] = ffma2(C0, A0[j], ffma2(C1, A1[j], ffma2(C2, A2[j], LP[j])));
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < NP; ++j) {
                unpack2(V[j], v[2 * j], v[2 * j + 1]);
                unpack2(GX[j], gx[2 * j], gx[2 * j + 1]);
                unpack2(GY[j], gy[2 * j], gy[2 * j + 1]);
                unpack2(GZ[j], gz[2 * j], gz[2 * j + 1]);
                unpack2(LP[j], lp[2 * j], lp[2 * j + 1]);
            }
        } else {
#pragma unroll
            for (int e = 0; e < E; ++e) v[e] = gx[e] = gy[e] = gz[e] = lp[e] = A(0);
#pragma unroll
            for (int l = 0; l < W; ++l) {
#pragma unroll
                for (int m = 0; m < W; ++m) {
                    const size_t col = (size_t)(xs[l] * p.ny + ys[m]) * colb + off;
                    const char* c0 = static_cast<const char*>(p.tab[0]) + col;
                    A a0[E], a1[E], a2[E], al[E];
#pragma unroll
                    for (int e = 0; e < E; ++e) a0[e] = a1[e] = a2[e] = al[e] = A(0);
#pragma unroll
                    for (int k = 0; k < W; ++k) {
                        A c[E];
                        unpack<T>(ldg_table(p, c0 + k * rowb), c);
#pragma unroll
                        for (int e = 0; e < E; ++e) {
                            a0[e] = fma(wz[k], c[e], a0[e]);
                            a1[e] = fma(dwz[k], c[e], a1[e]);
                            if (!LAPTAB) a2[e] = fma(d2wz[k], c[e], a2[e]);
                        }
                        if (LAPTAB) {
                            A cl[E];
                            unpack<T>(ldg_table(p, static_cast<const char*>(p.tab[1]) + col + k * rowb), cl);
#pragma unroll
                            for (int e = 0; e < E; ++e) al[e] = fma(wz[k], cl[e], al[e]);
                        }
                    }
                    const A w00 = wx[l] * wy[m], w10 = dwx[l] * wy[m], w01 = wx[l] * dwy[m];
                    A c0w = 0, c1w = 0, c2w = 0;
                    if (!LAPTAB) {
                        c0w = mlv[0] * (d2wx[l] * wy[m]) + mlv[1] * (wx[l] * d2wy[m]) + mlv[3] * (dwx[l] * dwy[m]);
                        c1w = mlv[4] * w10 + mlv[5] * w01;
                        c2w = mlv[2] * w00;
                    }
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        v[e] = fma(w00, a0[e], v[e]);
                        gx[e] = fma(w10, a0[e], gx[e]);
                        gy[e] = fma(w01, a0[e], gy[e]);
                        gz[e] = fma(w00, a1[e], gz[e]);
                        if (LAPTAB) lp[e] = fma(w00, al[e], lp[e]);
                        else lp[e] = fma(c0w, a0[e], fma(c1w, a1[e], fma(c2w, a2[e], lp[e])));
                    }
                }
            }
        }
        const int o0 = chunk * E;
        if (o0 >= p.n_orb) continue;
        const bool vec = p.vec_out != 0;
        A cg[3][E];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int e = 0; e < E; ++e) cg[a][e] = fma(mgv[3 * a], gx[e], fma(mgv[3 * a + 1], gy[e], mgv[3 * a + 2] * gz[e]));
        if (p.phase) bloch_apply<A, E>(p, ip, v, cg, lp, true, !LAPTAB);
        if (p.val) store_run<A, E>(static_cast<A*>(p.val) + ip * p.n_orb + o0, v, o0, p.n_orb, vec);
        if (p.grad)
#pragma unroll
            for (int a = 0; a < 3; ++a)
                store_run<A, E>(static_cast<A*>(p.grad) + (ip * 3 + a) * p.n_orb + o0, cg[a], o0, p.n_orb, vec);
        if (p.lap) store_run<A, E>(static_cast<A*>(p.lap) + ip * p.n_orb + o0, lp, o0, p.n_orb, vec);
    }
}

template <typename T, int DEG, bool NONUNI>
int launch_one(const EvalArgs& a, bool laptab, cudaStream_t st)
{
    void (*k)(EvalArgs) = laptab ? general_vgl_kernel<T, DEG, NONUNI, true> : general_vgl_kernel<T, DEG, NONUNI, false>;
    const int gpw = 32 >> a.lanes_log2;
    const long long warps = (a.n_pos * a.tiles + gpw - 1) / gpw;
    long long blocks = (warps + kEvalThreads / 32 - 1) / (kEvalThreads / 32);
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kEvalThreads, 0);
    if (e != cudaSuccess) return cuda_error(e, "occupancy query");
    if (per_sm < 1) per_sm = 1;
    const long long cap = (long long)sm_count() * per_sm;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k<<<(unsigned)blocks, kEvalThreads, 0, st>>>(a);
    return cuda_error(cudaGetLastError(), "general_vgl_kernel launch");
}

template <typename T>
int launch_typed(const Handle* h, const EvalArgs& a, cudaStream_t st)
{
    const bool lt = h->separate_lap != 0;
    if (h->nonuniform) {
        switch (h->degree) {
        case 1: return launch_one<T, 1, true>(a, lt, st);
        case 3: return launch_one<T, 3, true>(a, lt, st);
        case 5: return launch_one<T, 5, true>(a, lt, st);
        default: return launch_one<T, 7, true>(a, lt, st);
        }
    }
    switch (h->degree) {
    case 1: return launch_one<T, 1, false>(a, lt, st);
    case 3: return launch_one<T, 3, false>(a, lt, st);
    case 5: return launch_one<T, 5, false>(a, lt, st);
    default: return launch_one<T, 7, false>(a, lt, st);
    }
}

}  // namespace

// one translation unit per table type (eval_general_<type>.cu) keeps the build parallel
int launch_general_f64(const Handle* h, const EvalArgs& a, cudaStream_t st);
int launch_general_f32(const Handle* h, const EvalArgs& a, cudaStream_t st);
int launch_general_bf16(const Handle* h, const EvalArgs& a, cudaStream_t st);

}  // namespace qmcspl
