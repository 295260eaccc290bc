// backward_general.cuh -- adjoint of the general B-spline evaluation (eval_general.cuh):
// B-splines of odd degree n = 1, 3, 5, 7 on uniform grids and interpolating ones on graded
// (non-uniform) grids.  Not in the paper; the same transposition as the cubic adjoint of
// backward.cu, over the (n + 1)^3-point stencil:
//   dbeta     += wv B + g~ . D B + wl sum_ij M_ij D_i D_j B   (Hessian-derived Laplacian)
//   dbeta_lap += wl B                                         (separate Laplacian table)
//   dL/dr      = mg^T u,  u_i = sum_o [wv D_i phi + sum_j (D_i D_j phi) g~_j + wl D_i lap],
// with B = w_l(x) w_m(y) w_k(z) the general weights, D_i the derivative along axis i in the
// handle's coordinate (u = N s on uniform grids, s on graded ones; the handle's chain-rule
// constants mg, ml take the matching form), g~ = mg^T wg and D_i lap from third derivatives
// of the weights (general_basis.cuh) or from the gradient of the Laplacian table.  Bloch
// handles first take the upstream through the phase and the bracket (backward_common.cuh).
//
// Scalar arithmetic in the table's accumulation type, one group of L lanes per position and
// one 16-byte chunk of every row per lane, as the forward kernel; positions are reduced in
// FP64 here (no records).  Not a tuned path: up to (n + 1)^3 = 512 rows of vector atomics
// per position.
#pragma once

#include "backward_common.cuh"
#include "eval_general.cuh"

namespace qmcspl {
namespace {

template <typename T, int DEG, bool NONUNI, bool LAPTAB, bool BLOCH>
__global__ void __launch_bounds__(kEvalThreads) general_bwd_kernel(const BwdArgs b)
{
    using A = typename Traits<T>::A;
    constexpr int E = Traits<T>::E;
    constexpr int W = DEG + 1;
    constexpr int H = (DEG - 1) / 2;   // stencil points below the cell
    const EvalArgs& p = b.e;
    const int lane = threadIdx.x & 31;
    const int L = 1 << p.lanes_log2;
    const int sub = lane & (L - 1);
    const int gpw = 32 >> p.lanes_log2;
    const long long total = p.n_pos * p.tiles;
    const long long warp = (long long)blockIdx.x * (kEvalThreads / 32) + (threadIdx.x >> 5);
    const long long wstride = (long long)gridDim.x * (kEvalThreads / 32);
    const size_t rowb = (size_t)p.row_stride * sizeof(T);
    const size_t colb = (size_t)p.col_stride * sizeof(T);
    const int n_orb = p.n_orb;
    const A ml0 = (A)p.ml[0], ml1 = (A)p.ml[1], ml2 = (A)p.ml[2];
    const A ml3 = (A)p.ml[3], ml4 = (A)p.ml[4], ml5 = (A)p.ml[5];

    for (long long w0 = warp * gpw; w0 < total; w0 += wstride * gpw) {
        const long long gid = w0 + (lane >> p.lanes_log2);
        const bool active = gid < total;
        const long long ip = active ? gid / p.tiles : 0;
        const int tile = active ? (int)(gid - ip * p.tiles) : 0;
        // cell and local coordinate per axis, reduced in FP64 as the forward kernel does
        // without records
        int ci[3];
        A loc[3];
        bool ok = true;
        {
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
            }
        }
        if (active && !ok && sub == 0 && tile == 0) atomicOr(p.err, 1);
        const int ix = ci[0], iy = ci[1], iz = ci[2];
        A w[3][W], dw[3][W], d2w[3][W], d3w[3][W];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            if constexpr (NONUNI) {
                const int n = a == 0 ? p.nx : (a == 1 ? p.ny : p.nz);
                nonuniform_weights_local<A, A, DEG>(spacings<A>(p) + a * kMaxDim, n, ci[a], loc[a], (A)p.cdeg,
                                                    w[a], dw[a], d2w[a], d3w[a]);
            } else {
                uniform_weights<A, DEG>(loc[a], (A)p.cdeg, w[a], dw[a], d2w[a], d3w[a]);
            }
        }
        int xs[W], ys[W];
#pragma unroll
        for (int j = 0; j < W; ++j) {
            xs[j] = wrapn(ix + j - H, p.nx);
            ys[j] = wrapn(iy + j - H, p.ny);
        }

        const int chunk = tile * L + sub;
        const int o0 = chunk * E;
        A wv[E], wl[E], gt[3][E];
        A hv[E], hl[E], hg[3][E];   // Bloch: upstream of the bracket (phase term of dL/dr)
        {
            A wg[3][E];
            const A* gvp = static_cast<const A*>(b.gv);
            const A* ggp = static_cast<const A*>(b.gg);
            const A* glp = static_cast<const A*>(b.gl);
            const bool use = active && ok && o0 < n_orb;
            load_run<A>(use && gvp ? gvp + ip * n_orb + o0 : nullptr, wv, o0, n_orb, E);
            load_run<A>(use && glp ? glp + ip * n_orb + o0 : nullptr, wl, o0, n_orb, E);
            for (int a = 0; a < 3; ++a)
                load_run<A>(use && ggp ? ggp + (ip * 3 + a) * n_orb + o0 : nullptr, wg[a], o0, n_orb, E);
            if constexpr (BLOCH) bloch_upstream<A, E, LAPTAB>(p, p.pos + 3 * ip, wv, wg, wl, hv, hg, hl);
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int e = 0; e < E; ++e)
                    gt[i][e] = (A)p.mg[i] * wg[0][e] + (A)p.mg[3 + i] * wg[1][e] + (A)p.mg[6 + i] * wg[2][e];
        }

        // ---- coefficient adjoint: scatter into the W^3 stencil rows ----
        if (b.dcoef && active && ok && o0 < n_orb) {
            A* dc = static_cast<A*>(b.dcoef);
            A* dl = static_cast<A*>(b.dcoef_lap);
            const bool vec = b.vec_atomic != 0;
            for (int l = 0; l < W; ++l)
                for (int m = 0; m < W; ++m)
                    for (int n = 0; n < W; ++n) {
                        const int z = wrapn(iz + n - H, p.nz);
                        const A B = w[0][l] * w[1][m] * w[2][n];
                        const A Bx = dw[0][l] * w[1][m] * w[2][n];
                        const A By = w[0][l] * dw[1][m] * w[2][n];
                        const A Bz = w[0][l] * w[1][m] * dw[2][n];
                        A lapB = 0;
                        if (!LAPTAB)
                            lapB = ml0 * d2w[0][l] * w[1][m] * w[2][n] + ml1 * w[0][l] * d2w[1][m] * w[2][n] +
                                   ml2 * w[0][l] * w[1][m] * d2w[2][n] + ml3 * dw[0][l] * dw[1][m] * w[2][n] +
                                   ml4 * dw[0][l] * w[1][m] * dw[2][n] + ml5 * w[0][l] * dw[1][m] * dw[2][n];
                        A v[E], vl[E];
#pragma unroll
                        for (int e = 0; e < E; ++e) {
                            v[e] = wv[e] * B + gt[0][e] * Bx + gt[1][e] * By + gt[2][e] * Bz;
                            if (LAPTAB) vl[e] = wl[e] * B;
                            else v[e] += wl[e] * lapB;
                        }
                        const size_t row = (((size_t)xs[l] * p.ny + ys[m]) * p.nz + z) * n_orb + o0;
                        atomic_run<A, E>(dc + row, v, o0, n_orb, vec);
                        if (LAPTAB) atomic_run<A, E>(dl + row, vl, o0, n_orb, vec);
                    }
        }

        // ---- position adjoint ----
        if (b.dpos) {
            A g1[3][E], h2[6][E], d3[3][E];
            A u0[E], lam[E];
#pragma unroll
            for (int e = 0; e < E; ++e) {
                for (int i = 0; i < 3; ++i) g1[i][e] = d3[i][e] = A(0);
                for (int i = 0; i < 6; ++i) h2[i][e] = A(0);
                u0[e] = lam[e] = A(0);
            }
            // rows zz = z + H of the ghost-padded layout: the W rows of the stencil start at iz
            const char* t0 = static_cast<const char*>(p.tab[0]) + (size_t)chunk * 16 + (size_t)iz * rowb;
            const char* t1 = LAPTAB ? static_cast<const char*>(p.tab[1]) + (size_t)chunk * 16 + (size_t)iz * rowb
                                    : nullptr;
            for (int l = 0; l < W; ++l)
                for (int m = 0; m < W; ++m) {
                    const size_t col = (size_t)(xs[l] * p.ny + ys[m]) * colb;
                    A a[4][E], al[2][E];
#pragma unroll
                    for (int e = 0; e < E; ++e) a[0][e] = a[1][e] = a[2][e] = a[3][e] = al[0][e] = al[1][e] = A(0);
#pragma unroll
                    for (int n = 0; n < W; ++n) {
                        A c[E];
                        unpack<T>(ldg_table(p, t0 + col + n * rowb), c);
#pragma unroll
                        for (int e = 0; e < E; ++e) {
                            a[0][e] = fma(w[2][n], c[e], a[0][e]);
                            a[1][e] = fma(dw[2][n], c[e], a[1][e]);
                            a[2][e] = fma(d2w[2][n], c[e], a[2][e]);
                            a[3][e] = fma(d3w[2][n], c[e], a[3][e]);
                        }
                        if (LAPTAB) {
                            unpack<T>(ldg_table(p, t1 + col + n * rowb), c);
#pragma unroll
                            for (int e = 0; e < E; ++e) {
                                al[0][e] = fma(w[2][n], c[e], al[0][e]);
                                al[1][e] = fma(dw[2][n], c[e], al[1][e]);
                            }
                        }
                    }
                    const A bx = w[0][l], dbx = dw[0][l], d2bx = d2w[0][l], d3bx = d3w[0][l];
                    const A by = w[1][m], dby = dw[1][m], d2by = d2w[1][m], d3by = d3w[1][m];
                    // third-derivative weights contracted with the Laplacian metric
                    const A x0 = ml0 * d3bx * by + ml1 * dbx * d2by + ml3 * d2bx * dby;
                    const A x1 = ml4 * d2bx * by + ml5 * dbx * dby;
                    const A x2 = ml2 * dbx * by;
                    const A y0 = ml0 * d2bx * dby + ml1 * bx * d3by + ml3 * dbx * d2by;
                    const A y1 = ml4 * dbx * dby + ml5 * bx * d2by;
                    const A y2 = ml2 * bx * dby;
                    const A z1 = ml0 * d2bx * by + ml1 * bx * d2by + ml3 * dbx * dby;
                    const A z2 = ml4 * dbx * by + ml5 * bx * dby;
                    const A z3 = ml2 * bx * by;
                    if constexpr (BLOCH) {
#pragma unroll
                        for (int e = 0; e < E; ++e) {
                            u0[e] += bx * by * a[0][e];
                            if (LAPTAB) lam[e] += bx * by * al[0][e];
                        }
                    }
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        g1[0][e] += dbx * by * a[0][e];
                        g1[1][e] += bx * dby * a[0][e];
                        g1[2][e] += bx * by * a[1][e];
                        h2[0][e] += d2bx * by * a[0][e];
                        h2[1][e] += bx * d2by * a[0][e];
                        h2[2][e] += bx * by * a[2][e];
                        h2[3][e] += dbx * dby * a[0][e];
                        h2[4][e] += dbx * by * a[1][e];
                        h2[5][e] += bx * dby * a[1][e];
                        if (LAPTAB) {
                            d3[0][e] += dbx * by * al[0][e];
                            d3[1][e] += bx * dby * al[0][e];
                            d3[2][e] += bx * by * al[1][e];
                        } else {
                            d3[0][e] += x0 * a[0][e] + x1 * a[1][e] + x2 * a[2][e];
                            d3[1][e] += y0 * a[0][e] + y1 * a[1][e] + y2 * a[2][e];
                            d3[2][e] += z1 * a[1][e] + z2 * a[2][e] + z3 * a[3][e];
                        }
                    }
                }
            double u[3] = {0.0, 0.0, 0.0};
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const A hxx = h2[0][e], hyy = h2[1][e], hzz = h2[2][e];
                const A hxy = h2[3][e], hxz = h2[4][e], hyz = h2[5][e];
                u[0] += (double)(wv[e] * g1[0][e] + hxx * gt[0][e] + hxy * gt[1][e] + hxz * gt[2][e] + wl[e] * d3[0][e]);
                u[1] += (double)(wv[e] * g1[1][e] + hxy * gt[0][e] + hyy * gt[1][e] + hyz * gt[2][e] + wl[e] * d3[1][e]);
                u[2] += (double)(wv[e] * g1[2][e] + hxz * gt[0][e] + hyz * gt[1][e] + hzz * gt[2][e] + wl[e] * d3[2][e]);
            }
            double sph = 0.0;
            if constexpr (BLOCH) sph = bloch_phase_sum<A, E, LAPTAB>(p, u0, g1, h2, lam, hv, hg, hl);
            for (int off = L >> 1; off > 0; off >>= 1) {
#pragma unroll
                for (int i = 0; i < 3; ++i) u[i] += __shfl_xor_sync(kFullMask, u[i], off);
                sph += __shfl_xor_sync(kFullMask, sph, off);
            }
            if (active && sub == 0) {
                const double nan = __longlong_as_double(0x7ff8000000000000LL);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const double d = p.mg[3 * a] * u[0] + p.mg[3 * a + 1] * u[1] + p.mg[3 * a + 2] * u[2] -
                                     p.kc[a] * sph;
                    atomicAdd(b.dpos + 3 * ip + a, ok ? d : nan);
                }
            }
        }
    }
}

template <typename T, int DEG, bool NONUNI, bool LAPTAB, bool BLOCH>
int general_bwd_launch(const BwdArgs& a, cudaStream_t st)
{
    auto k = general_bwd_kernel<T, DEG, NONUNI, LAPTAB, BLOCH>;
    const int gpw = 32 >> a.e.lanes_log2;
    const long long warps = (a.e.n_pos * a.e.tiles + gpw - 1) / gpw;
    long long blocks = (warps + kEvalThreads / 32 - 1) / (kEvalThreads / 32);
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kEvalThreads, 0);
    if (e != cudaSuccess) return cuda_error(e, "occupancy query");
    if (per_sm < 1) per_sm = 1;
    const long long cap = (long long)sm_count() * per_sm;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    k<<<(unsigned)blocks, kEvalThreads, 0, st>>>(a);
    return cuda_error(cudaGetLastError(), "general_bwd_kernel launch");
}

template <typename T, int DEG, bool NONUNI>
int general_bwd_flags(const BwdArgs& a, bool laptab, cudaStream_t st)
{
    if (laptab)
        return a.bloch ? general_bwd_launch<T, DEG, NONUNI, true, true>(a, st)
                       : general_bwd_launch<T, DEG, NONUNI, true, false>(a, st);
    return a.bloch ? general_bwd_launch<T, DEG, NONUNI, false, true>(a, st)
                   : general_bwd_launch<T, DEG, NONUNI, false, false>(a, st);
}

// degree 3 on a uniform grid is the cubic adjoint of backward.cu, never dispatched here
template <typename T>
int general_bwd_typed(const Handle* h, const BwdArgs& a, cudaStream_t st)
{
    const bool lt = h->separate_lap != 0;
    if (h->nonuniform) {
        switch (h->degree) {
        case 1: return general_bwd_flags<T, 1, true>(a, lt, st);
        case 3: return general_bwd_flags<T, 3, true>(a, lt, st);
        case 5: return general_bwd_flags<T, 5, true>(a, lt, st);
        default: return general_bwd_flags<T, 7, true>(a, lt, st);
        }
    }
    switch (h->degree) {
    case 1: return general_bwd_flags<T, 1, false>(a, lt, st);
    case 5: return general_bwd_flags<T, 5, false>(a, lt, st);
    default: return general_bwd_flags<T, 7, false>(a, lt, st);
    }
}

}  // namespace

// one translation unit per table type (backward_general_<type>.cu) keeps the build parallel
int launch_general_backward_f64(const Handle* h, const BwdArgs& a, cudaStream_t st);
int launch_general_backward_f32(const Handle* h, const BwdArgs& a, cudaStream_t st);
int launch_general_backward_bf16(const Handle* h, const BwdArgs& a, cudaStream_t st);

}  // namespace qmcspl
