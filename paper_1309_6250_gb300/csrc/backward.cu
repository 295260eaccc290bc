// backward.cu -- adjoint of the evaluation (not part of the paper: gradients of a downstream
// scalar L for orbital optimisation and forces), for the tricubic B-splines below, and further
// down for the five-table handles (Lagrange, B-splines with separate gradient tables) and the
// pp-splines; B-splines of other degrees and on graded grids in backward_general.cuh.
//
// Given upstream weights wv = dL/dval, wg = dL/dgrad (Cartesian), wl = dL/dlap for one
// position and orbital, the chain rule of Sec. II (Coordinates) is transposed first:
//   g~_i = sum_a N_i (a^-1)_{i a} wg_a           (reduced-coordinate gradient weight)
// Coefficient adjoint (linear in beta, exact transpose of the evaluation): every
// stencil point (l, m, n) receives
//   dbeta     += wv B + g~ . grad_t B + wl lap(B)        (Hessian-derived Laplacian)
//   dbeta_lap += wl B                                     (separate Laplacian table)
// with B = b_l(tx) b_m(ty) b_n(tz) and lap(B) = sum_ij N_i N_j (a^-1 a^-T)_ij d2B/dt_i dt_j;
// the adds are vector atomics into the canonical table layout [Nx][Ny][Nz][O].
// Position adjoint: dL/dr = N (a^-1)^T u summed over orbitals, with
//   u_i = wv dphi/dt_i + sum_j H_ij g~_j + wl d(lap)/dt_i,
// where d(lap)/dt_i needs the third derivatives of the spline (Hessian-derived
// Laplacian) or the gradient of the Laplacian table.  The stencil weights are
// recomputed here, not stored by the forward pass.
//
// Bloch orbitals (Sec. II): the outputs are complex, z = e w with e = exp(i k.r) and w the
// bracket of bloch_apply (u; grad u + i k u; lap u + 2 i k.grad u - |k|^2 u, or the
// Laplacian table's value).  With upstream g = dL/dRe z + i dL/dIm z (complex, the layout of
// the outputs), the upstream of the bracket is h = conj(e) g, and transposing the bracket gives
// the upstream of the tabulated u (its real part for the Re u table, its imaginary part for Im u):
//   u:       h_val - i k.h_grad - |k|^2 h_lap      (the last term with the Hessian Laplacian)
//   grad u:  h_grad - 2 i k h_lap                  (the last term with the Hessian Laplacian)
//   lap u:   h_lap
// after which the real adjoint above applies unchanged.  The position adjoint gains the
// derivative of the phase, d e / d r = i k e:  dL/dr += -k sum_z Im(conj(h_z) w_z).
#include "backward_common.cuh"

namespace qmcspl {

// the general B-spline adjoint, one translation unit per table type (backward_general.cuh)
int launch_general_backward_f64(const Handle* h, const BwdArgs& a, cudaStream_t st);
int launch_general_backward_f32(const Handle* h, const BwdArgs& a, cudaStream_t st);
int launch_general_backward_bf16(const Handle* h, const BwdArgs& a, cudaStream_t st);

namespace {

// Grid cell and local coordinate t of position ip in the adjoint's arithmetic type A: from the
// per-position records when the launch has them (float records for float and bfloat16 tables,
// double records for double tables), else reduced here in FP64 and rounded to A -- the same
// values either way.  All 32 lanes must call it.
template <typename A>
__device__ __forceinline__ void bwd_coords(const EvalArgs& p, long long ip, int L, int sub, int gbase, int& ix,
                                           int& iy, int& iz, A& tx, A& ty, A& tz, bool& ok)
{
    if constexpr (sizeof(A) == 4) {
        float x, y, z;
        coords_float(p, ip, L, sub, gbase, ix, iy, iz, x, y, z, ok);
        tx = x;
        ty = y;
        tz = z;
    } else {
        double x, y, z;
        coords_double(p, ip, L, sub, gbase, ix, iy, iz, x, y, z, ok);
        tx = x;
        ty = y;
        tz = z;
    }
}

// One position's share of both adjoints for the lanes of one group (L lanes, lane `sub` owning the
// 16-byte chunk `chunk` of every stored row, E orbitals from o0 = chunk E): the coefficient adjoint's
// 64 stencil-point rows go to scatter(ix, iy, iz, l, m, n, o0, v, vl) (v for the value table, vl for
// the Laplacian table), the position adjoint is summed over the group and added to dpos[ip] by lane
// sub = 0.  COEF = false leaves the coefficient adjoint out (fewer registers for a pass that
// computes dL/dr alone).  first_part: this group's part is the one that reports a non-finite
// position.  All 32 lanes of the warp must call it (the group reductions shuffle).
template <typename T, bool LAPTAB, bool BLOCH, bool COEF, typename Scatter>
__device__ __forceinline__ void bwd_position(const BwdArgs& b, long long ip, bool active, bool first_part, int chunk,
                                             int L, int sub, int gbase, Scatter&& scatter)
{
    using A = typename Traits<T>::A;
    constexpr int E = Traits<T>::E;
    const EvalArgs& p = b.e;
    const size_t rowb = (size_t)p.row_stride * sizeof(T);
    const size_t colb = (size_t)p.col_stride * sizeof(T);
    const int n_orb = p.n_orb;
    int ix, iy, iz;
    A tx, ty, tz;
    bool ok;
    bwd_coords<A>(p, ip, L, sub, gbase, ix, iy, iz, tx, ty, tz, ok);
    if (active && !ok && sub == 0 && first_part) atomicOr(p.err, 1);

    A w[3][4], dw[3][4], d2w[3][4];
    bspline_weights<A>(tx, w[0], dw[0], d2w[0]);
    bspline_weights<A>(ty, w[1], dw[1], d2w[1]);
    bspline_weights<A>(tz, w[2], dw[2], d2w[2]);
    const A d3w[4] = {A(-1.5), A(4.5), A(-4.5), A(1.5)};

    const int o0 = chunk * E;
    // upstream weights of my orbitals (zero for inactive lanes and padding)
    A wv[E], wl[E], gt[3][E];
    A hv[E], hl[E], hg[3][E];   // Bloch: upstream of the bracket (phase term of dL/dr)
    {
        A wg[3][E];
        const A* gvp = static_cast<const A*>(b.gv);
        const A* ggp = static_cast<const A*>(b.gg);
        const A* glp = static_cast<const A*>(b.gl);
        const bool use = active && o0 < n_orb;
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
    const A ml0 = (A)p.ml[0], ml1 = (A)p.ml[1], ml2 = (A)p.ml[2];
    const A ml3 = (A)p.ml[3], ml4 = (A)p.ml[4], ml5 = (A)p.ml[5];
    int xs[4], ys[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        xs[j] = wrap1(ix + j - 1, p.nx);
        ys[j] = wrap1(iy + j - 1, p.ny);
    }

    // ---- coefficient adjoint: the weights of the 64 stencil points, handed to `scatter` ----
    // (a non-finite position adds nothing; its dL/dr comes out NaN)
    if (COEF && b.dcoef && active && ok && o0 < n_orb) {
        for (int l = 0; l < 4; ++l)
            for (int m = 0; m < 4; ++m)
                for (int n = 0; n < 4; ++n) {
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
                    scatter(ix, iy, iz, l, m, n, o0, v, vl);
                }
    }

    // ---- position adjoint ----
    if (b.dpos) {
        // reduced derivatives of my orbitals: gradient, Hessian, gradient of the Laplacian
        A g1[3][E], h2[6][E], d3[3][E];
        A u0[E], lam[E];   // Bloch: value of u and of the Laplacian table, for the phase term
#pragma unroll
        for (int e = 0; e < E; ++e) {
            for (int i = 0; i < 3; ++i) g1[i][e] = d3[i][e] = A(0);
            for (int i = 0; i < 6; ++i) h2[i][e] = A(0);
            u0[e] = lam[e] = A(0);
        }
        const char* t0 = static_cast<const char*>(p.tab[0]) + (size_t)chunk * 16 + (size_t)iz * rowb;
        const char* t1 = LAPTAB ? static_cast<const char*>(p.tab[1]) + (size_t)chunk * 16 + (size_t)iz * rowb
                                : nullptr;
        // a lane whose chunk lies past the stored row (a wide group on a short row) reads nothing
        const bool live = (size_t)chunk * 16 < rowb;
        for (int l = 0; l < 4; ++l)
            for (int m = 0; m < 4; ++m) {
                const size_t col = (size_t)(xs[l] * p.ny + ys[m]) * colb;
                A a[4][E], al[2][E];
#pragma unroll
                for (int e = 0; e < E; ++e) a[0][e] = a[1][e] = a[2][e] = a[3][e] = al[0][e] = al[1][e] = A(0);
#pragma unroll
                for (int n = 0; n < 4 && live; ++n) {
                    A c[E];
                    unpack<T>(ldg_table(p, t0 + col + n * rowb), c);
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        a[0][e] = fma(w[2][n], c[e], a[0][e]);
                        a[1][e] = fma(dw[2][n], c[e], a[1][e]);
                        a[2][e] = fma(d2w[2][n], c[e], a[2][e]);
                        a[3][e] = fma(d3w[n], c[e], a[3][e]);
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
                const A bx = w[0][l], dbx = dw[0][l], d2bx = d2w[0][l], d3bx = d3w[l];
                const A by = w[1][m], dby = dw[1][m], d2by = d2w[1][m], d3by = d3w[m];
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
        // u_i = wv g_i + sum_j H_ij g~_j + wl d3_i, summed over my orbitals (in FP64)
        double u[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const A hxx = h2[0][e], hyy = h2[1][e], hzz = h2[2][e];
            const A hxy = h2[3][e], hxz = h2[4][e], hyz = h2[5][e];
            u[0] += (double)(wv[e] * g1[0][e] + hxx * gt[0][e] + hxy * gt[1][e] + hxz * gt[2][e] + wl[e] * d3[0][e]);
            u[1] += (double)(wv[e] * g1[1][e] + hxy * gt[0][e] + hyy * gt[1][e] + hyz * gt[2][e] + wl[e] * d3[1][e]);
            u[2] += (double)(wv[e] * g1[2][e] + hxz * gt[0][e] + hyz * gt[1][e] + hzz * gt[2][e] + wl[e] * d3[2][e]);
        }
        // Bloch: the phase term, sum over outputs z of Im(conj(h_z) w_z) with the bracket w
        double sph = 0.0;
        if constexpr (BLOCH) sph = bloch_phase_sum<A, E, LAPTAB>(p, u0, g1, h2, lam, hv, hg, hl);
        // sum over the lanes of the group (all lanes of the warp take part)
        for (int off = L >> 1; off > 0; off >>= 1) {
#pragma unroll
            for (int i = 0; i < 3; ++i) u[i] += __shfl_xor_sync(kFullMask, u[i], off);
            sph += __shfl_xor_sync(kFullMask, sph, off);
        }
        if (active && sub == 0) {
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const double d = p.mg[3 * a] * u[0] + p.mg[3 * a + 1] * u[1] + p.mg[3 * a + 2] * u[2] -
                                 p.kc[a] * sph;
                atomicAdd(b.dpos + 3 * ip + a, d);
            }
        }
    }
}

template <typename T, bool LAPTAB, bool BLOCH, bool COEF>
__global__ void __launch_bounds__(kEvalThreads) bspline_bwd_kernel(const BwdArgs b)
{
    using A = typename Traits<T>::A;
    constexpr int E = Traits<T>::E;
    const EvalArgs& p = b.e;
    const int lane = threadIdx.x & 31;
    const int L = 1 << p.lanes_log2;
    const int sub = lane & (L - 1);
    const int gbase = lane & ~(L - 1);
    const int gpw = 32 >> p.lanes_log2;
    const long long total = p.n_pos * p.tiles;
    const long long warp = (long long)blockIdx.x * (kEvalThreads / 32) + (threadIdx.x >> 5);
    const long long wstride = (long long)gridDim.x * (kEvalThreads / 32);
    const int n_orb = p.n_orb;
    A* dc = static_cast<A*>(b.dcoef);
    A* dl = static_cast<A*>(b.dcoef_lap);
    const bool vec = b.vec_atomic != 0;
    // global vector atomics into the canonical table layout [Nx][Ny][Nz][O]
    auto scatter = [&](int ix, int iy, int iz, int l, int m, int n, int o0, const A* v, const A* vl) {
        const size_t row = (((size_t)wrap1(ix + l - 1, p.nx) * p.ny + wrap1(iy + m - 1, p.ny)) * p.nz +
                            wrap1(iz + n - 1, p.nz)) * n_orb + o0;
        atomic_run<A, E>(dc + row, v, o0, n_orb, vec);
        if (LAPTAB) atomic_run<A, E>(dl + row, vl, o0, n_orb, vec);
    };
    for (long long w0 = warp * gpw; w0 < total; w0 += wstride * gpw) {
        const long long gid = w0 + (lane >> p.lanes_log2);
        const bool active = gid < total;
        const long long q = active ? gid / p.tiles : 0;
        const int tile = active ? (int)(gid - q * p.tiles) : 0;
        const long long ip = active ? order_index(p, q) : 0;   // through the cell order, if any
        bwd_position<T, LAPTAB, BLOCH, COEF>(b, ip, active, tile == 0, tile * L + sub, L, sub, gbase, scatter);
    }
}

// ---- position adjoint alone, float and bfloat16 tables of real orbitals ----
// u_i = dL/dt_i = sum over the lane's orbitals of wv d_i phi + sum_j g~_j d_i d_j phi + wl d_i lap,
// with phi = sum over the 4 x 4 stencil columns (l, m) of bx_l by_m (sum_n bz_n c_n).  The upstream
// weights are contracted with each column's z sums first: with a_k = sum_n bz^(k)_n c_n (k-th
// derivative weights in z) and al_k the same for the Laplacian table, the column adds
//   u_x += bx' by (wv.a0 + wl.al0) + bx'' by (g~x.a0) + bx' by' (g~y.a0) + bx' by (g~z.a1)
//   u_y += bx by' (wv.a0 + wl.al0) + bx' by' (g~x.a0) + bx by'' (g~y.a0) + bx by' (g~z.a1)
//   u_z += bx by (wv.a1 + wl.al1) + bx' by (g~x.a1) + bx by' (g~y.a1) + bx by (g~z.a2)
// (without the Laplacian table the wl terms are the metric-weighted third derivatives of the
// Hessian Laplacian instead, from wl.a0 .. wl.a3), where "." sums over the lane's orbitals --
// eight or twelve dot products per column instead of twelve running sums per orbital.  Packed
// FP32 pairs.  The rows of the next two columns are in flight while one is contracted (the
// first two issued before the upstream weights are read): with 16 warps per SM one column
// ahead left the kernel waiting on its loads (4.2 ms against 2.2 ms on 524,288 positions x 128
// orbitals).
constexpr int kDposDepth = 2;
template <typename T, bool LAPTAB>
__device__ __forceinline__ void dpos_task_x2(const BwdArgs& b, long long w0, int lane)
{
    const EvalArgs& p = b.e;
    constexpr int E = Traits<T>::E;
    constexpr int NP = Pairs<T>::N;
    constexpr int R = LAPTAB ? 8 : 4;
    const int L = 1 << p.lanes_log2;
    const int sub = lane & (L - 1);
    const int gbase = lane & ~(L - 1);
    const long long total = p.n_pos * p.tiles;
    const size_t rowb = (size_t)p.row_stride * sizeof(T);
    const size_t colb = (size_t)p.col_stride * sizeof(T);
    const int n_orb = p.n_orb;

    const long long gid = w0 + (lane >> p.lanes_log2);
    const bool active = gid < total;
    const long long q = active ? gid / p.tiles : 0;
    const int tile = active ? (int)(gid - q * p.tiles) : 0;
    const long long ip = active ? order_index(p, q) : q;
    int ix, iy, iz;
    float tx, ty, tz;
    bool ok;
    coords_float(p, ip, L, sub, gbase, ix, iy, iz, tx, ty, tz, ok);
    if (active && !ok && sub == 0 && tile == 0) atomicOr(p.err, 1);

    float bx[4], dbx[4], d2bx[4], by[4], dby[4], d2by[4], bz[4], dbz[4], d2bz[4];
    bspline_weights<float>(tx, bx, dbx, d2bx);
    bspline_weights<float>(ty, by, dby, d2by);
    bspline_weights<float>(tz, bz, dbz, d2bz);
    const float d3w[4] = {-1.5f, 4.5f, -4.5f, 1.5f};
    f32x2 bz2[4], dbz2[4], d2bz2[4], d3z2[4];
#pragma unroll
    for (int n = 0; n < 4; ++n) {
        bz2[n] = pack2(bz[n], bz[n]);
        dbz2[n] = pack2(dbz[n], dbz[n]);
        d2bz2[n] = pack2(d2bz[n], d2bz[n]);
        if (!LAPTAB) d3z2[n] = pack2(d3w[n], d3w[n]);
    }
    const int chunk = tile * L + sub;
    const int o0 = chunk * E;
    const float ml0 = p.mlf[0], ml1 = p.mlf[1], ml2 = p.mlf[2];
    const float ml3 = p.mlf[3], ml4 = p.mlf[4], ml5 = p.mlf[5];
    int xs[4], ys[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        xs[j] = wrap1(ix + j - 1, p.nx);
        ys[j] = wrap1(iy + j - 1, p.ny);
    }
    const char* t0 = static_cast<const char*>(p.tab[0]) + (size_t)chunk * 16 + (size_t)iz * rowb;
    const char* t1 = LAPTAB ? static_cast<const char*>(p.tab[1]) + (size_t)chunk * 16 + (size_t)iz * rowb : nullptr;
    auto hsum = [](f32x2 v) {
        float lo, hi;
        unpack2(v, lo, hi);
        return lo + hi;
    };
    float ux = 0.f, uy = 0.f, uz = 0.f;
    // a ring of D + 1 columns of rows: column c + D is loaded while column c is contracted
    constexpr int D = kDposDepth;
    uint4 ring[D + 1][R];
    auto load_column = [&](int c, uint4 (&dst)[R]) {
        const size_t col = (size_t)(xs[c >> 2] * p.ny + ys[c & 3]) * colb;
#pragma unroll
        for (int n = 0; n < 4; ++n) dst[n] = ldg_table(p, t0 + col + n * rowb);
        if (LAPTAB) {
#pragma unroll
            for (int n = 0; n < 4; ++n) dst[4 + n] = ldg_table(p, t1 + col + n * rowb);
        }
    };
#pragma unroll
    for (int c = 0; c < D; ++c) load_column(c, ring[c]);
    // the lane's upstream weights (loaded while the first column's rows are in flight), the
    // gradient's through the transposed chain rule, as pairs
    f32x2 WV[NP], WL[NP], GX[NP], GY[NP], GZ[NP];
    {
        float wv[E], wl[E], wg[3][E];
        const float* gvp = static_cast<const float*>(b.gv);
        const float* ggp = static_cast<const float*>(b.gg);
        const float* glp = static_cast<const float*>(b.gl);
        const bool use = active && o0 < n_orb;
        load_run<float>(use && gvp ? gvp + ip * n_orb + o0 : nullptr, wv, o0, n_orb, E);
        load_run<float>(use && glp ? glp + ip * n_orb + o0 : nullptr, wl, o0, n_orb, E);
#pragma unroll
        for (int a = 0; a < 3; ++a)
            load_run<float>(use && ggp ? ggp + (ip * 3 + a) * n_orb + o0 : nullptr, wg[a], o0, n_orb, E);
        float gt[3][E];
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int e = 0; e < E; ++e)
                gt[i][e] = (float)p.mg[i] * wg[0][e] + (float)p.mg[3 + i] * wg[1][e] + (float)p.mg[6 + i] * wg[2][e];
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            WV[j] = pack2(wv[2 * j], wv[2 * j + 1]);
            WL[j] = pack2(wl[2 * j], wl[2 * j + 1]);
            GX[j] = pack2(gt[0][2 * j], gt[0][2 * j + 1]);
            GY[j] = pack2(gt[1][2 * j], gt[1][2 * j + 1]);
            GZ[j] = pack2(gt[2][2 * j], gt[2][2 * j + 1]);
        }
    }
#pragma unroll
    for (int c = 0; c < 16; ++c) {
        const int l = c >> 2, m = c & 3;
        if (c + D < 16) load_column(c + D, ring[(c + D) % (D + 1)]);
        const uint4 (&cur)[R] = ring[c % (D + 1)];
        // z sums of the column (value table; the Laplacian table's with the value weights)
        f32x2 A0[NP], A1[NP], A2[NP], A3[NP], AL0[NP], AL1[NP];
#pragma unroll
        for (int j = 0; j < NP; ++j) A0[j] = A1[j] = A2[j] = A3[j] = AL0[j] = AL1[j] = 0ull;
#pragma unroll
        for (int n = 0; n < 4; ++n) {
            f32x2 cv[NP];
            Pairs<T>::get(cur[n], cv);
#pragma unroll
            for (int j = 0; j < NP; ++j) {
                A0[j] = ffma2(bz2[n], cv[j], A0[j]);
                A1[j] = ffma2(dbz2[n], cv[j], A1[j]);
                A2[j] = ffma2(d2bz2[n], cv[j], A2[j]);
                if (!LAPTAB) A3[j] = ffma2(d3z2[n], cv[j], A3[j]);
            }
            if (LAPTAB) {
                Pairs<T>::get(cur[4 + n], cv);
#pragma unroll
                for (int j = 0; j < NP; ++j) {
                    AL0[j] = ffma2(bz2[n], cv[j], AL0[j]);
                    AL1[j] = ffma2(dbz2[n], cv[j], AL1[j]);
                }
            }
        }
        // the upstream against the z sums (pair accumulators, then the two halves added)
        f32x2 s0 = 0ull, s1 = 0ull, x0p = 0ull, x1p = 0ull, y0p = 0ull, y1p = 0ull, z1p = 0ull, z2p = 0ull;
        f32x2 w0p = 0ull, w1p = 0ull, w2p = 0ull, w3p = 0ull;
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            s0 = ffma2(WV[j], A0[j], s0);
            s1 = ffma2(WV[j], A1[j], s1);
            if (LAPTAB) {
                s0 = ffma2(WL[j], AL0[j], s0);
                s1 = ffma2(WL[j], AL1[j], s1);
            } else {
                w0p = ffma2(WL[j], A0[j], w0p);
                w1p = ffma2(WL[j], A1[j], w1p);
                w2p = ffma2(WL[j], A2[j], w2p);
                w3p = ffma2(WL[j], A3[j], w3p);
            }
            x0p = ffma2(GX[j], A0[j], x0p);
            x1p = ffma2(GX[j], A1[j], x1p);
            y0p = ffma2(GY[j], A0[j], y0p);
            y1p = ffma2(GY[j], A1[j], y1p);
            z1p = ffma2(GZ[j], A1[j], z1p);
            z2p = ffma2(GZ[j], A2[j], z2p);
        }
        const float S0 = hsum(s0), S1 = hsum(s1), X0 = hsum(x0p), X1 = hsum(x1p);
        const float Y0 = hsum(y0p), Y1 = hsum(y1p), Z1 = hsum(z1p), Z2 = hsum(z2p);
        const float bxl = bx[l], dbxl = dbx[l], d2bxl = d2bx[l];
        const float bym = by[m], dbym = dby[m], d2bym = d2by[m];
        ux += dbxl * bym * (S0 + Z1) + d2bxl * bym * X0 + dbxl * dbym * Y0;
        uy += bxl * dbym * (S0 + Z1) + dbxl * dbym * X0 + bxl * d2bym * Y0;
        uz += bxl * bym * (S1 + Z2) + dbxl * bym * X1 + bxl * dbym * Y1;
        if (!LAPTAB) {
            // d_i of the Hessian Laplacian: metric-weighted third derivatives
            const float W0 = hsum(w0p), W1 = hsum(w1p), W2 = hsum(w2p), W3 = hsum(w3p);
            const float d3bxl = d3w[l], d3bym = d3w[m];
            const float xx0 = ml0 * d3bxl * bym + ml1 * dbxl * d2bym + ml3 * d2bxl * dbym;
            const float xx1 = ml4 * d2bxl * bym + ml5 * dbxl * dbym;
            const float xx2 = ml2 * dbxl * bym;
            const float yy0 = ml0 * d2bxl * dbym + ml1 * bxl * d3bym + ml3 * dbxl * d2bym;
            const float yy1 = ml4 * dbxl * dbym + ml5 * bxl * d2bym;
            const float yy2 = ml2 * bxl * dbym;
            const float zz1 = ml0 * d2bxl * bym + ml1 * bxl * d2bym + ml3 * dbxl * dbym;
            const float zz2 = ml4 * dbxl * bym + ml5 * bxl * dbym;
            const float zz3 = ml2 * bxl * bym;
            ux += xx0 * W0 + xx1 * W1 + xx2 * W2;
            uy += yy0 * W0 + yy1 * W1 + yy2 * W2;
            uz += zz1 * W1 + zz2 * W2 + zz3 * W3;
        }
    }
    // sum over the lanes of the group (all lanes of the warp take part), FP32 pairwise
    for (int off = L >> 1; off > 0; off >>= 1) {
        ux += __shfl_xor_sync(kFullMask, ux, off);
        uy += __shfl_xor_sync(kFullMask, uy, off);
        uz += __shfl_xor_sync(kFullMask, uz, off);
    }
    if (active && sub == 0) {
        const double u[3] = {(double)ux, (double)uy, (double)uz};
#pragma unroll
        for (int a = 0; a < 3; ++a)
            atomicAdd(b.dpos + 3 * ip + a, p.mg[3 * a] * u[0] + p.mg[3 * a + 1] * u[1] + p.mg[3 * a + 2] * u[2]);
    }
}

// threads per block: 512 for float tables (128 registers); bfloat16 tables carry eight orbitals per
// lane (twice the upstream and z-sum pairs) and run 384 (168 registers; at 512 they spill)
template <typename T> struct DposShape {
    static constexpr int threads = sizeof(T) == 2 ? 384 : 512;
};

template <typename T, bool LAPTAB>
__global__ void __launch_bounds__(DposShape<T>::threads, 1) bspline_dpos_kernel(const BwdArgs b)
{
    constexpr int WPB = DposShape<T>::threads / 32;
    const EvalArgs& p = b.e;
    const int lane = threadIdx.x & 31;
    const int gpw = 32 >> p.lanes_log2;
    const long long total = p.n_pos * p.tiles;
    const long long warp = (long long)blockIdx.x * WPB + (threadIdx.x >> 5);
    const long long wstride = (long long)gridDim.x * WPB;
    for (long long w0 = warp * gpw; w0 < total; w0 += wstride * gpw) dpos_task_x2<T, LAPTAB>(b, w0, lane);
}

// ---- coefficient adjoint gathered per bin of cells (many positions, cell order) ----
// With positions sorted into bins of 4 x 4 x 4 grid cells, the positions of one bin touch only the
// 7 x 7 x 7 stencil points around the bin, each one by many of them.  One thread block takes one
// (bin, orbital slice): it stages a batch of the bin's positions in shared memory (local cell,
// 1-D weights, the upstream weights of the slice with the chain rule transposed), then each warp
// takes one (x, y) column of the block at a time and keeps the column's 7 z points in registers,
// lane c owning the c-th 16-byte chunk of the slice.  A position whose 4 x 4 (x, y) footprint holds
// the column (a ballot) adds to 4 consecutive z points of it; the product of its tensor weights
// factors as bz_n V + bz'_n W (+ bz''_n X for the Laplacian from the Hessian), with V, W, X sums of
// upstream weights scaled by the column's x and y weights, so the upstream chunks and the x/y
// products are read and formed once per column instead of once per point.  Each touched point
// row then goes to the coefficient gradient with one vector atomic per chunk: no shared-memory
// atomics, one global reduction per point row and batch.  The table is not read; the position
// adjoint is left to a second launch over the same cell order.
constexpr int kGatherThreads = 512;
constexpr int kGatherBatch = 64;                      // positions staged at a time
constexpr int kGatherSide = 7;                        // stencil points per axis of a 4-cell bin edge
constexpr int kGatherColumns = kGatherSide * kGatherSide;

// The (x, y) columns of the block in decreasing order of the cell columns of a bin that touch
// them, (4 - |lx - 3|) (4 - |ly - 3|) of 16, so that warps taking columns in turn finish together.
struct GatherColumnOrder {
    unsigned char c[kGatherColumns];
};
constexpr int gather_column_weight(int col)
{
    const int dx = col / kGatherSide - 3, dy = col % kGatherSide - 3;
    return (4 - (dx < 0 ? -dx : dx)) * (4 - (dy < 0 ? -dy : dy));
}
constexpr GatherColumnOrder make_gather_column_order()
{
    GatherColumnOrder r{};
    int n = 0;
    for (int w = 16; w >= 1; --w)
        for (int col = 0; col < kGatherColumns; ++col)
            if (gather_column_weight(col) == w) r.c[n++] = (unsigned char)col;
    return r;
}
__constant__ GatherColumnOrder kGatherColumnOrder = make_gather_column_order();

// four consecutive A values from 16-byte aligned shared memory
template <typename A>
__device__ __forceinline__ void lds4(const A* q, A (&v)[4])
{
    if constexpr (sizeof(A) == 4) {
        const float4 r = *reinterpret_cast<const float4*>(q);
        v[0] = r.x, v[1] = r.y, v[2] = r.z, v[3] = r.w;
    } else {
        const double2 r0 = reinterpret_cast<const double2*>(q)[0], r1 = reinterpret_cast<const double2*>(q)[1];
        v[0] = r0.x, v[1] = r0.y, v[2] = r1.x, v[3] = r1.y;
    }
}

// one position's share of a column: z points CZ .. CZ + 3 of the 7 (wz: bz[4], bz'[4], bz''[4])
template <typename A, int EA, bool LAPTAB, int CZ>
__device__ __forceinline__ void gather_column_add(A (&acc)[kGatherSide][EA], A (&accl)[kGatherSide][EA], const A* wz,
                                                  const A (&V)[EA], const A (&W)[EA], const A (&X)[EA], const A (&L)[EA])
{
    A bz[4], dbz[4], d2bz[4];
    lds4<A>(wz, bz);
    lds4<A>(wz + 4, dbz);
    if (!LAPTAB) lds4<A>(wz + 8, d2bz);
#pragma unroll
    for (int n = 0; n < 4; ++n) {
#pragma unroll
        for (int e = 0; e < EA; ++e) {
            A t = acc[CZ + n][e] + bz[n] * V[e];
            t = t + dbz[n] * W[e];
            if (!LAPTAB) t = t + d2bz[n] * X[e];
            acc[CZ + n][e] = t;
            if (LAPTAB) accl[CZ + n][e] = accl[CZ + n][e] + bz[n] * L[e];
        }
    }
}

struct GatherArgs {
    const int* bin_end;       // one past the last sorted position of every bin
    int nb[3];                // bins per axis (4 cells per edge)
    int n_bins, n_slices;
};

// staged data of one batch (dynamic shared memory)
template <typename A>
struct GatherStage {
    static constexpr int EA = 16 / sizeof(A);        // upstream values per 16-byte chunk
    A w[kGatherBatch][3][12];                        // per axis b[4], b'[4], b''[4]
    int cell[kGatherBatch];                          // local cell cx | cy << 8 | cz << 16, -1: none
    uint4 up[kGatherBatch][5][32];                   // wv, g~x, g~y, g~z, wl chunks of the slice
    int next;                                        // next column of the batch to take
};

template <typename A, bool LAPTAB>
__global__ void __launch_bounds__(kGatherThreads, 1) bspline_bwd_gather_kernel(const BwdArgs b, const GatherArgs g)
{
    constexpr int EA = GatherStage<A>::EA;
    constexpr int WARPS = kGatherThreads / 32;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    GatherStage<A>& S = *reinterpret_cast<GatherStage<A>*>(smem_raw);
    const EvalArgs& p = b.e;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n_orb = p.n_orb;
    const bool vec = b.vec_atomic != 0;
    A* dc = static_cast<A*>(b.dcoef);
    A* dl = static_cast<A*>(b.dcoef_lap);
    const A* gvp = static_cast<const A*>(b.gv);
    const A* ggp = static_cast<const A*>(b.gg);
    const A* glp = static_cast<const A*>(b.gl);
    const A ml0 = (A)p.ml[0], ml1 = (A)p.ml[1], ml2 = (A)p.ml[2];
    const A ml3 = (A)p.ml[3], ml4 = (A)p.ml[4], ml5 = (A)p.ml[5];
    const int items = g.n_bins * g.n_slices;
    for (int item = blockIdx.x; item < items; item += gridDim.x) {
        const int bin = item / g.n_slices, slice = item - bin * g.n_slices;
        const int start = bin ? g.bin_end[bin - 1] : 0, end = g.bin_end[bin];
        const int bz = bin % g.nb[2], by = (bin / g.nb[2]) % g.nb[1], bx = bin / (g.nb[2] * g.nb[1]);
        const int o0 = (slice * 32 + lane) * EA;     // this lane's first orbital of the slice
        for (int b0 = start; b0 < end; b0 += kGatherBatch) {
            const int nbat = min(kGatherBatch, end - b0);
            __syncthreads();                          // the previous batch is no longer read
            if (threadIdx.x == 0) S.next = 0;
            // ---- stage: warp w takes positions w, w + WARPS, ... of the batch ----
            for (int j = warp; j < nbat; j += WARPS) {
                const long long ip = order_index(p, b0 + j);
                int ix, iy, iz;
                A t[3];
                bool ok;
                bwd_coords<A>(p, ip, 32, lane, 0, ix, iy, iz, t[0], t[1], t[2], ok);
                if (lane < 3) {
                    A wv[4], dw[4], d2w[4];
                    bspline_weights<A>(t[lane], wv, dw, d2w);
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        S.w[j][lane][k] = wv[k];
                        S.w[j][lane][4 + k] = dw[k];
                        S.w[j][lane][8 + k] = d2w[k];
                    }
                }
                if (lane == 0)
                    S.cell[j] = ok ? ((ix - 4 * bx) | ((iy - 4 * by) << 8) | ((iz - 4 * bz) << 16)) : -1;
                A wv[EA], wl[EA], wg[3][EA], gt[3][EA];
                const bool use = ok && o0 < n_orb;
                load_run<A>(use && gvp ? gvp + ip * n_orb + o0 : nullptr, wv, o0, n_orb, EA);
                load_run<A>(use && glp ? glp + ip * n_orb + o0 : nullptr, wl, o0, n_orb, EA);
#pragma unroll
                for (int a = 0; a < 3; ++a)
                    load_run<A>(use && ggp ? ggp + (ip * 3 + a) * n_orb + o0 : nullptr, wg[a], o0, n_orb, EA);
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int e = 0; e < EA; ++e)
                        gt[i][e] = (A)p.mg[i] * wg[0][e] + (A)p.mg[3 + i] * wg[1][e] + (A)p.mg[6 + i] * wg[2][e];
                auto put = [&](int q, const A* v) {
                    A* d = reinterpret_cast<A*>(&S.up[j][q][lane]);
#pragma unroll
                    for (int e = 0; e < EA; ++e) d[e] = v[e];
                };
                put(0, wv);
                put(1, gt[0]);
                put(2, gt[1]);
                put(3, gt[2]);
                put(4, wl);
            }
            __syncthreads();
            // ---- gather: each warp takes (x, y) columns of the 7 x 7 x 7 block, heaviest first ----
            for (;;) {
                int k = 0;
                if (lane == 0) k = atomicAdd(&S.next, 1);
                k = __shfl_sync(kFullMask, k, 0);
                if (k >= kGatherSide * kGatherSide) break;
                const int col = kGatherColumnOrder.c[k];
                const int lx = col / kGatherSide, ly = col - lx * kGatherSide;
                A acc[kGatherSide][EA], accl[kGatherSide][EA];
#pragma unroll
                for (int z = 0; z < kGatherSide; ++z)
#pragma unroll
                    for (int e = 0; e < EA; ++e) acc[z][e] = accl[z][e] = A(0);
                unsigned zmask = 0u;                  // z points of the column some position touches
                for (int jb = 0; jb < nbat; jb += 32) {
                    const int jj = jb + lane;
                    bool member = false;
                    if (jj < nbat) {
                        const int c = S.cell[jj];
                        member = c >= 0 && (unsigned)(lx - (c & 255)) < 4u && (unsigned)(ly - ((c >> 8) & 255)) < 4u &&
                                 (c >> 16) < 4;
                    }
                    unsigned mask = __ballot_sync(kFullMask, member);
                    while (mask) {
                        const int j = jb + __ffs(mask) - 1;
                        mask &= mask - 1;
                        const int c = S.cell[j];
                        const int l = lx - (c & 255), m = ly - ((c >> 8) & 255), cz = c >> 16;
                        zmask |= 15u << cz;
                        const A bxl = S.w[j][0][l], dbxl = S.w[j][0][4 + l];
                        const A bym = S.w[j][1][m], dbym = S.w[j][1][4 + m];
                        const A bxby = bxl * bym, dxby = dbxl * bym, bxdy = bxl * dbym;
                        // the column's share of the position's rows: bz_n V + bz'_n W (+ bz''_n X),
                        // Laplacian table bz_n L
                        A V[EA], W[EA], X[EA], L[EA];
                        const A* u0 = reinterpret_cast<const A*>(&S.up[j][0][lane]);
                        const A* u1 = reinterpret_cast<const A*>(&S.up[j][1][lane]);
                        const A* u2 = reinterpret_cast<const A*>(&S.up[j][2][lane]);
                        const A* u3 = reinterpret_cast<const A*>(&S.up[j][3][lane]);
                        const A* u4 = reinterpret_cast<const A*>(&S.up[j][4][lane]);
                        if (LAPTAB) {
#pragma unroll
                            for (int e = 0; e < EA; ++e) {
                                V[e] = u0[e] * bxby + u1[e] * dxby + u2[e] * bxdy;
                                W[e] = u3[e] * bxby;
                                L[e] = u4[e] * bxby;
                                X[e] = A(0);
                            }
                        } else {
                            const A d2bxl = S.w[j][0][8 + l], d2bym = S.w[j][1][8 + m];
                            const A al = ml0 * d2bxl * bym + ml1 * bxl * d2bym + ml3 * dbxl * dbym;
                            const A be = ml2 * bxby;
                            const A ga = ml4 * dxby + ml5 * bxdy;
#pragma unroll
                            for (int e = 0; e < EA; ++e) {
                                V[e] = u0[e] * bxby + u1[e] * dxby + u2[e] * bxdy + u4[e] * al;
                                W[e] = u3[e] * bxby + u4[e] * ga;
                                X[e] = u4[e] * be;
                                L[e] = A(0);
                            }
                        }
                        const A* wz = &S.w[j][2][0];
                        switch (cz) {
                        case 0: gather_column_add<A, EA, LAPTAB, 0>(acc, accl, wz, V, W, X, L); break;
                        case 1: gather_column_add<A, EA, LAPTAB, 1>(acc, accl, wz, V, W, X, L); break;
                        case 2: gather_column_add<A, EA, LAPTAB, 2>(acc, accl, wz, V, W, X, L); break;
                        default: gather_column_add<A, EA, LAPTAB, 3>(acc, accl, wz, V, W, X, L); break;
                        }
                    }
                }
                if (o0 >= n_orb) continue;
                const size_t col_row = ((size_t)wrap1(4 * bx - 1 + lx, p.nx) * p.ny + wrap1(4 * by - 1 + ly, p.ny)) * p.nz;
#pragma unroll
                for (int z = 0; z < kGatherSide; ++z) {
                    if (!(zmask & (1u << z))) continue;
                    const size_t row = (col_row + wrap1(4 * bz - 1 + z, p.nz)) * n_orb + o0;
                    atomic_run<A, EA>(dc + row, acc[z], o0, n_orb, vec);
                    if (LAPTAB) atomic_run<A, EA>(dl + row, accl[z], o0, n_orb, vec);
                }
            }
        }
    }
}

template <typename T, bool LAPTAB, bool BLOCH, bool COEF>
int launch_one_kind(const BwdArgs& a, cudaStream_t st)
{
    const int gpw = 32 >> a.e.lanes_log2;
    const long long groups = a.e.n_pos * a.e.tiles;
    const long long warps = (groups + gpw - 1) / gpw;
    long long blocks = (warps + kEvalThreads / 32 - 1) / (kEvalThreads / 32);
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bspline_bwd_kernel<T, LAPTAB, BLOCH, COEF>,
                                                                  kEvalThreads, 0);
    if (e != cudaSuccess) return cuda_error(e, "occupancy query");
    if (per_sm < 1) per_sm = 1;
    const long long cap = (long long)sm_count() * per_sm;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    bspline_bwd_kernel<T, LAPTAB, BLOCH, COEF><<<(unsigned)blocks, kEvalThreads, 0, st>>>(a);
    return cuda_error(cudaGetLastError(), "bspline_bwd_kernel launch");
}

// the coefficient adjoint and the position adjoint in one pass, or (no dcoef) the position alone
template <typename T, bool LAPTAB, bool BLOCH>
int launch_one(const BwdArgs& a, cudaStream_t st)
{
    return a.dcoef ? launch_one_kind<T, LAPTAB, BLOCH, true>(a, st) : launch_one_kind<T, LAPTAB, BLOCH, false>(a, st);
}

template <typename T, bool LAPTAB>
int launch_dpos(const BwdArgs& a, cudaStream_t st)
{
    const int gpw = 32 >> a.e.lanes_log2;
    const long long warps = (a.e.n_pos * a.e.tiles + gpw - 1) / gpw;
    constexpr int threads = DposShape<T>::threads;
    long long blocks = (warps + threads / 32 - 1) / (threads / 32);
    if (blocks > sm_count()) blocks = sm_count();
    if (blocks < 1) blocks = 1;
    bspline_dpos_kernel<T, LAPTAB><<<(unsigned)blocks, threads, 0, st>>>(a);
    return cuda_error(cudaGetLastError(), "bspline_dpos_kernel launch");
}

template <typename A, bool LAPTAB>
int launch_gather(const BwdArgs& a, const GatherArgs& g, cudaStream_t st)
{
    constexpr size_t smem = sizeof(GatherStage<A>);
    cudaError_t e = cudaFuncSetAttribute(bspline_bwd_gather_kernel<A, LAPTAB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_error(e, "gathered adjoint shared memory");
    const int items = g.n_bins * g.n_slices;
    const int blocks = items < sm_count() ? items : sm_count();
    bspline_bwd_gather_kernel<A, LAPTAB><<<blocks > 0 ? blocks : 1, kGatherThreads, smem, st>>>(a, g);
    return cuda_error(cudaGetLastError(), "bspline_bwd_gather_kernel launch");
}

template <typename T, bool LAPTAB>
int launch_typed(const BwdArgs& a, cudaStream_t st)
{
    return a.bloch ? launch_one<T, LAPTAB, true>(a, st) : launch_one<T, LAPTAB, false>(a, st);
}

// ---- five tables (Lagrange; B-splines with separate gradient tables) ----
// The outputs are the values of five interpolants with one set of weights W = w_l w_m w_n
// (tables phi, d_x phi, d_y phi, d_z phi, lap phi, Sec. III C), so the adjoint of table t is
// dbeta_t += g_t W with g_t its output's upstream (value, the Cartesian gradient components,
// Laplacian), and dL/dr = N (a^-1)^T sum_t g_t grad_t(value of table t).  Bloch handles take
// the upstream through the phase first (h_t = conj(e) g_t; the tables hold the periodic parts
// of phi and of its derivatives) and add -k sum_t Im(conj(h_t) w_t) to dL/dr.
enum BwdFiveBasis : int { kBwdLagrange = 0, kBwdBSpline = 1 };

template <int BASIS, typename A>
__device__ __forceinline__ void five_weights(A t, A* w, A* dw)
{
    if constexpr (BASIS == kBwdLagrange) {   // Eq. (lagrangebasis) and its derivative
        const A tm1 = t - A(1), tm2 = t - A(2), tp1 = t + A(1);
        w[0] = A(-1.0 / 6.0) * t * tm1 * tm2;
        w[1] = A(0.5) * tp1 * tm1 * tm2;
        w[2] = A(-0.5) * tp1 * t * tm2;
        w[3] = A(1.0 / 6.0) * tp1 * t * tm1;
        const A t2 = t * t;
        dw[0] = A(-1.0 / 6.0) * (A(3) * t2 - A(6) * t + A(2));
        dw[1] = A(0.5) * (A(3) * t2 - A(4) * t - A(1));
        dw[2] = A(-0.5) * (A(3) * t2 - A(2) * t - A(2));
        dw[3] = A(1.0 / 6.0) * (A(3) * t2 - A(1));
    } else {
        bspline_weights<A>(t, w, dw, nullptr);
    }
}

template <typename T, int BASIS, bool BLOCH>
__global__ void __launch_bounds__(kEvalThreads) five_table_bwd_kernel(const BwdArgs b)
{
    using A = typename Traits<T>::A;
    constexpr int E = Traits<T>::E;
    const EvalArgs& p = b.e;
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
    const int n_orb = p.n_orb;
    const size_t canon = (size_t)p.nx * p.ny * p.nz * n_orb;   // one canonical table

    for (long long w0 = warp * gpw; w0 < total; w0 += wstride * gpw) {
        const long long gid = w0 + (lane >> p.lanes_log2);
        const bool active = gid < total;
        const long long ip = active ? gid / p.tiles : 0;
        const int tile = active ? (int)(gid - ip * p.tiles) : 0;
        const double r[3] = {p.pos[3 * ip], p.pos[3 * ip + 1], p.pos[3 * ip + 2]};
        int ix, iy, iz;
        double tx, ty, tz;
        bool ok;
        reduced_coordinates(p, r, L, sub, gbase, ix, iy, iz, tx, ty, tz, ok);
        if (active && !ok && sub == 0 && tile == 0) atomicOr(p.err, 1);
        A w[3][4], dw[3][4];
        five_weights<BASIS, A>((A)tx, w[0], dw[0]);
        five_weights<BASIS, A>((A)ty, w[1], dw[1]);
        five_weights<BASIS, A>((A)tz, w[2], dw[2]);
        const int chunk = tile * L + sub;
        const int o0 = chunk * E;
        const bool use = active && o0 < n_orb;
        // upstream of the five tables: value, Cartesian gradient components, Laplacian
        A up[5][E];
        {
            const A* gvp = static_cast<const A*>(b.gv);
            const A* ggp = static_cast<const A*>(b.gg);
            const A* glp = static_cast<const A*>(b.gl);
            load_run<A>(use && gvp ? gvp + ip * n_orb + o0 : nullptr, up[0], o0, n_orb, E);
            for (int a = 0; a < 3; ++a)
                load_run<A>(use && ggp ? ggp + (ip * 3 + a) * n_orb + o0 : nullptr, up[1 + a], o0, n_orb, E);
            load_run<A>(use && glp ? glp + ip * n_orb + o0 : nullptr, up[4], o0, n_orb, E);
        }
        if constexpr (BLOCH) {
            const double uk = __fma_rn(p.kred[0], r[0], __fma_rn(p.kred[1], r[1], __dmul_rn(p.kred[2], r[2])));
            double sn, cs;
            sincospi(2.0 * (uk - rint(uk)), &sn, &cs);
            const A c = (A)cs, sp = (A)sn;
#pragma unroll
            for (int t = 0; t < 5; ++t)
#pragma unroll
                for (int j = 0; j < E / 2; ++j) {
                    const A x = up[t][2 * j], y = up[t][2 * j + 1];
                    up[t][2 * j] = c * x + sp * y;
                    up[t][2 * j + 1] = c * y - sp * x;
                }
        }
        int xs[4], ys[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            xs[j] = wrap1(ix + j - 1, p.nx);
            ys[j] = wrap1(iy + j - 1, p.ny);
        }

        // ---- coefficient adjoint: scatter into 64 stencil rows of each table ----
        if (b.dcoef && use) {
            A* dc = static_cast<A*>(b.dcoef);
            const bool vec = b.vec_atomic != 0;
            for (int l = 0; l < 4; ++l)
                for (int m = 0; m < 4; ++m)
                    for (int n = 0; n < 4; ++n) {
                        const int z = wrap1(iz + n - 1, p.nz);
                        const A B = w[0][l] * w[1][m] * w[2][n];
                        const size_t row = (((size_t)xs[l] * p.ny + ys[m]) * p.nz + z) * n_orb + o0;
#pragma unroll
                        for (int t = 0; t < 5; ++t) {
                            A v[E];
#pragma unroll
                            for (int e = 0; e < E; ++e) v[e] = up[t][e] * B;
                            atomic_run<A, E>(dc + t * canon + row, v, o0, n_orb, vec);
                        }
                    }
        }

        // ---- position adjoint ----
        if (b.dpos) {
            double u[3] = {0.0, 0.0, 0.0};
            double sph = 0.0;
            const size_t off = (size_t)chunk * 16 + (size_t)iz * rowb;
            for (int l = 0; l < 4; ++l)
                for (int m = 0; m < 4; ++m) {
                    const size_t col = (size_t)(xs[l] * p.ny + ys[m]) * colb + off;
                    const A wdx = dw[0][l] * w[1][m], wdy = w[0][l] * dw[1][m], wxy = w[0][l] * w[1][m];
                    // sa = sum over tables and orbitals of upstream x (z-contracted value), sd the
                    // same with the z-derivative weights; sv the Bloch phase sum
                    A sa = 0, sd = 0, sv = 0;
#pragma unroll
                    for (int t = 0; t < 5; ++t) {
                        const char* base = static_cast<const char*>(p.tab[t]) + col;
                        A a[E], ad[E];
#pragma unroll
                        for (int e = 0; e < E; ++e) a[e] = ad[e] = A(0);
#pragma unroll
                        for (int n = 0; n < 4; ++n) {
                            A cvals[E];
                            unpack<T>(ldg_table(p, base + n * rowb), cvals);
#pragma unroll
                            for (int e = 0; e < E; ++e) {
                                a[e] = fma(w[2][n], cvals[e], a[e]);
                                ad[e] = fma(dw[2][n], cvals[e], ad[e]);
                            }
                        }
#pragma unroll
                        for (int e = 0; e < E; ++e) {
                            sa += up[t][e] * a[e];
                            sd += up[t][e] * ad[e];
                        }
                        if constexpr (BLOCH) {
#pragma unroll
                            for (int j = 0; j < E / 2; ++j)   // Im(conj(h) a)
                                sv += up[t][2 * j] * a[2 * j + 1] - up[t][2 * j + 1] * a[2 * j];
                        }
                    }
                    u[0] += (double)(wdx * sa);
                    u[1] += (double)(wdy * sa);
                    u[2] += (double)(wxy * sd);
                    if constexpr (BLOCH) sph += (double)(wxy * sv);
                }
            for (int o = L >> 1; o > 0; o >>= 1) {
#pragma unroll
                for (int i = 0; i < 3; ++i) u[i] += __shfl_xor_sync(kFullMask, u[i], o);
                sph += __shfl_xor_sync(kFullMask, sph, o);
            }
            if (active && sub == 0) {
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const double d = p.mg[3 * a] * u[0] + p.mg[3 * a + 1] * u[1] + p.mg[3 * a + 2] * u[2] -
                                     (BLOCH ? p.kc[a] * sph : 0.0);
                    atomicAdd(b.dpos + 3 * ip + a, d);
                }
            }
        }
    }
}

template <typename T, int BASIS, bool BLOCH>
int launch_five(const BwdArgs& a, cudaStream_t st)
{
    const int gpw = 32 >> a.e.lanes_log2;
    const long long warps = (a.e.n_pos * a.e.tiles + gpw - 1) / gpw;
    long long blocks = (warps + kEvalThreads / 32 - 1) / (kEvalThreads / 32);
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, five_table_bwd_kernel<T, BASIS, BLOCH>,
                                                                  kEvalThreads, 0);
    if (e != cudaSuccess) return cuda_error(e, "occupancy query");
    if (per_sm < 1) per_sm = 1;
    const long long cap = (long long)sm_count() * per_sm;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    five_table_bwd_kernel<T, BASIS, BLOCH><<<(unsigned)blocks, kEvalThreads, 0, st>>>(a);
    return cuda_error(cudaGetLastError(), "five_table_bwd_kernel launch");
}

template <typename T>
int launch_five_typed(const BwdArgs& a, bool lagrange, cudaStream_t st)
{
    if (lagrange)
        return a.bloch ? launch_five<T, kBwdLagrange, true>(a, st) : launch_five<T, kBwdLagrange, false>(a, st);
    return a.bloch ? launch_five<T, kBwdBSpline, true>(a, st) : launch_five<T, kBwdBSpline, false>(a, st);
}

// ---- pp-splines (Eq. pp-splineinterpolation3): eight coefficients sigma^{kappa mu nu} per grid
// point, a 2 x 2 x 2 corner stencil, weights s_i^kappa(t) (Eq. pp-splinebasis).  The outputs
// are derivatives of one spline with the chain rule, as for the B-splines with the Hessian
// Laplacian, so the adjoint has the same form with the pp weights and their derivatives up to
// the third (s^1 is linear, s^2 cubic: d3 s^2_0 = -1, d3 s^2_1 = 1); dcoef holds the eight
// tables [8][Nx][Ny][Nz][O], entry 4 kappa + 2 mu + nu.
template <typename A>
__device__ __forceinline__ void pp_bwd_weights(A t, A w[2][2], A dw[2][2], A d2w[2][2], A d3w[2][2])
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
    d3w[0][0] = A(0);
    d3w[0][1] = A(0);
    d3w[1][0] = A(-1);
    d3w[1][1] = A(1);
}

template <typename T, bool BLOCH>
__global__ void __launch_bounds__(kEvalThreads) pp_bwd_kernel(const BwdArgs b)
{
    using A = typename Traits<T>::A;
    constexpr int E = Traits<T>::E;
    const EvalArgs& p = b.e;
    const int lane = threadIdx.x & 31;
    const int L = 1 << p.lanes_log2;
    const int sub = lane & (L - 1);
    const int gbase = lane & ~(L - 1);
    const int gpw = 32 >> p.lanes_log2;
    const long long total = p.n_pos * p.tiles;
    const long long warp = (long long)blockIdx.x * (kEvalThreads / 32) + (threadIdx.x >> 5);
    const long long wstride = (long long)gridDim.x * (kEvalThreads / 32);
    const size_t rowb = (size_t)p.row_stride * sizeof(T);   // one z row: 8 entries x O_p
    const size_t entb = rowb / 8;
    const size_t colb = (size_t)p.col_stride * sizeof(T);
    const int n_orb = p.n_orb;
    const size_t canon = (size_t)p.nx * p.ny * p.nz * n_orb;
    const A ml0 = (A)p.ml[0], ml1 = (A)p.ml[1], ml2 = (A)p.ml[2];
    const A ml3 = (A)p.ml[3], ml4 = (A)p.ml[4], ml5 = (A)p.ml[5];

    for (long long w0 = warp * gpw; w0 < total; w0 += wstride * gpw) {
        const long long gid = w0 + (lane >> p.lanes_log2);
        const bool active = gid < total;
        const long long ip = active ? gid / p.tiles : 0;
        const int tile = active ? (int)(gid - ip * p.tiles) : 0;
        const double r[3] = {p.pos[3 * ip], p.pos[3 * ip + 1], p.pos[3 * ip + 2]};
        int ix, iy, iz;
        double tx, ty, tz;
        bool ok;
        reduced_coordinates(p, r, L, sub, gbase, ix, iy, iz, tx, ty, tz, ok);
        if (active && !ok && sub == 0 && tile == 0) atomicOr(p.err, 1);
        A w[3][2][2], dw[3][2][2], d2w[3][2][2], d3w[3][2][2];
        pp_bwd_weights<A>((A)tx, w[0], dw[0], d2w[0], d3w[0]);
        pp_bwd_weights<A>((A)ty, w[1], dw[1], d2w[1], d3w[1]);
        pp_bwd_weights<A>((A)tz, w[2], dw[2], d2w[2], d3w[2]);
        const int chunk = tile * L + sub;
        const int o0 = chunk * E;
        const bool use = active && o0 < n_orb;
        A wv[E], wl[E], gt[3][E];
        A hv[E], hl[E], hg[3][E];
        {
            A wg[3][E];
            const A* gvp = static_cast<const A*>(b.gv);
            const A* ggp = static_cast<const A*>(b.gg);
            const A* glp = static_cast<const A*>(b.gl);
            load_run<A>(use && gvp ? gvp + ip * n_orb + o0 : nullptr, wv, o0, n_orb, E);
            load_run<A>(use && glp ? glp + ip * n_orb + o0 : nullptr, wl, o0, n_orb, E);
            for (int a = 0; a < 3; ++a)
                load_run<A>(use && ggp ? ggp + (ip * 3 + a) * n_orb + o0 : nullptr, wg[a], o0, n_orb, E);
            if constexpr (BLOCH) bloch_upstream<A, E, false>(p, r, wv, wg, wl, hv, hg, hl);
#pragma unroll
            for (int i = 0; i < 3; ++i)
#pragma unroll
                for (int e = 0; e < E; ++e)
                    gt[i][e] = (A)p.mg[i] * wg[0][e] + (A)p.mg[3 + i] * wg[1][e] + (A)p.mg[6 + i] * wg[2][e];
        }
        int xs[2], ys[2], zs[2];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            xs[j] = ix + j < p.nx ? ix + j : 0;
            ys[j] = iy + j < p.ny ? iy + j : 0;
            zs[j] = iz + j < p.nz ? iz + j : 0;
        }

        // ---- coefficient adjoint: 8 corners x 8 entries ----
        if (b.dcoef && use) {
            A* dc = static_cast<A*>(b.dcoef);
            const bool vec = b.vec_atomic != 0;
            for (int i = 0; i < 2; ++i)
                for (int j = 0; j < 2; ++j)
                    for (int k = 0; k < 2; ++k) {
                        const size_t row = (((size_t)xs[i] * p.ny + ys[j]) * p.nz + zs[k]) * n_orb + o0;
                        for (int ent = 0; ent < 8; ++ent) {
                            const int kap = ent >> 2, mu = (ent >> 1) & 1, nu = ent & 1;
                            const A x0 = w[0][kap][i], x1 = dw[0][kap][i], x2 = d2w[0][kap][i];
                            const A y0 = w[1][mu][j], y1 = dw[1][mu][j], y2 = d2w[1][mu][j];
                            const A z0 = w[2][nu][k], z1 = dw[2][nu][k], z2 = d2w[2][nu][k];
                            const A B = x0 * y0 * z0, Bx = x1 * y0 * z0, By = x0 * y1 * z0, Bz = x0 * y0 * z1;
                            const A lapB = ml0 * x2 * y0 * z0 + ml1 * x0 * y2 * z0 + ml2 * x0 * y0 * z2 +
                                           ml3 * x1 * y1 * z0 + ml4 * x1 * y0 * z1 + ml5 * x0 * y1 * z1;
                            A v[E];
#pragma unroll
                            for (int e = 0; e < E; ++e)
                                v[e] = wv[e] * B + gt[0][e] * Bx + gt[1][e] * By + gt[2][e] * Bz + wl[e] * lapB;
                            atomic_run<A, E>(dc + ent * canon + row, v, o0, n_orb, vec);
                        }
                    }
        }

        // ---- position adjoint: gradient, Hessian and gradient of the Laplacian of the spline ----
        if (b.dpos) {
            A g1[3][E], h2[6][E], d3[3][E], u0[E];
#pragma unroll
            for (int e = 0; e < E; ++e) {
                for (int i = 0; i < 3; ++i) g1[i][e] = d3[i][e] = A(0);
                for (int i = 0; i < 6; ++i) h2[i][e] = A(0);
                u0[e] = A(0);
            }
            const size_t off = (size_t)chunk * 16 + (size_t)iz * rowb;
            for (int i = 0; i < 2; ++i)
                for (int j = 0; j < 2; ++j) {
                    const char* col = static_cast<const char*>(p.tab[0]) + (size_t)(xs[i] * p.ny + ys[j]) * colb + off;
                    for (int km = 0; km < 4; ++km) {
                        const int kap = km >> 1, mu = km & 1;
                        A a[4][E];
#pragma unroll
                        for (int e = 0; e < E; ++e) a[0][e] = a[1][e] = a[2][e] = a[3][e] = A(0);
#pragma unroll
                        for (int k = 0; k < 2; ++k)
#pragma unroll
                            for (int nu = 0; nu < 2; ++nu) {
                                A c[E];
                                unpack<T>(ldg_table(p, col + k * rowb + (size_t)(4 * kap + 2 * mu + nu) * entb), c);
#pragma unroll
                                for (int e = 0; e < E; ++e) {
                                    a[0][e] = fma(w[2][nu][k], c[e], a[0][e]);
                                    a[1][e] = fma(dw[2][nu][k], c[e], a[1][e]);
                                    a[2][e] = fma(d2w[2][nu][k], c[e], a[2][e]);
                                    a[3][e] = fma(d3w[2][nu][k], c[e], a[3][e]);
                                }
                            }
                        const A bx = w[0][kap][i], dbx = dw[0][kap][i], d2bx = d2w[0][kap][i], d3bx = d3w[0][kap][i];
                        const A by = w[1][mu][j], dby = dw[1][mu][j], d2by = d2w[1][mu][j], d3by = d3w[1][mu][j];
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
#pragma unroll
                        for (int e = 0; e < E; ++e) {
                            if constexpr (BLOCH) u0[e] += bx * by * a[0][e];
                            g1[0][e] += dbx * by * a[0][e];
                            g1[1][e] += bx * dby * a[0][e];
                            g1[2][e] += bx * by * a[1][e];
                            h2[0][e] += d2bx * by * a[0][e];
                            h2[1][e] += bx * d2by * a[0][e];
                            h2[2][e] += bx * by * a[2][e];
                            h2[3][e] += dbx * dby * a[0][e];
                            h2[4][e] += dbx * by * a[1][e];
                            h2[5][e] += bx * dby * a[1][e];
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
            if constexpr (BLOCH) sph = bloch_phase_sum<A, E, false>(p, u0, g1, h2, u0, hv, hg, hl);
            for (int o = L >> 1; o > 0; o >>= 1) {
#pragma unroll
                for (int i = 0; i < 3; ++i) u[i] += __shfl_xor_sync(kFullMask, u[i], o);
                sph += __shfl_xor_sync(kFullMask, sph, o);
            }
            if (active && sub == 0) {
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const double d = p.mg[3 * a] * u[0] + p.mg[3 * a + 1] * u[1] + p.mg[3 * a + 2] * u[2] -
                                     (BLOCH ? p.kc[a] * sph : 0.0);
                    atomicAdd(b.dpos + 3 * ip + a, d);
                }
            }
        }
    }
}

template <typename T, bool BLOCH>
int launch_pp_bwd(const BwdArgs& a, cudaStream_t st)
{
    const int gpw = 32 >> a.e.lanes_log2;
    const long long warps = (a.e.n_pos * a.e.tiles + gpw - 1) / gpw;
    long long blocks = (warps + kEvalThreads / 32 - 1) / (kEvalThreads / 32);
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pp_bwd_kernel<T, BLOCH>, kEvalThreads, 0);
    if (e != cudaSuccess) return cuda_error(e, "occupancy query");
    if (per_sm < 1) per_sm = 1;
    const long long cap = (long long)sm_count() * per_sm;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    pp_bwd_kernel<T, BLOCH><<<(unsigned)blocks, kEvalThreads, 0, st>>>(a);
    return cuda_error(cudaGetLastError(), "pp_bwd_kernel launch");
}

template <typename T>
int launch_pp_typed(const BwdArgs& a, cudaStream_t st)
{
    return a.bloch ? launch_pp_bwd<T, true>(a, st) : launch_pp_bwd<T, false>(a, st);
}

}  // namespace

int launch_bspline_backward(Handle* h, const double* pos, long long n_pos, const void* gv,
                            const void* gg, const void* gl, void* dcoef, void* dcoef_lap, double* dpos,
                            cudaStream_t st)
{
    BwdArgs a;
    fill_eval_args(h, &a.e);
    a.e.pos = pos;
    a.e.n_pos = n_pos;
    a.gv = gv;
    a.gg = gg;
    a.gl = gl;
    a.dcoef = dcoef;
    a.dcoef_lap = dcoef_lap;
    a.dpos = dpos;
    a.bloch = h->bloch;
    const size_t ob = (h->storage == QMCSPL_F64 || h->storage == QMCSPL_DF64) ? 8 : 4;
    const uintptr_t al = (uintptr_t)dcoef | (uintptr_t)dcoef_lap;
    a.vec_atomic = ((h->n_orb * ob) % 16 == 0) && (al % 16 == 0);
    if (dpos) {
        cudaError_t e = cudaMemsetAsync(dpos, 0, sizeof(double) * 3 * (size_t)n_pos, st);
        if (e != cudaSuccess) return cuda_error(e, "cudaMemsetAsync(dpos)");
    }
    if (!dcoef && !dpos) return QMCSPL_OK;
    if (is_general(h)) {   // other degrees, graded grids: backward_general.cuh
        switch (h->storage) {
        case QMCSPL_F64: return launch_general_backward_f64(h, a, st);
        case QMCSPL_F32: return launch_general_backward_f32(h, a, st);
        default: return launch_general_backward_bf16(h, a, st);
        }
    }
    if (h->method == QMCSPL_PPSPLINE) {
        switch (h->storage) {
        case QMCSPL_F64: return launch_pp_typed<double>(a, st);
        case QMCSPL_F32: return launch_pp_typed<float>(a, st);
        default: return launch_pp_typed<__nv_bfloat16>(a, st);
        }
    }
    if (h->n_tables == 5) {   // Lagrange, or B-splines with separate gradient tables
        const bool lag = h->method == QMCSPL_LAGRANGE;
        switch (h->storage) {
        case QMCSPL_F64: return launch_five_typed<double>(a, lag, st);
        case QMCSPL_F32: return launch_five_typed<float>(a, lag, st);
        case QMCSPL_DF64: return launch_five_typed<DF64Tag>(a, false, st);   // B-splines only
        default: return launch_five_typed<__nv_bfloat16>(a, lag, st);
        }
    }
    // cubic B-splines: positions in cell order (neighbouring positions scatter into the same
    // stencil rows one after the other, so the atomics meet in L2 rather than in HBM) and their
    // coordinates from per-position records (no FP64 in the kernel); double-float tables keep the
    // FP64 reduction in the kernel
    if (use_cell_order(h, n_pos)) {
        Prepared pr;
        const BinGeometry g = bin_geometry(h);
        const int rc = prepare_positions(h, pos, n_pos, true, &pr, st);
        if (rc != QMCSPL_OK) return rc;
        a.e.perm = pr.perm;
        a.e.rec = h->storage == QMCSPL_DF64 ? nullptr : pr.rec;
        // real orbitals, bins of 4 cells per edge: the coefficient adjoint gathered per bin
        // (bspline_bwd_gather_kernel), then the position adjoint alone (below: its own kernel for
        // float tables, the one-pass kernel without the coefficient part otherwise)
        const bool edge4 = g.edge[0] == 4 && g.edge[1] == 4 && g.edge[2] == 4;
        if (dcoef && edge4 && !h->bloch && h->storage != QMCSPL_DF64) {
            GatherArgs ga;
            ga.bin_end = pr.bin_end;
            for (int i = 0; i < 3; ++i) ga.nb[i] = g.nb[i];
            ga.n_bins = g.n_bins;
            const bool lt = h->separate_lap != 0;
            int rc2;
            if (h->storage == QMCSPL_F64) {
                ga.n_slices = (h->n_orb + 64 - 1) / 64;      // 32 lanes x 2 doubles
                rc2 = lt ? launch_gather<double, true>(a, ga, st) : launch_gather<double, false>(a, ga, st);
            } else {
                ga.n_slices = (h->n_orb + 128 - 1) / 128;    // 32 lanes x 4 floats
                rc2 = lt ? launch_gather<float, true>(a, ga, st) : launch_gather<float, false>(a, ga, st);
            }
            if (rc2 != QMCSPL_OK || !dpos) return rc2;
            a.dcoef = a.dcoef_lap = nullptr;   // the position adjoint alone, below
        }
    }
    const bool lt = h->separate_lap != 0;
    // the position adjoint alone, float and bfloat16 tables of real orbitals: its own kernel
    if (!a.dcoef && !h->bloch && h->storage == QMCSPL_F32)
        return lt ? launch_dpos<float, true>(a, st) : launch_dpos<float, false>(a, st);
    if (!a.dcoef && !h->bloch && h->storage == QMCSPL_BF16)
        return lt ? launch_dpos<__nv_bfloat16, true>(a, st) : launch_dpos<__nv_bfloat16, false>(a, st);
    switch (h->storage) {
    case QMCSPL_F64: return lt ? launch_typed<double, true>(a, st) : launch_typed<double, false>(a, st);
    case QMCSPL_F32: return lt ? launch_typed<float, true>(a, st) : launch_typed<float, false>(a, st);
    // double-float tables: the FP64 adjoint on the stored pairs read as doubles
    case QMCSPL_DF64: return lt ? launch_typed<DF64Tag, true>(a, st) : launch_typed<DF64Tag, false>(a, st);
    default:
        return lt ? launch_typed<__nv_bfloat16, true>(a, st) : launch_typed<__nv_bfloat16, false>(a, st);
    }
}

}  // namespace qmcspl
