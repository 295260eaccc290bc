// eval_bspline.cu -- tricubic B-spline value / gradient / Laplacian evaluation.
//
// Computes, for every position r and orbital n (Appendix, Eq. b-splineapproximation):
//   phi(r)   = sum_{l,m,n=-1..2} b_l(tx) b_m(ty) b_n(tz) beta[ix+l][iy+m][iz+n]
//   grad phi = N_i (a^-1)^T grad_t phi               (chain rule, Sec. II Coordinates)
//   lap phi  = sum_ij N_i N_j (a^-1 a^-T)_ij d2phi/dt_i dt_j, or, with the separate
//              Laplacian table of Sec. III C, the same tricubic sum over beta_lap.
// For Bloch orbitals (Sec. II) the stored functions are Re u and Im u of each orbital and
// the epilogue multiplies by exp(i k.r) with the product rule (bloch_apply).
//
// Work mapping.  A group of L = 2^k lanes shares one position; each lane owns one
// 16-byte chunk of every stored row (2, 4 or 8 orbitals for f64, f32, bf16), the
// group covers one orbital tile of L chunks, and tiles x groups cover the orbitals.
// Per position the group computes the reduced coordinate in FP64 (one lane per axis,
// broadcast by shuffles) and the 1-D weights in registers, then walks the 16 (x, y)
// stencil columns.  Each column is four contiguous z rows (ghost planes make them
// contiguous), read with coalesced 16-byte loads: a warp-wide load instruction moves
// 32 x 16 B of one row.  The z sum is done first, then the (x, y) weights; the
// Hessian-derived Laplacian folds the metric N_i N_j (a^-1 a^-T)_ij into the per-column
// weights so only one accumulator per orbital is needed.
//
// Every warp task (32 lanes x one chunk x 64 rows per table) moves the same number of
// bytes whatever the orbital count, which is what lets the batched kernel mix cells
// with different orbital counts and grids in one launch with a static schedule.
//
// The kernel is a gather bounded by memory bandwidth: no tensor cores, since each
// position gathers its own stencil.
#include <type_traits>

#include "eval_common.cuh"

namespace qmcspl {
namespace {

// Evaluate the groups [w0, w0 + groups per warp) of one cell.  Called by all 32 lanes.
template <typename T, bool LAPTAB>
__device__ __forceinline__ void bspline_warp_task(const EvalArgs& p, long long w0, int lane)
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
    double tx, ty, tz;
    bool ok;
    coords_double(p, ip, L, sub, gbase, ix, iy, iz, tx, ty, tz, ok);
    if (!active) return;
    if (!ok && sub == 0 && tile == 0) atomicOr(p.err, 1);

    A bx[4], dbx[4], d2bx[4], by[4], dby[4], d2by[4], bz[4], dbz[4], d2bz[4];
    bspline_weights<A>((A)tx, bx, dbx, LAPTAB ? nullptr : d2bx);
    bspline_weights<A>((A)ty, by, dby, LAPTAB ? nullptr : d2by);
    bspline_weights<A>((A)tz, bz, dbz, LAPTAB ? nullptr : d2bz);

    int xs[4], ys[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        xs[j] = wrap1(ix + j - 1, p.nx);
        ys[j] = wrap1(iy + j - 1, p.ny);
    }
    const int chunk = tile * L + sub;
    const char* t0 = static_cast<const char*>(p.tab[0]) + (size_t)chunk * 16 + (size_t)iz * rowb;
    const char* t1 = LAPTAB ? static_cast<const char*>(p.tab[1]) + (size_t)chunk * 16 + (size_t)iz * rowb
                            : nullptr;

    A v[E], gx[E], gy[E], gz[E], lp[E];
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = gx[e] = gy[e] = gz[e] = lp[e] = A(0);

    A ml0 = 0, ml1 = 0, ml2 = 0, ml3 = 0, ml4 = 0, ml5 = 0;
    if (!LAPTAB) {
        ml0 = (A)p.ml[0]; ml1 = (A)p.ml[1]; ml2 = (A)p.ml[2];
        ml3 = (A)p.ml[3]; ml4 = (A)p.ml[4]; ml5 = (A)p.ml[5];
    }

#pragma unroll
    for (int l = 0; l < 4; ++l) {
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const size_t col = (size_t)(xs[l] * p.ny + ys[m]) * colb;
            uint4 raw[4], rawl[4];
#pragma unroll
            for (int n = 0; n < 4; ++n) raw[n] = ldg_table(p, t0 + col + n * rowb);
            if (LAPTAB) {
#pragma unroll
                for (int n = 0; n < 4; ++n) rawl[n] = ldg_table(p, t1 + col + n * rowb);
            }
            A a0[E], a1[E], a2[E], al[E];
#pragma unroll
            for (int e = 0; e < E; ++e) a0[e] = a1[e] = a2[e] = al[e] = A(0);
#pragma unroll
            for (int n = 0; n < 4; ++n) {
                A c[E];
                unpack<T>(raw[n], c);
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    a0[e] = fma(bz[n], c[e], a0[e]);
                    a1[e] = fma(dbz[n], c[e], a1[e]);
                    if (!LAPTAB) a2[e] = fma(d2bz[n], c[e], a2[e]);
                }
                if (LAPTAB) {
                    A cl[E];
                    unpack<T>(rawl[n], cl);
#pragma unroll
                    for (int e = 0; e < E; ++e) al[e] = fma(bz[n], cl[e], al[e]);
                }
            }
            const A w00 = bx[l] * by[m];
            const A w10 = dbx[l] * by[m];
            const A w01 = bx[l] * dby[m];
            A c0 = 0, c1 = 0, c2 = 0;
            if (!LAPTAB) {
                c0 = ml0 * (d2bx[l] * by[m]) + ml1 * (bx[l] * d2by[m]) + ml3 * (dbx[l] * dby[m]);
                c1 = ml4 * w10 + ml5 * w01;
                c2 = ml2 * w00;
            }
#pragma unroll
            for (int e = 0; e < E; ++e) {
                v[e] = fma(w00, a0[e], v[e]);
                gx[e] = fma(w10, a0[e], gx[e]);
                gy[e] = fma(w01, a0[e], gy[e]);
                gz[e] = fma(w00, a1[e], gz[e]);
                if (LAPTAB) {
                    lp[e] = fma(w00, al[e], lp[e]);
                } else {
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
        const A m0 = (A)p.mg[3 * a], m1 = (A)p.mg[3 * a + 1], m2 = (A)p.mg[3 * a + 2];
#pragma unroll
        for (int e = 0; e < E; ++e) cg[a][e] = fma(m0, gx[e], fma(m1, gy[e], m2 * gz[e]));
    }
    if (p.phase) bloch_apply<A, E>(p, ip, v, cg, lp, true, !LAPTAB);
    if (p.val) store_run<A, E>(static_cast<A*>(p.val) + ip * p.n_orb + o0, v, o0, p.n_orb, vec);
    if (p.grad) {
        A* g = static_cast<A*>(p.grad) + ip * 3 * p.n_orb + o0;
#pragma unroll
        for (int a = 0; a < 3; ++a) store_run<A, E>(g + (size_t)a * p.n_orb, cg[a], o0, p.n_orb, vec);
    }
    if (p.lap) store_run<A, E>(static_cast<A*>(p.lap) + ip * p.n_orb + o0, lp, o0, p.n_orb, vec);
}

// The same computation for float and bfloat16 tables with packed FP32 arithmetic
// (fma.rn.f32x2: two orbitals per instruction) and the next stencil column's rows
// loaded before the current column is contracted.
template <typename T, bool LAPTAB>
__device__ __forceinline__ void bspline_warp_task_x2(const EvalArgs& p, long long w0, int lane)
{
    constexpr int E = Traits<T>::E;          // orbitals per lane (4 float, 8 bfloat16)
    constexpr int NP = Pairs<T>::N;          // packed pairs per lane
    constexpr int R = LAPTAB ? 8 : 4;        // rows loaded per column
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
    // (the bfloat16 kernel runs fastest with the rolled form of the reduction, the float one with
    // the written-out form; both give the same bits)
    coords_float<std::is_same<T, __nv_bfloat16>::value>(p, ip, L, sub, gbase, ix, iy, iz, tx, ty, tz, ok);
    if (!active) return;
    if (!ok && sub == 0 && tile == 0) atomicOr(p.err, 1);

    float bx[4], dbx[4], d2bx[4], by[4], dby[4], d2by[4], bz[4], dbz[4], d2bz[4];
    bspline_weights<float>(tx, bx, dbx, LAPTAB ? nullptr : d2bx);
    bspline_weights<float>(ty, by, dby, LAPTAB ? nullptr : d2by);
    bspline_weights<float>(tz, bz, dbz, LAPTAB ? nullptr : d2bz);
    f32x2 bz2[4], dbz2[4], d2bz2[4];
#pragma unroll
    for (int n = 0; n < 4; ++n) {
        bz2[n] = pack2(bz[n], bz[n]);
        dbz2[n] = pack2(dbz[n], dbz[n]);
        if (!LAPTAB) d2bz2[n] = pack2(d2bz[n], d2bz[n]);
    }
    float ml0 = 0.f, ml1 = 0.f, ml2 = 0.f, ml3 = 0.f, ml4 = 0.f, ml5 = 0.f;
    if (!LAPTAB) {
        ml0 = p.mlf[0]; ml1 = p.mlf[1]; ml2 = p.mlf[2];
        ml3 = p.mlf[3]; ml4 = p.mlf[4]; ml5 = p.mlf[5];
    }
    int xs[4], ys[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        xs[j] = wrap1(ix + j - 1, p.nx);
        ys[j] = wrap1(iy + j - 1, p.ny);
    }
    const int chunk = tile * L + sub;
    const char* t0 = static_cast<const char*>(p.tab[0]) + (size_t)chunk * 16 + (size_t)iz * rowb;
    const char* t1 = LAPTAB ? static_cast<const char*>(p.tab[1]) + (size_t)chunk * 16 + (size_t)iz * rowb
                            : nullptr;

    f32x2 V[NP], GX[NP], GY[NP], GZ[NP], LP[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) V[j] = GX[j] = GY[j] = GZ[j] = LP[j] = 0ull;

    uint4 cur[R], nxt[R];
    {
        const size_t col = (size_t)(xs[0] * p.ny + ys[0]) * colb;
#pragma unroll
        for (int n = 0; n < 4; ++n) cur[n] = ldg_table(p, t0 + col + n * rowb);
        if (LAPTAB) {
#pragma unroll
            for (int n = 0; n < 4; ++n) cur[4 + n] = ldg_table(p, t1 + col + n * rowb);
        }
    }
#pragma unroll
    for (int c = 0; c < 16; ++c) {
        const int l = c >> 2, m = c & 3;
        if (c < 15) {   // next column's rows in flight while this one is contracted
            const int ln = (c + 1) >> 2, mn = (c + 1) & 3;
            const size_t col = (size_t)(xs[ln] * p.ny + ys[mn]) * colb;
#pragma unroll
            for (int n = 0; n < 4; ++n) nxt[n] = ldg_table(p, t0 + col + n * rowb);
            if (LAPTAB) {
#pragma unroll
                for (int n = 0; n < 4; ++n) nxt[4 + n] = ldg_table(p, t1 + col + n * rowb);
            }
        }
        f32x2 A0[NP], A1[NP], A2[NP], AL[NP];
#pragma unroll
        for (int j = 0; j < NP; ++j) A0[j] = A1[j] = A2[j] = AL[j] = 0ull;
#pragma unroll
        for (int n = 0; n < 4; ++n) {
            f32x2 cv[NP];
            Pairs<T>::get(cur[n], cv);
#pragma unroll
            for (int j = 0; j < NP; ++j) {
                A0[j] = ffma2(bz2[n], cv[j], A0[j]);
                A1[j] = ffma2(dbz2[n], cv[j], A1[j]);
                if (!LAPTAB) A2[j] = ffma2(d2bz2[n], cv[j], A2[j]);
            }
            if (LAPTAB) {
                Pairs<T>::get(cur[4 + n], cv);
#pragma unroll
                for (int j = 0; j < NP; ++j) AL[j] = ffma2(bz2[n], cv[j], AL[j]);
            }
        }
        const float w00 = bx[l] * by[m], w10 = dbx[l] * by[m], w01 = bx[l] * dby[m];
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
            const float c0 = ml0 * (d2bx[l] * by[m]) + ml1 * (bx[l] * d2by[m]) + ml3 * (dbx[l] * dby[m]);
            const float c1 = ml4 * w10 + ml5 * w01;
            const float c2 = ml2 * w00;
            const f32x2 C0 = pack2(c0, c0), C1 = pack2(c1, c1), C2 = pack2(c2, c2);
#pragma unroll
            for (int j = 0; j < NP; ++j) LP[j] = ffma2(C0, A0[j], ffma2(C1, A1[j], ffma2(C2, A2[j], LP[j])));
        }
        if (c < 15) {
#pragma unroll
            for (int k = 0; k < R; ++k) cur[k] = nxt[k];
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
    if (p.phase) bloch_apply<float, E>(p, ip, v, cg, lp, true, !LAPTAB);
    if (p.val) store_run<float, E>(static_cast<float*>(p.val) + ip * p.n_orb + o0, v, o0, p.n_orb, vec);
    if (p.grad) {
        float* g = static_cast<float*>(p.grad) + ip * 3 * p.n_orb + o0;
#pragma unroll
        for (int a = 0; a < 3; ++a) store_run<float, E>(g + (size_t)a * p.n_orb, cg[a], o0, p.n_orb, vec);
    }
    if (p.lap) store_run<float, E>(static_cast<float*>(p.lap) + ip * p.n_orb + o0, lp, o0, p.n_orb, vec);
}

// Double-float tables (DF64Tag chunks, see eval_common.cuh): the same stencil walk with every
// product and sum carried as a double-float pair on the FP32 pipe (see df_fma2), results
// converted to double at the store.

template <bool LAPTAB>
__device__ __forceinline__ void bspline_warp_task_df(const EvalArgs& p, long long w0, int lane)
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
    dfloat tx, ty, tz;
    bool ok;
    if (p.rec) {   // kind-3 record: cell and double-float t, no FP64 work here
        const float4* qr = static_cast<const float4*>(p.rec) + 2 * ip;
        const float4 a = __ldg(qr), b = __ldg(qr + 1);
        unpack_cell(__float_as_int(a.x), ix, iy, iz, ok);
        tx = {a.y, a.z};
        ty = {a.w, b.x};
        tz = {b.y, b.z};
    } else {
        const double r[3] = {p.pos[3 * ip], p.pos[3 * ip + 1], p.pos[3 * ip + 2]};
        double dx, dy, dz;
        reduced_coordinates(p, r, L, sub, gbase, ix, iy, iz, dx, dy, dz, ok);
        tx = df_from_double(dx);
        ty = df_from_double(dy);
        tz = df_from_double(dz);
    }
    if (!active) return;
    if (!ok && sub == 0 && tile == 0) atomicOr(p.err, 1);

    dfloat bx[4], dbx[4], d2bx[4], by[4], dby[4], d2by[4], bz[4], dbz[4], d2bz[4];
    bspline_weights_df(tx, bx, dbx, LAPTAB ? nullptr : d2bx);
    bspline_weights_df(ty, by, dby, LAPTAB ? nullptr : d2by);
    bspline_weights_df(tz, bz, dbz, LAPTAB ? nullptr : d2bz);
    dfloat ml[6];
    if (!LAPTAB)
#pragma unroll
        for (int k = 0; k < 6; ++k) ml[k] = {p.mlh[k], p.mll[k]};
    int xs[4], ys[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        xs[j] = wrap1(ix + j - 1, p.nx);
        ys[j] = wrap1(iy + j - 1, p.ny);
    }
    const int chunk = tile * L + sub;
    const char* t0 = static_cast<const char*>(p.tab[0]) + (size_t)chunk * 16 + (size_t)iz * rowb;
    const char* t1 = LAPTAB ? static_cast<const char*>(p.tab[1]) + (size_t)chunk * 16 + (size_t)iz * rowb
                            : nullptr;
    // accumulators (h, l) for value, reduced gradient, Laplacian-table value
    f32x2 Vh = 0, Vl = 0, Xh = 0, Xl = 0, Yh = 0, Yl = 0, Zh = 0, Zl = 0, Lh = 0, Ll = 0;
#pragma unroll 1
    for (int c = 0; c < 16; ++c) {
        const int l = c >> 2, m = c & 3;
        const size_t col = (size_t)(xs[l] * p.ny + ys[m]) * colb;
        uint4 raw[4], rawl[4];
#pragma unroll
        for (int n = 0; n < 4; ++n) raw[n] = ldg_table(p, t0 + col + n * rowb);
        if (LAPTAB) {
#pragma unroll
            for (int n = 0; n < 4; ++n) rawl[n] = ldg_table(p, t1 + col + n * rowb);
        }
        f32x2 A0h = 0, A0l = 0, A1h = 0, A1l = 0, A2h = 0, A2l = 0, ALh = 0, ALl = 0;
#pragma unroll
        for (int n = 0; n < 4; ++n) {
            const f32x2 Bh = pack2u(raw[n].x, raw[n].y), Bl = pack2u(raw[n].z, raw[n].w);
            const f32x2 wh = pack2(bz[n].h, bz[n].h), wl = pack2(bz[n].l, bz[n].l), nwh = pack2(-bz[n].h, -bz[n].h);
            df_fma2(A0h, A0l, wh, wl, nwh, Bh, Bl);
            const f32x2 dh = pack2(dbz[n].h, dbz[n].h), dl = pack2(dbz[n].l, dbz[n].l),
                        ndh = pack2(-dbz[n].h, -dbz[n].h);
            df_fma2(A1h, A1l, dh, dl, ndh, Bh, Bl);
            if (!LAPTAB) {
                const f32x2 eh = pack2(d2bz[n].h, d2bz[n].h), el = pack2(d2bz[n].l, d2bz[n].l),
                            neh = pack2(-d2bz[n].h, -d2bz[n].h);
                df_fma2(A2h, A2l, eh, el, neh, Bh, Bl);
            }
            if (LAPTAB) {
                const f32x2 Ch = pack2u(rawl[n].x, rawl[n].y), Cl = pack2u(rawl[n].z, rawl[n].w);
                df_fma2(ALh, ALl, wh, wl, nwh, Ch, Cl);
            }
        }
        const dfloat w00 = df_mul(bx[l], by[m]), w10 = df_mul(dbx[l], by[m]), w01 = df_mul(bx[l], dby[m]);
        const f32x2 h00 = pack2(w00.h, w00.h), l00 = pack2(w00.l, w00.l), n00 = pack2(-w00.h, -w00.h);
        const f32x2 h10 = pack2(w10.h, w10.h), l10 = pack2(w10.l, w10.l), n10 = pack2(-w10.h, -w10.h);
        const f32x2 h01 = pack2(w01.h, w01.h), l01 = pack2(w01.l, w01.l), n01 = pack2(-w01.h, -w01.h);
        df_fma2(Vh, Vl, h00, l00, n00, A0h, A0l);
        df_fma2(Xh, Xl, h10, l10, n10, A0h, A0l);
        df_fma2(Yh, Yl, h01, l01, n01, A0h, A0l);
        df_fma2(Zh, Zl, h00, l00, n00, A1h, A1l);
        if (LAPTAB) {
            df_fma2(Lh, Ll, h00, l00, n00, ALh, ALl);
        } else {
            // metric folded into per-column weights: lap += c0 A0 + c1 A1 + c2 A2
            const dfloat c0 = df_add(df_add(df_mul(ml[0], df_mul(d2bx[l], by[m])), df_mul(ml[1], df_mul(bx[l], d2by[m]))),
                                     df_mul(ml[3], df_mul(dbx[l], dby[m])));
            const dfloat c1 = df_add(df_mul(ml[4], w10), df_mul(ml[5], w01));
            const dfloat c2 = df_mul(ml[2], w00);
            df_fma2(Lh, Ll, pack2(c0.h, c0.h), pack2(c0.l, c0.l), pack2(-c0.h, -c0.h), A0h, A0l);
            df_fma2(Lh, Ll, pack2(c1.h, c1.h), pack2(c1.l, c1.l), pack2(-c1.h, -c1.h), A1h, A1l);
            df_fma2(Lh, Ll, pack2(c2.h, c2.h), pack2(c2.l, c2.l), pack2(-c2.h, -c2.h), A2h, A2l);
        }
    }

    constexpr int E = 2;
    const int o0 = chunk * E;
    if (o0 >= p.n_orb) return;
    const bool vec = p.vec_out != 0;
    float a0, a1, b0, b1;
    dfloat dv[E], dl[E], dg[3][E];
    unpack2(Vh, a0, a1); unpack2(Vl, b0, b1);
    dv[0] = {a0, b0}; dv[1] = {a1, b1};
    unpack2(Lh, a0, a1); unpack2(Ll, b0, b1);
    dl[0] = {a0, b0}; dl[1] = {a1, b1};
    if (p.grad || p.phase) {
        // chain rule in double-float: grad_a = sum_i mg[a][i] grad_t[i]
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            f32x2 Gh = 0, Gl = 0;
            const float m0h = p.mgh[3 * a], m1h = p.mgh[3 * a + 1], m2h = p.mgh[3 * a + 2];
            const float m0l = p.mgl[3 * a], m1l = p.mgl[3 * a + 1], m2l = p.mgl[3 * a + 2];
            df_fma2(Gh, Gl, pack2(m0h, m0h), pack2(m0l, m0l), pack2(-m0h, -m0h), Xh, Xl);
            df_fma2(Gh, Gl, pack2(m1h, m1h), pack2(m1l, m1l), pack2(-m1h, -m1h), Yh, Yl);
            df_fma2(Gh, Gl, pack2(m2h, m2h), pack2(m2l, m2l), pack2(-m2h, -m2h), Zh, Zl);
            unpack2(Gh, a0, a1); unpack2(Gl, b0, b1);
            dg[a][0] = {a0, b0};
            dg[a][1] = {a1, b1};
        }
    }
    if (p.phase) {   // one complex orbital per lane, in double-float
        const double2 ph = __ldg(p.phase + ip);
        const dfloat c = df_from_double(ph.x), sn = df_from_double(ph.y);
        const dfloat k[3] = {df_from_double(p.kc[0]), df_from_double(p.kc[1]), df_from_double(p.kc[2])};
        const dfloat kk = df_add(df_add(df_mul(k[0], k[0]), df_mul(k[1], k[1])), df_mul(k[2], k[2]));
        dfloat gr[3] = {dg[0][0], dg[1][0], dg[2][0]}, gi[3] = {dg[0][1], dg[1][1], dg[2][1]};
        bloch_one<dfloat>(dv[0], dv[1], gr, gi, dl[0], dl[1], k, kk, c, sn, true, !LAPTAB);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            dg[a][0] = gr[a];
            dg[a][1] = gi[a];
        }
    }
    double v[E], lp[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        v[e] = df_to_double(dv[e].h, dv[e].l);
        lp[e] = df_to_double(dl[e].h, dl[e].l);
    }
    if (p.val) store_run<double, E>(static_cast<double*>(p.val) + ip * p.n_orb + o0, v, o0, p.n_orb, vec);
    if (p.grad) {
        double* g = static_cast<double*>(p.grad) + ip * 3 * p.n_orb + o0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double cg[E];
#pragma unroll
            for (int e = 0; e < E; ++e) cg[e] = df_to_double(dg[a][e].h, dg[a][e].l);
            store_run<double, E>(g + (size_t)a * p.n_orb, cg, o0, p.n_orb, vec);
        }
    }
    if (p.lap) store_run<double, E>(static_cast<double*>(p.lap) + ip * p.n_orb + o0, lp, o0, p.n_orb, vec);
}

// float and bfloat16 tables take the packed path, double tables the scalar one
template <typename T, bool LAPTAB>
__device__ __forceinline__ void warp_task(const EvalArgs& p, long long w0, int lane)
{
    if constexpr (std::is_same<T, DF64Tag>::value) bspline_warp_task_df<LAPTAB>(p, w0, lane);
    else if constexpr (sizeof(T) == 8) bspline_warp_task<T, LAPTAB>(p, w0, lane);
    else bspline_warp_task_x2<T, LAPTAB>(p, w0, lane);
}

#ifndef QMCSPL_EVAL_THREADS
#define QMCSPL_EVAL_THREADS 512
#endif
#ifndef QMCSPL_EVAL_THREADS_F32_LAP
#define QMCSPL_EVAL_THREADS_F32_LAP 640
#endif
// Threads per block of the B-spline evaluation kernels (one block per SM).  With cell-ordered
// positions the warps of one block evaluate consecutive (neighbouring) positions on one SM, so
// their shared stencil rows hit in that SM's L1; two smaller blocks on an SM would work on
// positions far apart in the order.  512 threads x 128 registers fill the register file; the
// single-cell FP32 kernel with the Laplacian table also comes in a 640-thread shape that fits in
// 96 registers (16 bytes spilled) and runs 20 warps, which hides more of the L1/L2 latency on
// large launches (1.205 vs 1.262 ms on the 128-orbital step; 576, 672 and 768 threads were
// slower).  Launches of only a few rounds of warp tasks keep 512 threads: their last, partly
// filled round costs more with the bigger block.  The batched kernel keeps 512.
template <typename T, bool LAPTAB> struct BspBlock {
    static constexpr int large = QMCSPL_EVAL_THREADS;   // threads of the shape for large launches
};
template <> struct BspBlock<float, true> {
    static constexpr int large = QMCSPL_EVAL_THREADS_F32_LAP;
};
constexpr int kLargeLaunchRounds = 4;   // warp-task rounds from which the large shape is used

template <typename T, bool LAPTAB, int THREADS>
__global__ void __launch_bounds__(THREADS, 1) bspline_vgl_kernel(const EvalArgs p)
{
    constexpr int WPB = THREADS / 32;
    const int lane = threadIdx.x & 31;
    const int gpw = 32 >> p.lanes_log2;
    const long long total = p.n_pos * p.tiles;
    const long long warp = (long long)blockIdx.x * WPB + (threadIdx.x >> 5);
    const long long wstride = (long long)gridDim.x * WPB;
    for (long long w0 = warp * gpw; w0 < total; w0 += wstride * gpw)
        warp_task<T, LAPTAB>(p, w0, lane);
}

// Several cells in one launch: warp task w belongs to the cell c with
// start[c] <= w < start[c + 1]; tasks are handed out round-robin over all warps.
struct BatchArgs {
    int n_cells;
    long long start[QMCSPL_MAX_BATCH + 1];   // prefix sums of warp tasks per cell
    EvalArgs cell[QMCSPL_MAX_BATCH];
};
static_assert(sizeof(BatchArgs) <= 32000, "batched kernel parameters exceed the 32 KB limit");

template <typename T, bool LAPTAB, int THREADS>
__global__ void __launch_bounds__(THREADS, 1) bspline_vgl_batched_kernel(const __grid_constant__ BatchArgs b)
{
    constexpr int WPB = THREADS / 32;
    const int lane = threadIdx.x & 31;
    const long long warp = (long long)blockIdx.x * WPB + (threadIdx.x >> 5);
    const long long wstride = (long long)gridDim.x * WPB;
    const long long total = b.start[b.n_cells];
    int c = 0;
    for (long long w = warp; w < total; w += wstride) {
        while (w >= b.start[c + 1]) ++c;          // tasks only move forward
        const EvalArgs& p = b.cell[c];
        const long long local = w - b.start[c];
        warp_task<T, LAPTAB>(p, local * (32 >> p.lanes_log2), lane);
    }
}

template <typename K>
long long grid_for(K kernel, int threads, long long warps)
{
    long long blocks = (warps + threads / 32 - 1) / (threads / 32);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess)
        per_sm = 1;
    if (per_sm < 1) per_sm = 1;
    const long long cap = (long long)sm_count() * per_sm;
    if (blocks > cap) blocks = cap;
    return blocks < 1 ? 1 : blocks;
}

template <typename T, bool LAPTAB, int THREADS>
int launch_shape(const EvalArgs& a, long long warps, cudaStream_t st)
{
    const long long blocks = grid_for(bspline_vgl_kernel<T, LAPTAB, THREADS>, THREADS, warps);
    bspline_vgl_kernel<T, LAPTAB, THREADS><<<(unsigned)blocks, THREADS, 0, st>>>(a);
    return cuda_error(cudaGetLastError(), "bspline_vgl_kernel launch");
}

// Block shapes a caller may choose (qmcspl_set_block, the batched launch plan): 512 threads for
// every table type, 640 for float and bfloat16 tables (96 registers).
template <typename T> constexpr bool kHas640 = std::is_same<T, float>::value || std::is_same<T, __nv_bfloat16>::value;

// `threads` = 0: the automatic rule (the large shape from kLargeLaunchRounds rounds of warp tasks
// on); 512 or 640: that shape.
template <typename T, bool LAPTAB>
int launch_typed(const EvalArgs& a, int threads, cudaStream_t st)
{
    const int gpw = 32 >> a.lanes_log2;
    const long long warps = (a.n_pos * a.tiles + gpw - 1) / gpw;
    if constexpr (kHas640<T>) {
        if (threads == 640) return launch_shape<T, LAPTAB, 640>(a, warps, st);
    }
    if (threads == QMCSPL_EVAL_THREADS) return launch_shape<T, LAPTAB, QMCSPL_EVAL_THREADS>(a, warps, st);
    constexpr int large = BspBlock<T, LAPTAB>::large;
    if constexpr (large != QMCSPL_EVAL_THREADS) {
        if (warps >= (long long)kLargeLaunchRounds * sm_count() * (large / 32))
            return launch_shape<T, LAPTAB, large>(a, warps, st);
    }
    return launch_shape<T, LAPTAB, QMCSPL_EVAL_THREADS>(a, warps, st);
}

template <typename T, bool LAPTAB, int THREADS>
int launch_batched_shape(const BatchArgs& b, cudaStream_t st)
{
    const long long blocks = grid_for(bspline_vgl_batched_kernel<T, LAPTAB, THREADS>, THREADS, b.start[b.n_cells]);
    bspline_vgl_batched_kernel<T, LAPTAB, THREADS><<<(unsigned)blocks, THREADS, 0, st>>>(b);
    return cuda_error(cudaGetLastError(), "bspline_vgl_batched_kernel launch");
}

template <typename T, bool LAPTAB>
int launch_batched_typed(const BatchArgs& b, int threads, cudaStream_t st)
{
    if constexpr (kHas640<T>) {
        if (threads == 640) return launch_batched_shape<T, LAPTAB, 640>(b, st);
    }
    return launch_batched_shape<T, LAPTAB, QMCSPL_EVAL_THREADS>(b, st);
}

void set_outputs(const Handle* h, EvalArgs& a, void* val, void* grad, void* lap)
{
    a.val = val;
    a.grad = grad;
    a.lap = lap;
    const size_t ob = (h->storage == QMCSPL_F64 || h->storage == QMCSPL_DF64) ? 8 : 4;
    const uintptr_t al = (uintptr_t)val | (uintptr_t)grad | (uintptr_t)lap;
    a.vec_out = ((h->n_orb * ob) % 16 == 0) && (al % 16 == 0);
}

}  // namespace

int launch_bspline_vgl(const Handle* h, const double* pos, const Prepared& pr, long long n_pos, void* val,
                       void* grad, void* lap, cudaStream_t st)
{
    EvalArgs a;
    fill_eval_args(h, &a);
    a.pos = pos;
    a.rec = pr.rec;
    a.perm = pr.perm;
    a.phase = pr.phase;
    a.n_pos = n_pos;
    set_outputs(h, a, val, grad, lap);
    const bool lt = h->separate_lap != 0;
    const int th = h->block_threads;
    switch (h->storage) {
    case QMCSPL_F64: return lt ? launch_typed<double, true>(a, th, st) : launch_typed<double, false>(a, th, st);
    case QMCSPL_F32: return lt ? launch_typed<float, true>(a, th, st) : launch_typed<float, false>(a, th, st);
    case QMCSPL_DF64: return lt ? launch_typed<DF64Tag, true>(a, th, st) : launch_typed<DF64Tag, false>(a, th, st);
    default:
        return lt ? launch_typed<__nv_bfloat16, true>(a, th, st) : launch_typed<__nv_bfloat16, false>(a, th, st);
    }
}

int launch_batched(int n_cells, const Handle* const* hs, const double* const* pos, const Prepared* pr,
                   const long long* n_pos, void* const* val, void* const* grad, void* const* lap,
                   int launch, int threads, cudaStream_t st)
{
    thread_local BatchArgs B;   // about 16 KB: kept off the stack, one per calling thread
    // QMCSPL_BATCH_AUTO: cells of at least kLargeLaunchRounds rounds of warp tasks (512-thread
    // blocks on every SM) get their own launch, the others share one batched launch;
    // QMCSPL_BATCH_SINGLE: every cell in the batched launch; QMCSPL_BATCH_SPLIT: every cell alone
    const long long large = (long long)kLargeLaunchRounds * sm_count() * (QMCSPL_EVAL_THREADS / 32);
    int nb = 0;
    B.start[0] = 0;
    for (int c = 0; c < n_cells; ++c) {
        EvalArgs& a = B.cell[nb];
        fill_eval_args(hs[c], &a);
        a.pos = pos[c];
        a.rec = pr[c].rec;
        a.perm = pr[c].perm;
        a.phase = pr[c].phase;
        a.n_pos = n_pos[c];
        set_outputs(hs[c], a, val[c], grad[c], lap[c]);
        const int gpw = 32 >> a.lanes_log2;
        const long long warps = (a.n_pos * a.tiles + gpw - 1) / gpw;
        const bool alone = launch == QMCSPL_BATCH_SPLIT || (launch == QMCSPL_BATCH_AUTO && warps >= large);
        if (alone) {
            if (warps == 0) continue;
            const int rc = launch_bspline_vgl(hs[c], pos[c], pr[c], n_pos[c], val[c], grad[c], lap[c], st);
            if (rc != QMCSPL_OK) return rc;
            continue;
        }
        B.start[nb + 1] = B.start[nb] + warps;
        ++nb;
    }
    B.n_cells = nb;
    if (nb == 0 || B.start[nb] == 0) return QMCSPL_OK;
    const bool lt = hs[0]->separate_lap != 0;
    switch (hs[0]->storage) {
    case QMCSPL_DF64:
        return lt ? launch_batched_typed<DF64Tag, true>(B, threads, st) : launch_batched_typed<DF64Tag, false>(B, threads, st);
    case QMCSPL_F64:
        return lt ? launch_batched_typed<double, true>(B, threads, st) : launch_batched_typed<double, false>(B, threads, st);
    case QMCSPL_F32:
        return lt ? launch_batched_typed<float, true>(B, threads, st) : launch_batched_typed<float, false>(B, threads, st);
    default:
        return lt ? launch_batched_typed<__nv_bfloat16, true>(B, threads, st)
                  : launch_batched_typed<__nv_bfloat16, false>(B, threads, st);
    }
}

}  // namespace qmcspl
