// eval_common.cuh -- device helpers shared by the evaluation kernels of this library.
#pragma once

#include "qmcspl_internal.cuh"

namespace qmcspl {

constexpr unsigned kFullMask = 0xffffffffu;

// Storage type traits: accumulation type A and elements per 16-byte chunk E.
template <typename T> struct Traits;
template <> struct Traits<double> { using A = double; static constexpr int E = 2; };
template <> struct Traits<float> { using A = float; static constexpr int E = 4; };
template <> struct Traits<__nv_bfloat16> { using A = float; static constexpr int E = 8; };
// Double-float tables: a 16-byte chunk holds two orbitals as hi0, hi1, lo0, lo1 (value =
// hi + lo).  The evaluation kernel computes in double-float; code that computes in double
// (the adjoint) reads the pairs as doubles through Traits / unpack.
struct DF64Tag {
    float v[2];   // 8 bytes per stored coefficient
};
template <> struct Traits<DF64Tag> { using A = double; static constexpr int E = 2; };

// 16-byte read-only load of table data.
__device__ __forceinline__ uint4 ldg16(const void* p)
{
    return __ldg(reinterpret_cast<const uint4*>(p));
}

// A table load.  In a QMCSPL_DEBUG_BOUNDS build every address is checked against the
// handle's table allocation (and 16-byte alignment); a bad one sets bit 1 of the error word
// and reads zeros instead of memory (never a trap).  Other builds load directly.
__device__ __forceinline__ uint4 ldg_table(const EvalArgs& p, const char* a)
{
#ifdef QMCSPL_DEBUG_BOUNDS
    if (a < p.tab_lo || a + 16 > p.tab_hi || (reinterpret_cast<uintptr_t>(a) & 15)) {
        atomicOr(p.err, 2);
        return make_uint4(0u, 0u, 0u, 0u);
    }
#endif
    return ldg16(a);
}

// The position evaluated q-th (through the evaluation order when there is one); range
// checked in QMCSPL_DEBUG_BOUNDS builds (bit 1 of the error word, position 0 used instead).
__device__ __forceinline__ long long order_index(const EvalArgs& p, long long q)
{
    long long ip = p.perm ? (long long)p.perm[q] : q;
#ifdef QMCSPL_DEBUG_BOUNDS
    if (ip < 0 || ip >= p.n_pos) {
        atomicOr(p.err, 2);
        ip = 0;
    }
#endif
    return ip;
}

template <typename T>
__device__ __forceinline__ void unpack(const uint4& r, typename Traits<T>::A* v);

template <> __device__ __forceinline__ void unpack<double>(const uint4& r, double* v)
{
    v[0] = __hiloint2double((int)r.y, (int)r.x);
    v[1] = __hiloint2double((int)r.w, (int)r.z);
}
template <> __device__ __forceinline__ void unpack<float>(const uint4& r, float* v)
{
    v[0] = __uint_as_float(r.x);
    v[1] = __uint_as_float(r.y);
    v[2] = __uint_as_float(r.z);
    v[3] = __uint_as_float(r.w);
}
template <> __device__ __forceinline__ void unpack<DF64Tag>(const uint4& r, double* v)
{
    v[0] = (double)__uint_as_float(r.x) + (double)__uint_as_float(r.z);
    v[1] = (double)__uint_as_float(r.y) + (double)__uint_as_float(r.w);
}
// bfloat16 is the top half of a float: widen by shifting into the high 16 bits.
template <> __device__ __forceinline__ void unpack<__nv_bfloat16>(const uint4& r, float* v)
{
    const unsigned w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        v[2 * j] = __uint_as_float(w[j] << 16);
        v[2 * j + 1] = __uint_as_float(w[j] & 0xffff0000u);
    }
}

// Eq. (reducedcoordinate) for one axis: s -> (grid index below the point, t in [0,1)).
// `ok` is false for a non-finite coordinate (then i = 0 and t = NaN).
__device__ __forceinline__ void reduce_axis(double s, int N, int& i, double& t, bool& ok)
{
    const double f = s - floor(s);
    ok = isfinite(f);
    const double u = (double)N * f;
    const double fl = floor(u);
    t = u - fl;
    int k = ok ? (int)fl : 0;
    if (k >= N) k -= N;        // f rounded up to 1.0
    i = k;
    if (!ok) t = __longlong_as_double(0x7ff8000000000000LL);
}

// Crystal coordinate s_i = sum_j ainv[i][j] r_j with a fixed rounding sequence, so that
// every kernel that reduces a position gets the same bits.
__device__ __forceinline__ double crystal(double a0, double a1, double a2, const double* r)
{
    return __fma_rn(a0, r[0], __fma_rn(a1, r[1], __dmul_rn(a2, r[2])));
}

// Reduced coordinates of position r for every lane of a group of L lanes.  With
// L >= 4 lane j < 3 of the group reduces axis j and the results are broadcast by
// shuffles; smaller groups reduce all three axes in every lane.  Must be called by
// all 32 lanes of the warp.
__device__ __forceinline__ void reduced_coordinates(const EvalArgs& p, const double* r, int L,
                                                    int sub, int gbase, int& ix, int& iy,
                                                    int& iz, double& tx, double& ty,
                                                    double& tz, bool& ok)
{
    if (L >= 4) {
        const int ax = sub < 3 ? sub : 2;
        const double a0 = ax == 0 ? p.ainv[0] : (ax == 1 ? p.ainv[3] : p.ainv[6]);
        const double a1 = ax == 0 ? p.ainv[1] : (ax == 1 ? p.ainv[4] : p.ainv[7]);
        const double a2 = ax == 0 ? p.ainv[2] : (ax == 1 ? p.ainv[5] : p.ainv[8]);
        const int N = ax == 0 ? p.nx : (ax == 1 ? p.ny : p.nz);
        int i;
        double t;
        bool o;
        reduce_axis(crystal(a0, a1, a2, r), N, i, t, o);
        ix = __shfl_sync(kFullMask, i, gbase);
        iy = __shfl_sync(kFullMask, i, gbase + 1);
        iz = __shfl_sync(kFullMask, i, gbase + 2);
        tx = __shfl_sync(kFullMask, t, gbase);
        ty = __shfl_sync(kFullMask, t, gbase + 1);
        tz = __shfl_sync(kFullMask, t, gbase + 2);
        const int okb = o ? 1 : 0;
        ok = (__shfl_sync(kFullMask, okb, gbase) & __shfl_sync(kFullMask, okb, gbase + 1) &
              __shfl_sync(kFullMask, okb, gbase + 2)) != 0;
    } else {
        bool o0, o1, o2;
        reduce_axis(crystal(p.ainv[0], p.ainv[1], p.ainv[2], r), p.nx, ix, tx, o0);
        reduce_axis(crystal(p.ainv[3], p.ainv[4], p.ainv[5], r), p.ny, iy, ty, o1);
        reduce_axis(crystal(p.ainv[6], p.ainv[7], p.ainv[8], r), p.nz, iz, tz, o2);
        ok = o0 && o1 && o2;
    }
}

// ---- coordinates of position ip: from its record when the launch has records,
// otherwise reduced here (all 32 lanes must call these) ----
__device__ __forceinline__ void unpack_cell(int c, int& ix, int& iy, int& iz, bool& ok)
{
    ok = c >= 0;
    const int cc = ok ? c : 0;
    ix = cc & 1023;
    iy = (cc >> 10) & 1023;
    iz = (cc >> 20) & 1023;
}

// the reduced coordinates of float and bfloat16 tables (double-float arithmetic), defined below
template <bool ROLLED>
__device__ __forceinline__ void reduced_coordinates_df(const EvalArgs& p, const double* r, int L, int sub,
                                                       int gbase, int& ix, int& iy, int& iz, float& tx,
                                                       float& ty, float& tz, bool& ok);

// ROLLED: the form of the reduction without records (see reduced_coordinates_df); both forms give
// the same bits
template <bool ROLLED = false>
__device__ __forceinline__ void coords_float(const EvalArgs& p, long long ip, int L, int sub, int gbase,
                                             int& ix, int& iy, int& iz, float& tx, float& ty, float& tz,
                                             bool& ok)
{
    if (p.rec) {
        const float4 q = __ldg(static_cast<const float4*>(p.rec) + ip);
        unpack_cell(__float_as_int(q.x), ix, iy, iz, ok);
        tx = q.y;
        ty = q.z;
        tz = q.w;
    } else {
        const double r[3] = {p.pos[3 * ip], p.pos[3 * ip + 1], p.pos[3 * ip + 2]};
        reduced_coordinates_df<ROLLED>(p, r, L, sub, gbase, ix, iy, iz, tx, ty, tz, ok);
    }
}

__device__ __forceinline__ void coords_double(const EvalArgs& p, long long ip, int L, int sub, int gbase,
                                              int& ix, int& iy, int& iz, double& tx, double& ty, double& tz,
                                              bool& ok)
{
    if (p.rec) {
        const double2* q = static_cast<const double2*>(p.rec) + 2 * ip;
        const double2 a = __ldg(q), b = __ldg(q + 1);
        tx = a.x;
        ty = a.y;
        tz = b.x;
        unpack_cell(__double2loint(b.y), ix, iy, iz, ok);
    } else {
        const double r[3] = {p.pos[3 * ip], p.pos[3 * ip + 1], p.pos[3 * ip + 2]};
        reduced_coordinates(p, r, L, sub, gbase, ix, iy, iz, tx, ty, tz, ok);
    }
}

__device__ __forceinline__ int wrap1(int x, int n)
{
    return x < 0 ? x + n : (x >= n ? x - n : x);
}

// Cubic B-spline weights of the Appendix, Eq. (b-splinebasis), for stencil offsets
// -1..2 (index 0..3), and their first and second t-derivatives.
template <typename A>
__device__ __forceinline__ void bspline_weights(A t, A* w, A* dw, A* d2w)
{
    const A s = A(1) - t;
    const A t2 = t * t;
    w[0] = A(0.25) * s * s * s;
    w[1] = (A(0.75) * t - A(1.5)) * t2 + A(1);
    w[2] = ((A(-0.75) * t + A(0.75)) * t + A(0.75)) * t + A(0.25);
    w[3] = A(0.25) * t2 * t;
    dw[0] = A(-0.75) * s * s;
    dw[1] = (A(2.25) * t - A(3)) * t;
    dw[2] = (A(-2.25) * t + A(1.5)) * t + A(0.75);
    dw[3] = A(0.75) * t2;
    if (d2w) {
        d2w[0] = A(1.5) * s;
        d2w[1] = A(4.5) * t - A(3);
        d2w[2] = A(-4.5) * t + A(1.5);
        d2w[3] = A(1.5) * t;
    }
}

// ---- packed FP32 pairs (fma.rn.f32x2 on sm_100+): two orbitals per instruction ----
typedef unsigned long long f32x2;

__device__ __forceinline__ f32x2 pack2(float lo, float hi)
{
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ f32x2 pack2u(unsigned lo, unsigned hi)
{
    f32x2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "r"(lo), "r"(hi));
    return r;
}
__device__ __forceinline__ void unpack2(f32x2 v, float& lo, float& hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
// d = a * b + c, lane-wise on the two halves, round to nearest
__device__ __forceinline__ f32x2 ffma2(f32x2 a, f32x2 b, f32x2 c)
{
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

// A 16-byte chunk as float pairs: 2 pairs (4 floats) or 4 pairs (8 bfloat16 widened).
template <typename T> struct Pairs;
template <> struct Pairs<float> {
    static constexpr int N = 2;
    __device__ __forceinline__ static void get(const uint4& r, f32x2* c)
    {
        c[0] = pack2u(r.x, r.y);
        c[1] = pack2u(r.z, r.w);
    }
};
template <> struct Pairs<__nv_bfloat16> {
    static constexpr int N = 4;
    __device__ __forceinline__ static void get(const uint4& r, f32x2* c)
    {
        c[0] = pack2u(r.x << 16, r.x & 0xffff0000u);
        c[1] = pack2u(r.y << 16, r.y & 0xffff0000u);
        c[2] = pack2u(r.z << 16, r.z & 0xffff0000u);
        c[3] = pack2u(r.w << 16, r.w & 0xffff0000u);
    }
};

__device__ __forceinline__ f32x2 add2(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b)
{
    f32x2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// ---- double-float numbers x = h + l (two floats, ~48 significant bits) ----
// Error-free transformations (Dekker / Knuth): the rounded product or sum plus its
// exact rounding error.  Only the _rn intrinsics and explicit fma are used, so the
// compiler cannot contract or reassociate them.
struct dfloat {
    float h, l;
};

__device__ __forceinline__ dfloat df_from_double(double x)
{
    const float h = __double2float_rn(x);
    return {h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double df_to_double(float h, float l) { return (double)h + (double)l; }
// renormalise so that |l| <= ulp(h)/2 (requires |h| >= |l|)
__device__ __forceinline__ dfloat df_norm(float h, float l)
{
    const float s = __fadd_rn(h, l);
    return {s, __fsub_rn(l, __fsub_rn(s, h))};
}
__device__ __forceinline__ dfloat df_mul(dfloat a, dfloat b)
{
    const float p = __fmul_rn(a.h, b.h);
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    return df_norm(p, e);
}
__device__ __forceinline__ dfloat df_mulf(dfloat a, float c)
{
    const float p = __fmul_rn(a.h, c);
    float e = fmaf(a.h, c, -p);
    e = fmaf(a.l, c, e);
    return df_norm(p, e);
}
__device__ __forceinline__ dfloat df_add(dfloat a, dfloat b)
{
    const float s = __fadd_rn(a.h, b.h);
    const float bb = __fsub_rn(s, a.h);
    float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));
    e = __fadd_rn(e, __fadd_rn(a.l, b.l));
    return df_norm(s, e);
}
__device__ __forceinline__ dfloat df_neg(dfloat a) { return {-a.h, -a.l}; }

// floor of a double-float value (|l| <= ulp(h)/2): that of h, one less where h is an integer
// and the value lies just below it
__device__ __forceinline__ float df_floor(dfloat x)
{
    const float f = floorf(x.h);
    return (f == x.h && x.l < 0.0f) ? f - 1.0f : f;
}

// Reduced coordinate of one axis for float and bfloat16 tables (Eq. reducedcoordinate, the
// steps of reduce_axis) in double-float arithmetic on the FP32 pipe: crystal coordinate
// s = sum_j a^-1_ij r_j, wrap to [0, 1), scale by N, split into cell i and offset t, the offset
// rounded to float at the end.  About 48 significant bits: t to about N 2^-38 within 1024 lattice
// vectors of the origin (|s| < 1024), far below the float it is rounded to; a position further
// out takes the FP64 steps.  rh, rl: the position as
// double-float pairs; ah, al: row `ax` of a^-1 as double-float pairs.
__device__ __forceinline__ void reduce_axis_df(const double* r, const float* rh, const float* rl, const double* ad,
                                               const float* ah, const float* al, int N, int& i, float& t, bool& ok)
{
    dfloat s = df_mul({ah[0], al[0]}, {rh[0], rl[0]});
    s = df_add(s, df_mul({ah[1], al[1]}, {rh[1], rl[1]}));
    s = df_add(s, df_mul({ah[2], al[2]}, {rh[2], rl[2]}));
    if (!(fabsf(s.h) < 1024.0f)) {   // far outside the cell, or not finite
        double td;
        reduce_axis(crystal(ad[0], ad[1], ad[2], r), N, i, td, ok);
        t = (float)td;
        return;
    }
    ok = true;
    const dfloat f = df_add(s, {-df_floor(s), 0.0f});
    const dfloat u = df_mulf(f, (float)N);
    const float fl = df_floor(u);
    const dfloat d = df_add(u, {-fl, 0.0f});
    t = __fadd_rn(d.h, d.l);
    int k = (int)fl;
    if (k >= N) k -= N;
    i = k;
}

// a row of a^-1 as double-float pairs: the same split as df_from_double, so that the host's split
// of the same doubles (the records' arguments) gives the same floats
__device__ __forceinline__ void df_row(const double* ad, float* ah, float* al)
{
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const dfloat d = df_from_double(ad[j]);
        ah[j] = d.h;
        al[j] = d.l;
    }
}

// reduced_coordinates() for float and bfloat16 tables, with reduce_axis_df per axis: with L >= 4
// lane j < 3 of the group takes axis j (the results broadcast by shuffles), smaller groups reduce
// all three axes in every lane.  Two forms of the same arithmetic, chosen per kernel by what its
// code layout runs fastest with: the axes written out (ROLLED = false), or one copy of the steps
// in a loop over the axes (ROLLED = true).
template <bool ROLLED>
__device__ __forceinline__ void reduced_coordinates_df(const EvalArgs& p, const double* r, int L, int sub,
                                                       int gbase, int& ix, int& iy, int& iz, float& tx,
                                                       float& ty, float& tz, bool& ok)
{
    float rh[3], rl[3];
    df_row(r, rh, rl);
    const bool shared = L >= 4;
    if (!ROLLED) {
        if (shared) {
            const int ax = sub < 3 ? sub : 2;
            const double ad[3] = {ax == 0 ? p.ainv[0] : (ax == 1 ? p.ainv[3] : p.ainv[6]),
                                  ax == 0 ? p.ainv[1] : (ax == 1 ? p.ainv[4] : p.ainv[7]),
                                  ax == 0 ? p.ainv[2] : (ax == 1 ? p.ainv[5] : p.ainv[8])};
            const int N = ax == 0 ? p.nx : (ax == 1 ? p.ny : p.nz);
            float ah[3], al[3];
            df_row(ad, ah, al);
            int i;
            float t;
            bool o;
            reduce_axis_df(r, rh, rl, ad, ah, al, N, i, t, o);
            ix = __shfl_sync(kFullMask, i, gbase);
            iy = __shfl_sync(kFullMask, i, gbase + 1);
            iz = __shfl_sync(kFullMask, i, gbase + 2);
            tx = __shfl_sync(kFullMask, t, gbase);
            ty = __shfl_sync(kFullMask, t, gbase + 1);
            tz = __shfl_sync(kFullMask, t, gbase + 2);
            const int okb = o ? 1 : 0;
            ok = (__shfl_sync(kFullMask, okb, gbase) & __shfl_sync(kFullMask, okb, gbase + 1) &
                  __shfl_sync(kFullMask, okb, gbase + 2)) != 0;
        } else {
            bool o0, o1, o2;
            float ah[9], al[9];
            df_row(p.ainv, ah, al);
            df_row(p.ainv + 3, ah + 3, al + 3);
            df_row(p.ainv + 6, ah + 6, al + 6);
            reduce_axis_df(r, rh, rl, p.ainv, ah, al, p.nx, ix, tx, o0);
            reduce_axis_df(r, rh, rl, p.ainv + 3, ah + 3, al + 3, p.ny, iy, ty, o1);
            reduce_axis_df(r, rh, rl, p.ainv + 6, ah + 6, al + 6, p.nz, iz, tz, o2);
            ok = o0 && o1 && o2;
        }
        return;
    }
    int i0 = 0, i1 = 0, i2 = 0;
    float t0 = 0.f, t1 = 0.f, t2 = 0.f;
    bool o0 = true, o1 = true, o2 = true;
#pragma unroll 1
    for (int k = 0; k < (shared ? 1 : 3); ++k) {
        const int ax = shared ? (sub < 3 ? sub : 2) : k;
        const double ad[3] = {ax == 0 ? p.ainv[0] : (ax == 1 ? p.ainv[3] : p.ainv[6]),
                              ax == 0 ? p.ainv[1] : (ax == 1 ? p.ainv[4] : p.ainv[7]),
                              ax == 0 ? p.ainv[2] : (ax == 1 ? p.ainv[5] : p.ainv[8])};
        const int N = ax == 0 ? p.nx : (ax == 1 ? p.ny : p.nz);
        float ah[3], al[3];
        df_row(ad, ah, al);
        int i;
        float t;
        bool o;
        reduce_axis_df(r, rh, rl, ad, ah, al, N, i, t, o);
        if (k == 0) {
            i0 = i;
            t0 = t;
            o0 = o;
        } else if (k == 1) {
            i1 = i;
            t1 = t;
            o1 = o;
        } else {
            i2 = i;
            t2 = t;
            o2 = o;
        }
    }
    if (shared) {
        ix = __shfl_sync(kFullMask, i0, gbase);
        iy = __shfl_sync(kFullMask, i0, gbase + 1);
        iz = __shfl_sync(kFullMask, i0, gbase + 2);
        tx = __shfl_sync(kFullMask, t0, gbase);
        ty = __shfl_sync(kFullMask, t0, gbase + 1);
        tz = __shfl_sync(kFullMask, t0, gbase + 2);
        const int okb = o0 ? 1 : 0;
        ok = (__shfl_sync(kFullMask, okb, gbase) & __shfl_sync(kFullMask, okb, gbase + 1) &
              __shfl_sync(kFullMask, okb, gbase + 2)) != 0;
    } else {
        ix = i0;
        iy = i1;
        iz = i2;
        tx = t0;
        ty = t1;
        tz = t2;
        ok = o0 && o1 && o2;
    }
}

// Cubic B-spline weights (Eq. b-splinebasis) and first derivatives in double-float
// from a reduced coordinate given in double.
__device__ __forceinline__ void bspline_weights_df(dfloat t, dfloat* w, dfloat* dw, dfloat* d2w)
{
    const dfloat s = df_add({1.0f, 0.0f}, df_neg(t));
    const dfloat t2 = df_mul(t, t), t3 = df_mul(t2, t);
    const dfloat s2 = df_mul(s, s), s3 = df_mul(s2, s);
    w[0] = {0.25f * s3.h, 0.25f * s3.l};                                        // (1-t)^3/4
    w[1] = df_add(df_add(df_mulf(t3, 0.75f), df_mulf(t2, -1.5f)), {1.0f, 0.0f});
    w[2] = df_add(df_add(df_mulf(t3, -0.75f), df_mulf(t2, 0.75f)), df_add(df_mulf(t, 0.75f), {0.25f, 0.0f}));
    w[3] = {0.25f * t3.h, 0.25f * t3.l};
    dw[0] = df_mulf(s2, -0.75f);
    dw[1] = df_add(df_mulf(t2, 2.25f), df_mulf(t, -3.0f));
    dw[2] = df_add(df_add(df_mulf(t2, -2.25f), df_mulf(t, 1.5f)), {0.75f, 0.0f});
    dw[3] = df_mulf(t2, 0.75f);
    if (d2w) {
        d2w[0] = df_mulf(s, 1.5f);
        d2w[1] = df_add(df_mulf(t, 4.5f), {-3.0f, 0.0f});
        d2w[2] = df_add(df_mulf(t, -4.5f), {1.5f, 0.0f});
        d2w[3] = df_mulf(t, 1.5f);
    }
}

// Packed double-float accumulation of two orbitals: (Ah, Al) += w * (Bh, Bl), where w is
// a double-float scalar given as the packed pairs wh = (w.h, w.h), wl = (w.l, w.l) and
// nwh = -wh.  The rounded products enter Ah through an exact two-sum; the product's
// rounding error, the cross terms and the sum's rounding error go to Al.
__device__ __forceinline__ void df_fma2(f32x2& Ah, f32x2& Al, f32x2 wh, f32x2 wl, f32x2 nwh, f32x2 Bh, f32x2 Bl)
{
    const f32x2 nP = mul2(nwh, Bh);                 // -(rounded w.h * Bh)
    f32x2 E = ffma2(wh, Bh, nP);                     // its exact rounding error
    E = ffma2(wh, Bl, E);
    E = ffma2(wl, Bh, E);
    const f32x2 S = sub2(Ah, nP);                    // Ah + P
    const f32x2 BB = sub2(S, Ah);
    const f32x2 T1 = sub2(Ah, sub2(S, BB));
    const f32x2 T2 = add2(nP, BB);                   // -(P - BB)
    Al = add2(Al, add2(sub2(T1, T2), E));
    Ah = S;
}

// ---- Bloch orbitals (Sec. II): phi = u exp(i k.r) ----
// The same arithmetic in float, double and double-float through one set of names.
__device__ __forceinline__ float nadd(float a, float b) { return a + b; }
__device__ __forceinline__ double nadd(double a, double b) { return a + b; }
__device__ __forceinline__ dfloat nadd(dfloat a, dfloat b) { return df_add(a, b); }
__device__ __forceinline__ float nsub(float a, float b) { return a - b; }
__device__ __forceinline__ double nsub(double a, double b) { return a - b; }
__device__ __forceinline__ dfloat nsub(dfloat a, dfloat b) { return df_add(a, df_neg(b)); }
__device__ __forceinline__ float nmul(float a, float b) { return a * b; }
__device__ __forceinline__ double nmul(double a, double b) { return a * b; }
__device__ __forceinline__ dfloat nmul(dfloat a, dfloat b) { return df_mul(a, b); }

// (x + i y) <- (x + i y)(c + i s)
template <typename N>
__device__ __forceinline__ void crot(N& x, N& y, N c, N s)
{
    const N r = nsub(nmul(x, c), nmul(y, s));
    y = nadd(nmul(x, s), nmul(y, c));
    x = r;
}

// One complex orbital.  In: value (vr, vi), Cartesian gradient (gr, gi) and Laplacian
// (lr, li) of the periodic part u; where grad_u / lap_u is false the gradient / Laplacian
// given is already the periodic part of grad phi / lap phi (a separate table).  Out: the
// same of phi, with c + i s = exp(i k.r), kk = |k|^2:
//   phi = (c + i s) u
//   grad phi = (c + i s)(grad u + i k u)
//   lap phi = (c + i s)(lap u + 2 i k.grad u - |k|^2 u)
template <typename N>
__device__ __forceinline__ void bloch_one(N& vr, N& vi, N* gr, N* gi, N& lr, N& li, const N* k, N kk, N c,
                                          N s, bool grad_u, bool lap_u)
{
    if (lap_u) {   // uses grad u, so before the gradient is completed
        const N kgr = nadd(nadd(nmul(k[0], gr[0]), nmul(k[1], gr[1])), nmul(k[2], gr[2]));
        const N kgi = nadd(nadd(nmul(k[0], gi[0]), nmul(k[1], gi[1])), nmul(k[2], gi[2]));
        lr = nsub(nsub(lr, nadd(kgi, kgi)), nmul(kk, vr));
        li = nsub(nadd(li, nadd(kgr, kgr)), nmul(kk, vi));
    }
    if (grad_u) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const N r = nsub(gr[a], nmul(k[a], vi));
            gi[a] = nadd(gi[a], nmul(k[a], vr));
            gr[a] = r;
        }
    }
    crot(vr, vi, c, s);
#pragma unroll
    for (int a = 0; a < 3; ++a) crot(gr[a], gi[a], c, s);
    crot(lr, li, c, s);
}

// A lane's E outputs of type A (float or double): E/2 complex orbitals with Re and Im
// adjacent; g[a] holds Cartesian gradient component a.  Position ip's factor is read
// from p.phase (computed in FP64 by the per-position pass).
template <typename A, int E>
__device__ __forceinline__ void bloch_apply(const EvalArgs& p, long long ip, A* v, A (*g)[E], A* lp, bool grad_u,
                                            bool lap_u)
{
    const double2 ph = __ldg(p.phase + ip);
    A k[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if constexpr (sizeof(A) == 8) k[a] = p.kc[a];
        else k[a] = p.kcf[a];
    }
    const A kk = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
    const A c = (A)ph.x, s = (A)ph.y;
#pragma unroll
    for (int j = 0; j < E / 2; ++j) {
        A gr[3], gi[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            gr[a] = g[a][2 * j];
            gi[a] = g[a][2 * j + 1];
        }
        bloch_one<A>(v[2 * j], v[2 * j + 1], gr, gi, lp[2 * j], lp[2 * j + 1], k, kk, c, s, grad_u, lap_u);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            g[a][2 * j] = gr[a];
            g[a][2 * j + 1] = gi[a];
        }
    }
}

// Streaming stores of E consecutive outputs (vector when allowed).
template <typename A, int E>
__device__ __forceinline__ void store_run(A* dst, const A* v, int o0, int n_orb, bool vec)
{
    if (vec && o0 + E <= n_orb) {
        if constexpr (sizeof(A) == 8) {
#pragma unroll
            for (int j = 0; j < E; j += 2)
                __stcs(reinterpret_cast<double2*>(dst + j), make_double2(v[j], v[j + 1]));
        } else {
#pragma unroll
            for (int j = 0; j < E; j += 4)
                __stcs(reinterpret_cast<float4*>(dst + j), make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]));
        }
    } else {
#pragma unroll
        for (int j = 0; j < E; ++j)
            if (o0 + j < n_orb) __stcs(dst + j, v[j]);
    }
}

}  // namespace qmcspl
