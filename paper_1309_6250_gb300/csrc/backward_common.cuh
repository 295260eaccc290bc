// backward_common.cuh -- argument block and helpers shared by the adjoint kernels
// (backward.cu: cubic B-splines, five tables, pp; backward_general.cuh: B-splines of any odd
// degree on uniform and graded grids).  The Bloch helpers transpose the phase and the
// bracket of the forward epilogue (see backward.cu's header).
#pragma once

#include "eval_common.cuh"

namespace qmcspl {

// Arguments of every adjoint kernel (a named type: the launchers of the general adjoint live
// in other translation units).
struct BwdArgs {
    EvalArgs e;               // tables, geometry, positions (outputs unused)
    const void* gv;           // [P][O] output dtype, may be null
    const void* gg;           // [P][3][O]
    const void* gl;           // [P][O]
    void* dcoef;              // [Nx][Ny][Nz][O] output dtype, accumulated ([5][..] five tables, [8][..] pp)
    void* dcoef_lap;
    double* dpos;             // [P][3], zeroed before the launch, accumulated
    int vec_atomic;           // dcoef rows allow 16-byte vector atomics
    int bloch;                // complex Bloch outputs: pairs (Re u, Im u) of stored functions (selects the kernel)
};

namespace {

template <typename A>
__device__ __forceinline__ void load_run(const A* src, A* v, int o0, int n_orb, int E)
{
    for (int j = 0; j < E; ++j) v[j] = (src && o0 + j < n_orb) ? src[j] : A(0);
}

template <typename A, int E>
__device__ __forceinline__ void atomic_run(A* dst, const A* v, int o0, int n_orb, bool vec)
{
    if constexpr (sizeof(A) == 4) {
        if (vec && o0 + E <= n_orb) {
#pragma unroll
            for (int j = 0; j < E; j += 4)
                atomicAdd(reinterpret_cast<float4*>(dst + j), make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]));
            return;
        }
    }
#pragma unroll
    for (int j = 0; j < E; ++j)
        if (o0 + j < n_orb) atomicAdd(dst + j, v[j]);
}

// ---- Bloch handles: the upstream through the phase and the bracket, and the phase term ----
// (see the header).  Per lane: E stored functions = E/2 complex orbitals (Re, Im adjacent).

// In: g (complex upstream of the outputs) in wv, wg (Cartesian), wl.  Out: h = conj(e) g in
// hv, hg, hl; the upstream of the tabulated u in wv, wg, wl.
template <typename A, int E, bool LAPTAB>
__device__ __forceinline__ void bloch_upstream(const EvalArgs& p, const double* rr, A* wv, A (*wg)[E], A* wl,
                                               A* hv, A (*hg)[E], A* hl)
{
    const double uk = __fma_rn(p.kred[0], rr[0], __fma_rn(p.kred[1], rr[1], __dmul_rn(p.kred[2], rr[2])));
    double sn, cs;
    sincospi(2.0 * (uk - rint(uk)), &sn, &cs);
    const A c = (A)cs, sph = (A)sn;
    const A ka[3] = {(A)p.kc[0], (A)p.kc[1], (A)p.kc[2]};
    const A kk = ka[0] * ka[0] + ka[1] * ka[1] + ka[2] * ka[2];
    auto rot = [&](A& x, A& y) {   // (x + i y) <- conj(e) (x + i y)
        const A xr = c * x + sph * y, yi = c * y - sph * x;
        x = xr;
        y = yi;
    };
#pragma unroll
    for (int j = 0; j < E / 2; ++j) {
        const int r = 2 * j, q = 2 * j + 1;
        rot(wv[r], wv[q]);
        rot(wl[r], wl[q]);
#pragma unroll
        for (int a = 0; a < 3; ++a) rot(wg[a][r], wg[a][q]);
        hv[r] = wv[r];
        hv[q] = wv[q];
        hl[r] = wl[r];
        hl[q] = wl[q];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            hg[a][r] = wg[a][r];
            hg[a][q] = wg[a][q];
        }
        // -i k.h_grad = (k.Im h_grad, -k.Re h_grad)
        const A khr = ka[0] * wg[0][r] + ka[1] * wg[1][r] + ka[2] * wg[2][r];
        const A khi = ka[0] * wg[0][q] + ka[1] * wg[1][q] + ka[2] * wg[2][q];
        wv[r] += khi;
        wv[q] -= khr;
        if (!LAPTAB) {
            wv[r] -= kk * hl[r];
            wv[q] -= kk * hl[q];
            // -2 i k_a h_lap = (2 k_a Im h_lap, -2 k_a Re h_lap)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                wg[a][r] += A(2) * ka[a] * hl[q];
                wg[a][q] -= A(2) * ka[a] * hl[r];
            }
        }
    }
}

// sum over the lane's complex orbitals and the outputs z of Im(conj(h_z) w_z), the bracket w
// rebuilt from the value u0, the reduced gradient g1 and Hessian h2 (xx, yy, zz, xy, xz, yz) of u,
// or the Laplacian table's value lam
template <typename A, int E, bool LAPTAB>
__device__ __forceinline__ double bloch_phase_sum(const EvalArgs& p, const A* u0, const A (*g1)[E],
                                                  const A (*h2)[E], const A* lam, const A* hv,
                                                  const A (*hg)[E], const A* hl)
{
    const A ka[3] = {(A)p.kc[0], (A)p.kc[1], (A)p.kc[2]};
    const A kk = ka[0] * ka[0] + ka[1] * ka[1] + ka[2] * ka[2];
    const A ml0 = (A)p.ml[0], ml1 = (A)p.ml[1], ml2 = (A)p.ml[2];
    const A ml3 = (A)p.ml[3], ml4 = (A)p.ml[4], ml5 = (A)p.ml[5];
    auto imc = [](A hr, A hi, A wr, A wi) { return hr * wi - hi * wr; };   // Im(conj(h) w)
    double sph = 0.0;
#pragma unroll
    for (int j = 0; j < E / 2; ++j) {
        const int r = 2 * j, q = 2 * j + 1;
        A gc[3][2];   // Cartesian gradient of Re u, Im u
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            gc[a][0] = (A)p.mg[3 * a] * g1[0][r] + (A)p.mg[3 * a + 1] * g1[1][r] + (A)p.mg[3 * a + 2] * g1[2][r];
            gc[a][1] = (A)p.mg[3 * a] * g1[0][q] + (A)p.mg[3 * a + 1] * g1[1][q] + (A)p.mg[3 * a + 2] * g1[2][q];
        }
        const A ur = u0[r], ui = u0[q];
        A acc = imc(hv[r], hv[q], ur, ui);
#pragma unroll
        for (int a = 0; a < 3; ++a) acc += imc(hg[a][r], hg[a][q], gc[a][0] - ka[a] * ui, gc[a][1] + ka[a] * ur);
        A lr, li;
        if (LAPTAB) {
            lr = lam[r];
            li = lam[q];
        } else {
            const A hl_r = ml0 * h2[0][r] + ml1 * h2[1][r] + ml2 * h2[2][r] + ml3 * h2[3][r] + ml4 * h2[4][r] +
                           ml5 * h2[5][r];
            const A hl_i = ml0 * h2[0][q] + ml1 * h2[1][q] + ml2 * h2[2][q] + ml3 * h2[3][q] + ml4 * h2[4][q] +
                           ml5 * h2[5][q];
            const A kgr = ka[0] * gc[0][0] + ka[1] * gc[1][0] + ka[2] * gc[2][0];
            const A kgi = ka[0] * gc[0][1] + ka[1] * gc[1][1] + ka[2] * gc[2][1];
            lr = hl_r - A(2) * kgi - kk * ur;
            li = hl_i + A(2) * kgr - kk * ui;
        }
        acc += imc(hl[r], hl[q], lr, li);
        sph += (double)acc;
    }
    return sph;
}

}  // namespace
}  // namespace qmcspl
