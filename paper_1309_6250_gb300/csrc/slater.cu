// slater.cu -- a consumer of the orbital outputs: Slater matrices, log-determinant, local
// kinetic energy and drift of every walker (Sec. I).
//
// Sec. I writes the trial wave function as a Jastrow factor times a Slater determinant of
// the single-particle orbitals.  Without the Jastrow factor and with the electrons of a
// walker split into spin blocks, Psi = det A_up det A_dn, A_s[i][j] = phi_j(r_i) over the
// block's electrons i and its first n_s orbitals j.  Jacobi's formula (row i of A replaced
// by its Laplacian or gradient) gives, with X = A^-1,
//   lap_i det A / det A = sum_j X_ji lap phi_j(r_i),   grad_i ln|det A| = sum_j X_ji grad phi_j(r_i),
// so the kinetic part of the local energy E_L = H Psi / Psi is
//   T_L = -1/2 sum_s tr(A_s^-1 L_s),  L_s[i][j] = lap phi_j(r_i).
//
// One thread block per walker handles its two spin blocks in turn: the block's Slater
// matrix is gathered from the val rows of qmcspl_eval_vgl (walker-major positions, so the
// matrix is n_s consecutive rows) into shared memory as FP64 and inverted in place by
// Gauss-Jordan elimination with row pivoting; the pivots give ln|det A| and its sign; the
// row swaps become a column permutation of the inverse, applied by index.  The kinetic
// term and the drift then read lap and grad rows once, coalesced.
//
// The elimination is n^3 multiply-adds per block (2.1 M for n = 128).  Two arithmetic
// modes: FP64 (GB300's FP64 pipe bounds it), and double-float, where every matrix entry is
// a pair of floats (hi + lo, ~48 significant bits) and each elimination update is an
// error-free FP32 multiply-add done two columns at a time with fma.rn.f32x2 (see df_fma2):
// the FP32 pipe carries it, several times faster on this part.  Every loop is bounded by n.
// Complex orbitals (Bloch functions) take a complex elimination, in FP64 (slater_complex_kernel)
// or in double-float (slater_cdf_kernel).
#include <cmath>

#include "eval_common.cuh"

namespace qmcspl {
namespace {

constexpr int kSlaterThreads = 256;
#ifndef QMCSPL_SLATER_DF_THREADS
#define QMCSPL_SLATER_DF_THREADS 512
#endif
// double-float kernel: one CTA per SM (its matrix fills shared memory), so the CTA itself
// must bring the warps that hide the latency of the dependent FP32 chains
constexpr int kSlaterDfThreads = QMCSPL_SLATER_DF_THREADS;
constexpr int kSlaterMaxBlock = QMCSPL_SLATER_MAX_BLOCK;

struct SlaterArgs {
    const void* val;
    const void* grad;
    const void* lap;
    long long n_walkers;
    int n_elec, n_up, n_orb;
    double* logdet;
    double* sign;
    double* kinetic;
    double* drift;
    int arith;                // 0: FP64, 1: double-float
};

template <typename T>
__device__ __forceinline__ double ld(const void* p, long long i)
{
    return (double)__ldg(static_cast<const T*>(p) + i);
}

// Block-wide sum of one double per thread (NT threads); every thread gets the total.
template <int NT = kSlaterThreads>
__device__ double block_sum(double v, double* red)
{
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < NT / 32; ++w) t += red[w];
    return t;
}

// ln|det| = sum_k ln|pivot_k| over the block's pivots (one logarithm per pivot, spread over
// the threads); sgn is multiplied by the sign of the determinant (pivot signs and row swaps).
// Called by all threads.
template <int NT = kSlaterThreads>
__device__ double pivot_logdet(const double* pivd, const int* piv, int n, double& sgn, double* red)
{
    double part = 0.0;
    int neg = 0;
    for (int k = threadIdx.x; k < n; k += NT) {
        part += log(fabs(pivd[k]));
        neg += (pivd[k] < 0.0) + (piv[k] != k);
    }
    const double ld = block_sum<NT>(part, red);
    const double nn = block_sum<NT>((double)neg, red);
    if (((long long)nn) & 1) sgn = -sgn;
    return ld;
}

template <typename T>
__global__ void __launch_bounds__(kSlaterThreads) slater_kernel(const SlaterArgs a)
{
    extern __shared__ double smem[];
    __shared__ double red[kSlaterThreads / 32];
    __shared__ int piv[kSlaterMaxBlock];
    __shared__ int colmap[kSlaterMaxBlock];
    __shared__ double fcol[kSlaterMaxBlock];
    __shared__ double rowk[kSlaterMaxBlock];
    __shared__ int s_p;
    __shared__ double s_d;
    __shared__ double pivd[kSlaterMaxBlock];   // pivot values: ln|det| and sign at the end

    const long long w = blockIdx.x;
    if (w >= a.n_walkers) return;
    const int tid = threadIdx.x;
    const int lane = tid & 31, wid = tid >> 5;
    const long long O = a.n_orb;
    double logdet = 0.0, sgn = 1.0, kin = 0.0;
    bool singular = false;

    for (int blk = 0; blk < 2; ++blk) {
        const int e0 = blk == 0 ? 0 : a.n_up;
        const int n = blk == 0 ? a.n_up : a.n_elec - a.n_up;
        if (n == 0) continue;
        const int ns = n + 1;                              // padded row stride (banks)
        const long long base = w * a.n_elec + e0;          // first position of the block
        double* A = smem;                                   // [n][n + 1]

        __syncthreads();                                    // smem reuse between blocks
        for (int i = wid; i < n; i += kSlaterThreads / 32)  // warps over rows, lanes over columns
            for (int j = lane; j < n; j += 32) A[i * ns + j] = ld<T>(a.val, (base + i) * O + j);
        __syncthreads();

        bool sing = false;
        for (int k = 0; k < n; ++k) {
            // pivot: the largest |A[i][k]| over i >= k (first one on ties)
            if (wid == 0) {
                double best = -1.0;
                int bi = k;
                for (int i = k + lane; i < n; i += 32) {
                    const double v = fabs(A[i * ns + k]);
                    if (v > best) {
                        best = v;
                        bi = i;
                    }
                }
                for (int off = 16; off > 0; off >>= 1) {
                    const double ob = __shfl_xor_sync(0xffffffffu, best, off);
                    const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
                    if (ob > best || (ob == best && oi < bi)) {
                        best = ob;
                        bi = oi;
                    }
                }
                if (lane == 0) {
                    s_p = bi;
                    s_d = A[bi * ns + k];   // the pivot value (the swap below moves, not changes, it)
                    piv[k] = bi;
                    pivd[k] = s_d;
                }
            }
            __syncthreads();
            const int p = s_p;
            const double d = s_d;
            if (p != k)
                for (int j = tid; j < n; j += kSlaterThreads) {
                    const double t = A[k * ns + j];
                    A[k * ns + j] = A[p * ns + j];
                    A[p * ns + j] = t;
                }
            __syncthreads();   // the swapped rows are read by other threads below
            if (d == 0.0) {   // exactly singular (uniform: every thread reads the same value)
                sing = true;
                break;
            }
            // scaled pivot row (its pivot entry becomes 1/d) and the pivot column
            for (int j = tid; j < n; j += kSlaterThreads) {
                const double r = (j == k ? 1.0 : A[k * ns + j]) / d;
                rowk[j] = r;
                A[k * ns + j] = r;
            }
            for (int i = tid; i < n; i += kSlaterThreads)
                if (i != k) fcol[i] = A[i * ns + k];
            __syncthreads();
            // eliminate column k from every other row
            for (int i = wid; i < n; i += kSlaterThreads / 32) {
                if (i == k) continue;
                const double f = fcol[i];
                for (int j = lane; j < n; j += 32) {
                    const double x = (j == k) ? 0.0 : A[i * ns + j];
                    A[i * ns + j] = fma(-f, rowk[j], x);
                }
            }
            __syncthreads();
        }
        if (sing) {
            singular = true;
            break;
        }
        logdet += pivot_logdet(pivd, piv, n, sgn, red);
        // The row swaps of the elimination permute the columns of the inverse: undoing
        // them in reverse order maps column c of A^-1 to column colmap[c] of A.
        if (tid == 0) {
            for (int c = 0; c < n; ++c) colmap[c] = c;
            for (int k = n - 1; k >= 0; --k) {
                const int t = colmap[k];
                colmap[k] = colmap[piv[k]];
                colmap[piv[k]] = t;
            }
        }
        __syncthreads();
        // T_s = -1/2 sum_ij (A^-1)_ji L_ij, (A^-1)_ji = A[j][colmap[i]]
        if (a.kinetic) {
            double part = 0.0;
            for (int i = wid; i < n; i += kSlaterThreads / 32) {
                const int ci = colmap[i];
                for (int j = lane; j < n; j += 32) part = fma(A[j * ns + ci], ld<T>(a.lap, (base + i) * O + j), part);
            }
            kin += -0.5 * block_sum(part, red);
        }
        // drift_i[c] = sum_j (A^-1)_ji d_c phi_j(r_i): one warp per (i, c)
        if (a.drift) {
            for (int ic = wid; ic < 3 * n; ic += kSlaterThreads / 32) {
                const int i = ic / 3, c = ic - (ic / 3) * 3;
                const int ci = colmap[i];
                double s = 0.0;
                for (int j = lane; j < n; j += 32)
                    s = fma(A[j * ns + ci], ld<T>(a.grad, ((base + i) * 3 + c) * O + j), s);
                for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
                if (lane == 0) a.drift[((w * a.n_elec) + e0 + i) * 3 + c] = s;
            }
        }
    }
    if (tid == 0) {
        const double nan = __longlong_as_double(0x7ff8000000000000LL);
        const double inf = __longlong_as_double(0x7ff0000000000000LL);
        if (a.logdet) a.logdet[w] = singular ? -inf : logdet;
        if (a.sign) a.sign[w] = singular ? 0.0 : sgn;
        if (a.kinetic) a.kinetic[w] = singular ? nan : kin;
    }
    if (singular && a.drift) {
        const double nan = __longlong_as_double(0x7ff8000000000000LL);
        for (int e = tid; e < 3 * a.n_elec; e += kSlaterThreads) a.drift[w * a.n_elec * 3 + e] = nan;
    }
}

// 1 / d in double-float: one Newton step on the float reciprocal, e = 1 - d y to ~2^-48.
__device__ __forceinline__ dfloat df_recip(dfloat d)
{
    const float y = 1.0f / d.h;
    const float p = __fmul_rn(d.h, y);
    const float pe = fmaf(d.h, y, -p);                  // d.h y = p + pe exactly
    const float e = __fsub_rn(__fsub_rn(__fsub_rn(1.0f, p), pe), __fmul_rn(d.l, y));
    return df_norm(y, __fmul_rn(y, e));
}

// The same computation in double-float.  Shared memory holds the matrix as two float arrays
// Ah, Al of [n][ns] with ns = n rounded up to even, plus 2 (zero padding columns stay zero
// through the elimination), so that column pairs (j, j+1) are one 8-byte word of each.
template <typename T, int NT>
__global__ void __launch_bounds__(NT, NT <= 256 ? 2 : 1) slater_df_kernel(const SlaterArgs a)
{
    extern __shared__ float fsm[];
    __shared__ double red[NT / 32];
    __shared__ int piv[kSlaterMaxBlock];
    __shared__ int colmap[kSlaterMaxBlock];
    __shared__ f32x2 fw[3][kSlaterMaxBlock];   // per row: (-f_h, -f_h), (-f_l, -f_l), (f_h, f_h)
    __shared__ __align__(8) float rkh[kSlaterMaxBlock + 2], rkl[kSlaterMaxBlock + 2];
    __shared__ int s_p;
    __shared__ float s_dh, s_dl;
    __shared__ double pivd[kSlaterMaxBlock];

    const long long w = blockIdx.x;
    if (w >= a.n_walkers) return;
    const int tid = threadIdx.x;
    const int lane = tid & 31, wid = tid >> 5;
    const long long O = a.n_orb;
    double logdet = 0.0, sgn = 1.0, kin = 0.0;
    bool singular = false;

    for (int blk = 0; blk < 2; ++blk) {
        const int e0 = blk == 0 ? 0 : a.n_up;
        const int n = blk == 0 ? a.n_up : a.n_elec - a.n_up;
        if (n == 0) continue;
        const int nw = (n + 1) & ~1;                        // columns processed, in pairs
        const int ns = nw + 2;                              // row stride (floats)
        const long long base = w * a.n_elec + e0;
        float* Ah = fsm;
        float* Al = fsm + (size_t)n * ns;

        __syncthreads();
        for (int i = wid; i < n; i += NT / 32)
            for (int j = lane; j < ns; j += 32) {
                const double v = j < n ? ld<T>(a.val, (base + i) * O + j) : 0.0;
                const dfloat x = df_from_double(v);
                Ah[i * ns + j] = x.h;
                Al[i * ns + j] = x.l;
            }
        __syncthreads();

        bool sing = false;
        for (int k = 0; k < n; ++k) {
            if (wid == 0) {
                float best = -1.0f;
                int bi = k;
                for (int i = k + lane; i < n; i += 32) {
                    const float v = fabsf(Ah[i * ns + k]);
                    if (v > best) {
                        best = v;
                        bi = i;
                    }
                }
                for (int off = 16; off > 0; off >>= 1) {
                    const float ob = __shfl_xor_sync(0xffffffffu, best, off);
                    const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
                    if (ob > best || (ob == best && oi < bi)) {
                        best = ob;
                        bi = oi;
                    }
                }
                if (lane == 0) {
                    s_p = bi;
                    s_dh = Ah[bi * ns + k];
                    s_dl = Al[bi * ns + k];
                    piv[k] = bi;
                    pivd[k] = (double)s_dh + (double)s_dl;
                }
            }
            __syncthreads();
            const int p = s_p;
            const dfloat d = {s_dh, s_dl};
            if (p != k)
                for (int j = tid; j < nw; j += NT) {
                    float t = Ah[k * ns + j];
                    Ah[k * ns + j] = Ah[p * ns + j];
                    Ah[p * ns + j] = t;
                    t = Al[k * ns + j];
                    Al[k * ns + j] = Al[p * ns + j];
                    Al[p * ns + j] = t;
                }
            __syncthreads();
            if (d.h == 0.0f) {   // exactly singular (uniform)
                sing = true;
                break;
            }
            const dfloat inv = df_recip(d);
            for (int j = tid; j < nw; j += NT) {
                const dfloat x = (j == k) ? dfloat{1.0f, 0.0f} : dfloat{Ah[k * ns + j], Al[k * ns + j]};
                const dfloat r = df_mul(x, inv);
                rkh[j] = r.h;
                rkl[j] = r.l;
                Ah[k * ns + j] = r.h;
                Al[k * ns + j] = r.l;
            }
            // pivot column of the other rows: the multipliers, packed for the update, and the
            // entries set to 0 so that the update leaves -f_i / d there (Gauss-Jordan)
            for (int i = tid; i < n; i += NT)
                if (i != k) {
                    const float fh = Ah[i * ns + k], fl = Al[i * ns + k];
                    Ah[i * ns + k] = 0.0f;
                    Al[i * ns + k] = 0.0f;
                    fw[0][i] = pack2(-fh, -fh);
                    fw[1][i] = pack2(-fl, -fl);
                    fw[2][i] = pack2(fh, fh);
                }
            __syncthreads();
            // A[i][j] += (-f_i) rowk[j], two columns per packed operation.  A lane holds two
            // column pairs of rowk in registers and updates four rows for each (eight
            // independent error-free chains), loads first, then arithmetic, then stores.
            {
                constexpr int R = 4, NW = NT / 32;
                const f32x2* rh2 = reinterpret_cast<const f32x2*>(rkh);
                const f32x2* rl2 = reinterpret_cast<const f32x2*>(rkl);
                const int np = nw / 2;
                for (int m0 = lane; m0 < np; m0 += 64) {
                    const int m1 = m0 + 32;
                    const bool v1 = m1 < np;
                    const f32x2 Bh0 = rh2[m0], Bl0 = rl2[m0];
                    const f32x2 Bh1 = v1 ? rh2[m1] : 0ull, Bl1 = v1 ? rl2[m1] : 0ull;
                    for (int ib = wid; ib < n; ib += R * NW) {
                        f32x2 Xh[2 * R], Xl[2 * R];
                        bool act[R];
#pragma unroll
                        for (int u = 0; u < R; ++u) {
                            const int i = ib + u * NW;
                            act[u] = i < n && i != k;
                            const f32x2* ph = reinterpret_cast<const f32x2*>(Ah + i * ns);
                            const f32x2* pl = reinterpret_cast<const f32x2*>(Al + i * ns);
                            Xh[2 * u] = act[u] ? ph[m0] : 0ull;
                            Xl[2 * u] = act[u] ? pl[m0] : 0ull;
                            Xh[2 * u + 1] = (act[u] && v1) ? ph[m1] : 0ull;
                            Xl[2 * u + 1] = (act[u] && v1) ? pl[m1] : 0ull;
                        }
#pragma unroll
                        for (int u = 0; u < R; ++u) {
                            const int i = ib + u * NW;
                            const int ii = act[u] ? i : 0;
                            const f32x2 wh = fw[0][ii], wl = fw[1][ii], nwh = fw[2][ii];
#pragma unroll
                            for (int q = 0; q < 2; ++q) {
                                f32x2& H = Xh[2 * u + q];
                                f32x2& Lo = Xl[2 * u + q];
                                df_fma2(H, Lo, wh, wl, nwh, q ? Bh1 : Bh0, q ? Bl1 : Bl0);
                                // renormalise (two-sum): entries are updated n times and reused
                                // as pivots, multipliers and reciprocals (|lo| << |hi| assumed)
                                const f32x2 S = add2(H, Lo);
                                const f32x2 BB = sub2(S, H);
                                Lo = add2(sub2(H, sub2(S, BB)), sub2(Lo, BB));
                                H = S;
                            }
                        }
#pragma unroll
                        for (int u = 0; u < R; ++u) {
                            const int i = ib + u * NW;
                            if (!act[u]) continue;
                            f32x2* ph = reinterpret_cast<f32x2*>(Ah + i * ns);
                            f32x2* pl = reinterpret_cast<f32x2*>(Al + i * ns);
                            ph[m0] = Xh[2 * u];
                            pl[m0] = Xl[2 * u];
                            if (v1) {
                                ph[m1] = Xh[2 * u + 1];
                                pl[m1] = Xl[2 * u + 1];
                            }
                        }
                    }
                }
            }
            __syncthreads();
        }
        if (sing) {
            singular = true;
            break;
        }
        logdet += pivot_logdet<NT>(pivd, piv, n, sgn, red);
        if (tid == 0) {
            for (int c = 0; c < n; ++c) colmap[c] = c;
            for (int k = n - 1; k >= 0; --k) {
                const int t = colmap[k];
                colmap[k] = colmap[piv[k]];
                colmap[piv[k]] = t;
            }
        }
        __syncthreads();
        // the inverse entries as doubles (h + l) for the final dot products
        if (a.kinetic) {
            double part = 0.0;
            for (int i = wid; i < n; i += NT / 32) {
                const int ci = colmap[i];
                for (int j = lane; j < n; j += 32) {
                    const double x = (double)Ah[j * ns + ci] + (double)Al[j * ns + ci];
                    part = fma(x, ld<T>(a.lap, (base + i) * O + j), part);
                }
            }
            kin += -0.5 * block_sum<NT>(part, red);
        }
        if (a.drift) {
            for (int ic = wid; ic < 3 * n; ic += NT / 32) {
                const int i = ic / 3, c = ic - (ic / 3) * 3;
                const int ci = colmap[i];
                double s = 0.0;
                for (int j = lane; j < n; j += 32) {
                    const double x = (double)Ah[j * ns + ci] + (double)Al[j * ns + ci];
                    s = fma(x, ld<T>(a.grad, ((base + i) * 3 + c) * O + j), s);
                }
                for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
                if (lane == 0) a.drift[((w * a.n_elec) + e0 + i) * 3 + c] = s;
            }
        }
    }
    if (tid == 0) {
        const double nan = __longlong_as_double(0x7ff8000000000000LL);
        const double inf = __longlong_as_double(0x7ff0000000000000LL);
        if (a.logdet) a.logdet[w] = singular ? -inf : logdet;
        if (a.sign) a.sign[w] = singular ? 0.0 : sgn;
        if (a.kinetic) a.kinetic[w] = singular ? nan : kin;
    }
    if (singular && a.drift) {
        const double nan = __longlong_as_double(0x7ff8000000000000LL);
        for (int e = tid; e < 3 * a.n_elec; e += NT) a.drift[w * a.n_elec * 3 + e] = nan;
    }
}

// ---- complex orbitals (Bloch functions, Sec. II) ----
// The same elimination on complex FP64 entries (double2), for outputs of a Bloch handle
// (complex val, grad, lap: pairs (re, im) of T).  The pivot is the entry of largest modulus;
// ln|det A| = sum_k ln|d_k| and the phase of det A is sum_k arg d_k + pi (number of row swaps),
// reported as (cos, sin).  The kinetic term and the drift are complex (Jacobi's formula).
constexpr int kSlaterCplxMaxBlock = QMCSPL_SLATER_MAX_COMPLEX_BLOCK;
// complex double-float kernel: blocks small enough for two CTAs per SM in shared memory run
// 256-thread CTAs, two per SM, so that one walker's barriers and pivot search overlap the
// other's updates (64 + 64 electrons: 15.5 -> 10.2 ms for 4,096 walkers); larger blocks run one
// 512-thread CTA per SM
constexpr int kSlaterCdfThreadsSmall = 256;
constexpr int kSlaterCdfThreadsLarge = 512;

__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}

template <typename T>
__device__ __forceinline__ double2 ldc(const void* p, long long i)   // complex element i
{
    const T* q = static_cast<const T*>(p) + 2 * i;
    return make_double2((double)__ldg(q), (double)__ldg(q + 1));
}

template <typename T>
__global__ void __launch_bounds__(kSlaterThreads) slater_complex_kernel(const SlaterArgs a)
{
    extern __shared__ double2 csm[];
    __shared__ double red[kSlaterThreads / 32];
    __shared__ int piv[kSlaterCplxMaxBlock];
    __shared__ int colmap[kSlaterCplxMaxBlock];
    __shared__ double2 fcol[kSlaterCplxMaxBlock];
    __shared__ double2 rowk[kSlaterCplxMaxBlock];
    __shared__ double2 pivd[kSlaterCplxMaxBlock];
    __shared__ int s_p;
    __shared__ double2 s_d;

    const long long w = blockIdx.x;
    if (w >= a.n_walkers) return;
    const int tid = threadIdx.x;
    const int lane = tid & 31, wid = tid >> 5;
    const long long O = a.n_orb;
    double logdet = 0.0, arg = 0.0;
    double2 kin = make_double2(0.0, 0.0);
    bool singular = false;

    for (int blk = 0; blk < 2; ++blk) {
        const int e0 = blk == 0 ? 0 : a.n_up;
        const int n = blk == 0 ? a.n_up : a.n_elec - a.n_up;
        if (n == 0) continue;
        const int ns = n + 1;
        const long long base = w * a.n_elec + e0;
        double2* A = csm;   // [n][n + 1]

        __syncthreads();
        for (int i = wid; i < n; i += kSlaterThreads / 32)
            for (int j = lane; j < n; j += 32) A[i * ns + j] = ldc<T>(a.val, (base + i) * O + j);
        __syncthreads();

        bool sing = false;
        for (int k = 0; k < n; ++k) {
            if (wid == 0) {   // pivot: largest |A[i][k]|^2 over i >= k (first one on ties)
                double best = -1.0;
                int bi = k;
                for (int i = k + lane; i < n; i += 32) {
                    const double2 z = A[i * ns + k];
                    const double v = fma(z.x, z.x, z.y * z.y);
                    if (v > best) {
                        best = v;
                        bi = i;
                    }
                }
                for (int off = 16; off > 0; off >>= 1) {
                    const double ob = __shfl_xor_sync(0xffffffffu, best, off);
                    const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
                    if (ob > best || (ob == best && oi < bi)) {
                        best = ob;
                        bi = oi;
                    }
                }
                if (lane == 0) {
                    s_p = bi;
                    s_d = A[bi * ns + k];
                    piv[k] = bi;
                    pivd[k] = s_d;
                }
            }
            __syncthreads();
            const int p = s_p;
            const double2 d = s_d;
            if (p != k)
                for (int j = tid; j < n; j += kSlaterThreads) {
                    const double2 t = A[k * ns + j];
                    A[k * ns + j] = A[p * ns + j];
                    A[p * ns + j] = t;
                }
            __syncthreads();
            if (d.x == 0.0 && d.y == 0.0) {
                sing = true;
                break;
            }
            // 1/d = conj(d) / |d|^2
            const double m2 = fma(d.x, d.x, d.y * d.y);
            const double2 inv = make_double2(d.x / m2, -d.y / m2);
            for (int j = tid; j < n; j += kSlaterThreads) {
                const double2 r = cmul(j == k ? make_double2(1.0, 0.0) : A[k * ns + j], inv);
                rowk[j] = r;
                A[k * ns + j] = r;
            }
            for (int i = tid; i < n; i += kSlaterThreads)
                if (i != k) fcol[i] = A[i * ns + k];
            __syncthreads();
            for (int i = wid; i < n; i += kSlaterThreads / 32) {
                if (i == k) continue;
                const double2 f = fcol[i];
                for (int j = lane; j < n; j += 32) {
                    const double2 x = (j == k) ? make_double2(0.0, 0.0) : A[i * ns + j];
                    const double2 r = rowk[j];
                    A[i * ns + j] = make_double2(x.x - fma(f.x, r.x, -f.y * r.y), x.y - fma(f.x, r.y, f.y * r.x));
                }
            }
            __syncthreads();
        }
        if (sing) {
            singular = true;
            break;
        }
        {   // ln|det| and the phase from the pivots and the row swaps
            double lp = 0.0, ap = 0.0;
            int swaps = 0;
            for (int k = tid; k < n; k += kSlaterThreads) {
                const double2 z = pivd[k];
                lp += 0.5 * log(fma(z.x, z.x, z.y * z.y));
                ap += atan2(z.y, z.x);
                swaps += piv[k] != k;
            }
            logdet += block_sum(lp, red);
            arg += block_sum(ap, red);
            if (((long long)block_sum((double)swaps, red)) & 1) arg += M_PI;
        }
        if (tid == 0) {
            for (int c = 0; c < n; ++c) colmap[c] = c;
            for (int k = n - 1; k >= 0; --k) {
                const int t = colmap[k];
                colmap[k] = colmap[piv[k]];
                colmap[piv[k]] = t;
            }
        }
        __syncthreads();
        if (a.kinetic) {   // T_s = -1/2 sum_ij (A^-1)_ji L_ij
            double pr = 0.0, pi = 0.0;
            for (int i = wid; i < n; i += kSlaterThreads / 32) {
                const int ci = colmap[i];
                for (int j = lane; j < n; j += 32) {
                    const double2 t = cmul(A[j * ns + ci], ldc<T>(a.lap, (base + i) * O + j));
                    pr += t.x;
                    pi += t.y;
                }
            }
            kin.x += -0.5 * block_sum(pr, red);
            kin.y += -0.5 * block_sum(pi, red);
        }
        if (a.drift) {
            for (int ic = wid; ic < 3 * n; ic += kSlaterThreads / 32) {
                const int i = ic / 3, c = ic - (ic / 3) * 3;
                const int ci = colmap[i];
                double sr = 0.0, si = 0.0;
                for (int j = lane; j < n; j += 32) {
                    const double2 t = cmul(A[j * ns + ci], ldc<T>(a.grad, ((base + i) * 3 + c) * O + j));
                    sr += t.x;
                    si += t.y;
                }
                for (int off = 16; off > 0; off >>= 1) {
                    sr += __shfl_xor_sync(0xffffffffu, sr, off);
                    si += __shfl_xor_sync(0xffffffffu, si, off);
                }
                if (lane == 0) {
                    double* q = a.drift + 2 * (((w * a.n_elec) + e0 + i) * 3 + c);
                    q[0] = sr;
                    q[1] = si;
                }
            }
        }
    }
    if (tid == 0) {
        const double nan = __longlong_as_double(0x7ff8000000000000LL);
        const double inf = __longlong_as_double(0x7ff0000000000000LL);
        if (a.logdet) a.logdet[w] = singular ? -inf : logdet;
        if (a.sign) {
            double sn, cs;
            sincos(arg, &sn, &cs);
            a.sign[2 * w] = singular ? 0.0 : cs;
            a.sign[2 * w + 1] = singular ? 0.0 : sn;
        }
        if (a.kinetic) {
            a.kinetic[2 * w] = singular ? nan : kin.x;
            a.kinetic[2 * w + 1] = singular ? nan : kin.y;
        }
    }
    if (singular && a.drift) {
        const double nan = __longlong_as_double(0x7ff8000000000000LL);
        for (int e = tid; e < 6 * a.n_elec; e += kSlaterThreads) a.drift[w * a.n_elec * 6 + e] = nan;
    }
}

// Complex entries in double-float: four float arrays Rh, Rl, Ih, Il of [n][ns] (real and
// imaginary parts, each a pair h + l), ns = n rounded up to even, plus 2, as in
// slater_df_kernel.  The update A[i][j] -= f_i r_j of a complex multiplier f and row entry r is
// four error-free packed multiply-adds (re += (-f.re) r.re + f.im r.im, im += (-f.re) r.im +
// (-f.im) r.re), renormalised; 1/d = conj(d) / |d|^2 with the double-float reciprocal.
template <typename T, int NT>
__global__ void __launch_bounds__(NT, NT <= 256 ? 2 : 1) slater_cdf_kernel(const SlaterArgs a)
{
    extern __shared__ float csf[];
    __shared__ double red[NT / 32];
    __shared__ int piv[kSlaterCplxMaxBlock];
    __shared__ int colmap[kSlaterCplxMaxBlock];
    // per row: -f.re as (wh, wl, -wh), +f.im as (wh, wl, -wh), and -f.im's low part
    __shared__ f32x2 fw[7][kSlaterCplxMaxBlock];
    __shared__ __align__(8) float rrh[kSlaterCplxMaxBlock + 2], rrl[kSlaterCplxMaxBlock + 2];
    __shared__ __align__(8) float rih[kSlaterCplxMaxBlock + 2], ril[kSlaterCplxMaxBlock + 2];
    __shared__ int s_p;
    __shared__ float s_d[4];
    __shared__ double2 pivd[kSlaterCplxMaxBlock];

    const long long w = blockIdx.x;
    if (w >= a.n_walkers) return;
    const int tid = threadIdx.x;
    const int lane = tid & 31, wid = tid >> 5;
    const long long O = a.n_orb;
    double logdet = 0.0, arg = 0.0;
    double2 kin = make_double2(0.0, 0.0);
    bool singular = false;

    for (int blk = 0; blk < 2; ++blk) {
        const int e0 = blk == 0 ? 0 : a.n_up;
        const int n = blk == 0 ? a.n_up : a.n_elec - a.n_up;
        if (n == 0) continue;
        const int nw = (n + 1) & ~1;
        const int ns = nw + 2;
        const long long base = w * a.n_elec + e0;
        const size_t plane = (size_t)n * ns;
        float* Rh = csf;
        float* Rl = csf + plane;
        float* Ih = csf + 2 * plane;
        float* Il = csf + 3 * plane;

        __syncthreads();
        for (int i = wid; i < n; i += NT / 32)
            for (int j = lane; j < ns; j += 32) {
                const double2 z = j < n ? ldc<T>(a.val, (base + i) * O + j) : make_double2(0.0, 0.0);
                const dfloat xr = df_from_double(z.x), xi = df_from_double(z.y);
                Rh[i * ns + j] = xr.h;
                Rl[i * ns + j] = xr.l;
                Ih[i * ns + j] = xi.h;
                Il[i * ns + j] = xi.l;
            }
        __syncthreads();

        bool sing = false;
        for (int k = 0; k < n; ++k) {
            if (wid == 0) {   // pivot: largest |A[i][k]|^2 (high parts) over i >= k, first on ties
                float best = -1.0f;
                int bi = k;
                for (int i = k + lane; i < n; i += 32) {
                    const float re = Rh[i * ns + k], im = Ih[i * ns + k];
                    const float v = fmaf(re, re, im * im);
                    if (v > best) {
                        best = v;
                        bi = i;
                    }
                }
                for (int off = 16; off > 0; off >>= 1) {
                    const float ob = __shfl_xor_sync(0xffffffffu, best, off);
                    const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
                    if (ob > best || (ob == best && oi < bi)) {
                        best = ob;
                        bi = oi;
                    }
                }
                if (lane == 0) {
                    s_p = bi;
                    s_d[0] = Rh[bi * ns + k];
                    s_d[1] = Rl[bi * ns + k];
                    s_d[2] = Ih[bi * ns + k];
                    s_d[3] = Il[bi * ns + k];
                    piv[k] = bi;
                    pivd[k] = make_double2((double)s_d[0] + (double)s_d[1], (double)s_d[2] + (double)s_d[3]);
                }
            }
            __syncthreads();
            const int p = s_p;
            const dfloat dr = {s_d[0], s_d[1]}, di = {s_d[2], s_d[3]};
            if (p != k)
                for (int j = tid; j < nw; j += NT) {
                    float* arr[4] = {Rh, Rl, Ih, Il};
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float t = arr[q][k * ns + j];
                        arr[q][k * ns + j] = arr[q][p * ns + j];
                        arr[q][p * ns + j] = t;
                    }
                }
            __syncthreads();
            if (dr.h == 0.0f && di.h == 0.0f) {   // exactly singular (uniform)
                sing = true;
                break;
            }
            // 1/d = (d.re - i d.im) / |d|^2
            const dfloat m2 = df_add(df_mul(dr, dr), df_mul(di, di));
            const dfloat rm = df_recip(m2);
            const dfloat ir = df_mul(dr, rm), ii = df_neg(df_mul(di, rm));
            for (int j = tid; j < nw; j += NT) {
                const dfloat xr = (j == k) ? dfloat{1.0f, 0.0f} : dfloat{Rh[k * ns + j], Rl[k * ns + j]};
                const dfloat xi = (j == k) ? dfloat{0.0f, 0.0f} : dfloat{Ih[k * ns + j], Il[k * ns + j]};
                const dfloat zr = df_add(df_mul(xr, ir), df_neg(df_mul(xi, ii)));
                const dfloat zi = df_add(df_mul(xr, ii), df_mul(xi, ir));
                rrh[j] = zr.h;
                rrl[j] = zr.l;
                rih[j] = zi.h;
                ril[j] = zi.l;
                Rh[k * ns + j] = zr.h;
                Rl[k * ns + j] = zr.l;
                Ih[k * ns + j] = zi.h;
                Il[k * ns + j] = zi.l;
            }
            // the multipliers of the other rows, packed for the update; their pivot-column
            // entries set to 0 so that the update leaves -f_i / d there (Gauss-Jordan)
            for (int i = tid; i < n; i += NT)
                if (i != k) {
                    const float frh = Rh[i * ns + k], frl = Rl[i * ns + k];
                    const float fih = Ih[i * ns + k], fil = Il[i * ns + k];
                    Rh[i * ns + k] = 0.0f;
                    Rl[i * ns + k] = 0.0f;
                    Ih[i * ns + k] = 0.0f;
                    Il[i * ns + k] = 0.0f;
                    fw[0][i] = pack2(-frh, -frh);
                    fw[1][i] = pack2(-frl, -frl);
                    fw[2][i] = pack2(frh, frh);
                    fw[3][i] = pack2(fih, fih);
                    fw[4][i] = pack2(fil, fil);
                    fw[5][i] = pack2(-fih, -fih);
                    fw[6][i] = pack2(-fil, -fil);
                }
            __syncthreads();
            {   // a lane holds one column pair of the pivot row and updates R rows
                constexpr int R = 4, NW = NT / 32;
                const f32x2* brh = reinterpret_cast<const f32x2*>(rrh);
                const f32x2* brl = reinterpret_cast<const f32x2*>(rrl);
                const f32x2* bih = reinterpret_cast<const f32x2*>(rih);
                const f32x2* bil = reinterpret_cast<const f32x2*>(ril);
                const int np = nw / 2;
                for (int m = lane; m < np; m += 32) {
                    const f32x2 Brh = brh[m], Brl = brl[m], Bih = bih[m], Bil = bil[m];
                    for (int ib = wid; ib < n; ib += R * NW) {
                        f32x2 Xrh[R], Xrl[R], Xih[R], Xil[R];
                        bool act[R];
#pragma unroll
                        for (int u = 0; u < R; ++u) {
                            const int i = ib + u * NW;
                            act[u] = i < n && i != k;
                            Xrh[u] = act[u] ? reinterpret_cast<const f32x2*>(Rh + i * ns)[m] : 0ull;
                            Xrl[u] = act[u] ? reinterpret_cast<const f32x2*>(Rl + i * ns)[m] : 0ull;
                            Xih[u] = act[u] ? reinterpret_cast<const f32x2*>(Ih + i * ns)[m] : 0ull;
                            Xil[u] = act[u] ? reinterpret_cast<const f32x2*>(Il + i * ns)[m] : 0ull;
                        }
#pragma unroll
                        for (int u = 0; u < R; ++u) {
                            const int i = ib + u * NW;
                            const int q = act[u] ? i : 0;
                            const f32x2 nrh = fw[0][q], nrl = fw[1][q], prh = fw[2][q];
                            const f32x2 pih = fw[3][q], pil = fw[4][q], nih = fw[5][q], nil = fw[6][q];
                            df_fma2(Xrh[u], Xrl[u], nrh, nrl, prh, Brh, Brl);   // re += (-f.re) r.re
                            df_fma2(Xrh[u], Xrl[u], pih, pil, nih, Bih, Bil);   // re += f.im r.im
                            df_fma2(Xih[u], Xil[u], nrh, nrl, prh, Bih, Bil);   // im += (-f.re) r.im
                            df_fma2(Xih[u], Xil[u], nih, nil, pih, Brh, Brl);   // im += (-f.im) r.re
                            // renormalise both parts (two-sum), as in slater_df_kernel
                            f32x2 S = add2(Xrh[u], Xrl[u]);
                            f32x2 BB = sub2(S, Xrh[u]);
                            Xrl[u] = add2(sub2(Xrh[u], sub2(S, BB)), sub2(Xrl[u], BB));
                            Xrh[u] = S;
                            S = add2(Xih[u], Xil[u]);
                            BB = sub2(S, Xih[u]);
                            Xil[u] = add2(sub2(Xih[u], sub2(S, BB)), sub2(Xil[u], BB));
                            Xih[u] = S;
                        }
#pragma unroll
                        for (int u = 0; u < R; ++u) {
                            const int i = ib + u * NW;
                            if (!act[u]) continue;
                            reinterpret_cast<f32x2*>(Rh + i * ns)[m] = Xrh[u];
                            reinterpret_cast<f32x2*>(Rl + i * ns)[m] = Xrl[u];
                            reinterpret_cast<f32x2*>(Ih + i * ns)[m] = Xih[u];
                            reinterpret_cast<f32x2*>(Il + i * ns)[m] = Xil[u];
                        }
                    }
                }
            }
            __syncthreads();
        }
        if (sing) {
            singular = true;
            break;
        }
        {   // ln|det| and the phase from the pivots and the row swaps
            double lp = 0.0, ap = 0.0;
            int swaps = 0;
            for (int k = tid; k < n; k += NT) {
                const double2 z = pivd[k];
                lp += 0.5 * log(fma(z.x, z.x, z.y * z.y));
                ap += atan2(z.y, z.x);
                swaps += piv[k] != k;
            }
            logdet += block_sum<NT>(lp, red);
            arg += block_sum<NT>(ap, red);
            if (((long long)block_sum<NT>((double)swaps, red)) & 1) arg += M_PI;
        }
        if (tid == 0) {
            for (int c = 0; c < n; ++c) colmap[c] = c;
            for (int k = n - 1; k >= 0; --k) {
                const int t = colmap[k];
                colmap[k] = colmap[piv[k]];
                colmap[piv[k]] = t;
            }
        }
        __syncthreads();
        // the inverse entries as complex doubles for the final dot products
        auto inv_at = [&](int j, int c) {
            return make_double2((double)Rh[j * ns + c] + (double)Rl[j * ns + c],
                                (double)Ih[j * ns + c] + (double)Il[j * ns + c]);
        };
        if (a.kinetic) {   // T_s = -1/2 sum_ij (A^-1)_ji L_ij
            double pr = 0.0, pi = 0.0;
            for (int i = wid; i < n; i += NT / 32) {
                const int ci = colmap[i];
                for (int j = lane; j < n; j += 32) {
                    const double2 t = cmul(inv_at(j, ci), ldc<T>(a.lap, (base + i) * O + j));
                    pr += t.x;
                    pi += t.y;
                }
            }
            kin.x += -0.5 * block_sum<NT>(pr, red);
            kin.y += -0.5 * block_sum<NT>(pi, red);
        }
        if (a.drift) {
            for (int ic = wid; ic < 3 * n; ic += NT / 32) {
                const int i = ic / 3, c = ic - (ic / 3) * 3;
                const int ci = colmap[i];
                double sr = 0.0, si = 0.0;
                for (int j = lane; j < n; j += 32) {
                    const double2 t = cmul(inv_at(j, ci), ldc<T>(a.grad, ((base + i) * 3 + c) * O + j));
                    sr += t.x;
                    si += t.y;
                }
                for (int off = 16; off > 0; off >>= 1) {
                    sr += __shfl_xor_sync(0xffffffffu, sr, off);
                    si += __shfl_xor_sync(0xffffffffu, si, off);
                }
                if (lane == 0) {
                    double* q = a.drift + 2 * (((w * a.n_elec) + e0 + i) * 3 + c);
                    q[0] = sr;
                    q[1] = si;
                }
            }
        }
    }
    if (tid == 0) {
        const double nan = __longlong_as_double(0x7ff8000000000000LL);
        const double inf = __longlong_as_double(0x7ff0000000000000LL);
        if (a.logdet) a.logdet[w] = singular ? -inf : logdet;
        if (a.sign) {
            double sn, cs;
            sincos(arg, &sn, &cs);
            a.sign[2 * w] = singular ? 0.0 : cs;
            a.sign[2 * w + 1] = singular ? 0.0 : sn;
        }
        if (a.kinetic) {
            a.kinetic[2 * w] = singular ? nan : kin.x;
            a.kinetic[2 * w + 1] = singular ? nan : kin.y;
        }
    }
    if (singular && a.drift) {
        const double nan = __longlong_as_double(0x7ff8000000000000LL);
        for (int e = tid; e < 6 * a.n_elec; e += NT) a.drift[w * a.n_elec * 6 + e] = nan;
    }
}

template <typename T>
int launch_slater_complex(const SlaterArgs& a, int nmax, cudaStream_t st)
{
    if (a.arith == 1) {
        const int ns = ((nmax + 1) & ~1) + 2;
        const size_t smem = 4 * (size_t)nmax * ns * sizeof(float);
        // static shared memory of the kernel is under 11 KB; 227 KB per SM
        const bool two = 2 * (smem + 11 * 1024) <= 227 * 1024;
        auto k = two ? slater_cdf_kernel<T, kSlaterCdfThreadsSmall> : slater_cdf_kernel<T, kSlaterCdfThreadsLarge>;
        const int nt = two ? kSlaterCdfThreadsSmall : kSlaterCdfThreadsLarge;
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute(slater_cdf_kernel)");
        k<<<(unsigned)a.n_walkers, nt, smem, st>>>(a);
        return cuda_error(cudaGetLastError(), "slater_cdf_kernel launch");
    }
    const size_t smem = (size_t)nmax * (nmax + 1) * sizeof(double2);
    cudaError_t e = cudaFuncSetAttribute(slater_complex_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute(slater_complex_kernel)");
    slater_complex_kernel<T><<<(unsigned)a.n_walkers, kSlaterThreads, smem, st>>>(a);
    return cuda_error(cudaGetLastError(), "slater_complex_kernel launch");
}

template <typename T>
int launch_slater(const SlaterArgs& a, int nmax, cudaStream_t st)
{
    if (a.arith == 1) {
        const int ns = ((nmax + 1) & ~1) + 2;
        const size_t smem = 2 * (size_t)nmax * ns * sizeof(float);
        // blocks that fit twice in shared memory: two 256-thread CTAs per SM, as for the
        // complex double-float kernel (static shared memory under 9 KB; 227 KB per SM)
        const bool two = 2 * (smem + 9 * 1024) <= 227 * 1024;
        auto k = two ? slater_df_kernel<T, 256> : slater_df_kernel<T, kSlaterDfThreads>;
        const int nt = two ? 256 : kSlaterDfThreads;
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute(slater_df_kernel)");
        k<<<(unsigned)a.n_walkers, nt, smem, st>>>(a);
        return cuda_error(cudaGetLastError(), "slater_df_kernel launch");
    }
    const size_t smem = (size_t)nmax * (nmax + 1) * sizeof(double);
    cudaError_t e = cudaFuncSetAttribute(slater_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute(slater_kernel)");
    slater_kernel<T><<<(unsigned)a.n_walkers, kSlaterThreads, smem, st>>>(a);
    return cuda_error(cudaGetLastError(), "slater_kernel launch");
}

}  // namespace
}  // namespace qmcspl

using namespace qmcspl;

extern "C" int qmcspl_slater_kinetic(const void* val, const void* grad, const void* lap, int dtype, int arith,
                                     long long n_walkers, int n_elec, int n_up, int n_orb, double* logdet,
                                     double* sign, double* kinetic, double* drift, void* stream)
{
    if (dtype < 0 || dtype > 3)
        return set_error(QMCSPL_ERR_ARG, "dtype must be 0 (double), 1 (float), 2 (complex double) or 3 (complex float)");
    if (arith != QMCSPL_SLATER_FP64 && arith != QMCSPL_SLATER_DF64)
        return set_error(QMCSPL_ERR_ARG, "arith must be QMCSPL_SLATER_FP64 or QMCSPL_SLATER_DF64");
    const bool cplx = dtype >= 2;
    if (n_walkers < 0) return set_error(QMCSPL_ERR_ARG, "n_walkers < 0");
    if (n_elec < 1 || n_up < 0 || n_up > n_elec) return set_error(QMCSPL_ERR_ARG, "need n_elec >= 1, 0 <= n_up <= n_elec");
    const int n_dn = n_elec - n_up;
    const int nmax = n_up > n_dn ? n_up : n_dn;
    if (nmax > (cplx ? kSlaterCplxMaxBlock : kSlaterMaxBlock))
        return set_error(QMCSPL_ERR_UNSUPPORTED, cplx ? "spin block larger than QMCSPL_SLATER_MAX_COMPLEX_BLOCK"
                                                      : "spin block larger than QMCSPL_SLATER_MAX_BLOCK");
    if (n_orb < nmax) return set_error(QMCSPL_ERR_ARG, "n_orb (the output row length) is smaller than a spin block");
    if (!val) return set_error(QMCSPL_ERR_ARG, "val is NULL");
    if (kinetic && !lap) return set_error(QMCSPL_ERR_ARG, "kinetic needs lap");
    if (drift && !grad) return set_error(QMCSPL_ERR_ARG, "drift needs grad");
    if (n_walkers > 0x7fffffffLL) return set_error(QMCSPL_ERR_ARG, "n_walkers too large");
    if (n_walkers == 0) return QMCSPL_OK;
    SlaterArgs a;
    a.val = val;
    a.grad = grad;
    a.lap = lap;
    a.n_walkers = n_walkers;
    a.n_elec = n_elec;
    a.n_up = n_up;
    a.n_orb = n_orb;
    a.logdet = logdet;
    a.sign = sign;
    a.kinetic = kinetic;
    a.drift = drift;
    a.arith = arith;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    switch (dtype) {
    case 0: return launch_slater<double>(a, nmax, st);
    case 1: return launch_slater<float>(a, nmax, st);
    case 2: return launch_slater_complex<double>(a, nmax, st);
    default: return launch_slater_complex<float>(a, nmax, st);
    }
}
