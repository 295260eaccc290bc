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
// The elimination is n^3 FP64 FMAs per block (2.1 M for n = 128), so this consumer runs on
// GB300's FP64 pipe; every loop is bounded by n.
#include <cmath>

#include "qmcspl_internal.cuh"

namespace qmcspl {
namespace {

constexpr int kSlaterThreads = 256;
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
};

template <typename T>
__device__ __forceinline__ double ld(const void* p, long long i)
{
    return (double)__ldg(static_cast<const T*>(p) + i);
}

// Block-wide sum of one double per thread; every thread gets the total.
__device__ double block_sum(double v, double* red)
{
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < kSlaterThreads / 32; ++w) t += red[w];
    return t;
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
            logdet += log(fabs(d));
            if (d < 0.0) sgn = -sgn;
            if (p != k) sgn = -sgn;
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

}  // namespace
}  // namespace qmcspl

using namespace qmcspl;

extern "C" int qmcspl_slater_kinetic(const void* val, const void* grad, const void* lap, int dtype,
                                     long long n_walkers, int n_elec, int n_up, int n_orb, double* logdet,
                                     double* sign, double* kinetic, double* drift, void* stream)
{
    if (dtype != 0 && dtype != 1) return set_error(QMCSPL_ERR_ARG, "dtype must be 0 (double) or 1 (float)");
    if (n_walkers < 0) return set_error(QMCSPL_ERR_ARG, "n_walkers < 0");
    if (n_elec < 1 || n_up < 0 || n_up > n_elec) return set_error(QMCSPL_ERR_ARG, "need n_elec >= 1, 0 <= n_up <= n_elec");
    const int n_dn = n_elec - n_up;
    const int nmax = n_up > n_dn ? n_up : n_dn;
    if (nmax > kSlaterMaxBlock)
        return set_error(QMCSPL_ERR_UNSUPPORTED, "spin block larger than QMCSPL_SLATER_MAX_BLOCK");
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
    const size_t smem = (size_t)nmax * (nmax + 1) * sizeof(double);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (dtype == 0) {
        e = cudaFuncSetAttribute(slater_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute(slater_kernel)");
        slater_kernel<double><<<(unsigned)n_walkers, kSlaterThreads, smem, st>>>(a);
    } else {
        e = cudaFuncSetAttribute(slater_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute(slater_kernel)");
        slater_kernel<float><<<(unsigned)n_walkers, kSlaterThreads, smem, st>>>(a);
    }
    return cuda_error(cudaGetLastError(), "slater_kernel launch");
}
