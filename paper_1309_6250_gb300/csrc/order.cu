// order.cu -- cell ordering of positions (not in the paper; a memory-locality step).
//
// Each position's stencil touches 4 x 4 x 4 grid points; positions in nearby grid cells
// share most of them.  Evaluating the positions grouped by cell lets those shared rows
// be served by L1/L2 instead of HBM.  The order is a counting sort of the positions
// into bins of `edge`^3 grid cells, bins swept x-major (z fastest), so the warps
// resident on the GPU at any moment cover a compact slab of the cell.  Within a bin
// the order is whatever the atomics give; it does not change any result, since each
// position is computed the same way and written to its own output rows.
#include "qmcspl_internal.cuh"

namespace qmcspl {
namespace {

#ifndef QMCSPL_BIN_EDGE
#define QMCSPL_BIN_EDGE 4      // grid cells per bin edge (a bin is edge^3 cells)
#endif
constexpr int kMaxBins = 1 << 16;
constexpr int kScanThreads = 1024;

__device__ __forceinline__ int cell_index(double s, int N)
{
    const double f = s - floor(s);
    if (!isfinite(f)) return 0;
    int k = (int)floor((double)N * f);
    return k >= N ? k - N : (k < 0 ? 0 : k);
}

struct BinArgs {
    const double* pos;
    long long n;
    double ainv[9];
    int dims[3];
    int edge;
    int nb[3];
    int* bin;
    int* count;
};

__global__ void bin_kernel(const BinArgs a)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    const double r0 = a.pos[3 * i], r1 = a.pos[3 * i + 1], r2 = a.pos[3 * i + 2];
    const int ix = cell_index(a.ainv[0] * r0 + a.ainv[1] * r1 + a.ainv[2] * r2, a.dims[0]);
    const int iy = cell_index(a.ainv[3] * r0 + a.ainv[4] * r1 + a.ainv[5] * r2, a.dims[1]);
    const int iz = cell_index(a.ainv[6] * r0 + a.ainv[7] * r1 + a.ainv[8] * r2, a.dims[2]);
    const int b = ((ix / a.edge) * a.nb[1] + iy / a.edge) * a.nb[2] + iz / a.edge;
    a.bin[i] = b;
    atomicAdd(a.count + b, 1);
}

// In-place exclusive scan of count[0 .. n) by one block; count[n] receives the total.
__global__ void __launch_bounds__(kScanThreads) scan_kernel(int* count, int n)
{
    __shared__ int warp_sum[kScanThreads / 32];
    const int per = (n + kScanThreads - 1) / kScanThreads;
    const int lo = threadIdx.x * per;
    const int hi = min(lo + per, n);
    int s = 0;
    for (int i = lo; i < hi; ++i) s += count[i];
    // block-wide exclusive scan of the per-thread sums
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = s;
    for (int off = 1; off < 32; off <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += v;
    }
    if (lane == 31) warp_sum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int w = warp_sum[lane];
        for (int off = 1; off < 32; off <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, w, off);
            if (lane >= off) w += v;
        }
        warp_sum[lane] = w;   // inclusive over warps
    }
    __syncthreads();
    int run = incl - s + (wid > 0 ? warp_sum[wid - 1] : 0);
    for (int i = lo; i < hi; ++i) {
        const int c = count[i];
        count[i] = run;
        run += c;
    }
    if (threadIdx.x == kScanThreads - 1) count[n] = run;
}

__global__ void place_kernel(const int* bin, long long n, int* offset, int* perm)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int slot = atomicAdd(offset + bin[i], 1);
    perm[slot] = (int)i;
}

}  // namespace

BinGeometry bin_geometry(const Handle* h)
{
    BinGeometry g;
    g.edge = QMCSPL_BIN_EDGE;
    for (;;) {
        long long nb = 1;
        for (int a = 0; a < 3; ++a) {
            g.nb[a] = (h->dims[a] + g.edge - 1) / g.edge;
            nb *= g.nb[a];
        }
        if (nb <= kMaxBins) {
            g.n_bins = (int)nb;
            return g;
        }
        g.edge *= 2;
    }
}

bool use_cell_order(const Handle* h, long long n_pos)
{
    if (n_pos >= (1LL << 31) - 1) return false;
    switch (h->order_mode) {
    case QMCSPL_ORDER_INPUT: return false;
    case QMCSPL_ORDER_CELL: return true;
    default: return n_pos >= 8192;
    }
}

int build_cell_order(const Handle* h, const double* pos, long long n_pos, int* bin, int* count,
                     int* perm, const BinGeometry& g, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int) * (size_t)(g.n_bins + 1), st);
    if (e != cudaSuccess) return cuda_error(e, "cudaMemsetAsync(bin counts)");
    BinArgs a;
    a.pos = pos;
    a.n = n_pos;
    for (int i = 0; i < 9; ++i) a.ainv[i] = h->ainv[i];
    for (int i = 0; i < 3; ++i) {
        a.dims[i] = h->dims[i];
        a.nb[i] = g.nb[i];
    }
    a.edge = g.edge;
    a.bin = bin;
    a.count = count;
    const unsigned blocks = (unsigned)((n_pos + 255) / 256);
    bin_kernel<<<blocks, 256, 0, st>>>(a);
    scan_kernel<<<1, kScanThreads, 0, st>>>(count, g.n_bins);
    place_kernel<<<blocks, 256, 0, st>>>(bin, n_pos, count, perm);
    return cuda_error(cudaGetLastError(), "cell-order kernels");
}

int cell_order(Handle* h, const double* pos, long long n_pos, const int** perm, cudaStream_t st)
{
    const BinGeometry g = bin_geometry(h);
    if (n_pos > h->ord_cap || g.n_bins + 1 > h->ord_nbins) {
        // grow the scratch; cudaFree waits for kernels that may still read the old arrays
        if (h->ord_bin) cudaFree(h->ord_bin);
        if (h->ord_perm) cudaFree(h->ord_perm);
        if (h->ord_count) cudaFree(h->ord_count);
        h->ord_bin = h->ord_perm = h->ord_count = nullptr;
        h->ord_cap = 0;
        h->ord_nbins = 0;
        const long long cap = n_pos > h->ord_cap ? n_pos : h->ord_cap;
        cudaError_t e = cudaMalloc((void**)&h->ord_bin, sizeof(int) * (size_t)cap);
        if (e == cudaSuccess) e = cudaMalloc((void**)&h->ord_perm, sizeof(int) * (size_t)cap);
        if (e == cudaSuccess) e = cudaMalloc((void**)&h->ord_count, sizeof(int) * (size_t)(g.n_bins + 1));
        if (e != cudaSuccess) return cuda_error(e, "cudaMalloc(cell-order scratch)");
        h->ord_cap = cap;
        h->ord_nbins = g.n_bins + 1;
    }
    const int rc = build_cell_order(h, pos, n_pos, h->ord_bin, h->ord_count, h->ord_perm, g, st);
    *perm = h->ord_perm;
    return rc;
}

}  // namespace qmcspl
