// order.cu -- per-position preparation before evaluation (not in the paper).
//
// 1. Coordinate records.  Eq. (reducedcoordinate) needs more than FP32 (an FP32 product N*s
//    loses ~N*6e-8 of t), and GB300 runs FP64 at a small fraction of its FP32 rate: the
//    records of float and bfloat16 tables (kind 1) are reduced in double-float arithmetic
//    on the FP32 pipe (reduce_axis_df, about 48 bits), the others in FP64.
//    Inside the evaluation kernels a group of lanes shares one position, so a warp-wide
//    FP64 instruction there serves one position; here one thread reduces one position,
//    so the same instruction serves 32.  The result (grid cell and t, see
//    record_kind) is read by the evaluation kernels, which then do no FP64 work.
// 2. Cell order.  Each position's stencil touches 4 x 4 x 4 grid points; positions in
//    nearby grid cells share most of them.  Evaluating the positions grouped by cell
//    lets those shared rows be served by L1/L2 instead of HBM.  The order is a counting
//    sort of the positions into bins of edge^3 grid cells, bins swept x-major (z
//    fastest), so the warps resident on the GPU at any moment cover a compact slab of
//    the cell.  Within a bin the order is whatever the atomics give; it does not change
//    any result, since each position is computed the same way and written to its own
//    output rows.
// 3. Bloch phase factors (Sec. II, phi = u exp(i k.r)).  exp(i k.r) at the unwrapped
//    position, in FP64, once per position, for the evaluation epilogues.
#include "eval_common.cuh"
#include "general_basis.cuh"

namespace qmcspl {
namespace {

#ifndef QMCSPL_BIN_EDGE
#define QMCSPL_BIN_EDGE 4      // grid cells per bin edge (a bin is edge^3 cells)
#endif
constexpr int kScanThreads = 1024;

struct PrepArgs {
    const double* pos;
    long long n;
    double ainv[9];
    float ainv_h[9], ainv_l[9];   // a^-1 as double-float pairs (records of kind 1)
    int dims[3];
    int edge[3];              // grid cells per bin edge, per axis
    int nb[3];
    void* rec;                // records (kind 1, 2 or 3), may be null
    double2* phase;           // Bloch phase factors, may be null
    const double* knots;      // non-uniform grids: [3][kMaxDim] grid points (record kinds 4, 5)
    double kred[3];           // a^-T kpoint: k.r = 2 pi (kred . r)
    int* bin;                 // per-position bin (with count)
    int* count;               // bin counters, null: no binning
};

// Reduce position i; the same arithmetic as reduced_coordinates() in the kernels.
__device__ __forceinline__ void reduce_position(const PrepArgs& a, long long i, int& ix, int& iy, int& iz,
                                                double& tx, double& ty, double& tz, bool& ok)
{
    const double r[3] = {a.pos[3 * i], a.pos[3 * i + 1], a.pos[3 * i + 2]};
    bool o0, o1, o2;
    reduce_axis(crystal(a.ainv[0], a.ainv[1], a.ainv[2], r), a.dims[0], ix, tx, o0);
    reduce_axis(crystal(a.ainv[3], a.ainv[4], a.ainv[5], r), a.dims[1], iy, ty, o1);
    reduce_axis(crystal(a.ainv[6], a.ainv[7], a.ainv[8], r), a.dims[2], iz, tz, o2);
    ok = o0 && o1 && o2;
}

// Float records (kind 1): the double-float steps of the float kernels' own reduction
// (reduced_coordinates_df), so that a record holds the bits those kernels would compute.
__device__ __forceinline__ void reduce_position_df(const PrepArgs& a, long long i, int& ix, int& iy, int& iz,
                                                   float& tx, float& ty, float& tz, bool& ok)
{
    const double r[3] = {a.pos[3 * i], a.pos[3 * i + 1], a.pos[3 * i + 2]};
    float rh[3], rl[3];
    df_row(r, rh, rl);
    bool o0, o1, o2;
    reduce_axis_df(r, rh, rl, a.ainv, a.ainv_h, a.ainv_l, a.dims[0], ix, tx, o0);
    reduce_axis_df(r, rh, rl, a.ainv + 3, a.ainv_h + 3, a.ainv_l + 3, a.dims[1], iy, ty, o1);
    reduce_axis_df(r, rh, rl, a.ainv + 6, a.ainv_h + 6, a.ainv_l + 6, a.dims[2], iz, tz, o2);
    ok = o0 && o1 && o2;
}

// Non-uniform grids: per axis the interval of the grid points that holds the position and
// the offset from its left point (reduced units).
__device__ __forceinline__ void locate_position(const PrepArgs& a, long long i, int& ix, int& iy, int& iz,
                                                double& tx, double& ty, double& tz, bool& ok)
{
    const double r[3] = {a.pos[3 * i], a.pos[3 * i + 1], a.pos[3 * i + 2]};
    int c[3];
    double d[3];
    ok = true;
    for (int ax = 0; ax < 3; ++ax) {
        const double s = crystal(a.ainv[3 * ax], a.ainv[3 * ax + 1], a.ainv[3 * ax + 2], r);
        double f = s - floor(s);
        const bool o = isfinite(f);
        ok = ok && o;
        if (o) {
            const double* kn = a.knots + ax * kMaxDim;
            c[ax] = knot_interval(kn, a.dims[ax], f);
            d[ax] = f - kn[c[ax]];
        } else {
            c[ax] = 0;
            d[ax] = __longlong_as_double(0x7ff8000000000000LL);
        }
    }
    ix = c[0];
    iy = c[1];
    iz = c[2];
    tx = d[0];
    ty = d[1];
    tz = d[2];
}

template <int KIND>
__global__ void prepare_kernel(const PrepArgs a)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    int ix, iy, iz;
    double tx = 0.0, ty = 0.0, tz = 0.0;
    float fx = 0.f, fy = 0.f, fz = 0.f;
    bool ok;
    // kinds 4, 5 and binning alone (kind 0) on a non-uniform grid: the grid interval that holds
    // the position, so that bins group positions by the knot intervals they evaluate in
    if (KIND >= 4 || (KIND == 0 && a.knots)) locate_position(a, i, ix, iy, iz, tx, ty, tz, ok);
    else if (KIND == 1) reduce_position_df(a, i, ix, iy, iz, fx, fy, fz, ok);
    else reduce_position(a, i, ix, iy, iz, tx, ty, tz, ok);
    const int cell = ok ? (ix | (iy << 10) | (iz << 20)) : -1;
    if (KIND == 1) {
        static_cast<float4*>(a.rec)[i] = make_float4(__int_as_float(cell), fx, fy, fz);
    } else if (KIND == 4) {
        static_cast<float4*>(a.rec)[i] = make_float4(__int_as_float(cell), (float)tx, (float)ty, (float)tz);
    } else if (KIND == 2 || KIND == 5) {
        double2* q = static_cast<double2*>(a.rec) + 2 * i;
        q[0] = make_double2(tx, ty);
        q[1] = make_double2(tz, __hiloint2double(0, cell));
    } else if (KIND == 3) {
        const dfloat x = df_from_double(tx), y = df_from_double(ty), z = df_from_double(tz);
        float4* q = static_cast<float4*>(a.rec) + 2 * i;
        q[0] = make_float4(__int_as_float(cell), x.h, x.l, y.h);
        q[1] = make_float4(y.l, z.h, z.l, 0.0f);
    }
    if (a.phase) {
        // k.r / (2 pi) = kred . r; only its fractional part matters
        const double* r = a.pos + 3 * i;
        const double u = __fma_rn(a.kred[0], r[0], __fma_rn(a.kred[1], r[1], __dmul_rn(a.kred[2], r[2])));
        const double f = u - rint(u);
        double sn, cs;
        sincospi(2.0 * f, &sn, &cs);
        a.phase[i] = make_double2(cs, sn);
    }
    if (a.count) {
        const int b = ((ix / a.edge[0]) * a.nb[1] + iy / a.edge[1]) * a.nb[2] + iz / a.edge[2];
        a.bin[i] = b;
        atomicAdd(a.count + b, 1);
    }
}

// In-place exclusive scan of count[0 .. n) by one block; count[n] receives the total.
// Each warp owns one contiguous segment and walks it 32 entries at a time (coalesced):
// first the segment sums, then, from the block-wide prefix of those, the scan itself.
__global__ void __launch_bounds__(kScanThreads) scan_kernel(int* count, int n)
{
    constexpr int kWarps = kScanThreads / 32;
    __shared__ int seg_sum[kWarps];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int per = ((n + kScanThreads - 1) / kScanThreads) * 32;   // a multiple of 32
    const int lo = min(wid * per, n), hi = min(lo + per, n);
    int s = 0;
#pragma unroll 4
    for (int i = lo + lane; i < hi; i += 32) s += count[i];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) seg_sum[wid] = s;
    __syncthreads();
    if (wid == 0) {
        const int v = seg_sum[lane];
        int incl = v;
        for (int off = 1; off < 32; off <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += u;
        }
        seg_sum[lane] = incl - v;   // exclusive over segments
        if (lane == 31) count[n] = incl;
    }
    __syncthreads();
    int carry = seg_sum[wid];
    for (int base = lo; base < hi; base += 32) {
        const int i = base + lane;
        const int c = i < hi ? count[i] : 0;
        int incl = c;
        for (int off = 1; off < 32; off <<= 1) {
            const int u = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += u;
        }
        if (i < hi) count[i] = carry + incl - c;
        carry += __shfl_sync(0xffffffffu, incl, 31);
    }
}

__global__ void place_kernel(const int* bin, long long n, int* offset, int* perm)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int slot = atomicAdd(offset + bin[i], 1);
    perm[slot] = (int)i;
}

PrepArgs prep_args(const Handle* h, const double* pos, long long n, void* rec, double2* phase, int* bin,
                   int* count, const BinGeometry* g)
{
    PrepArgs a;
    a.pos = pos;
    a.n = n;
    a.phase = phase;
    a.knots = h->nonuniform ? h->d_knots : nullptr;
    for (int i = 0; i < 3; ++i) a.kred[i] = h->kred[i];
    for (int i = 0; i < 9; ++i) {
        a.ainv[i] = h->ainv[i];
        a.ainv_h[i] = (float)h->ainv[i];
        a.ainv_l[i] = (float)(h->ainv[i] - (double)a.ainv_h[i]);
    }
    for (int i = 0; i < 3; ++i) {
        a.dims[i] = h->dims[i];
        a.nb[i] = g ? g->nb[i] : 1;
        a.edge[i] = g ? g->edge[i] : 1;
    }
    a.rec = rec;
    a.bin = bin;
    a.count = count;
    return a;
}

int launch_prepare(const PrepArgs& a, int kind, cudaStream_t st)
{
    const unsigned blocks = (unsigned)((a.n + 255) / 256);
    switch (kind) {
    case 1: prepare_kernel<1><<<blocks, 256, 0, st>>>(a); break;
    case 2: prepare_kernel<2><<<blocks, 256, 0, st>>>(a); break;
    case 3: prepare_kernel<3><<<blocks, 256, 0, st>>>(a); break;
    case 4: prepare_kernel<4><<<blocks, 256, 0, st>>>(a); break;
    case 5: prepare_kernel<5><<<blocks, 256, 0, st>>>(a); break;
    default: prepare_kernel<0><<<blocks, 256, 0, st>>>(a); break;
    }
    return cuda_error(cudaGetLastError(), "prepare_kernel launch");
}

}  // namespace

BinGeometry bin_geometry(const Handle* h)
{
    BinGeometry g;
    int edge = QMCSPL_BIN_EDGE;
    for (;;) {
        long long nb = 1;
        for (int a = 0; a < 3; ++a) {
            g.edge[a] = edge;
            g.nb[a] = (h->dims[a] + edge - 1) / edge;
            nb *= g.nb[a];
        }
        if (nb <= kMaxBins) {
            g.n_bins = (int)nb;
            return g;
        }
        edge *= 2;
    }
}

// QMCSPL_ORDER_AUTO.  Cell order costs three short kernels (bin counts, scan, placement) and pays
// back through the L1 reuse of stencil rows among neighbouring positions.  A table larger than L2
// is re-read from HBM in input order, and sorting wins from 8192 positions on.  A table that fits
// in L2 is gathered from there in input order too, so sorting pays only once enough positions
// share each bin of cells -- the fewer, the more of L2 the table takes.  Break-even points
// measured on GB300 (FP32 tables with the Laplacian table, 16 to 128 orbitals, 48^3 to 96^3
// grids): about 170 positions per 4^3-cell bin for a table filling 11% of L2, 25 to 30 at 45 to
// 50%, 7 at 75%; tables of 400 MB and more (3 to 7 times L2) were faster sorted from 8192.
bool use_cell_order(const Handle* h, long long n_pos)
{
    if (n_pos >= (1LL << 31) - 1) return false;
    switch (h->order_mode) {
    case QMCSPL_ORDER_INPUT: return false;
    case QMCSPL_ORDER_CELL:
    case QMCSPL_ORDER_PENCIL: return true;   // pencil order where staged evaluation does not apply
    default: {
        if (n_pos < 8192) return false;
        const double share = (double)h->table_elems * h->elem_bytes * h->n_tables / (double)l2_cache_bytes();
        if (share > 1.0) return true;
        const double per_bin = (double)n_pos / bin_geometry(h).n_bins;
        return per_bin >= (share > 0.6 ? 8.0 : share > 0.3 ? 32.0 : 192.0);
    }
    }
}

int record_kind(const Handle* h)
{
    if (h->nonuniform) return h->storage == QMCSPL_F64 ? 5 : 4;
    if (h->storage == QMCSPL_DF64) return 3;
    if (h->storage == QMCSPL_F64) return 2;
    return 1;
}

int build_records(const Handle* h, const double* pos, long long n_pos, void* rec, double2* phase, int* bin,
                  int* count, const BinGeometry* g, cudaStream_t st)
{
    if (count) {
        cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int) * (size_t)(g->n_bins + 1), st);
        if (e != cudaSuccess) return cuda_error(e, "cudaMemsetAsync(bin counts)");
    }
    return launch_prepare(prep_args(h, pos, n_pos, rec, phase, bin, count, g), rec ? record_kind(h) : 0, st);
}

// Cell order without records (the positions are reduced again by the evaluation kernel).
int build_cell_order(const Handle* h, const double* pos, long long n_pos, int* bin, int* count,
                     int* perm, const BinGeometry& g, cudaStream_t st)
{
    int rc = build_records(h, pos, n_pos, nullptr, nullptr, bin, count, &g, st);
    if (rc != QMCSPL_OK) return rc;
    const unsigned blocks = (unsigned)((n_pos + 255) / 256);
    scan_kernel<<<1, kScanThreads, 0, st>>>(count, g.n_bins);
    place_kernel<<<blocks, 256, 0, st>>>(bin, n_pos, count, perm);
    return cuda_error(cudaGetLastError(), "cell-order kernels");
}

static int grow_scratch(Handle* h, long long n_pos, int n_bins)
{
    if (n_pos <= h->ord_cap && n_bins + 1 <= h->ord_nbins) return QMCSPL_OK;
    // cudaFree waits for kernels that may still read the old arrays
    const long long cap = n_pos > h->ord_cap ? n_pos : h->ord_cap;
    const int nb = n_bins + 1 > h->ord_nbins ? n_bins + 1 : h->ord_nbins;
    if (h->ord_bin) cudaFree(h->ord_bin);
    if (h->ord_perm) cudaFree(h->ord_perm);
    if (h->ord_count) cudaFree(h->ord_count);
    if (h->ord_rec) cudaFree(h->ord_rec);
    if (h->ord_phase) cudaFree(h->ord_phase);
    h->ord_bin = h->ord_perm = h->ord_count = nullptr;
    h->ord_rec = nullptr;
    h->ord_phase = nullptr;
    h->ord_cap = 0;
    h->ord_nbins = 0;
    cudaError_t e = dev_malloc((void**)&h->ord_bin, sizeof(int) * (size_t)cap);
    if (e == cudaSuccess) e = dev_malloc((void**)&h->ord_perm, sizeof(int) * (size_t)cap);
    if (e == cudaSuccess) e = dev_malloc((void**)&h->ord_count, sizeof(int) * (size_t)nb);
    if (e == cudaSuccess) e = dev_malloc(&h->ord_rec, 32 * (size_t)cap);
    if (e == cudaSuccess && h->bloch) e = dev_malloc((void**)&h->ord_phase, sizeof(double2) * (size_t)cap);
    if (e != cudaSuccess) return cuda_error(e, "cudaMalloc(position scratch)");
    h->ord_cap = cap;
    h->ord_nbins = nb;
    return QMCSPL_OK;
}

int prepare_positions(Handle* h, const double* pos, long long n_pos, bool sort, Prepared* out,
                      cudaStream_t st, const BinGeometry* geom)
{
    const BinGeometry g = geom ? *geom : bin_geometry(h);
    int rc = grow_scratch(h, n_pos, g.n_bins);
    if (rc != QMCSPL_OK) return rc;
    out->rec = h->ord_rec;
    out->perm = nullptr;
    out->phase = h->bloch ? h->ord_phase : nullptr;
    double2* phase = h->bloch ? h->ord_phase : nullptr;
    if (!sort) return build_records(h, pos, n_pos, h->ord_rec, phase, nullptr, nullptr, nullptr, st);
    rc = build_records(h, pos, n_pos, h->ord_rec, phase, h->ord_bin, h->ord_count, &g, st);
    if (rc != QMCSPL_OK) return rc;
    const unsigned blocks = (unsigned)((n_pos + 255) / 256);
    scan_kernel<<<1, kScanThreads, 0, st>>>(h->ord_count, g.n_bins);
    place_kernel<<<blocks, 256, 0, st>>>(h->ord_bin, n_pos, h->ord_count, h->ord_perm);
    out->perm = h->ord_perm;
    out->bin_end = h->ord_count;
    return cuda_error(cudaGetLastError(), "cell-order kernels");
}

}  // namespace qmcspl
