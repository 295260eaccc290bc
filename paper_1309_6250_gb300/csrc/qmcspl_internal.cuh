// qmcspl_internal.cuh -- private declarations of the qmcspl CUDA library.
//
// Stored table layout (all methods), orbital-innermost so that one position's stencil
// is a handful of long contiguous runs:
//
//   B-spline, Lagrange:  T[x][y][zz][O_p],     zz = z + 1, z in [-1, Nz + 1]
//   pp-spline:           T[x][y][zz][8][O_p],  zz = z,     z in [0, Nz]
//
// The z ghost planes repeat planes Nz-1, 0 and 1 (pp: plane 0), so the four (two)
// z rows of a stencil column are contiguous and only x and y need a periodic wrap.
// O_p pads the orbital count so that each row is a whole number of 16-byte chunks
// split evenly over the lanes that share a position.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>

#include "../../include/qmcspl.h"

struct qmcspl_s;

namespace qmcspl {

using Handle = ::qmcspl_s;

constexpr int kMaxDim = 512;          // grid points per axis accepted by qmcspl_create
constexpr int kEvalThreads = 256;     // eval kernels: 8 warps per block
constexpr int kProfCalls = 4096;      // calls qmcspl_profile can record
constexpr long long kRecordMinPositions = 8192;   // from here on positions are reduced in a pass of their own
constexpr int kMaxBins = 1 << 16;     // cell-order bins: bin_geometry widens the bins to stay within this

// Per-planewave multiplier of a table sum (construct.cu) = basis factor x derivative
// factor.  For Bloch orbitals every G in a derivative factor stands for k + G.
enum BuildBasis : int {
    kBasisSmooth = 0,        // 1 / gamma_G                       (smoothing B-spline)
    kBasisInterp = 1,        // 1 / prod(1 + cos(th)/2)           (interpolating B-spline)
    kBasisGrid = 2,          // 1                                 (grid values: Lagrange)
    kBasisPP = 3,            // prod over label-2 axes of 6(cos th - 1)/(2 + cos th)
    kBasisInterpN = 4,       // 1 / prod S_n(th), S_n = sum_m C_n B_n(m) e^{i m th}: interpolating
                             // B-spline of odd degree n on a uniform grid
    kBasisSmoothN = 5,       // 1 / prod C_n sinc^{n+1}(th/2): smoothing B-spline of odd degree n
};
enum BuildDeriv : int {
    kDerivValue = 0,         // 1          (phi)
    kDerivX = 1,             // i G_x      (d_x phi)
    kDerivY = 2,             // i G_y
    kDerivZ = 3,             // i G_z
    kDerivLap = 4,           // -|G|^2     (lap phi)
};

// Eval parameters shared by the B-spline, Lagrange and pp kernels (passed by value).
struct EvalArgs {
    const void* tab[5];       // tables (B-spline: value[, Laplacian]; five-table: phi, d_x, d_y,
                              // d_z, lap phi; pp: 1)
    long long col_stride;     // elements between successive (x, y) columns
    int row_stride;           // elements between successive z rows (O_p, or 8 O_p for pp)
    int nx, ny, nz;
    int n_orb;
    int lanes_log2;           // lanes sharing one position
    int tiles;                // orbital tiles per position
    double ainv[9];           // s = a^-1 r (row-major)
    double mg[9];             // grad_cart[a] = sum_i mg[3a+i] grad_t[i]
    double ml[6];             // lap = ml0 Hxx + ml1 Hyy + ml2 Hzz + ml3 Hxy + ml4 Hxz + ml5 Hyz
    float mgf[9], mlf[6];     // the same rounded to float (float kernels)
    float mgh[9], mgl[9];     // double-float split of mg: mg = mgh + mgl
    float mlh[6], mll[6];     // double-float split of ml
    const double* pos;
    const void* rec;          // per-position coordinate records (null: compute from pos), see order.cu
    const int* perm;          // evaluation order: position perm[i] is the i-th evaluated (null: input order)
    long long n_pos;
    void* val;
    void* grad;
    void* lap;
    int vec_out;              // outputs may use 16-byte vector stores
    int* err;                 // device error word (bit 0: non-finite position)
    // Bloch orbitals (Sec. II): the n_orb stored functions are Re u, Im u of n_orb / 2
    // complex orbitals; phase[ip] = (cos k.r, sin k.r) at the unwrapped position
    const double2* phase;     // null: real orbitals
    double kc[3];             // Cartesian k (1/bohr)
    float kcf[3];
    double kred[3];           // a^-T kpoint: k.r = 2 pi (kred . r)
    // general B-splines (degree other than 3, or non-uniform grids)
    const double* knots[3];   // per-axis grid points in [0, 1) (non-uniform grids), else null
    double cdeg;              // degree-0 constant C of the recurrence
    const char* tab_lo;       // the handle's table allocation [tab_lo, tab_hi): every table
    const char* tab_hi;       // load is checked against it in QMCSPL_DEBUG_BOUNDS builds
};

}  // namespace qmcspl

// The handle behind the opaque qmcspl_t of the C ABI.
struct qmcspl_s {
    int device = 0;
    int method = 0, storage = 0, separate_lap = 0;
    int separate_grad = 0;    // B-splines: tables of d_x, d_y, d_z phi too (five tables)
    int degree = 3;           // odd B-spline degree (interpolating B-splines may use 1, 3, 5, 7)
    int nonuniform = 0;       // 1: per-axis grid points (cubic interpolating B-splines)
    int zshift = 1;           // ghost planes below z = 0: (degree - 1) / 2 (pp: 0)
    double* d_knots = nullptr;            // device: grid points [3][kMaxDim], their periodic
                                          // spacings [3][kMaxDim] (double), then as float
    double knots[3][qmcspl::kMaxDim];     // host copy (non-uniform grids)
    int dims[3] = {0, 0, 0};
    int n_orb = 0, n_orb_p = 0;   // stored real functions per row (2 per orbital when bloch)
    int n_tables = 0;
    int entries = 1;          // 8 for pp
    int rows_z = 0;
    int lanes_log2 = 0, tiles = 1;
    long long n_pw = 0;
    int bloch = 0;            // complex Bloch orbitals: phi = u exp(i k.r)
    double kpoint[3] = {0.0, 0.0, 0.0};   // k in units of the reciprocal vectors
    double kcart[3] = {0.0, 0.0, 0.0};    // Cartesian k = 2 pi a^-T kpoint
    double kred[3] = {0.0, 0.0, 0.0};     // a^-T kpoint: k.r = 2 pi (kred . r)
    double lattice[9];
    double ainv[9];
    double mg[9];
    double ml[6];
    size_t elem_bytes = 4;
    size_t table_elems = 0;   // elements per table
    void* tables = nullptr;   // one allocation, n_tables * table_elems elements
    int* d_err = nullptr;
    // staging for qmcspl_eval_vgl_host
    double* st_pos[2] = {nullptr, nullptr};
    void* st_out[2] = {nullptr, nullptr};
    void* st_half[2] = {nullptr, nullptr};   // 16-bit copies of st_out (reduced output types)
    long long st_cap = 0;     // positions per staging chunk
    cudaStream_t st_stream[2] = {nullptr, nullptr};
    cudaEvent_t st_ev[6] = {};
    bool st_ready = false;
    // cell-ordering scratch (device): per-position bin, bin counts/offsets, permutation
    int* ord_bin = nullptr;
    int* ord_count = nullptr;
    int* ord_perm = nullptr;
    void* ord_rec = nullptr;  // per-position coordinate records (32 bytes each)
    double2* ord_phase = nullptr;   // Bloch handles: exp(i k.r) per position
    long long ord_cap = 0;    // positions the scratch can hold
    int ord_nbins = 0;        // bins the count array can hold
    int order_mode = 0;       // QMCSPL_ORDER_AUTO / INPUT / CELL
    int block_threads = 0;    // cubic B-spline kernels: 0 = automatic, else threads per block (512, 640)
    // kernel timing (qmcspl_profile): per call, events before ordering, before and
    // after the evaluation kernel
    bool prof_on = false;
    int prof_n = 0;           // calls recorded
    cudaEvent_t* prof_ev = nullptr;   // 3 * kProfCalls events, created on first enable

    const void* table(int t) const
    {
        return static_cast<const char*>(tables) + (size_t)t * table_elems * elem_bytes;
    }
    void* table(int t)
    {
        return static_cast<char*>(tables) + (size_t)t * table_elems * elem_bytes;
    }
};

namespace qmcspl {

// ---- error reporting (thread-local message) ----
int set_error(int code, const std::string& msg);
void clear_error();   // every entry point calls this first: "" until something fails
int cuda_error(cudaError_t e, const char* what);

// ---- device allocations: every one goes through these, so that the test hook
// qmcspl_debug_fail_alloc can make a chosen one fail ----
cudaError_t dev_malloc(void** p, size_t bytes);
cudaError_t dev_malloc_async(void** p, size_t bytes, cudaStream_t stream);

// ---- construction (construct.cu) ----
int build_tables(Handle* h, int n_pw, const int* miller_host, const double* coef_host,
                 cudaStream_t stream);
// Overwrite stored table `table` (pp: entry `table`) from a device array in canonical layout
// [Nx][Ny][Nz][n_orb stored functions], double (src_double = 1) or float.
int launch_set_table(Handle* h, int table, const void* src, int src_double, cudaStream_t stream);

// ---- evaluation launchers ----
// Prepared per-position data of one evaluation: coordinate records, the evaluation
// order and (Bloch handles) the phase factors; any may be null.
struct Prepared {
    const void* rec = nullptr;
    const int* perm = nullptr;
    const double2* phase = nullptr;
    const int* bin_end = nullptr;   // sorted: one past the last position of every bin
};
int launch_bspline_vgl(const Handle* h, const double* pos, const Prepared& pr, long long n_pos, void* val,
                       void* grad, void* lap, cudaStream_t stream);
// Five tables (phi, d_x phi, d_y phi, d_z phi, lap phi) interpolated with one set of
// weights: Lagrange, and B-splines with separate gradient tables.
int launch_five_table_vgl(const Handle* h, const double* pos, const Prepared& pr, long long n_pos, void* val,
                          void* grad, void* lap, cudaStream_t stream);
int launch_pp_vgl(const Handle* h, const double* pos, const Prepared& pr, long long n_pos, void* val,
                  void* grad, void* lap, cudaStream_t stream);
// B-splines of degree other than 3, or on non-uniform grids (eval_general.cu)
int launch_general_vgl(const Handle* h, const double* pos, const Prepared& pr, long long n_pos, void* val,
                       void* grad, void* lap, cudaStream_t stream);
inline bool is_general(const Handle* h) { return h->degree != 3 || h->nonuniform; }
int launch_bspline_backward(Handle* h, const double* pos, long long n_pos,
                            const void* gv, const void* gg, const void* gl, void* dcoef,
                            void* dcoef_lap, double* dpos, cudaStream_t stream);
// launch: QMCSPL_BATCH_AUTO / SINGLE / SPLIT; threads: block shape of the batched launch (0 = 512)
int launch_batched(int n_cells, const Handle* const* hs, const double* const* pos, const Prepared* pr,
                   const long long* n_pos, void* const* val, void* const* grad, void* const* lap,
                   int launch, int threads, cudaStream_t stream);

// ---- cell ordering (order.cu) ----
// Bin geometry of a handle: bins of edge[a] grid cells along axis a, nb[a] bins along it;
// bins are numbered x-major, z fastest.
struct BinGeometry {
    int edge[3];
    int nb[3];
    int n_bins;
};
BinGeometry bin_geometry(const Handle* h);
// True when the evaluation of n_pos positions should run in cell order.
bool use_cell_order(const Handle* h, long long n_pos);
// Build the cell-order permutation of `pos` into the scratch arrays given (device
// pointers sized for n_pos positions and g.n_bins + 1 counters) on `stream`.
int build_cell_order(const Handle* h, const double* pos, long long n_pos, int* bin, int* count,
                     int* perm, const BinGeometry& g, cudaStream_t stream);

// Per-position coordinate records: the grid cell and reduced coordinate t of every
// position, computed once (FP64) so that the evaluation kernels need no FP64 work.
//   kind 1 (float / bfloat16 tables): 16 bytes {int cell, float tx, ty, tz}
//   kind 2 (double tables):           32 bytes {double tx, ty, tz; int cell, pad}
//   kind 3 (double-float tables):     32 bytes {int cell, float txh, txl, tyh, tyl, tzh, tzl, pad}
//   kind 4, 5: as kinds 1, 2 for non-uniform grids, with the offset of the position from the
//              left grid point of its interval (reduced units) in place of t
// cell = ix | iy << 10 | iz << 20, or -1 for a non-finite position.
// With `count` non-null the kernel also bins the positions for the cell order.
int record_kind(const Handle* h);
// With `phase` non-null (Bloch handles) the same pass writes exp(i k.r) per position.
int build_records(const Handle* h, const double* pos, long long n_pos, void* rec, double2* phase, int* bin,
                  int* count, const BinGeometry* g, cudaStream_t stream);
// Records, phase factors (Bloch handles) and, when sorting, the cell order in the
// handle's scratch: bins of the handle's bin_geometry, or of `geom` when given.
int prepare_positions(Handle* h, const double* pos, long long n_pos, bool sort, Prepared* out,
                      cudaStream_t stream, const BinGeometry* geom = nullptr);

// Convert n float outputs to bfloat16 (to_bf16) or IEEE half, round to nearest even.
int launch_convert_outputs(const float* src, void* dst, long long n, bool to_bf16, cudaStream_t stream);

// Allocate (once) and fill the device grid-point buffer of a non-uniform handle.
int upload_grid_points(Handle* h, cudaStream_t stream);

// fill the common part of EvalArgs from a handle
void fill_eval_args(const Handle* h, EvalArgs* a);

// number of SMs of the current device (cached)
int sm_count();
long long l2_cache_bytes();   // L2 size of the current device

}  // namespace qmcspl
