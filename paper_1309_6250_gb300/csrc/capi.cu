// capi.cu -- the extern "C" entry points declared in include/qmcspl.h.
//
// Host-side work only: argument validation, the Hermitian check of the planewave
// coefficients (real Gamma-point orbitals, Sec. III), the chain-rule matrices of
// Sec. II (Coordinates), the Cartesian k of Bloch orbitals, table sizing, and dispatch
// to the kernels.
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "general_basis.cuh"
#include "qmcspl_internal.cuh"
#include "staged.cuh"

namespace qmcspl {

static thread_local std::string g_err;

int set_error(int code, const std::string& msg)
{
    g_err = msg;
    return code;
}

void clear_error() { g_err.clear(); }

int cuda_error(cudaError_t e, const char* what)
{
    if (e == cudaSuccess) return QMCSPL_OK;
    cudaGetLastError();   // clear a sticky launch error so later calls can proceed
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? QMCSPL_ERR_OOM : QMCSPL_ERR_CUDA;
}

// Allocation failure injection (tests): -1 = off; n >= 0 = the allocation after n more
// successful ones fails once, then injection switches itself off.
static std::atomic<long long> g_fail_countdown{-1};

static bool inject_failure()
{
    long long v = g_fail_countdown.load();
    while (v >= 0) {
        const long long next = v == 0 ? -1 : v - 1;
        if (g_fail_countdown.compare_exchange_weak(v, next)) return v == 0;
    }
    return false;
}

cudaError_t dev_malloc(void** p, size_t bytes)
{
    if (inject_failure()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

cudaError_t dev_malloc_async(void** p, size_t bytes, cudaStream_t st)
{
    if (inject_failure()) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMallocAsync(p, bytes, st);
}

int sm_count()
{
    static int cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 152;
    if (!cached[dev]) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = n > 0 ? n : 152;
    }
    return cached[dev];
}

long long l2_cache_bytes()
{
    static long long cached[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 128LL << 20;
    if (!cached[dev]) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrL2CacheSize, dev);
        cached[dev] = n > 0 ? n : (128LL << 20);
    }
    return cached[dev];
}

void fill_eval_args(const Handle* h, EvalArgs* a)
{
    std::memset(a, 0, sizeof(*a));
    for (int t = 0; t < 5; ++t) a->tab[t] = t < h->n_tables ? h->table(t) : nullptr;
    a->row_stride = h->n_orb_p * h->entries;
    a->col_stride = (long long)h->rows_z * a->row_stride;
    a->nx = h->dims[0];
    a->ny = h->dims[1];
    a->nz = h->dims[2];
    a->n_orb = h->n_orb;
    a->lanes_log2 = h->lanes_log2;
    a->tiles = h->tiles;
    std::memcpy(a->ainv, h->ainv, sizeof(a->ainv));
    std::memcpy(a->mg, h->mg, sizeof(a->mg));
    std::memcpy(a->ml, h->ml, sizeof(a->ml));
    for (int i = 0; i < 9; ++i) {
        a->mgf[i] = (float)h->mg[i];
        a->mgh[i] = (float)h->mg[i];
        a->mgl[i] = (float)(h->mg[i] - (double)a->mgh[i]);
    }
    for (int i = 0; i < 6; ++i) {
        a->mlf[i] = (float)h->ml[i];
        a->mlh[i] = (float)h->ml[i];
        a->mll[i] = (float)(h->ml[i] - (double)a->mlh[i]);
    }
    a->err = h->d_err;
    a->tab_lo = static_cast<const char*>(h->tables);
    a->tab_hi = a->tab_lo + h->table_elems * h->elem_bytes * h->n_tables;
    for (int i = 0; i < 3; ++i) {
        a->kc[i] = h->kcart[i];
        a->kcf[i] = (float)h->kcart[i];
        a->kred[i] = h->kred[i];
        a->knots[i] = h->nonuniform ? h->d_knots + (size_t)i * kMaxDim : nullptr;
    }
    a->cdeg = degree_constant(h->degree);
}

bool inv3(const double m[9], double out[9]);

int upload_grid_points(Handle* h, cudaStream_t st)
{
    const size_t nd = 3 * (size_t)kMaxDim;
    std::vector<double> buf(nd * 2 + nd / 2 + 1, 0.0);
    float* fs = reinterpret_cast<float*>(buf.data() + 2 * nd);
    for (int a = 0; a < 3; ++a) {
        const int n = h->dims[a];
        for (int i = 0; i < n; ++i) {
            buf[a * kMaxDim + i] = h->knots[a][i];
            const double sp = periodic_knot(h->knots[a], n, i + 1) - h->knots[a][i];
            buf[nd + a * kMaxDim + i] = sp;
            fs[a * kMaxDim + i] = (float)sp;
        }
    }
    cudaError_t e = cudaSuccess;
    if (!h->d_knots) e = dev_malloc((void**)&h->d_knots, sizeof(double) * buf.size());
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->d_knots, buf.data(), sizeof(double) * buf.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return cuda_error(e, "grid point upload");
}

// Lattice, inverse and the chain-rule matrices of Sec. II (Coordinates):
//   grad_cart[a] = sum_i N_i ainv[i][a] grad_t[i]
//   lap = sum_ij N_i N_j (a^-1 a^-T)_ij H_ij, off-diagonal terms counted twice.
bool handle_geometry(Handle* h, const double lattice[9])
{
    double ainv[9];
    if (!inv3(lattice, ainv)) return false;
    std::memcpy(h->lattice, lattice, sizeof(h->lattice));
    std::memcpy(h->ainv, ainv, sizeof(h->ainv));
    // uniform grids differentiate with respect to u = N s (factor N_i), non-uniform ones
    // with respect to s itself
    double nf[3];
    for (int i = 0; i < 3; ++i) nf[i] = h->nonuniform ? 1.0 : (double)h->dims[i];
    for (int a = 0; a < 3; ++a)
        for (int i = 0; i < 3; ++i) h->mg[3 * a + i] = nf[i] * ainv[3 * i + a];
    double M[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int a = 0; a < 3; ++a) s += ainv[3 * i + a] * ainv[3 * j + a];
            M[3 * i + j] = nf[i] * nf[j] * s;
        }
    h->ml[0] = M[0];
    h->ml[1] = M[4];
    h->ml[2] = M[8];
    h->ml[3] = 2.0 * M[1];
    h->ml[4] = 2.0 * M[2];
    h->ml[5] = 2.0 * M[5];
    // Bloch k (Sec. II): k = 2 pi a^-T kpoint; kred = a^-T kpoint so that k.r = 2 pi kred.r
    for (int a = 0; a < 3; ++a) {
        double s = 0.0;
        for (int i = 0; i < 3; ++i) s += ainv[3 * i + a] * h->kpoint[i];
        h->kred[a] = h->bloch ? s : 0.0;
        h->kcart[a] = h->bloch ? 2.0 * M_PI * s : 0.0;
    }
    return true;
}

bool inv3(const double m[9], double out[9])
{
    const double c00 = m[4] * m[8] - m[5] * m[7];
    const double c01 = m[5] * m[6] - m[3] * m[8];
    const double c02 = m[3] * m[7] - m[4] * m[6];
    const double det = m[0] * c00 + m[1] * c01 + m[2] * c02;
    // singular (or nearly) relative to the product of the column lengths
    double vol = 1.0;
    for (int j = 0; j < 3; ++j) vol *= std::sqrt(m[j] * m[j] + m[3 + j] * m[3 + j] + m[6 + j] * m[6 + j]);
    if (!std::isfinite(det) || std::fabs(det) <= 1e-12 * vol) return false;
    const double id = 1.0 / det;
    out[0] = c00 * id;
    out[1] = (m[2] * m[7] - m[1] * m[8]) * id;
    out[2] = (m[1] * m[5] - m[2] * m[4]) * id;
    out[3] = c01 * id;
    out[4] = (m[0] * m[8] - m[2] * m[6]) * id;
    out[5] = (m[2] * m[3] - m[0] * m[5]) * id;
    out[6] = c02 * id;
    out[7] = (m[1] * m[6] - m[0] * m[7]) * id;
    out[8] = (m[0] * m[4] - m[1] * m[3]) * id;
    return true;
}

namespace {

inline long long miller_key(int a, int b, int c)
{
    const long long off = 1LL << 20;
    return ((a + off) << 42) | ((b + off) << 21) | (c + off);
}

// Distinct, in-range Miller indices and finite coefficients; real (Gamma-point)
// orbitals also need every -G and c_{-G} = conj(c_G).
int check_planewaves(int n_pw, const int* miller, int n_orb, const double* coef, bool hermitian)
{
    std::unordered_map<long long, int> index;
    index.reserve((size_t)n_pw * 2);
    for (int g = 0; g < n_pw; ++g) {
        const int a = miller[3 * g], b = miller[3 * g + 1], c = miller[3 * g + 2];
        if (std::abs(a) >= (1 << 20) || std::abs(b) >= (1 << 20) || std::abs(c) >= (1 << 20))
            return set_error(QMCSPL_ERR_ARG, "Miller index out of range");
        if (!index.emplace(miller_key(a, b, c), g).second)
            return set_error(QMCSPL_ERR_ARG, "duplicate Miller index " + std::to_string(g));
    }
    double cmax = 0.0;
    for (long long i = 0; i < 2LL * n_pw * n_orb; ++i) {
        if (!std::isfinite(coef[i])) return set_error(QMCSPL_ERR_ARG, "non-finite coefficient");
        cmax = std::fmax(cmax, std::fabs(coef[i]));
    }
    if (!hermitian) return QMCSPL_OK;
    const double tol = 1e-12 * (cmax > 0 ? cmax : 1.0);
    for (int g = 0; g < n_pw; ++g) {
        auto it = index.find(miller_key(-miller[3 * g], -miller[3 * g + 1], -miller[3 * g + 2]));
        if (it == index.end())
            return set_error(QMCSPL_ERR_NOT_HERMITIAN, "planewave " + std::to_string(g) + " has no -G partner");
        const int m = it->second;
        for (int o = 0; o < n_orb; ++o) {
            const double* c1 = coef + 2 * ((size_t)o * n_pw + g);
            const double* c2 = coef + 2 * ((size_t)o * n_pw + m);
            if (std::fabs(c1[0] - c2[0]) > tol || std::fabs(c1[1] + c2[1]) > tol)
                return set_error(QMCSPL_ERR_NOT_HERMITIAN,
                                 "c_{-G} != conj(c_G) for planewave " + std::to_string(g) +
                                     ", orbital " + std::to_string(o));
        }
    }
    return QMCSPL_OK;
}

// Lanes per position and orbital tiles: rows of n 16-byte chunks are split over
// L = 2^k lanes and ceil(n / L) tiles, taking the widest L whose padding stays
// within 1/8 of the row.
void choose_lanes(int n_chunks, int& lanes_log2, int& tiles)
{
    for (int lg = 5; lg >= 0; --lg) {
        const int L = 1 << lg;
        const long long padded = (long long)((n_chunks + L - 1) / L) * L;
        if (L == 1 || padded * 8 <= (long long)n_chunks * 9) {
            lanes_log2 = lg;
            tiles = (n_chunks + L - 1) / L;
            return;
        }
    }
}

void free_handle(Handle* h)
{
    if (!h) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    if (h->tables) cudaFree(h->tables);
    if (h->d_err) cudaFree(h->d_err);
    for (int b = 0; b < 2; ++b) {
        if (h->st_pos[b]) cudaFree(h->st_pos[b]);
        if (h->st_out[b]) cudaFree(h->st_out[b]);
        if (h->st_half[b]) cudaFree(h->st_half[b]);
        if (h->st_stream[b]) cudaStreamDestroy(h->st_stream[b]);
    }
    if (h->st_ready)
        for (int i = 0; i < 6; ++i) cudaEventDestroy(h->st_ev[i]);
    if (h->ord_bin) cudaFree(h->ord_bin);
    if (h->ord_perm) cudaFree(h->ord_perm);
    if (h->ord_count) cudaFree(h->ord_count);
    if (h->ord_rec) cudaFree(h->ord_rec);
    if (h->ord_phase) cudaFree(h->ord_phase);
    if (h->d_knots) cudaFree(h->d_knots);
    if (h->prof_ev) {
        for (int i = 0; i < 3 * kProfCalls; ++i) cudaEventDestroy(h->prof_ev[i]);
        delete[] h->prof_ev;
    }
    delete h;
    cudaSetDevice(prev);
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace
}  // namespace qmcspl

using namespace qmcspl;

extern "C" {

int qmcspl_version(void) { return 10000 * 1 + 100 * 0 + 0; }

int qmcspl_debug_fail_alloc(long long n)
{
    g_fail_countdown.store(n < 0 ? -1 : n);
    return QMCSPL_OK;
}

const char* qmcspl_last_error(void) { return g_err.c_str(); }

int qmcspl_create(qmcspl_t* out, const double lattice[9], const int dims[3], int n_pw,
                  const int* miller, int n_orb, const double* coef, const qmcspl_opts* opts,
                  void* stream)
{
    return qmcspl_create_grid(out, lattice, dims, n_pw, miller, n_orb, coef, opts, nullptr, stream);
}

int qmcspl_create_grid(qmcspl_t* out, const double lattice[9], const int dims[3], int n_pw,
                       const int* miller, int n_orb, const double* coef, const qmcspl_opts* opts,
                       const qmcspl_grid_opts* grid, void* stream)
{
    g_err.clear();
    if (!out) return set_error(QMCSPL_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!lattice || !dims || !miller || !coef || !opts)
        return set_error(QMCSPL_ERR_ARG, "NULL argument");
    if (n_pw < 1) return set_error(QMCSPL_ERR_ARG, "n_pw must be >= 1");
    if (n_orb < 1) return set_error(QMCSPL_ERR_ARG, "n_orb must be >= 1");
    for (int a = 0; a < 3; ++a)
        if (dims[a] < 4 || dims[a] > kMaxDim)
            return set_error(QMCSPL_ERR_ARG, "grid dims must be in [4, 512]");
    if (opts->method < QMCSPL_BSPLINE_SMOOTH || opts->method > QMCSPL_PPSPLINE)
        return set_error(QMCSPL_ERR_ARG, "unknown method");
    if (opts->storage < QMCSPL_F64 || opts->storage > QMCSPL_DF64)
        return set_error(QMCSPL_ERR_ARG, "unknown storage type");
    if (opts->storage == QMCSPL_DF64 && opts->method != QMCSPL_BSPLINE_SMOOTH &&
        opts->method != QMCSPL_BSPLINE_INTERP)
        return set_error(QMCSPL_ERR_UNSUPPORTED, "double-float tables are for the B-spline methods");
    for (int i = 0; i < 9; ++i)
        if (!std::isfinite(lattice[i])) return set_error(QMCSPL_ERR_ARG, "non-finite lattice");
    double ainv[9];
    if (!inv3(lattice, ainv)) return set_error(QMCSPL_ERR_ARG, "singular lattice");
    if (opts->bloch != 0 && opts->bloch != 1) return set_error(QMCSPL_ERR_ARG, "bloch must be 0 or 1");
    const bool is_bspline = opts->method == QMCSPL_BSPLINE_SMOOTH || opts->method == QMCSPL_BSPLINE_INTERP;
    if (is_bspline && opts->separate_grad) {
        if (!opts->separate_lap)
            return set_error(QMCSPL_ERR_ARG, "separate_grad needs separate_lap (the five-table layout)");
    }
    if (opts->bloch)
        for (int i = 0; i < 3; ++i)
            if (!std::isfinite(opts->kpoint[i])) return set_error(QMCSPL_ERR_ARG, "non-finite kpoint");
    if (opts->bloch && n_orb > (1 << 29)) return set_error(QMCSPL_ERR_ARG, "n_orb too large");
    int degree = 3;
    bool nonuni = false;
    if (grid) {
        degree = grid->degree == 0 ? 3 : grid->degree;
        if (degree != 1 && degree != 3 && degree != 5 && degree != 7)
            return set_error(QMCSPL_ERR_ARG, "degree must be 1, 3, 5 or 7");
        for (int a = 0; a < 3; ++a) nonuni = nonuni || grid->knots[a] != nullptr;
        // other degrees: interpolating or smoothing B-splines; non-uniform grids: interpolating
        const bool ok_method = nonuni ? opts->method == QMCSPL_BSPLINE_INTERP
                                      : (opts->method == QMCSPL_BSPLINE_INTERP || opts->method == QMCSPL_BSPLINE_SMOOTH);
        if ((degree != 3 || nonuni) && (!ok_method || opts->storage == QMCSPL_DF64 || opts->separate_grad))
            return set_error(QMCSPL_ERR_UNSUPPORTED,
                             "other degrees are for B-splines, non-uniform grids for interpolating ones "
                             "(f64, f32 or bf16 tables, no separate gradient tables)");
        for (int a = 0; a < 3; ++a) {
            if (dims[a] < degree + 1) return set_error(QMCSPL_ERR_ARG, "grid too small for the degree");
            const double* k = grid->knots[a];
            if (!nonuni) continue;
            if (!k) return set_error(QMCSPL_ERR_ARG, "non-uniform grids need the points of all three axes");
            for (int i = 0; i < dims[a]; ++i) {
                if (!std::isfinite(k[i]) || k[i] < 0.0 || k[i] >= 1.0)
                    return set_error(QMCSPL_ERR_ARG, "grid points must lie in [0, 1)");
                if (i > 0 && !(k[i] > k[i - 1]))
                    return set_error(QMCSPL_ERR_ARG, "grid points must be strictly increasing");
            }
        }
    }
    int rc = check_planewaves(n_pw, miller, n_orb, coef, opts->bloch == 0);
    if (rc != QMCSPL_OK) return rc;

    Handle* h = new (std::nothrow) Handle();
    if (!h) return set_error(QMCSPL_ERR_OOM, "host allocation failed");
    cudaGetDevice(&h->device);
    h->method = opts->method;
    h->storage = opts->storage;
    const bool bspline = h->method == QMCSPL_BSPLINE_SMOOTH || h->method == QMCSPL_BSPLINE_INTERP;
    h->separate_lap = bspline ? (opts->separate_lap != 0) : (h->method == QMCSPL_LAGRANGE);
    h->separate_grad = bspline ? (opts->separate_grad != 0) : (h->method == QMCSPL_LAGRANGE);
    h->degree = degree;
    h->nonuniform = nonuni ? 1 : 0;
    h->zshift = (h->method == QMCSPL_PPSPLINE) ? 0 : (degree - 1) / 2;
    if (nonuni)
        for (int a = 0; a < 3; ++a)
            for (int i = 0; i < dims[a]; ++i) h->knots[a][i] = grid->knots[a][i];
    for (int a = 0; a < 3; ++a) h->dims[a] = dims[a];
    h->bloch = opts->bloch;
    for (int i = 0; i < 3; ++i) h->kpoint[i] = h->bloch ? opts->kpoint[i] : 0.0;
    h->n_orb = n_orb << h->bloch;   // stored real functions: Re u, Im u per Bloch orbital
    h->n_pw = n_pw;
    handle_geometry(h, lattice);

    h->elem_bytes = (h->storage == QMCSPL_F64 || h->storage == QMCSPL_DF64) ? 8 : (h->storage == QMCSPL_F32 ? 4 : 2);
    const int E = (int)(16 / h->elem_bytes);
    const int n_chunks = (h->n_orb + E - 1) / E;
    if (opts->lanes == 0) {
        choose_lanes(n_chunks, h->lanes_log2, h->tiles);
    } else {
        int lg = -1;
        for (int k = 0; k <= 5; ++k)
            if (opts->lanes == (1 << k)) lg = k;
        if (lg < 0) {
            delete h;
            return set_error(QMCSPL_ERR_ARG, "lanes must be 0, 1, 2, 4, 8, 16 or 32");
        }
        h->lanes_log2 = lg;
        h->tiles = (n_chunks + (1 << lg) - 1) >> lg;
    }
    h->n_orb_p = h->tiles * (1 << h->lanes_log2) * E;
    switch (h->method) {
    case QMCSPL_LAGRANGE: h->n_tables = 5; h->entries = 1; h->rows_z = dims[2] + 3; break;
    case QMCSPL_PPSPLINE: h->n_tables = 1; h->entries = 8; h->rows_z = dims[2] + 1; break;
    default:
        h->n_tables = h->separate_grad ? 5 : (h->separate_lap ? 2 : 1);
        h->entries = 1;
        h->rows_z = dims[2] + degree;   // (degree - 1)/2 ghost planes below, (degree + 1)/2 above
        break;
    }
    h->table_elems = (size_t)dims[0] * dims[1] * h->rows_z * h->entries * h->n_orb_p;

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t bytes = h->table_elems * h->elem_bytes * h->n_tables;
    cudaError_t e = dev_malloc(&h->tables, bytes);
    if (e != cudaSuccess) {
        rc = cuda_error(e, "cudaMalloc(tables)");
        free_handle(h);
        return rc;
    }
    e = dev_malloc((void**)&h->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_err, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->tables, 0, bytes, st);
    if (e != cudaSuccess) {
        rc = cuda_error(e, "table initialisation");
        free_handle(h);
        return rc;
    }
    if (nonuni && (rc = upload_grid_points(h, st)) != QMCSPL_OK) {
        free_handle(h);
        return rc;
    }
    rc = build_tables(h, n_pw, miller, coef, st);
    if (rc != QMCSPL_OK) {
        free_handle(h);
        return rc;
    }
    *out = h;
    return QMCSPL_OK;
}

int qmcspl_destroy(qmcspl_t h)
{
    g_err.clear();
    free_handle(h);
    return QMCSPL_OK;
}

int qmcspl_info(qmcspl_t h, qmcspl_info_t* out)
{
    g_err.clear();
    if (!h || !out) return set_error(QMCSPL_ERR_ARG, "NULL argument");
    std::memset(out, 0, sizeof(*out));
    for (int a = 0; a < 3; ++a) out->dims[a] = h->dims[a];
    out->n_orb = h->n_orb >> h->bloch;
    out->n_orb_padded = h->n_orb_p;
    out->method = h->method;
    out->storage = h->storage;
    out->separate_lap = h->separate_lap;
    out->n_tables = h->n_tables;
    out->entries_per_point = h->entries;
    out->rows_z = h->rows_z;
    out->lanes = 1 << h->lanes_log2;
    out->tiles = h->tiles;
    out->table_bytes = (long long)(h->table_elems * h->elem_bytes * h->n_tables);
    out->n_pw = h->n_pw;
    out->bloch = h->bloch;
    out->separate_grad = h->separate_grad;
    out->degree = h->degree;
    out->nonuniform = h->nonuniform;
    out->staged = staged_eligible(h) ? 1 : 0;
    out->block_threads = h->block_threads;
    for (int i = 0; i < 3; ++i) out->kpoint[i] = h->kpoint[i];
    return QMCSPL_OK;
}

static int eval_dispatch(Handle* h, const double* pos, long long n_pos, void* val, void* grad,
                         void* lap, cudaStream_t st)
{
    cudaEvent_t* ev = nullptr;
    if (h->prof_on && h->prof_n < kProfCalls) ev = h->prof_ev + 3 * h->prof_n++;
    if (ev) cudaEventRecord(ev[0], st);
    Prepared pr;
    BinGeometry pg;
    StagedArgs sa;
    if (use_staged(h, n_pos) && staged_plan(h, n_pos, &pg, &sa)) {
        int rc = prepare_positions(h, pos, n_pos, true, &pr, st, &pg);
        if (rc != QMCSPL_OK) return rc;
        if (ev) cudaEventRecord(ev[1], st);
        rc = launch_bspline_vgl_staged(h, pr, n_pos, val, grad, lap, sa, st);
        if (ev) cudaEventRecord(ev[2], st);
        return rc;
    }
    const bool sort = use_cell_order(h, n_pos);
    // Bloch handles always take the per-position pass: it computes the phase factors
    if (sort || n_pos >= kRecordMinPositions || h->bloch) {
        const int rc = prepare_positions(h, pos, n_pos, sort, &pr, st);
        if (rc != QMCSPL_OK) return rc;
    }
    if (ev) cudaEventRecord(ev[1], st);
    int rc;
    switch (h->method) {
    case QMCSPL_LAGRANGE: rc = launch_five_table_vgl(h, pos, pr, n_pos, val, grad, lap, st); break;
    case QMCSPL_PPSPLINE: rc = launch_pp_vgl(h, pos, pr, n_pos, val, grad, lap, st); break;
    default:
        rc = h->separate_grad  ? launch_five_table_vgl(h, pos, pr, n_pos, val, grad, lap, st)
             : is_general(h) ? launch_general_vgl(h, pos, pr, n_pos, val, grad, lap, st)
                               : launch_bspline_vgl(h, pos, pr, n_pos, val, grad, lap, st);
        break;
    }
    if (ev) cudaEventRecord(ev[2], st);
    return rc;
}

int qmcspl_eval_vgl(qmcspl_t h, const double* pos, long long n_pos, void* val, void* grad,
                    void* lap, void* stream)
{
    g_err.clear();
    if (!h) return set_error(QMCSPL_ERR_ARG, "NULL handle");
    if (n_pos < 0) return set_error(QMCSPL_ERR_ARG, "n_pos < 0");
    if (n_pos == 0) return QMCSPL_OK;
    if (!pos) return set_error(QMCSPL_ERR_ARG, "pos is NULL");
    if (n_pos > (1LL << 40)) return set_error(QMCSPL_ERR_ARG, "n_pos too large");
    DeviceGuard dg(h->device);
    return eval_dispatch(h, pos, n_pos, val, grad, lap, static_cast<cudaStream_t>(stream));
}

int qmcspl_eval_vgl_host_ex(qmcspl_t h, const double* pos_host, long long n_pos, void* val_host,
                            void* grad_host, void* lap_host, const qmcspl_host_opts* opts, void* stream)
{
    g_err.clear();
    if (!h) return set_error(QMCSPL_ERR_ARG, "NULL handle");
    if (n_pos < 0) return set_error(QMCSPL_ERR_ARG, "n_pos < 0");
    const int out_type = opts ? opts->out_type : QMCSPL_OUT_NATIVE;
    if (out_type < QMCSPL_OUT_NATIVE || out_type > QMCSPL_OUT_F16) return set_error(QMCSPL_ERR_ARG, "unknown out_type");
    const bool reduced = out_type != QMCSPL_OUT_NATIVE;
    if (reduced && (h->storage == QMCSPL_F64 || h->storage == QMCSPL_DF64 || h->bloch))
        return set_error(QMCSPL_ERR_UNSUPPORTED, "16-bit outputs are for real orbitals with float or bfloat16 tables");
    if (n_pos == 0) return QMCSPL_OK;
    if (!pos_host) return set_error(QMCSPL_ERR_ARG, "pos_host is NULL");
    DeviceGuard dg(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t ob = (h->storage == QMCSPL_F64 || h->storage == QMCSPL_DF64) ? 8 : 4;
    const size_t row = (size_t)h->n_orb * ob;          // bytes of one output row on the device
    const size_t hrow = reduced ? (size_t)h->n_orb * 2 : row;   // ... and in the host buffers
    const long long cap = 1LL << 16;                   // positions per chunk
    cudaError_t e;
    if (!h->st_ready) {
        // all or nothing: on a failure everything created so far is released again
        cudaStream_t ss[2] = {nullptr, nullptr};
        cudaEvent_t ee[6] = {};
        double* sp[2] = {nullptr, nullptr};
        void* so[2] = {nullptr, nullptr};
        int n_ev = 0;
        e = cudaSuccess;
        for (int b = 0; b < 2 && e == cudaSuccess; ++b) e = cudaStreamCreateWithFlags(&ss[b], cudaStreamNonBlocking);
        for (; n_ev < 6 && e == cudaSuccess; ++n_ev) {
            e = cudaEventCreateWithFlags(&ee[n_ev], cudaEventDisableTiming);
            if (e != cudaSuccess) break;
        }
        for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
            e = dev_malloc((void**)&sp[b], sizeof(double) * 3 * cap);
            if (e == cudaSuccess) e = dev_malloc(&so[b], row * 5 * cap);
        }
        if (e != cudaSuccess) {
            const int rc = cuda_error(e, "host staging set-up");
            for (int b = 0; b < 2; ++b) {
                if (ss[b]) cudaStreamDestroy(ss[b]);
                if (sp[b]) cudaFree(sp[b]);
                if (so[b]) cudaFree(so[b]);
            }
            for (int i = 0; i < n_ev; ++i) cudaEventDestroy(ee[i]);
            return rc;
        }
        for (int b = 0; b < 2; ++b) {
            h->st_stream[b] = ss[b];
            h->st_pos[b] = sp[b];
            h->st_out[b] = so[b];
        }
        for (int i = 0; i < 6; ++i) h->st_ev[i] = ee[i];
        h->st_cap = cap;
        h->st_ready = true;
    }
    if (reduced && !h->st_half[0]) {
        void* sh[2] = {nullptr, nullptr};
        e = dev_malloc(&sh[0], (size_t)h->n_orb * 2 * 5 * h->st_cap);
        if (e == cudaSuccess) e = dev_malloc(&sh[1], (size_t)h->n_orb * 2 * 5 * h->st_cap);
        if (e != cudaSuccess) {
            if (sh[0]) cudaFree(sh[0]);
            return cuda_error(e, "16-bit output staging");
        }
        h->st_half[0] = sh[0];
        h->st_half[1] = sh[1];
    }
    cudaStream_t s_in = h->st_stream[0], s_out = h->st_stream[1];
    cudaEvent_t* ev_in = h->st_ev;          // positions of buffer b are on the device
    cudaEvent_t* ev_done = h->st_ev + 2;    // kernel writing buffer b finished
    cudaEvent_t* ev_free = h->st_ev + 4;    // outputs of buffer b copied out
    // order the staging streams after the work already queued on `stream`
    e = cudaEventRecord(ev_free[0], st);
    if (e == cudaSuccess) e = cudaEventRecord(ev_free[1], st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s_in, ev_free[0], 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s_out, ev_free[0], 0);
    if (e != cudaSuccess) return cuda_error(e, "stream ordering");
    char* hv = static_cast<char*>(val_host);
    char* hg = static_cast<char*>(grad_host);
    char* hl = static_cast<char*>(lap_host);
    int rc = QMCSPL_OK;
    int chunk_i = 0;
    for (long long p0 = 0; p0 < n_pos; p0 += h->st_cap, ++chunk_i) {
        const int b = chunk_i & 1;
        const long long n = (n_pos - p0 < h->st_cap) ? n_pos - p0 : h->st_cap;
        char* dv = static_cast<char*>(h->st_out[b]);
        char* dg_ = dv + row * n;
        char* dl = dg_ + row * 3 * n;
        // what the host copies come from: the outputs, or their 16-bit conversion (same layout)
        char* cv = reduced ? static_cast<char*>(h->st_half[b]) : dv;
        char* cg = cv + hrow * n;
        char* cl = cg + hrow * 3 * n;
        if ((e = cudaStreamWaitEvent(s_in, ev_free[b], 0)) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(h->st_pos[b], pos_host + 3 * p0, sizeof(double) * 3 * n,
                                 cudaMemcpyHostToDevice, s_in)) != cudaSuccess) break;
        if ((e = cudaEventRecord(ev_in[b], s_in)) != cudaSuccess) break;
        if ((e = cudaStreamWaitEvent(st, ev_in[b], 0)) != cudaSuccess) break;
        rc = eval_dispatch(h, h->st_pos[b], n, hv ? dv : nullptr, hg ? dg_ : nullptr,
                           hl ? dl : nullptr, st);
        if (rc != QMCSPL_OK) break;
        if (reduced) {   // the requested outputs of the chunk, converted on the device
            const bool bf = out_type == QMCSPL_OUT_BF16;
            const long long m = n * (long long)h->n_orb;
            if (hv && (rc = launch_convert_outputs(reinterpret_cast<const float*>(dv), cv, m, bf, st)) != QMCSPL_OK) break;
            if (hg && (rc = launch_convert_outputs(reinterpret_cast<const float*>(dg_), cg, 3 * m, bf, st)) != QMCSPL_OK) break;
            if (hl && (rc = launch_convert_outputs(reinterpret_cast<const float*>(dl), cl, m, bf, st)) != QMCSPL_OK) break;
        }
        if ((e = cudaEventRecord(ev_done[b], st)) != cudaSuccess) break;
        if ((e = cudaStreamWaitEvent(s_out, ev_done[b], 0)) != cudaSuccess) break;
        if (hv && (e = cudaMemcpyAsync(hv + hrow * p0, cv, hrow * n, cudaMemcpyDeviceToHost, s_out)) != cudaSuccess) break;
        if (hg && (e = cudaMemcpyAsync(hg + hrow * 3 * p0, cg, hrow * 3 * n, cudaMemcpyDeviceToHost, s_out)) != cudaSuccess) break;
        if (hl && (e = cudaMemcpyAsync(hl + hrow * p0, cl, hrow * n, cudaMemcpyDeviceToHost, s_out)) != cudaSuccess) break;
        if ((e = cudaEventRecord(ev_free[b], s_out)) != cudaSuccess) break;
    }
    if (rc == QMCSPL_OK && e != cudaSuccess) rc = cuda_error(e, "host staging pipeline");
    cudaError_t e2 = cudaStreamSynchronize(s_out);
    cudaError_t e3 = cudaStreamSynchronize(st);
    if (rc == QMCSPL_OK && e2 != cudaSuccess) rc = cuda_error(e2, "host staging copy-out");
    if (rc == QMCSPL_OK && e3 != cudaSuccess) rc = cuda_error(e3, "host staging kernels");
    return rc;
}

int qmcspl_eval_vgl_host(qmcspl_t h, const double* pos_host, long long n_pos, void* val_host,
                         void* grad_host, void* lap_host, void* stream)
{
    return qmcspl_eval_vgl_host_ex(h, pos_host, n_pos, val_host, grad_host, lap_host, nullptr, stream);
}

int qmcspl_eval_vgl_backward(qmcspl_t h, const double* pos, long long n_pos, const void* gv,
                             const void* gg, const void* gl, void* dcoef, void* dcoef_lap,
                             double* dpos, void* stream)
{
    g_err.clear();
    if (!h) return set_error(QMCSPL_ERR_ARG, "NULL handle");
    if (n_pos < 0) return set_error(QMCSPL_ERR_ARG, "n_pos < 0");
    // five-table and pp handles: dcoef holds all their tables (5, or the 8 pp entries)
    const bool multi = h->n_tables == 5 || h->method == QMCSPL_PPSPLINE;
    if (dcoef_lap && (multi || !(h->separate_lap && dcoef)))
        return set_error(QMCSPL_ERR_ARG, multi ? "five-table or pp handle: dcoef holds all tables, dcoef_lap must be NULL"
                                               : "dcoef_lap needs a separate-Laplacian handle and dcoef");
    if (dcoef && !multi && h->separate_lap && !dcoef_lap)
        return set_error(QMCSPL_ERR_ARG, "separate-Laplacian handle: dcoef_lap is required with dcoef");
    if (n_pos == 0) return QMCSPL_OK;
    if (!pos) return set_error(QMCSPL_ERR_ARG, "pos is NULL");
    DeviceGuard dg(h->device);
    return launch_bspline_backward(h, pos, n_pos, gv, gg, gl, dcoef, dcoef_lap, dpos,
                                   static_cast<cudaStream_t>(stream));
}

int qmcspl_eval_batched_ex(int n_cells, const qmcspl_t* hs, const double* const* pos,
                           const long long* n_pos, void* const* val, void* const* grad,
                           void* const* lap, const qmcspl_batch_opts* opts, void* stream)
{
    g_err.clear();
    if (n_cells < 1 || n_cells > QMCSPL_MAX_BATCH)
        return set_error(QMCSPL_ERR_ARG, "n_cells must be in [1, QMCSPL_MAX_BATCH]");
    const int launch = opts ? opts->launch : QMCSPL_BATCH_AUTO;
    const int threads = opts ? opts->threads : 0;
    if (launch < QMCSPL_BATCH_AUTO || launch > QMCSPL_BATCH_SPLIT) return set_error(QMCSPL_ERR_ARG, "unknown batch launch plan");
    if (threads != 0 && threads != 512 && threads != 640) return set_error(QMCSPL_ERR_ARG, "batch threads must be 0, 512 or 640");
    if (!hs || !pos || !n_pos || !val || !grad || !lap) return set_error(QMCSPL_ERR_ARG, "NULL argument");
    for (int c = 0; c < n_cells; ++c) {
        if (!hs[c]) return set_error(QMCSPL_ERR_ARG, "NULL handle in batch");
        if (hs[c]->device != hs[0]->device) return set_error(QMCSPL_ERR_ARG, "handles on different devices");
        if (hs[c]->storage != hs[0]->storage || hs[c]->separate_lap != hs[0]->separate_lap ||
            hs[c]->bloch != hs[0]->bloch)
            return set_error(QMCSPL_ERR_ARG, "handles of a batch must share storage type, separate_lap and bloch");
        if ((hs[c]->method != QMCSPL_BSPLINE_SMOOTH && hs[c]->method != QMCSPL_BSPLINE_INTERP) ||
            hs[c]->separate_grad || is_general(hs[c]))
            return set_error(QMCSPL_ERR_UNSUPPORTED,
                             "batched evaluation is for B-spline handles without separate gradient tables");
        if (n_pos[c] < 0) return set_error(QMCSPL_ERR_ARG, "n_pos < 0");
        if (n_pos[c] > 0 && !pos[c]) return set_error(QMCSPL_ERR_ARG, "pos is NULL");
    }
    if (threads == 640 && hs[0]->storage != QMCSPL_F32 && hs[0]->storage != QMCSPL_BF16)
        return set_error(QMCSPL_ERR_UNSUPPORTED, "640-thread blocks are for float and bfloat16 tables");
    // each cell's order lives in its handle's scratch: a handle twice would overwrite its own
    for (int c = 0; c < n_cells; ++c)
        for (int d = 0; d < c; ++d)
            if (hs[d] == hs[c]) return set_error(QMCSPL_ERR_ARG, "a handle appears twice in the batch");
    DeviceGuard dg(hs[0]->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Prepared prs[QMCSPL_MAX_BATCH];
    for (int c = 0; c < n_cells; ++c) {
        const bool sort = n_pos[c] > 0 && use_cell_order(hs[c], n_pos[c]);
        if (n_pos[c] > 0 && (sort || n_pos[c] >= kRecordMinPositions || hs[c]->bloch)) {
            const int rc = prepare_positions(hs[c], pos[c], n_pos[c], sort, &prs[c], st);
            if (rc != QMCSPL_OK) return rc;
        }
    }
    return launch_batched(n_cells, reinterpret_cast<const Handle* const*>(hs), pos, prs, n_pos, val, grad, lap,
                          launch, threads, st);
}

int qmcspl_eval_batched(int n_cells, const qmcspl_t* hs, const double* const* pos,
                        const long long* n_pos, void* const* val, void* const* grad,
                        void* const* lap, void* stream)
{
    return qmcspl_eval_batched_ex(n_cells, hs, pos, n_pos, val, grad, lap, nullptr, stream);
}

int qmcspl_set_block(qmcspl_t h, int threads)
{
    g_err.clear();
    if (!h) return set_error(QMCSPL_ERR_ARG, "NULL handle");
    if (threads != 0 && threads != 512 && threads != 640) return set_error(QMCSPL_ERR_ARG, "threads must be 0, 512 or 640");
    if (threads == 640 && h->storage != QMCSPL_F32 && h->storage != QMCSPL_BF16)
        return set_error(QMCSPL_ERR_UNSUPPORTED, "640-thread blocks are for float and bfloat16 tables");
    h->block_threads = threads;
    return QMCSPL_OK;
}

int qmcspl_get_table(qmcspl_t h, int table, double* out_host, void* stream)
{
    g_err.clear();
    if (!h || !out_host) return set_error(QMCSPL_ERR_ARG, "NULL argument");
    const int n_avail = (h->method == QMCSPL_PPSPLINE) ? 8 : h->n_tables;
    if (table < 0 || table >= n_avail) return set_error(QMCSPL_ERR_ARG, "table index out of range");
    DeviceGuard dg(h->device);
    const int tab = (h->method == QMCSPL_PPSPLINE) ? 0 : table;
    const int entry = (h->method == QMCSPL_PPSPLINE) ? table : 0;
    const size_t bytes = h->table_elems * h->elem_bytes;
    char* raw = new (std::nothrow) char[bytes];
    if (!raw) return set_error(QMCSPL_ERR_OOM, "host allocation failed");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(raw, h->table(tab), bytes, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        delete[] raw;
        return cuda_error(e, "table copy");
    }
    const int N1 = h->dims[0], N2 = h->dims[1], N3 = h->dims[2];
    const int zshift = h->zshift;
    for (int x = 0; x < N1; ++x)
        for (int y = 0; y < N2; ++y)
            for (int z = 0; z < N3; ++z) {
                const size_t src = ((((size_t)x * N2 + y) * h->rows_z + z + zshift) * h->entries + entry) *
                                   h->n_orb_p;
                double* dst = out_host + (((size_t)x * N2 + y) * N3 + z) * h->n_orb;
                for (int o = 0; o < h->n_orb; ++o) {
                    double v;
                    if (h->storage == QMCSPL_DF64) {
                        // 16-byte chunk of two orbitals: hi0, hi1, lo0, lo1
                        const size_t fl = (src + (o & ~1)) * 2 + (o & 1);
                        float hi, lo;
                        std::memcpy(&hi, raw + fl * 4, 4);
                        std::memcpy(&lo, raw + (fl + 2) * 4, 4);
                        v = (double)hi + (double)lo;
                    } else if (h->storage == QMCSPL_F64) {
                        std::memcpy(&v, raw + (src + o) * 8, 8);
                    } else if (h->storage == QMCSPL_F32) {
                        float f;
                        std::memcpy(&f, raw + (src + o) * 4, 4);
                        v = f;
                    } else {
                        uint16_t b;
                        std::memcpy(&b, raw + (src + o) * 2, 2);
                        const uint32_t u = (uint32_t)b << 16;
                        float f;
                        std::memcpy(&f, &u, 4);
                        v = f;
                    }
                    dst[o] = v;
                }
            }
    delete[] raw;
    return QMCSPL_OK;
}

int qmcspl_set_table(qmcspl_t h, int table, const void* src, int src_dtype, void* stream)
{
    g_err.clear();
    if (!h || !src) return set_error(QMCSPL_ERR_ARG, "NULL argument");
    const int n_avail = (h->method == QMCSPL_PPSPLINE) ? 8 : h->n_tables;
    if (table < 0 || table >= n_avail) return set_error(QMCSPL_ERR_ARG, "table index out of range");
    if (src_dtype != QMCSPL_F64 && src_dtype != QMCSPL_F32)
        return set_error(QMCSPL_ERR_ARG, "src_dtype must be QMCSPL_F64 (double) or QMCSPL_F32 (float)");
    const size_t esz = src_dtype == QMCSPL_F64 ? 8 : 4;
    if (reinterpret_cast<uintptr_t>(src) % esz) return set_error(QMCSPL_ERR_ARG, "src is not aligned to its element size");
    DeviceGuard dg(h->device);
    return launch_set_table(h, table, src, src_dtype == QMCSPL_F64 ? 1 : 0, static_cast<cudaStream_t>(stream));
}

int qmcspl_profile(qmcspl_t h, int enable)
{
    g_err.clear();
    if (!h) return set_error(QMCSPL_ERR_ARG, "NULL handle");
    DeviceGuard dg(h->device);
    if (enable && !h->prof_ev) {
        h->prof_ev = new (std::nothrow) cudaEvent_t[3 * kProfCalls];
        if (!h->prof_ev) return set_error(QMCSPL_ERR_OOM, "host allocation failed");
        for (int i = 0; i < 3 * kProfCalls; ++i) {
            cudaError_t e = cudaEventCreate(&h->prof_ev[i]);
            if (e != cudaSuccess) {
                for (int j = 0; j < i; ++j) cudaEventDestroy(h->prof_ev[j]);
                delete[] h->prof_ev;
                h->prof_ev = nullptr;
                return cuda_error(e, "cudaEventCreate");
            }
        }
    }
    h->prof_on = enable != 0;
    if (enable) h->prof_n = 0;
    return QMCSPL_OK;
}

int qmcspl_profile_read(qmcspl_t h, double* eval_ms, double* order_ms, long long* launches)
{
    g_err.clear();
    if (!h) return set_error(QMCSPL_ERR_ARG, "NULL handle");
    DeviceGuard dg(h->device);
    double te = 0.0, to = 0.0;
    for (int i = 0; i < h->prof_n; ++i) {
        cudaEvent_t* ev = h->prof_ev + 3 * i;
        cudaError_t e = cudaEventSynchronize(ev[2]);
        float a = 0.f, b = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&a, ev[0], ev[1]);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&b, ev[1], ev[2]);
        if (e != cudaSuccess) return cuda_error(e, "profile events");
        to += a;
        te += b;
    }
    if (eval_ms) *eval_ms = te;
    if (order_ms) *order_ms = to;
    if (launches) *launches = h->prof_n;
    return QMCSPL_OK;
}

int qmcspl_set_order(qmcspl_t h, int mode)
{
    g_err.clear();
    if (!h) return set_error(QMCSPL_ERR_ARG, "NULL handle");
    if (mode < QMCSPL_ORDER_AUTO || mode > QMCSPL_ORDER_PENCIL) return set_error(QMCSPL_ERR_ARG, "unknown order mode");
    h->order_mode = mode;
    return QMCSPL_OK;
}

int qmcspl_get_order(qmcspl_t h, long long n_pos, int* order)
{
    g_err.clear();
    if (!h) return set_error(QMCSPL_ERR_ARG, "NULL handle");
    if (!order) return set_error(QMCSPL_ERR_ARG, "order is NULL");
    if (n_pos < 0) return set_error(QMCSPL_ERR_ARG, "n_pos < 0");
    DeviceGuard dg(h->device);
    BinGeometry g;
    StagedArgs sa;
    if (n_pos > 0 && use_staged(h, n_pos) && staged_plan(h, n_pos, &g, &sa)) *order = QMCSPL_ORDER_PENCIL;
    else *order = n_pos > 0 && use_cell_order(h, n_pos) ? QMCSPL_ORDER_CELL : QMCSPL_ORDER_INPUT;
    return QMCSPL_OK;
}

int qmcspl_sync(qmcspl_t h, void* stream)
{
    g_err.clear();
    if (!h) return set_error(QMCSPL_ERR_ARG, "NULL handle");
    DeviceGuard dg(h->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_error(e, "cudaStreamSynchronize");
    int flag = 0;
    e = cudaMemcpy(&flag, h->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_error(e, "error word read");
    if (flag) {
        cudaMemset(h->d_err, 0, sizeof(int));
        if (flag & 4)
            return set_error(QMCSPL_ERR_TIMEOUT, "a wait of the staged evaluation pipeline gave up");
        if (flag & 2)
            return set_error(QMCSPL_ERR_DEVICE, "a kernel caught an out-of-range table, plane or position "
                                                "index");
        return set_error(QMCSPL_ERR_DEVICE, "a kernel saw a non-finite position");
    }
    return QMCSPL_OK;
}

}  // extern "C"
