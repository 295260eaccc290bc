// checkpoint.cu -- qmcspl_save / qmcspl_load: built tables to and from a file.
//
// File layout (little-endian, as the host writes it):
//   FileHeader (fixed size, below); for a non-uniform grid the grid points of the three
//   axes (dims[0] + dims[1] + dims[2] doubles); then n_tables * table_elems * elem_bytes
//   bytes of tables exactly as they sit on the device.  The checksum covers both.
#include <cerrno>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "qmcspl_internal.cuh"

namespace qmcspl {
namespace {

constexpr char kMagic[8] = {'Q', 'M', 'C', 'S', 'P', 'L', 'T', 'B'};
constexpr int kFormatVersion = 3;   // 2: Bloch flag and k point; 3: degree and grid points
constexpr int kLayoutVersion = 1;   // ghost planes, padding and chunk order of the tables

struct FileHeader {
    char magic[8];
    int format_version, layout_version;
    int dims[3];
    int n_orb, n_orb_p;
    int method, storage, separate_lap, separate_grad;
    int lanes_log2, tiles;
    int n_tables, entries, rows_z;
    int bloch;
    int degree, nonuniform;
    long long n_pw;
    long long table_elems;
    long long elem_bytes;
    double lattice[9];
    double kpoint[3];
    unsigned long long checksum;   // FNV-1a 64 of the table bytes
};

unsigned long long fnv1a(const unsigned char* p, size_t n, unsigned long long h = 1469598103934665603ULL)
{
    for (size_t i = 0; i < n; ++i) {
        h ^= p[i];
        h *= 1099511628211ULL;
    }
    return h;
}

int io_error(const char* what, const char* path)
{
    return set_error(QMCSPL_ERR_ARG, std::string(what) + " '" + path + "': " + std::strerror(errno));
}

}  // namespace

// Geometry-derived fields of a handle (inverse lattice and chain-rule matrices).
bool handle_geometry(Handle* h, const double lattice[9]);

}  // namespace qmcspl

using namespace qmcspl;

extern "C" int qmcspl_save(qmcspl_t h, const char* path)
{
    if (!h || !path) return set_error(QMCSPL_ERR_ARG, "NULL argument");
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(h->device);
    const size_t bytes = h->table_elems * h->elem_bytes * h->n_tables;
    std::vector<unsigned char> buf;
    try {
        buf.resize(bytes);
    } catch (...) {
        cudaSetDevice(prev);
        return set_error(QMCSPL_ERR_OOM, "host allocation failed");
    }
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(buf.data(), h->tables, bytes, cudaMemcpyDeviceToHost);
    cudaSetDevice(prev);
    if (e != cudaSuccess) return cuda_error(e, "table download");
    FileHeader hd;
    std::memset(&hd, 0, sizeof(hd));
    std::memcpy(hd.magic, kMagic, 8);
    hd.format_version = kFormatVersion;
    hd.layout_version = kLayoutVersion;
    for (int a = 0; a < 3; ++a) hd.dims[a] = h->dims[a];
    hd.n_orb = h->n_orb;
    hd.n_orb_p = h->n_orb_p;
    hd.method = h->method;
    hd.storage = h->storage;
    hd.separate_lap = h->separate_lap;
    hd.separate_grad = h->separate_grad;
    hd.lanes_log2 = h->lanes_log2;
    hd.tiles = h->tiles;
    hd.n_tables = h->n_tables;
    hd.entries = h->entries;
    hd.rows_z = h->rows_z;
    hd.n_pw = h->n_pw;
    hd.table_elems = (long long)h->table_elems;
    hd.elem_bytes = (long long)h->elem_bytes;
    std::memcpy(hd.lattice, h->lattice, sizeof(hd.lattice));
    hd.bloch = h->bloch;
    hd.degree = h->degree;
    hd.nonuniform = h->nonuniform;
    std::memcpy(hd.kpoint, h->kpoint, sizeof(hd.kpoint));
    std::vector<double> pts;
    if (h->nonuniform)
        for (int a = 0; a < 3; ++a) pts.insert(pts.end(), h->knots[a], h->knots[a] + h->dims[a]);
    const size_t pbytes = pts.size() * sizeof(double);
    hd.checksum = fnv1a(buf.data(), buf.size(),
                        fnv1a(reinterpret_cast<const unsigned char*>(pts.data()), pbytes));
    FILE* f = std::fopen(path, "wb");
    if (!f) return io_error("cannot open", path);
    const bool ok = std::fwrite(&hd, sizeof(hd), 1, f) == 1 &&
                    (pbytes == 0 || std::fwrite(pts.data(), 1, pbytes, f) == pbytes) &&
                    std::fwrite(buf.data(), 1, bytes, f) == bytes;
    const bool closed = std::fclose(f) == 0;
    if (!ok || !closed) return io_error("cannot write", path);
    return QMCSPL_OK;
}

extern "C" int qmcspl_load(qmcspl_t* out, const char* path, void* stream)
{
    if (!out || !path) return set_error(QMCSPL_ERR_ARG, "NULL argument");
    *out = nullptr;
    FILE* f = std::fopen(path, "rb");
    if (!f) return io_error("cannot open", path);
    FileHeader hd;
    if (std::fread(&hd, sizeof(hd), 1, f) != 1) {
        std::fclose(f);
        return set_error(QMCSPL_ERR_ARG, "truncated table file (header)");
    }
    if (std::memcmp(hd.magic, kMagic, 8) != 0) {
        std::fclose(f);
        return set_error(QMCSPL_ERR_ARG, "not a qmcspl table file");
    }
    if (hd.format_version != kFormatVersion || hd.layout_version != kLayoutVersion) {
        std::fclose(f);
        return set_error(QMCSPL_ERR_ARG, "table file format or layout version not supported by this library");
    }
    // sizes must agree with what qmcspl_create would have built
    bool sane = hd.n_orb >= 1 && hd.n_orb_p >= hd.n_orb && hd.method >= QMCSPL_BSPLINE_SMOOTH &&
                hd.method <= QMCSPL_PPSPLINE && hd.storage >= QMCSPL_F64 && hd.storage <= QMCSPL_DF64 &&
                hd.lanes_log2 >= 0 && hd.lanes_log2 <= 5 && hd.tiles >= 1 && hd.n_tables >= 1 && hd.n_tables <= 5 &&
                (hd.entries == 1 || hd.entries == 8);
    for (int a = 0; a < 3; ++a) sane = sane && hd.dims[a] >= 4 && hd.dims[a] <= kMaxDim;
    const long long eb = hd.storage == QMCSPL_BF16 ? 2 : (hd.storage == QMCSPL_F32 ? 4 : 8);
    sane = sane && hd.elem_bytes == eb && (long long)hd.n_orb_p * hd.elem_bytes % 16 == 0 &&
           hd.n_orb_p == hd.tiles * (1 << hd.lanes_log2) * (int)(16 / eb) &&
           (hd.degree == 1 || hd.degree == 3 || hd.degree == 5 || hd.degree == 7) &&
           (hd.nonuniform == 0 || hd.nonuniform == 1) &&
           hd.rows_z == hd.dims[2] + (hd.method == QMCSPL_PPSPLINE ? 1 : hd.degree) &&
           hd.table_elems == (long long)hd.dims[0] * hd.dims[1] * hd.rows_z * hd.entries * hd.n_orb_p;
    for (int i = 0; i < 9; ++i) sane = sane && std::isfinite(hd.lattice[i]);
    sane = sane && (hd.bloch == 0 || (hd.bloch == 1 && hd.n_orb % 2 == 0));
    sane = sane && (hd.separate_grad == 0 || hd.separate_grad == 1) && (hd.separate_lap == 0 || hd.separate_lap == 1);
    {
        const int want = hd.method == QMCSPL_PPSPLINE ? 1
                         : (hd.method == QMCSPL_LAGRANGE || hd.separate_grad) ? 5
                         : (hd.separate_lap ? 2 : 1);
        sane = sane && hd.n_tables == want && hd.entries == (hd.method == QMCSPL_PPSPLINE ? 8 : 1);
    }
    for (int i = 0; i < 3; ++i) sane = sane && std::isfinite(hd.kpoint[i]) && (hd.bloch || hd.kpoint[i] == 0.0);
    if (!sane) {
        std::fclose(f);
        return set_error(QMCSPL_ERR_ARG, "inconsistent table file header");
    }
    const size_t bytes = (size_t)hd.table_elems * (size_t)hd.elem_bytes * (size_t)hd.n_tables;
    std::vector<double> pts(hd.nonuniform ? (size_t)hd.dims[0] + hd.dims[1] + hd.dims[2] : 0);
    const size_t pbytes = pts.size() * sizeof(double);
    if (pbytes && std::fread(pts.data(), 1, pbytes, f) != pbytes) {
        std::fclose(f);
        return set_error(QMCSPL_ERR_ARG, "truncated table file (grid points)");
    }
    std::vector<unsigned char> buf;
    try {
        buf.resize(bytes);
    } catch (...) {
        std::fclose(f);
        return set_error(QMCSPL_ERR_OOM, "host allocation failed");
    }
    const size_t got = std::fread(buf.data(), 1, bytes, f);
    const bool extra = std::fgetc(f) != EOF;
    std::fclose(f);
    if (got != bytes || extra) return set_error(QMCSPL_ERR_ARG, "table file has the wrong size");
    if (fnv1a(buf.data(), buf.size(), fnv1a(reinterpret_cast<const unsigned char*>(pts.data()), pbytes)) !=
        hd.checksum)
        return set_error(QMCSPL_ERR_ARG, "table file checksum mismatch");
    {
        size_t o = 0;
        for (int a = 0; a < 3 && hd.nonuniform; ++a)
            for (int i = 0; i < hd.dims[a]; ++i, ++o) {
                const double v = pts[o];
                if (!std::isfinite(v) || v < 0.0 || v >= 1.0 || (i > 0 && !(v > pts[o - 1])))
                    return set_error(QMCSPL_ERR_ARG, "table file has invalid grid points");
            }
    }

    Handle* h = new (std::nothrow) Handle();
    if (!h) return set_error(QMCSPL_ERR_OOM, "host allocation failed");
    cudaGetDevice(&h->device);
    for (int a = 0; a < 3; ++a) h->dims[a] = hd.dims[a];
    h->n_orb = hd.n_orb;
    h->n_orb_p = hd.n_orb_p;
    h->method = hd.method;
    h->storage = hd.storage;
    h->separate_lap = hd.separate_lap;
    h->separate_grad = hd.separate_grad;
    h->lanes_log2 = hd.lanes_log2;
    h->tiles = hd.tiles;
    h->n_tables = hd.n_tables;
    h->entries = hd.entries;
    h->rows_z = hd.rows_z;
    h->n_pw = hd.n_pw;
    h->bloch = hd.bloch;
    for (int i = 0; i < 3; ++i) h->kpoint[i] = hd.kpoint[i];
    h->degree = hd.degree;
    h->nonuniform = hd.nonuniform;
    h->zshift = hd.method == QMCSPL_PPSPLINE ? 0 : (hd.degree - 1) / 2;
    {
        size_t o = 0;
        for (int a = 0; a < 3 && hd.nonuniform; ++a)
            for (int i = 0; i < hd.dims[a]; ++i) h->knots[a][i] = pts[o++];
    }
    h->table_elems = (size_t)hd.table_elems;
    h->elem_bytes = (size_t)hd.elem_bytes;
    if (!handle_geometry(h, hd.lattice)) {
        delete h;
        return set_error(QMCSPL_ERR_ARG, "singular lattice in table file");
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = dev_malloc(&h->tables, bytes);
    if (e == cudaSuccess) e = dev_malloc((void**)&h->d_err, sizeof(int));
    if (e == cudaSuccess && h->nonuniform && upload_grid_points(h, st) != QMCSPL_OK) e = cudaErrorMemoryAllocation;
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_err, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->tables, buf.data(), bytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        const int rc = cuda_error(e, "table upload");
        qmcspl_destroy(h);
        return rc;
    }
    *out = h;
    return QMCSPL_OK;
}
