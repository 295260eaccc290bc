// noalloc.cu -- qmcspl_eval_vgl_noalloc: cell-ordered evaluation with a fixed scratch
// array instead of allocated memory (for callers that cannot allocate device memory).
//
// The scratch of the cell-order sort lives in g_noalloc_scratch below, a file-scope
// __device__ array that every GPU loading the library holds until the process exits:
//   [0, max_pos)                    bin of each position
//   [max_pos, 2 max_pos)            evaluation order (permutation)
//   [2 max_pos, 2 max_pos + bins+1) bin counters, cleared by every call
// Host code must not pass the symbol itself to a kernel (on the host it only names a
// stand-in); the device address is looked up once per device with
// cudaGetSymbolAddress while that device is current.
#include <mutex>

#include "qmcspl_internal.cuh"

namespace qmcspl {
namespace {

constexpr long long kNoAllocMaxPos = QMCSPL_NOALLOC_MAX_POS;
// bin_geometry never makes more than kMaxBins bins; the counters take one more entry (the total)
constexpr size_t kScratchInts = (size_t)(2 * kNoAllocMaxPos + kMaxBins + 1);
constexpr int kMaxDevices = 64;
static_assert(kScratchInts * sizeof(int) < (16u << 20), "the fixed scratch array stays modest");

static __device__ __align__(256) int g_noalloc_scratch[kScratchInts];

std::mutex g_scratch_mutex;
int* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on device `dev`, which must be the current device
// (looked up once per device and cached).
int scratch_on_device(int dev, int** out)
{
    if (dev < 0 || dev >= kMaxDevices) return set_error(QMCSPL_ERR_UNSUPPORTED, "device index out of range");
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[dev]) {
        int cur = -1;
        cudaError_t e = cudaGetDevice(&cur);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
        if (cur != dev) return set_error(QMCSPL_ERR_CUDA, "noalloc scratch looked up on the wrong device");
        int* p = nullptr;
        e = cudaGetSymbolAddress((void**)&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(noalloc scratch)");
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return QMCSPL_OK;
}

}  // namespace
}  // namespace qmcspl

using namespace qmcspl;

extern "C" int qmcspl_eval_vgl_noalloc(qmcspl_t h, const double* pos, long long n_pos, void* val,
                                       void* grad, void* lap, void* stream)
{
    clear_error();
    if (!h) return set_error(QMCSPL_ERR_ARG, "NULL handle");
    if (n_pos < 0) return set_error(QMCSPL_ERR_ARG, "n_pos < 0");
    if (n_pos > kNoAllocMaxPos)
        return set_error(QMCSPL_ERR_ARG, "qmcspl_eval_vgl_noalloc: n_pos " + std::to_string(n_pos) +
                                             " exceeds QMCSPL_NOALLOC_MAX_POS (" +
                                             std::to_string(kNoAllocMaxPos) + ")");
    if (h->bloch)
        return set_error(QMCSPL_ERR_UNSUPPORTED, "qmcspl_eval_vgl_noalloc: Bloch handles need per-position phase scratch");
    if (n_pos == 0) return QMCSPL_OK;
    if (!pos) return set_error(QMCSPL_ERR_ARG, "pos is NULL");
    const BinGeometry g = bin_geometry(h);
    if (g.n_bins > kMaxBins) return set_error(QMCSPL_ERR_UNSUPPORTED, "cell-order bins exceed the scratch array");
    int prev = -1;
    cudaError_t e = cudaGetDevice(&prev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    if (prev != h->device && (e = cudaSetDevice(h->device)) != cudaSuccess) return cuda_error(e, "cudaSetDevice");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int* scratch = nullptr;
    int rc = scratch_on_device(h->device, &scratch);
    if (rc == QMCSPL_OK) {
        int* bin = scratch;
        int* perm = scratch + kNoAllocMaxPos;
        int* count = scratch + 2 * kNoAllocMaxPos;
        rc = build_cell_order(h, pos, n_pos, bin, count, perm, g, st);
        if (rc == QMCSPL_OK) {
            Prepared pr;
            pr.perm = perm;
            switch (h->method) {
            case QMCSPL_LAGRANGE: rc = launch_five_table_vgl(h, pos, pr, n_pos, val, grad, lap, st); break;
            case QMCSPL_PPSPLINE: rc = launch_pp_vgl(h, pos, pr, n_pos, val, grad, lap, st); break;
            default:
                rc = h->separate_grad  ? launch_five_table_vgl(h, pos, pr, n_pos, val, grad, lap, st)
                     : is_general(h) ? launch_general_vgl(h, pos, pr, n_pos, val, grad, lap, st)
                                       : launch_bspline_vgl(h, pos, pr, n_pos, val, grad, lap, st);
                break;
            }
        }
    }
    if (prev >= 0 && prev != h->device) {
        e = cudaSetDevice(prev);
        if (rc == QMCSPL_OK && e != cudaSuccess) rc = cuda_error(e, "cudaSetDevice (restore)");
    }
    return rc;
}
