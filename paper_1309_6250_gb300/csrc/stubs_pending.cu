// Entry points whose kernels are not written yet report QMCSPL_ERR_UNSUPPORTED.
#include "qmcspl_internal.cuh"

namespace qmcspl {

int launch_lagrange_vgl(const Handle*, const double*, long long, void*, void*, void*, cudaStream_t)
{
    return set_error(QMCSPL_ERR_UNSUPPORTED, "Lagrange evaluation not available in this build");
}

int launch_pp_vgl(const Handle*, const double*, long long, void*, void*, void*, cudaStream_t)
{
    return set_error(QMCSPL_ERR_UNSUPPORTED, "pp-spline evaluation not available in this build");
}

int launch_bspline_backward(const Handle*, const double*, long long, const void*, const void*,
                            const void*, void*, void*, double*, cudaStream_t)
{
    return set_error(QMCSPL_ERR_UNSUPPORTED, "backward not available in this build");
}

int launch_batched(int, const Handle* const*, const double* const*, const long long*, void* const*,
                   void* const*, void* const*, cudaStream_t)
{
    return set_error(QMCSPL_ERR_UNSUPPORTED, "batched evaluation not available in this build");
}

}  // namespace qmcspl
