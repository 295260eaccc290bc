// backward_general_f64.cu -- the general B-spline adjoint kernels (backward_general.cuh) for
// f64 tables.
#include "backward_general.cuh"

namespace qmcspl {

int launch_general_backward_f64(const Handle* h, const BwdArgs& a, cudaStream_t st)
{
    return general_bwd_typed<double>(h, a, st);
}

}  // namespace qmcspl
