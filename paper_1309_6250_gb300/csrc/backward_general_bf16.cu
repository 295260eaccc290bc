// backward_general_bf16.cu -- the general B-spline adjoint kernels (backward_general.cuh) for
// bf16 tables.
#include "backward_general.cuh"

namespace qmcspl {

int launch_general_backward_bf16(const Handle* h, const BwdArgs& a, cudaStream_t st)
{
    return general_bwd_typed<__nv_bfloat16>(h, a, st);
}

}  // namespace qmcspl
