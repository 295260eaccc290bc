// backward_general_f32.cu -- the general B-spline adjoint kernels (backward_general.cuh) for
// f32 tables.
#include "backward_general.cuh"

namespace qmcspl {

int launch_general_backward_f32(const Handle* h, const BwdArgs& a, cudaStream_t st)
{
    return general_bwd_typed<float>(h, a, st);
}

}  // namespace qmcspl
