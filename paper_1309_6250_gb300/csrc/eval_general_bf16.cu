// eval_general_bf16.cu -- the general B-spline evaluation kernels (eval_general.cuh) for BF16
// tables.
#include "eval_general.cuh"

namespace qmcspl {

int launch_general_bf16(const Handle* h, const EvalArgs& a, cudaStream_t st)
{
    return launch_typed<__nv_bfloat16>(h, a, st);
}

}  // namespace qmcspl
