// eval_general_f32.cu -- the general B-spline evaluation kernels (eval_general.cuh) for FP32
// tables.
#include "eval_general.cuh"

namespace qmcspl {

int launch_general_f32(const Handle* h, const EvalArgs& a, cudaStream_t st)
{
    return launch_typed<float>(h, a, st);
}

}  // namespace qmcspl
