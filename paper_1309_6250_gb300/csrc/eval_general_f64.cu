// eval_general_f64.cu -- the general B-spline evaluation kernels (eval_general.cuh) for FP64
// tables.
#include "eval_general.cuh"

namespace qmcspl {

int launch_general_f64(const Handle* h, const EvalArgs& a, cudaStream_t st)
{
    return launch_typed<double>(h, a, st);
}

}  // namespace qmcspl
