// eval_general.cu -- entry of the general B-spline evaluation (eval_general.cuh): the
// kernels of each table type are compiled in their own translation unit.
#include "eval_general.cuh"

namespace qmcspl {

int launch_general_vgl(const Handle* h, const double* pos, const Prepared& pr, long long n_pos, void* val,
                       void* grad, void* lap, cudaStream_t st)
{
    EvalArgs a;
    fill_eval_args(h, &a);
    a.pos = pos;
    a.rec = pr.rec;           // records of kind 1/2 (uniform) or 4/5 (non-uniform), or none
    a.perm = pr.perm;
    a.phase = pr.phase;
    a.n_pos = n_pos;
    a.val = val;
    a.grad = grad;
    a.lap = lap;
    const size_t ob = (h->storage == QMCSPL_F64) ? 8 : 4;
    const uintptr_t al = (uintptr_t)val | (uintptr_t)grad | (uintptr_t)lap;
    a.vec_out = ((h->n_orb * ob) % 16 == 0) && (al % 16 == 0);
    switch (h->storage) {
    case QMCSPL_F64: return launch_general_f64(h, a, st);
    case QMCSPL_F32: return launch_general_f32(h, a, st);
    default: return launch_general_bf16(h, a, st);
    }
}

}  // namespace qmcspl
