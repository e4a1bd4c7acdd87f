// heat_sweeps_f64.cu -- instantiation of the sweep kernels for the FP64 path (literal form of eqs. "scheme_eq_1", "scheme_eq_2").
#include "heat_kernels.cuh"

namespace heat {

cudaError_t plan_fp64(SweepArgs<double> *h, int n, const Tuning &req, SweepPlan &plan)
{
    return plan_mode<double, MODE_LIT>(h, n, req, plan);
}

}  // namespace heat
