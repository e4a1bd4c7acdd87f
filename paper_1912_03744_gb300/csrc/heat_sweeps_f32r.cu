// heat_sweeps_f32r.cu -- instantiation of the sweep kernels for the refined FP32 path (increment form + FP64 residual correction).
#include "heat_kernels.cuh"

namespace heat {

cudaError_t plan_fp32_refined(SweepArgs<float> *h, int n, const Tuning &req, SweepPlan &plan)
{
    return plan_mode<float, MODE_REFINE>(h, n, req, plan);
}

}  // namespace heat
