// heat_sweeps_f32.cu -- instantiation of the sweep kernels for the FP32 path (increment form).
#include "heat_kernels.cuh"

namespace heat {

cudaError_t plan_fp32(SweepArgs<float> *h, int n, const Tuning &req, SweepPlan &plan)
{
    return plan_mode<float, MODE_DELTA>(h, n, req, plan);
}

}  // namespace heat
