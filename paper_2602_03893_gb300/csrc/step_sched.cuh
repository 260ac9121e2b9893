// step_sched.cuh -- per-step scalars of the reconstruction step (Algorithm 2), kept on the device
// so that every step launches the same kernels with the same arguments (step.cu, gpair_abi.cu).
#pragma once

namespace gp {

struct StepSched {
    int t;                       // steps taken
    float eta, inv_c1, inv_sqrt_c2;
    double b1t, b2t;             // beta1^t, beta2^t (running products)
};
struct SchedParams {
    double eta_max, eta_min, T_mult, beta1, beta2;
    int T0;
};

}  // namespace gp
