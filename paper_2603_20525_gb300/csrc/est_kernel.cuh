// est_kernel.cuh - launcher of the planar (EST) rollout and argmin kernel.
// The kernel takes the SRB kernel's parameter block: x0 and x0_soa hold the
// 7-component EST state, xf receives 7 rows, margin is the lateral-
// acceleration margin, and the vehicle's EST constants (Kzzf, Kzzr, Kzx, abar)
// and the cost's inv_eps (1 / eps of that constraint) must be set.
#pragma once

#include "plan_kernel.cuh"

namespace atp {

cudaError_t launch_est(const PlanParams &p, bool reduce, cudaStream_t stream);

}  // namespace atp
