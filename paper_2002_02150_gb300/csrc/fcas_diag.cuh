// Launchers of the per-particle diagnostics (defined in fcas_diag.cu).
#pragma once

#include "fcas_internal.cuh"

namespace fcas {

// Condition number of the antenna-pattern matrix per particle (+inf for rank one, NaN for a
// non-finite angle).
cudaError_t launch_condition(const double* theta, int64_t n, const double* det9, int n_det, double* kappa,
                             cudaStream_t s);

}  // namespace fcas
