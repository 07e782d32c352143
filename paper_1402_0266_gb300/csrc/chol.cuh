// chol.cuh -- the direct subdomain solves (chol.cu).
#pragma once

#include "common.cuh"

namespace sdd {

// Whether an mx x my subdomain fits the direct solve, and the launch (one block
// per system of a.sys, both fields; a.iters 1 per system, max_iter + 1 and the
// status bit when the residual misses rtol).
bool chol_fits(int mx, int my);
cudaError_t launch_chol(const SolveArgs& a, int mx_max, int my_max, cudaStream_t s);

}  // namespace sdd
