// sb_precheck.cuh -- launch interface of the preprocessing probe (Sec. 3.4).
#pragma once
#include "sb_internal.cuh"

namespace sb {

// Doubles of scratch the probe needs for dimension d and K components.
size_t precheck_scratch_elems(int d, int K);
// Sensitivities s[d], classes cls[d] (0 active, 1 flat, 2 soft), the flagged coordinates'
// marginal log-integral and log-volume, and the active count, from pv's a_k, c, half.
void launch_precheck(const ProbView &pv, double eps_flat, double eps_soft, double *scratch, double *s, int8_t *cls,
                     double *log_int, double *log_vol, int32_t *n_active, cudaStream_t st);

}  // namespace sb
