// sb_segments.cuh -- launch interface of the V2V / V2E / W2W rays and their two-pass sampling
// (Sec. 3.5.1-3.5.2).
#pragma once
#include "sb_internal.cuh"

namespace sb {

// Doubles of scratch for n_rays rays of n_steps coarse samples (d, K of the problem).
size_t segments_scratch_elems(int n_rays, int n_steps, int d, int K);
// ends: [2][n_rays][d] (starts, then ends); ell_coarse: [n_rays][n_steps]; t_ref, ell_ref:
// [n_rays][n_ref]. pv needs a_k (launch_setup).
void launch_segments(const ProbView &pv, int family, uint64_t seed, int n_rays, int n_steps, double delta, int n_ref,
                     double *scratch, double *ends, double *ell_coarse, double *t_ref, double *ell_ref,
                     cudaStream_t s);

}  // namespace sb
