// sb_raysq.cuh -- sunburst ray likelihoods from three scalars per (ray, component).
#pragma once
#include "sb_internal.cuh"

namespace sb {

// t_exit,r = min_i half_i / |u_ri| of each direction u [n_rays][d] from the box centre.
void launch_ray_texit(const ProbView &pv, const double *u, int n_rays, double *texit, cudaStream_t s);
// Doubles of scratch for n_rays directions; form 0 = FP64 GEMM, 1 = FP32 SIMT GEMM.
size_t rayq_scratch_elems(int n_rays, int d, int K, int form);
// ell[r][j] = l(c + ((j + 1) / n_steps) t_exit,r u_r) for directions u [n_rays][d]; pv needs a_k,
// c and half (launch_setup).
void launch_ray_loglik_quad(const ProbView &pv, int form, const double *u, int n_rays, int n_steps, double *scratch,
                            double *ell, cudaStream_t s);

}  // namespace sb
