// sb_tc.cuh -- mixed-precision (tcgen05 tensor-core) log-likelihood and gradient.
#pragma once
#include <cuda.h>

#include "sb_internal.cuh"

namespace sb {

// Scratch of the tensor-core path: converted L_k copies (GEMM1 / GEMM2 layouts),
// FP32 means and box centre, z rows, |z|^2 partials, responsibilities, and the
// TMA descriptors of the two L_k copies (host-side, rebuilt per call).
struct TcWs {
    void *p[20];
    size_t rows;
    int prec, bn, d, K, ldz;
    CUtensorMap mapT, mapB;    // B operands: L_k^T (GEMM1) and L_k (GEMM2)
    CUtensorMap mapA1, mapZ;   // A operands: centred points (GEMM1) and scaled z (GEMM2)
};

bool tc_available(int prec);
void carve_tc(Carver &cv, TcWs &t, int rows, int d, int K, int prec);
int tc_ray_chunk(int d, int K, int64_t total);
// Encodes the A-operand tensor maps of this scratch (depends on its row capacity).
bool tc_maps_for_rows(TcWs &t);
// Tile width the autotuner chose for (d, K, prec) in this process (0: not tuned yet).
// A first call made inside a stream capture cannot time the candidates: it takes the
// heuristic width and leaves the shape untuned.
int tc_tuned_tile(int d, int K, int prec);
// Converts L_k / mu / c into the tensor-core copies, picks the tile width
// (autotuned once per shape; that first call synchronises the stream) and
// encodes the tensor maps. skip_bounds: also the |L_k|_2 bounds the walker
// rounds' component skip reads (one |z|^2 pass over the columns of every L_k).
sb_status tc_prepare(const ProbView &pv, TcWs &t, cudaStream_t s, bool skip_bounds = true);
// l at every ray sample x_rj = c + t_j t_exit,r u_r from the FP32 directions
// u32 [n_rays][d]; chunks of the scratch row capacity.
sb_status tc_ray_loglik(const ProbView &pv, const sb_config *c, const TcWs &t, const float *u32,
                        const double *texit, double *ell_all, cudaStream_t s);
// l at the ray samples of flat indices [f_begin, f_end) (ray = flat / n_steps,
// j = flat % n_steps): x = o_ray + ((j + 1) / n_steps) t_exit,ray u_ray formed in FP32
// inside the centring pass, o32 [rays][d] the rays' origins (the box centre when
// null); ell[flat - f_begin]. Chunks of the scratch row capacity.
sb_status tc_ray_samples(const ProbView &pv, const TcWs &t, const float *o32, const float *u32, const double *texit,
                         int n_steps, int64_t f_begin, int64_t f_end, double *ell, cudaStream_t s);
// One chunk of ray samples with the row count on the device (*n_rows_dev <= rows_max
// <= the scratch rows): flat indices f0 .. f0 + *n_rows_dev - 1, ell[flat - f0].
sb_status tc_ray_chunk(const ProbView &pv, const TcWs &t, const float *o32, const float *u32, const double *texit,
                       int n_steps, int64_t f0, int rows_max, const int32_t *n_rows_dev, double *ell, cudaStream_t s);
// y[e] = (float) x[e], e < n.
void tc_to_f32(const double *x, float *y, size_t n, cudaStream_t s);
// Clears the per-walker bounds of the component skip (before a refinement).
void tc_walkers_reset(const TcWs &t, int n, cudaStream_t s);
// Slot of TcWs.p holding the per-walker distance bound the L-BFGS step writes.
constexpr int kTcDistSlot = 14;
void tc_eval_walkers(const ProbView &pv, const sb_config *c, const TcWs &t, const float *XT, const int32_t *act,
                     const int32_t *n_act, int n, float *FT, float *GT, cudaStream_t s);
sb_status tc_loglik_points(const ProbView &pv, const sb_config *c, const TcWs &t, const double *x, int n, float *f,
                           float *g, double *ell, double *grad, cudaStream_t s);

}  // namespace sb
