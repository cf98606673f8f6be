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
// Rows of the scratch that holds the problem's tensor-core copies of L_k, mu and c
// (the autotuner's and the skip bounds' passes run on it), for total ray samples.
int tc_setup_rows(int64_t total);
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
// y[e] = (float) x[e], e < n.
void tc_to_f32(const double *x, float *y, size_t n, cudaStream_t s);

// The sunburst rays from the box centre c as a quadratic form (Sec. 3.5.1-3.5.2):
// along ray r, z_k(c + tau u_r) = z_k(c) + tau w_rk with w_rk = L_k^T u_r, so l at
// every sample of the ray follows from q0_k = |z_k(c)|^2, q1_rk = z_k(c) . w_rk and
// q2_rk = |w_rk|^2, tau = ((j + 1) / n_steps) t_exit,r. z_k(c) is FP64; w comes from
// one tensor-core GEMM of the n_rays directions (not of n_rays n_steps samples) whose
// operands are split into high and low parts, u_hi L_hi + u_lo L_hi + u_hi L_lo, close
// to FP32 accuracy: near a mode the three terms cancel (|z_k(c)|^2 ~ 1e6 at d = 1024).
struct TcQuadWs {
    void *A2, *B2;                   // [rows][2 dK] direction splits, [K][d][2 dK] L_k^T splits
    float *alpha, *qpart1, *qpart2;  // [K][ald] z_k(c) in FP32 (zero past d); partials [rows][K][nct]
    double *zc, *q0;                 // [K][d] z_k(c), [K] |z_k(c)|^2
    double2 *q12;                    // [n_rays][K] (z_k(c) . w_rk, |w_rk|^2) in FP64
    int rows, dK, ald;
    CUtensorMap mapU, mapL;
};
void carve_tc_quad(Carver &cv, TcQuadWs &q, int n_rays, int d, int K, int prec);
// l at every ray sample from the FP64 directions u [n_rays][d] and t_exit; ell_all[r n_steps + j].
// bn: the GEMM's column tile (64, 128 or 256; 0: the width tuned for (d, K, prec) in
// this process, else the heuristic one). pv needs a_k, mu, L and c.
sb_status tc_ray_loglik_quad(const ProbView &pv, int n_rays, int n_steps, int prec, int bn, TcQuadWs q,
                             const double *u, const double *texit, double *ell_all, cudaStream_t s);
// Rays from per-ray origins, x = o_r + tau u_r, in the same quadratic form:
// z_k(o_r + tau u_r) = z_k(o_r) + tau w_rk, z_k(o_r) = o_r L_k - mu_k L_k from a split
// GEMM of the origins (FP32 result, stored, with the FP32 -mu_k L_k added in the
// epilogue), w_rk from a split GEMM of the directions whose epilogue takes the
// dot products with the stored z_k(o_r).
struct TcOriginWs {
    float *zo, *off, *qp0;  // [rows][K][ald] z_k(o_r); [K][ald] -mu_k L_k (FP32); [rows][K][nct] |z|^2 partials
    double *negm, *q0k;     // [K][d] -mu_k L_k (FP64); [K] scratch
    double *q0r;            // [rows][K] |z_k(o_r)|^2
};
void carve_tc_origins(Carver &cv, TcOriginWs &o, int n_rays, int d, int K, int prec);
// Split L_k^T into q.B2 and -mu_k L_k into o.off (once per problem and call).
sb_status tc_quad_prepare_origins(const ProbView &pv, int prec, TcQuadWs q, TcOriginWs o, cudaStream_t s);
// l at sample j of ray r < *n_rays_dev (flat r n_steps + j < *n_samples_dev, both on
// the device, at most n_cap rays): ell[r n_steps + j], tau = ((j + 1) / n_steps)
// t_exit,r. O, U: [n_cap][d] FP64 origins and unit directions. q must hold n_cap rays.
sb_status tc_ray_origins_quad(const ProbView &pv, int n_cap, int n_steps, int prec, int bn, TcQuadWs q, TcOriginWs o,
                              const double *O, const double *U, const double *texit, const int32_t *n_rays_dev,
                              const int32_t *n_samples_dev, double *ell, cudaStream_t s);
// Clears the per-walker bounds of the component skip (before a refinement).
void tc_walkers_reset(const TcWs &t, int n, cudaStream_t s);
// Slot of TcWs.p holding the per-walker distance bound the L-BFGS step writes.
constexpr int kTcDistSlot = 14;
void tc_eval_walkers(const ProbView &pv, const sb_config *c, const TcWs &t, const float *XT, const int32_t *act,
                     const int32_t *n_act, int n, float *FT, float *GT, cudaStream_t s);
sb_status tc_loglik_points(const ProbView &pv, const sb_config *c, const TcWs &t, const double *x, int n, float *f,
                           float *g, double *ell, double *grad, cudaStream_t s);

}  // namespace sb
