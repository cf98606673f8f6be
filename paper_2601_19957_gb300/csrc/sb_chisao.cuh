// sb_chisao.cuh -- launch interface of the ChiSao oscillation kernels (Sec. 3.5.5).
#pragma once
#include "sb_internal.cuh"

namespace sb {

// Gradient test: conv[s] = l_s finite and |G_s|_inf <= eps (1 + |l_s|).
void launch_cs_conv(int n, int d, const double *G, const double *ell, double eps, uint8_t *conv, cudaStream_t s);
// Mixed-precision form of the test: conv[s] = l_s finite and status CONVERGED or STALLED.
void launch_cs_conv_status(int n, const int8_t *status, const double *ell, uint8_t *conv, cudaStream_t s);
// Stick test over all samples (one CTA): stuck[s] = conv[s] and l_s >= max_finite l + log 0.1.
void launch_cs_stick(int n, const double *ell, const uint8_t *conv, uint8_t *stuck, cudaStream_t s);
// After the dedup of the stuck samples: lost = stuck and not a representative; stuck = representative.
void launch_cs_split(int n, const int32_t *reps, const int32_t *n_reps, uint8_t *stuck, uint8_t *lost,
                     cudaStream_t s);
// Ordered lists (ascending sample index): lost, unconverged (finite l, conv == 0), moving (not stuck,
// status not NONFINITE); counts in cnt[0..2].
void launch_cs_lists(int n, const uint8_t *lost, const uint8_t *conv, const uint8_t *stuck, const int8_t *status,
                     const double *ell, int32_t *lost_list, int32_t *unconv_list, int32_t *moving_list, int32_t *cnt,
                     cudaStream_t s);
// Repulse Monkey rays: origin = unconverged sample (l mod n_unconv) clamped to the box, direction a
// unit Philox-normal vector (counter (pair, l, osc, 'RPMK')), t_exit to the box face.
void launch_cs_rm_rays(int n_lost, int d, uint64_t seed, int osc, const int32_t *unconv_list, int n_unconv,
                       const double *X, const double *lo, const double *hi, double *O, double *U, double *texit,
                       cudaStream_t s);
// Golden Rooster bases: job j fills cols[j] orthonormal columns (column c at Q + off[j] + c d) of basis
// b[j] of peak pk[j]: Philox normals (counter (pair, b d + c, osc << 16 | pk, 'GRST')) made orthonormal
// in column order (classical Gram-Schmidt, two passes).
void launch_cs_bases(int n_jobs, int d, uint64_t seed, int osc, const int32_t *job_pk, const int32_t *job_b,
                     const int32_t *job_cols, const int64_t *job_off, double *Q, bool fp32, cudaStream_t s);
// Golden Rooster rays: lost sample l -> peak pk = l mod n_peaks, direction c = (l / n_peaks) / 2 with sign
// + for even l / n_peaks, column c mod d of basis c / d; origin = the peak clamped to the box.
void launch_cs_gr_rays(int n_lost, int d, int n_peaks, const int32_t *reps, const double *X, const double *lo,
                       const double *hi, const int32_t *job_start, const int64_t *job_off, const double *Q, double *O,
                       double *U, double *texit, cudaStream_t s);
// Ray samples of lost samples l0 .. l0 + nl - 1: P[(l - l0) n_steps + j] = o_l + ((j+1)/n_steps) t_exit,l u_l.
void launch_cs_ray_points(int l0, int nl, int n_steps, int d, const double *O, const double *U, const double *texit,
                          double *P, cudaStream_t s);
// Best sample of each ray (past the first valley if past_valley) written to X[lost_list[l]].
void launch_cs_ray_pick(int l0, int nl, int n_steps, int d, int past_valley, const double *ellp,
                        const int32_t *lost_list, const double *O, const double *U, const double *texit, double *X,
                        cudaStream_t s);
// One momentum descent step of the moving samples: v <- m v - alpha grad l, x <- clamp(x + v).
void launch_cs_momentum(int n, int d, const int32_t *moving_list, const int32_t *n_moving, double momentum,
                        double alpha, const double *G, double *V, double *X, const double *lo, const double *hi,
                        cudaStream_t s);
// *dst += *src (when src is given) + v, on the device (evaluation counters).
void launch_cs_stat_add(int64_t *dst, const int64_t *src, int64_t v, cudaStream_t s);

}  // namespace sb
