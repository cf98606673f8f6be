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
// Device-side state of the oscillations (int32 [8] in the workspace): whether Golden
// Rooster is still on, whether the last reseeding used it, the previous peak count,
// the reseeding branch (0 none, 1 Repulse Monkey, 2 Golden Rooster) and its job count.
void launch_cs_state_init(int32_t *state, cudaStream_t s);
// After the stick test and dedup (n_peaks representatives): Golden Rooster switches off
// for good once an oscillation that used it ends with no more peaks than the one before.
void launch_cs_osc_state(const int32_t *n_peaks, int32_t *state, cudaStream_t s);
// The reseeding branch from the list counts cnt (lost, unconverged, moving): Repulse
// Monkey when at least min_unconv samples are unconverged, else Golden Rooster while
// on and with peaks, else none; for Golden Rooster the job tables of its orthonormal
// groups (lost sample l: peak l mod n_peaks, direction c = (l / n_peaks) / 2, column
// c mod G of group c / G, G = min(d, 64); job_start [n_peaks + 1]). Adds the ray
// samples to evaluate (lost x n_steps) to stats[0].
void launch_cs_branch(const int32_t *cnt, const int32_t *n_peaks, int min_unconv, int d, int n_steps, int32_t *state,
                      int32_t *job_start, int32_t *job_pk, int32_t *job_b, int32_t *job_cols, int64_t *job_off,
                      int64_t *stats, cudaStream_t s);
// Repulse Monkey rays (when the branch is 1; lost sample l < cnt[0], grid for n):
// origin = unconverged sample (l mod cnt[1]) clamped to the box, direction a unit
// Philox-normal vector (counter (pair, l, osc, 'RPMK')), t_exit to the box face.
// t_exit,l = min over u_li != 0 of (hi_i - o_li) / u_li or (lo_i - o_li) / u_li (0 when
// no coordinate moves): the distance from origin o_l along u_l to the box surface.
void launch_cs_exit(int n, int d, const double *O, const double *U, const double *lo, const double *hi, double *texit,
                    cudaStream_t s);
void launch_cs_rm_rays(int n, int d, uint64_t seed, int osc, const int32_t *unconv_list, const int32_t *cnt,
                       const int32_t *state, const double *X, const double *lo, const double *hi, double *O, double *U,
                       double *texit, cudaStream_t s);
// Golden Rooster groups (when the branch is 2; job j < the job count, grid for
// max_jobs): job j fills cols[j] orthonormal columns (column c at Q + off[j] + c d) of
// group b[j] of peak pk[j]: Philox normals (counter (pair, b G + c, osc << 16 | pk,
// 'GRST')) made orthonormal in column order (the Q factor of their QR, by Cholesky QR
// applied twice), in FP32 when fp32, else FP64.
void launch_cs_bases(int max_jobs, int d, uint64_t seed, int osc, const int32_t *job_pk, const int32_t *job_b,
                     const int32_t *job_cols, const int64_t *job_off, const int32_t *state, double *Q, bool fp32,
                     cudaStream_t s);
// Golden Rooster rays (when the branch is 2; lost sample l < cnt[0], grid for n): peak
// pk = l mod n_peaks, direction c = (l / n_peaks) / 2 with sign + for even
// l / n_peaks, column c mod G of group c / G; origin = the peak clamped to the box.
void launch_cs_gr_rays(int n, int d, const int32_t *n_peaks, const int32_t *reps, const double *X, const double *lo,
                       const double *hi, const int32_t *job_start, const int64_t *job_off, const double *Q,
                       const int32_t *cnt, const int32_t *state, double *O, double *U, double *texit,
                       cudaStream_t s);
// *rows = ray samples of the reseeding chunk of lost samples l0 .. l0 + lc - 1 (0 when
// there is no reseeding): min(max(cnt[0] - l0, 0), lc) n_steps.
void launch_cs_chunk_rows(const int32_t *cnt, const int32_t *state, int l0, int lc, int n_steps, int32_t *rows,
                          cudaStream_t s);
// Ray samples of the chunk from l0 (*rows of them, grid for lc rays):
// P[(l - l0) n_steps + j] = o_l + ((j+1)/n_steps) t_exit,l u_l.
void launch_cs_ray_points(int l0, int lc, int n_steps, int d, const double *O, const double *U, const double *texit,
                          const int32_t *rows, double *P, cudaStream_t s);
// Best sample of each ray of the chunk (past the first valley for Golden Rooster)
// written to X[lost_list[l]].
void launch_cs_ray_pick(int l0, int lc, int n_steps, int d, const int32_t *rows, const int32_t *state,
                        const double *ellp, const int32_t *lost_list, const double *O, const double *U,
                        const double *texit, double *X, cudaStream_t s);
// One momentum descent step of the moving samples: v <- m v - alpha grad l, x <- clamp(x + v).
void launch_cs_momentum(int n, int d, const int32_t *moving_list, const int32_t *n_moving, double momentum,
                        double alpha, const double *G, double *V, double *X, const double *lo, const double *hi,
                        cudaStream_t s);
// The mixed path's momentum step in FP32 on the moving samples: GT = grad f (= -grad l),
// v <- m v + alpha GT, x <- clamp(x + v); dist[s] = an upper bound on the move.
void launch_cs_momentum_f32(int n, int d, const int32_t *moving_list, const int32_t *n_moving, double momentum,
                            double alpha, const float *GT, float *V, float *X, const double *lo, const double *hi,
                            float *dist, cudaStream_t s);
// X[s] = (double) X32[s] for the moving samples.
void launch_cs_scatter_moving(int n, int d, const int32_t *moving_list, const int32_t *n_moving, const float *X32,
                              double *X, cudaStream_t s);
// *dst += *src (when src is given) + v, on the device (evaluation counters).
void launch_cs_stat_add(int64_t *dst, const int64_t *src, int64_t v, cudaStream_t s);
// *dst += *src mult, on the device.
void launch_cs_stat_add32(int64_t *dst, const int32_t *src, int64_t mult, cudaStream_t s);

}  // namespace sb
