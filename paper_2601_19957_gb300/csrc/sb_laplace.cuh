// sb_laplace.cuh -- launch interface of the FP64 Laplace-stage kernels.
#pragma once
#include "sb_internal.cuh"

namespace sb {

constexpr int kHalvings = 30;  // Newton step halvings (t = 1, 1/2, ..., 2^-29)

// Scratch of the grid-wide greedy dedup: per-CTA partials (two rounds) and the grid barrier.
constexpr int kDedupMaxGrid = 1024;
struct DedupScratch {
    double *part_l;   // [2 * kDedupMaxGrid]
    int32_t *part_i;  // [2 * kDedupMaxGrid]
    uint32_t *bar;    // [2] arrival count, generation
    int32_t *err;     // device status word (SB_DEV_TIMEOUT)
};
void launch_dedup(int n, int d, const double *X, const double *ell, const int8_t *status, const uint8_t *keep,
                  double tau_scale, const double *wmax, int cap, int32_t *reps, int32_t *n_reps, uint8_t *assigned,
                  const DedupScratch &sc, cudaStream_t s);
void launch_gather_rows(int d, int cap, const double *X, const int32_t *idx, const int32_t *n_idx, double *out,
                        const double *ell, double *ell_out, cudaStream_t s);
void launch_precision(int d, int K, const double *L, double *P, cudaStream_t s);
// P_k only for the components with r != 0 at some live candidate that are not
// formed yet (done[K] is cleared by the caller before the first call).
// onehot[c] = k when candidate c's responsibilities R[c] are exactly one-hot at k
// (then H = P_k and its Cholesky factor is L_k), else -1; for c < cap.
void launch_onehot(int K, const double *R, const int32_t *n_c, int cap, int32_t *onehot, cudaStream_t s);
// P_k for the components some candidate's Hessian reads (one-hot candidates read none).
void launch_precision_needed(int d, int K, const double *L, const double *R, const int32_t *n_c, int32_t *done,
                             int32_t *need, double *P, cudaStream_t s, const int32_t *onehot = nullptr);
// H and its lower Cholesky factor in place for every live candidate; with onehot,
// the one-hot candidates take L_k as their factor (no assembly, no factorisation).
// The factorisation is one cooperative launch (bar: 2 words of grid-barrier state; a
// barrier wait that runs out records SB_DEV_TIMEOUT in *err).
void launch_hessian_chol(int d, int K, int cap, const double *L, const double *P, const double *Z, const double *R,
                         const double *gbar, const int32_t *n_c, double *GK, double *H, int32_t *info,
                         uint32_t *bar, int32_t *err, cudaStream_t s, const int32_t *onehot = nullptr);
// Newton step (C C^T) delta = g and g^T delta / 2 for the live candidates, over
// co-resident CTAs (cooperative launch, one bounded grid barrier per 32-row block
// and direction; at most one per SM and 16 per candidate of the cap, divided among
// the *n_c candidates on the device).
void launch_chol_solve_coop(int d, int cap, const double *H, const double *g, const int32_t *n_c, const int32_t *info,
                            const uint8_t *active, double *delta, double *pred, uint32_t *bar, int32_t *err,
                            cudaStream_t s);
// *n_eff = *n_reps when *n_live > 0 (or n_live is null), else 0: the candidate count the
// rest of a Newton step runs on (zero once no candidate moves).
void launch_set_eff(int32_t *n_eff, const int32_t *n_reps, const int32_t *n_live, cudaStream_t s);
// Newton line search: mode 0 starts it (t = 1) for the candidates still polishing
// and counts them in *n_live (a candidate whose step is below 1e-11 (1 + |x|_inf)
// in max norm has converged and stops where it is); mode 1 decides on the trial.
void launch_newton_ls(int d, int cap, int mode, const int32_t *n_c, const int32_t *info, uint8_t *active,
                      uint8_t *searching, int32_t *halvings, double *t, double *XC, double *LC, const double *delta,
                      double *XN, const double *LN, const double *pred, int32_t *n_live, cudaStream_t s);
// Batched halvings h = 1..kHalvings-1 for the candidates still searching after t = 1.
void launch_ls_batch_setup(int d, int cap, const int32_t *n_c, const uint8_t *searching, const double *XC,
                           const double *delta, double *XN2, int32_t *rows2, int32_t *n_rows2, cudaStream_t s);
void launch_ls_batch_decide(int d, int cap, const int32_t *n_c, uint8_t *searching, uint8_t *active, double *XC,
                            double *LC, const double *XN2, const double *LN2, cudaStream_t s);
void launch_cand_stats(int d, int cap, const double *XC, const double *LC, const double *GC, const double *H,
                       const int32_t *info, const double *lo, const double *hi, double eps_grad, const int32_t *n_c,
                       uint8_t *keep, double *logZk, cudaStream_t s);
void launch_laplace_final(int d, const double *XC, const double *LC, const double *logZk_c, const int32_t *n_c,
                          const int32_t *reps, const int32_t *n_reps, const double *logV, int cap, double *modes,
                          double *logZk, double *ell_modes, int32_t *n_modes, double *logZ, int32_t *dev_status,
                          cudaStream_t s);

}  // namespace sb
