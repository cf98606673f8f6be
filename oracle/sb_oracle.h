/*
 * sb_oracle.h -- plain, slow, FP64 CPU oracle for the mode-centric evidence
 * hot path (SunBURST, arXiv 2601.19957).
 *
 * TEST INFRASTRUCTURE ONLY. Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library. It shares no code,
 * header, table or constant generator with the CUDA path.
 *
 * Notation: d dimensions, K mixture components, component k has log-weight
 * log_w[k], mean mu[k*d..], and the lower Cholesky factor L_k (row-major,
 * L[k*d*d + i*d + j], j <= i) of its precision P_k = L_k L_k^T. Prior box
 * [lo_i, hi_i]. z_k = L_k^T (x - mu_k); e_k = log w_k - (d/2) log 2pi +
 * sum_i log L_k,ii - |z_k|^2 / 2; l(x) = logsumexp_k e_k.
 */
#ifndef SB_ORACLE_H
#define SB_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int d, K;
    const double *log_w, *mu, *L, *lo, *hi;
} orc_problem;

typedef struct {
    int n_rays, n_steps, n_starts, m, max_iter, max_backtracks, newton_steps, cand_cap;
    double gtol, armijo_c1, backtrack, dedup_coarse, dedup_tol, eps_grad;
    uint64_t seed;
    int n_threads; /* OpenMP threads for the walker / ray loops; <= 0 means 1 */
} orc_config;

/* walker terminal states */
enum { ORC_RUNNING = 0, ORC_CONVERGED = 1, ORC_STALLED = 2, ORC_MAXITER = 3, ORC_NONFINITE = 4 };

/* Philox4x32-10 (Salmon et al., SC'11): one block of 4 x 32-bit outputs. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Unit ray directions u[r*d + i] for rays r = 0..n_rays-1 (Sec. 3.5.1 "Sunburst"). */
void orc_ray_directions(int d, int n_rays, uint64_t seed, double *u);

/* l(x); if grad != NULL writes grad l(x) (d); if hneg != NULL writes -hess l(x) (d*d, row-major). */
double orc_loglik(const orc_problem *p, const double *x, double *grad, double *hneg);

/* Coarse pass: l at every ray sample x_rj = c + ((j+1)/n_steps) t_exit_r u_r. ell[r*n_steps + j]. */
void orc_ray_loglik(const orc_problem *p, const orc_config *c, double *u, double *t_exit, double *ell);

/* Start selection by the tiered key (tier, rank-in-ray, -l, flat index); idx sorted ascending. */
int orc_select_starts(const orc_config *c, const double *ell, int64_t *idx);

/* Rays + coarse pass + start selection: starts[n_starts*d], ell_starts[n_starts]. */
int orc_discover(const orc_problem *p, const orc_config *c, double *starts, double *ell_starts);

/* L-BFGS two-loop recursion (App. A.5) on a history of `count` pairs, newest last:
 * S[i*d..], Y[i*d..], rho[i] for i = 0..count-1. Returns r = H_k q in r_out. */
void orc_two_loop(int d, int count, const double *S, const double *Y, const double *rho,
                  const double *q, double *r_out);

/* Batched L-BFGS with Armijo backtracking, one walker at a time. */
void orc_lbfgs(const orc_problem *p, const orc_config *c, const double *x0, int n,
               double *x_out, double *ell_out, int8_t *status_out, int32_t *iters_out,
               int64_t *evals_out);

/* Cholesky-Banachiewicz of an SPD matrix A (d*d) into lower C. Returns 0, or -1 if not PD. */
int orc_cholesky(int d, const double *A, double *C);

/* Laplace stage: coarse dedup, Newton polish, filters, final dedup, log Z_k, LSE - log V.
 * Returns the number of modes (also in *n_modes); modes beyond cap are dropped. */
int orc_laplace(const orc_problem *p, const orc_config *c, const double *x, const double *ell,
                const int8_t *status, int n, double *modes, double *logZk, double *ell_modes,
                int cap, int *n_modes, double *logZ);

/* discover + refine + laplace. Returns the number of modes. */
int orc_evidence(const orc_problem *p, const orc_config *c, double *modes, double *logZk,
                 int cap, int *n_modes, double *logZ);

/* ChiSao oscillation (Sec. 3.5.5) around the refinement; readings in sb_oracle.c. */
typedef struct {
    int n_osc, conv_iters, anti_steps, min_unconverged;
    double momentum, anti_alpha;
    int conv_from_status; /* 1: "converged" is the refinement's CONVERGED / STALLED state (mixed-precision reading) */
} orc_chisao_config;

/* anti-convergence of n samples in place: steps momentum descent steps of step size alpha */
void orc_chisao_anticonverge(const orc_problem *p, double *x, int n, int steps, double momentum, double alpha);
/* the first r <= min(d, 64) columns (Q[j*d..], j < r) of orthonormal group `basis` of oscillation osc, peak peak */
void orc_chisao_directions(int d, int r, uint64_t seed, int osc, int peak, int basis, double *Q);
/* best of n_steps samples on the ray from origin (clamped to the box) along dir to the box
 * boundary (past_valley: beyond the first valley); returns the sample index */
int orc_chisao_ray_best(const orc_problem *p, const double *origin, const double *dir, int n_steps, int past_valley,
                        double *x_out, double *ell_out);
/* ChiSao: returns the number of peaks (stuck representatives, flagged in stuck_out) */
int orc_chisao(const orc_problem *p, const orc_config *c, const orc_chisao_config *cc, const double *x0, int n,
               double *x_out, double *ell_out, int8_t *stuck_out);

/* Preprocessing (Sec. 3.4): sensitivities s[d], classes cls[d] (0 active, 1 flat, 2 soft), the flagged
 * coordinates' marginal log-integral *log_int and log-volume *log_vol; returns the active count. */
int orc_precheck(const orc_problem *p, double eps_flat, double eps_soft, double *s_out, int8_t *cls_out,
                 double *log_int, double *log_vol);

/* Central-difference derivatives of l (App. A.4), Hessians of l itself: gradient (2d evaluations),
 * diagonal (2d + 1), full d*d row-major (2 d^2 + 1). */
void orc_fd_grad(const orc_problem *p, const double *x, double eps, double *g);
void orc_fd_hess_diag(const orc_problem *p, const double *x, double eps, double *hdiag);
void orc_fd_hess_full(const orc_problem *p, const double *x, double eps, double *H);
/* Uniform-correlation probe b = (v^T H v - mean H_ii) / (d - 1), v = 1/sqrt(d) (Sec. 3.7.2). */
double orc_uniform_corr_probe(const orc_problem *p, const double *x, double eps, const double *hdiag);
/* Perpendicular step fraction of one step in coordinates whitened by sqrt(-H_ii) (Sec. 3.7.2). */
double orc_perp_fraction(int d, const double *dtheta, const double *grad, const double *hdiag);

/* Ray families (Sec. 3.5.1): segment of ray r from start to end; 0, or -1 for an unknown family. */
enum { ORC_RAY_V2V = 1, ORC_RAY_V2E = 2, ORC_RAY_W2W = 3 };
int orc_ray_segment(const orc_problem *p, int family, uint64_t seed, int r, double *start, double *end);
/* Two-pass sampling along a segment (Sec. 3.5.2): n coarse values, then n_ref points drawn with density
 * proportional to the likelihood on the active region l > max l - delta: parameters t_ref, values ell_ref. */
void orc_ray_two_pass(const orc_problem *p, const double *start, const double *end, int n, double delta, int n_ref,
                      double *ell_coarse, double *t_ref, double *ell_ref);

#ifdef __cplusplus
}
#endif
#endif
