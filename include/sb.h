/*
 * sb.h -- C ABI of the GB300 (sm_103a) evidence library `libsb.so`.
 *
 * The library computes Bayesian evidence log Z for a Gaussian-mixture
 * log-likelihood under a uniform box prior by the mode-centric method of
 * SunBURST (arXiv 2601.19957): sunburst rays from the prior centre (Sec. 3.5),
 * batched L-BFGS refinement (Sec. 3.6, App. A.5), and a Laplace term per
 * distinct mode combined by log-sum-exp (Sec. 3.7, App. A.3, A.8, A.10).
 *
 * Conventions for every entry point:
 *  - Pointers named in `sb_problem`, and every array argument, are DEVICE
 *    pointers unless the comment says "host". The caller owns all memory.
 *  - Arrays are dense, row-major, float64 unless stated: a point set is
 *    [n][d]; the precision Cholesky factors are [K][d][d] (lower triangle used).
 *  - `ws` is caller-owned device scratch of at least the size the matching
 *    *_workspace_bytes query returns (256-byte aligned base). The library
 *    allocates no device memory of its own; the one exception is the 32 MiB
 *    file-scope scratch array of sb_loglik_noalloc, which every GPU that loads
 *    the library holds until the process exits.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Work is enqueued on it. The solve entry points (sb_discover, sb_refine,
 *    sb_laplace, sb_evidence, sb_chisao, sb_evidence_chisao, sb_evidence_batched)
 *    read nothing back to the host: every count and stopping decision stays on the
 *    device (the refinement's loop is a WHILE conditional node of a CUDA graph),
 *    so a caller can capture them into a graph of its own. Called outside a
 *    capture they run as a CUDA graph the library captures once per distinct set
 *    of arguments and replays on `stream` ("graph mode"); with SB_EAGER=1 in the
 *    environment, or while per-launch profiling is on, they run eagerly instead
 *    (the host reads the active walker count after every 8 rounds). The first
 *    BF16 / TF32 call per (d, K, prec) runs the tile autotuner, which
 *    synchronises the stream: make it outside a capture (inside one, that shape
 *    takes the heuristic tile). Entry points that must observe device state
 *    (noted per function: host-buffer calls, sb_check, the statistics)
 *    synchronise that stream before returning.
 *  - Argument errors are detected on the host and returned before any launch.
 *    Problems only visible on the device (non-finite parameters, lo >= hi,
 *    non-positive Cholesky diagonal, zero modes) are recorded in a status word
 *    inside `ws`; `sb_check` reads it.
 *  - No C++ exception crosses this boundary.
 */
#ifndef SB_H
#define SB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum sb_status {
    SB_OK = 0,
    SB_ERR_INVALID_ARG = 1, /* bad sizes, null pointers, lo >= hi, L_kk <= 0 */
    SB_ERR_CUDA = 2,        /* a CUDA runtime call failed                      */
    SB_ERR_WORKSPACE = 3,   /* ws smaller than the query says                  */
    SB_ERR_NONFINITE = 4,   /* NaN/Inf in parameters or in a required result   */
    SB_ERR_NO_MODES = 5,    /* no candidate survived the Laplace filters       */
    SB_ERR_TIMEOUT = 6,     /* a bounded device loop ran out of iterations     */
    SB_ERR_UNSUPPORTED = 7  /* size or precision the library does not handle (d > 1024, ...) */
} sb_status;

/* Arithmetic of the log-likelihood / gradient contractions (discover, refine).
 * The Laplace stage (Newton polish, Hessian, Cholesky, log-sum-exp) is always FP64. */
typedef enum sb_precision {
    SB_PREC_FP64 = 0, /* FP64 on CUDA cores, FP64 L-BFGS state               */
    SB_PREC_TF32 = 1, /* tcgen05 kind::tf32, FP32 accumulate, FP32 state      */
    SB_PREC_BF16 = 2  /* tcgen05 kind::f16 (bf16), FP32 accumulate, FP32 state */
} sb_precision;

/* One evidence problem (Sec. 3.2): l(x) = log sum_k w_k N(x; mu_k, P_k^{-1}),
 * P_k = L_k L_k^T, uniform prior on prod_i [lo_i, hi_i]. */
typedef struct sb_problem {
    int32_t d;            /* dimension, 1 <= d <= 1024                      */
    int32_t K;            /* components, 1 <= K <= 64                       */
    const double *log_w;  /* [K]      log mixture weights                   */
    const double *mu;     /* [K][d]   component means                       */
    const double *L;      /* [K][d][d] lower Cholesky factors of precisions */
    const double *lo;     /* [d]      prior box lower edges                 */
    const double *hi;     /* [d]      prior box upper edges (hi > lo)       */
} sb_problem;

/* Knobs of one solve. Defaults used by the tests are in parentheses. */
typedef struct sb_config {
    int32_t n_rays;         /* sunburst rays from the prior centre (Sec. 3.5.1)           */
    int32_t n_steps;        /* coarse samples per ray, t_j = (j+1)/n_steps (Sec. 3.5.2)    */
    int32_t n_starts;       /* L-BFGS walkers, <= n_rays * n_steps                         */
    int32_t m;              /* L-BFGS history pairs, 1..64 (App. A.5)                      */
    int32_t max_iter;       /* accepted L-BFGS steps per walker (1000)                     */
    int32_t max_backtracks; /* Armijo halvings per line search (40)                        */
    int32_t newton_steps;   /* FP64 Newton polish steps per candidate (3)                  */
    int32_t cand_cap;       /* most candidates entering the Laplace stage (256)            */
    double gtol;            /* stop when |grad l|_inf <= gtol (1 + |l|) (1e-12)            */
    double armijo_c1;       /* sufficient-decrease constant (1e-4)                         */
    double backtrack;       /* step factor per backtrack (0.5)                             */
    double dedup_coarse;    /* coarse L-inf dedup radius / max_i (hi_i - lo_i) (1e-3)      */
    double dedup_tol;       /* final L-inf dedup radius / max_i (hi_i - lo_i) (1e-6)       */
    double eps_grad;        /* gradient filter |grad l|_inf <= eps_grad (1 + |l|) (1e-6)   */
    uint64_t seed;          /* Philox4x32-10 key for the ray directions                    */
    int32_t prec;           /* sb_precision of discover/refine                             */
    int32_t reserved;       /* must be 0                                                   */
} sb_config;

/* Walker terminal states written by sb_refine (int8 per walker). */
enum { SB_WALKER_RUNNING = 0, SB_WALKER_CONVERGED = 1, SB_WALKER_STALLED = 2,
       SB_WALKER_MAXITER = 3, SB_WALKER_NONFINITE = 4 };

/* Human-readable name of a status code (static storage). */
const char *sb_status_string(sb_status s);

/* Bytes of device scratch the solve stages need for this problem and config
 * (the maximum over sb_discover, sb_refine, sb_laplace and sb_evidence).
 * Host-only call: no allocation, no CUDA call. Returns 0 if the arguments are invalid. */
size_t sb_workspace_bytes(const sb_problem *prob, const sb_config *cfg);

/*
 * sb_loglik without a workspace, for callers that cannot allocate device
 * memory (for example code inside a host application that owns every device
 * allocation, or a plugin that may not call cudaMalloc). There is no
 * counterpart in the paper. Same arguments and results as sb_loglik minus
 * ws/ws_bytes: the scratch is a 32 MiB array inside this library, held by
 * every GPU that loads it until the process exits. Requests whose
 * sb_loglik_workspace_bytes exceed 32 MiB return SB_ERR_WORKSPACE before any
 * launch. Every call made outside a stream capture looks up this device's
 * address of the array (so the first call on a device must come before any
 * capture; a capture reuses the last address looked up). With SB_PREC_BF16 /
 * SB_PREC_TF32, the first call per (d, K, prec) in a process also runs the
 * tensor-core tile autotuner, which synchronises the stream: make that call
 * outside any capture too, or set SB_TUNE=0. Calls that overlap on the GPU
 * (concurrent streams, or several host threads) share the array and race;
 * serialise them. It allocates nothing: no cudaMalloc, no cudaFree.
 */
sb_status sb_loglik_noalloc(const sb_problem *prob, int32_t prec, const double *x, int32_t n, double *ell,
                            double *grad, void *stream);

/* The device status word of the last sb_loglik_noalloc call (non-finite parameters,
 * non-positive Cholesky diagonal), which lives in the library's array: synchronises
 * `stream`, returns it as sb_check does, and clears it. */
sb_status sb_loglik_noalloc_check(void *stream);

/* Bytes of scratch sb_loglik needs for n points at precision prec. */
size_t sb_loglik_workspace_bytes(const sb_problem *prob, int32_t prec, int32_t n);

/*
 * Batched log-likelihood (and gradient) of the mixture at n points:
 *   ell[p] = l(x_p) = LSE_k [log w_k - (d/2) log 2pi + sum_i log L_k,ii - |L_k^T (x_p - mu_k)|^2 / 2]
 *   grad[p*d + i] = d l / d x_i = -sum_k r_k (L_k L_k^T (x_p - mu_k))_i,  r = softmax_k
 * (Sec. 3.2 likelihood; the gradient replaces the finite differences of App. A.4.1).
 * x: [n][d]; ell: [n]; grad: [n][d] or NULL for values only. Asynchronous.
 */
sb_status sb_loglik(const sb_problem *prob, int32_t prec, const double *x, int32_t n, double *ell,
                    double *grad, void *ws, size_t ws_bytes, void *stream);

/*
 * Mode discovery (Sec. 3.5.1-3.5.2): n_rays unit directions u_r (Philox4x32-10
 * normals, key = seed, normalised), samples x_rj = c + ((j+1)/n_steps) t_exit,r u_r
 * with c the box centre and t_exit,r the distance to the box surface, l at every
 * sample, then the n_starts samples first in the order (tier: local maximum
 * along the ray first; rank of l inside the ray; -l; flat index r*n_steps+j),
 * written in ascending flat index.
 * starts: [n_starts][d]; ell: [n_starts] (l at each start). Asynchronous.
 */
sb_status sb_discover(const sb_problem *prob, const sb_config *cfg, double *starts, double *ell, void *ws,
                      size_t ws_bytes, void *stream);

/*
 * Batched L-BFGS refinement (Sec. 3.6.2, App. A.5) of n walkers maximising l:
 * two-loop recursion with history m, Armijo backtracking, terminal states in
 * status_out (SB_WALKER_*). starts: [n][d]; x_out: [n][d]; ell_out: [n];
 * status_out: int8 [n]; iters_out: int32 [n] accepted steps (may be NULL);
 * n_evals: int64 device scalar, total l+grad evaluations (may be NULL).
 * Asynchronous; the rounds run until no walker is active, decided on the device
 * (batches of 8 rounds; at most 2 + (max_iter + 1) 2 (max_backtracks + 2) rounds,
 * a bound no run reaches, else SB_ERR_TIMEOUT in the status word).
 */
sb_status sb_refine(const sb_problem *prob, const sb_config *cfg, const double *starts, int32_t n, double *x_out,
                    double *ell_out, int8_t *status_out, int32_t *iters_out, int64_t *n_evals, void *ws,
                    size_t ws_bytes, void *stream);

/*
 * Laplace stage in FP64 (Sec. 3.6.4 filters, Sec. 3.7.1 Laplace, App. A.8, A.10):
 * coarse L-inf dedup of the walkers (x, ell, status), FP64 Newton polish with
 * the analytic Hessian H = -hess l and its Cholesky factor (at most
 * newton_steps steps; a candidate whose step is below 1e-11 (1 + |x|_inf) in
 * max norm has converged and stays put, and the polish ends once none moves),
 * positive-definite /
 * gradient / in-box filters, final dedup, log Z_k = l(x*) + (d/2) log 2pi -
 * sum_i log C_ii (H = C C^T), log Z = LSE_k log Z_k - log V.
 * status may be NULL (all walkers eligible). modes: [cap][d]; logZk, ell_modes:
 * [cap] (ell_modes may be NULL); n_modes: int32 device scalar; logZ: device scalar.
 * Modes are ordered by decreasing l. Asynchronous: the candidate kernels are
 * sized by cand_cap and read the candidate count on the device, and a Newton step
 * after which no candidate moves leaves the remaining steps empty. At a candidate
 * whose FP64 responsibilities are exactly one-hot (component k), H = P_k and its
 * Cholesky factor is L_k itself (no factorisation). Zero modes give logZ = -inf
 * and set SB_ERR_NO_MODES in the status word.
 */
sb_status sb_laplace(const sb_problem *prob, const sb_config *cfg, const double *x, const double *ell,
                     const int8_t *status, int32_t n, double *modes, double *logZk, double *ell_modes, int32_t cap,
                     int32_t *n_modes, double *logZ, void *ws, size_t ws_bytes, void *stream);

/* discover + refine + laplace on device buffers (the whole hot path).
 * logZ, n_modes: device scalars; modes [cap][d]; logZk [cap]. Asynchronous and
 * capturable (see the conventions); sb_check reads the status word afterwards. */
sb_status sb_evidence(const sb_problem *prob, const sb_config *cfg, double *logZ, double *modes, double *logZk,
                      int32_t cap, int32_t *n_modes, void *ws, size_t ws_bytes, void *stream);

/* sb_evidence with HOST inputs and outputs: copies the problem arrays (host
 * pointers in `host_prob`) into `ws`, solves, and copies log Z, the modes and
 * their log Z_k back (host pointers; modes/logZk may be NULL). ws must hold
 * sb_evidence_host_workspace_bytes. Synchronises `stream`. */
size_t sb_evidence_host_workspace_bytes(const sb_problem *host_prob, const sb_config *cfg);
sb_status sb_evidence_host(const sb_problem *host_prob, const sb_config *cfg, double *logZ, double *modes,
                           double *logZk, int32_t cap, int32_t *n_modes, void *ws, size_t ws_bytes, void *stream);

/*
 * Adjoint of log Z with respect to the component means and precision Cholesky
 * factors, at the modes of a forward solve (FP64; not in the paper, which has
 * no gradient of log Z). For log Z = LSE_m log Z_m - log V and
 * pi = softmax_m log Z_m, writes
 *   dmu[k][i]    = grad_logZ * d log Z / d mu_k,i
 *   dL[k][i][j]  = grad_logZ * d log Z / d L_k,ij   (lower triangle; upper = 0)
 * including the implicit shift of each mode (its Hessian is recomputed, never
 * stored): d log Z_m/dphi = d/dphi [l - 1/2 log det H - 1/2 v^T grad l] at the
 * mode with v = H^-1 grad_x log det H. modes: [n_modes][d]; logZk: [n_modes]
 * (device, as written by sb_evidence); dmu: [K][d]; dL: [K][d][d] (device).
 * ws: sb_evidence_backward_workspace_bytes. Synchronises `stream`.
 */
size_t sb_evidence_backward_workspace_bytes(const sb_problem *prob);
sb_status sb_evidence_backward(const sb_problem *prob, const double *modes, const double *logZk, int32_t n_modes,
                               double grad_logZ, double *dmu, double *dL, void *ws, size_t ws_bytes, void *stream);

/*
 * Many independent evidence problems (uneven d and K) in one call: problem i
 * is solved as sb_evidence does on worker stream i % n_workers (forked from and
 * joined back into `stream`), each worker with its own workspace slice, so the
 * problems' kernels overlap on the GPU. In graph mode the whole batch is one
 * CUDA graph (captured once per distinct argument set, then one launch per
 * call). probs: HOST array of P problems (their arrays are device pointers);
 * logZ: device [P]; n_modes: device int32 [P]. Asynchronous. Device-side
 * conditions (e.g. zero modes) are per problem: logZ = -inf.
 */
size_t sb_evidence_batched_workspace_bytes(const sb_problem *probs, int32_t P, const sb_config *cfg,
                                           int32_t n_workers);
sb_status sb_evidence_batched(const sb_problem *probs, int32_t P, const sb_config *cfg, double *logZ,
                              int32_t *n_modes, int32_t n_workers, void *ws, size_t ws_bytes, void *stream);

/* Output tile width (64, 128 or 256 columns) the tensor-core GEMMs use for
 * (d, K, prec) in this process, as chosen by the library's autotuner on the
 * first mixed-precision call with that shape (which synchronises its stream);
 * 0 if that shape has not been tuned yet. SB_TUNE=0 in the environment skips
 * the timing (heuristic width); SB_TUNE_CACHE=<file> persists the choices. */
int32_t sb_tuned_tile(int32_t d, int32_t K, int32_t prec);

/* Synchronise `stream` and return the status word the device recorded in ws
 * (SB_OK if nothing went wrong); clears the word. */
sb_status sb_check(void *ws, size_t ws_bytes, void *stream);

/* Counters of the last sb_evidence call that used this workspace (synchronises
 * `stream`): out[0] ray samples evaluated (l only), out[1] l + grad evaluations
 * of the L-BFGS stage, out[2] coarse candidates polished, out[3] modes kept.
 * out: host int64[4]. */
sb_status sb_evidence_stats(const sb_problem *prob, const sb_config *cfg, void *ws, size_t ws_bytes, int64_t *out,
                            void *stream);

/* Number of kernel launches this process has issued through the library so far
 * (host counter, diagnostics only). */
int64_t sb_launch_count(void);

/* Device-time profiling of the main kernel classes (diagnostics). While enabled,
 * each launch of a class is bracketed by CUDA events on its stream.
 * sb_profile_read synchronises those events, writes per-class total
 * milliseconds and launch counts (host arrays of 8: 0 tensor-core z GEMM at
 * walkers, 1 tensor-core z GEMM at ray samples, 2 tensor-core gradient GEMM,
 * 3 L-BFGS step, 4 FP64 z GEMM, 5 FP64 gradient GEMM, 6 FP64 Cholesky,
 * 7 other), clears the record and returns the number of unreadable events. */
void sb_profile_enable(int on);
int32_t sb_profile_read(double *ms, int64_t *launches);
/* Profiling of some classes only: bit c of `mask` times the launches of class c
 * (sb_profile_enable(1) is mask 0xFF, sb_profile_enable(0) mask 0). Timing one
 * class keeps the events off every other launch. */
void sb_profile_classes(uint32_t mask);

/* Algorithmic bytes moved by the launches of profiling class `cls` while
 * profiling was enabled, then clears that count. Only class 3 (the FP32 L-BFGS
 * step) counts bytes: per walker visited, the vectors it reads and writes
 * (x, grad, trial point and gradient, direction, state) and, for a new
 * direction, every stored pair read in both passes of the two-loop recursion
 * (4 m d history elements at a full history, the figure of the limited-memory
 * update of Nocedal & Wright, Alg. 7.4). Other classes return 0. Synchronises
 * the device; returns -1 on a CUDA error. */
double sb_profile_bytes(int32_t cls);

/* FP64 FMA throughput of the current device in TFLOP/s, the peak the FP64 kernels are
 * measured against: independent FMA chains on every SM, timed with CUDA events on
 * `stream`, best of five launches after a warm-up (diagnostics; synchronises the
 * stream; -1 on a CUDA error). */
double sb_fp64_fma_peak(void *stream);

/* Knobs of the ChiSao oscillation (Sec. 3.5.5, Algorithm 1). */
typedef struct sb_chisao_config {
    int32_t n_osc;           /* oscillations, 1..1024 (3)                                   */
    int32_t conv_iters;      /* accepted L-BFGS steps per convergence phase (1000)          */
    int32_t anti_steps;      /* momentum descent steps per anti-convergence phase (10)      */
    int32_t min_unconverged; /* Repulse Monkey needs this many unconverged samples, >= 1 (5)*/
    double momentum;         /* mu of the momentum step (0.9)                               */
    double anti_alpha;       /* step size alpha of the momentum step (0.1)                  */
} sb_chisao_config;

/* Bytes of device scratch sb_chisao needs (the solve stages' scratch plus its own). */
size_t sb_chisao_workspace_bytes(const sb_problem *prob, const sb_config *cfg);

/*
 * ChiSao oscillation (Sec. 3.5.5) of n <= cfg->n_starts samples. With
 * cfg->prec = SB_PREC_FP64 everything is FP64; with TF32 / BF16 the refinement is
 * sb_refine's mixed path, the ray samples and momentum gradients come from the
 * tensor-core likelihood, and n_starts must be at least n_steps (else
 * SB_ERR_UNSUPPORTED). n_osc times:
 *   convergence: sb_refine's L-BFGS from the current positions, at most
 *     conv_iters accepted steps;
 *   stick test: converged and l >= max l + log 0.1, converged meaning
 *     |grad l|_inf <= eps_grad (1 + |l|) in FP64, and the refinement's
 *     CONVERGED / STALLED state on the mixed path (whose gradients are too
 *     coarse for that test);
 *   dedup of the stuck samples (greedy L-inf, radius dedup_coarse
 *     max_i (hi_i - lo_i), decreasing l): representatives stay stuck (the
 *     peaks), the other stuck samples are lost;
 *   unless this is the last oscillation, reseeding of the lost samples and
 *   anti-convergence:
 *     Repulse Monkey (at least min_unconverged samples fail the gradient
 *       test): lost sample l (index order) casts a ray from unconverged sample
 *       l mod n_unconv, clamped to the box, in a Philox-normal unit direction
 *       (counter (pair, l, oscillation, 'RPMK'), key = seed) to the box face,
 *       sampled at t_j = (j+1)/n_steps t_exit, and moves to its best sample;
 *     Golden Rooster (otherwise, while it keeps finding peaks): lost sample l
 *       goes to peak l mod n_peaks along +-column c mod G of orthonormal group
 *       c / G of that peak, G = min(d, 64), c = (l / n_peaks) / 2 (+ for even
 *       l / n_peaks), a group the QR of G Philox-normal vectors (counter (pair,
 *       group G + column, oscillation << 16 | peak, 'GRST')), to the best sample past the first
 *       valley of the ray (the exit sample when l never rises); it stays off
 *       after an oscillation that used it ends with no more peaks than before;
 *     anti-convergence: every sample that is not stuck (and not NONFINITE)
 *       takes anti_steps steps v <- momentum v - anti_alpha grad l,
 *       x <- x + v (v = 0 at the start), clamped to the box.
 * x0: [n][d] device; x_out: [n][d]; ell_out: [n] l after the last
 * convergence phase; stuck_out: int8 [n], 1 at the peaks; n_peaks: int32
 * device scalar. ws: sb_chisao_workspace_bytes. Asynchronous: the stick test,
 * the lists, the branch and the Golden Rooster groups are decided on the device
 * (the mixed path forms its Golden Rooster groups in FP32).
 */
sb_status sb_chisao(const sb_problem *prob, const sb_config *cfg, const sb_chisao_config *cc, const double *x0,
                    int32_t n, double *x_out, double *ell_out, int8_t *stuck_out, int32_t *n_peaks, void *ws,
                    size_t ws_bytes, void *stream);

/* Bytes of device scratch sb_fd_derivatives needs (full != 0: with the full Hessian). */
size_t sb_fd_workspace_bytes(const sb_problem *prob, int32_t full);

/*
 * Black-box derivatives of l at one point by central differences (App. A.4), FP64, and the
 * uniform-correlation probe (Sec. 3.7.2). l is only evaluated, at the perturbed points
 *   x +- eps_g e_i (gradient), x and x +- eps_h e_i (Hessian diagonal), x +- eps_h v with
 *   v = (1, ..., 1)/sqrt(d) (probe), and, when full, x +- eps_h e_i +- eps_h e_j for i < j,
 * 4d + 3 points plus 2 d (d - 1) for the full Hessian, in batches of the likelihood:
 *   grad_i = (l(x + eps_g e_i) - l(x - eps_g e_i)) / (2 eps_g)
 *   H_ii = (l(x + eps_h e_i) - 2 l(x) + l(x - eps_h e_i)) / eps_h^2
 *   H_ij = H_ji = (l_++ - l_+- - l_-+ + l_--) / (4 eps_h^2)
 *   b = (v^T H v - mean_i H_ii) / (d - 1) (0 for d = 1), v^T H v the second difference along v.
 * The Hessians are of l itself (negative definite at a maximum).
 * x: [d] device; grad: [d] or NULL; hdiag: [d]; H: [d][d] (required when full); b: device
 * scalar or NULL. eps_g, eps_h > 0 (1e-5 and 1e-4 suit FP64). ws: sb_fd_workspace_bytes.
 * Asynchronous.
 */
sb_status sb_fd_derivatives(const sb_problem *prob, const double *x, double eps_g, double eps_h, int32_t full,
                            double *grad, double *hdiag, double *H, double *b, void *ws, size_t ws_bytes,
                            void *stream);

/* Ray families besides the sunburst (Sec. 3.5.1). */
enum { SB_RAY_V2V = 1, SB_RAY_V2E = 2, SB_RAY_W2W = 3 };

/* Bytes of device scratch sb_segments needs for n_rays rays of n_steps coarse samples. */
size_t sb_segments_workspace_bytes(const sb_problem *prob, int32_t n_rays, int32_t n_steps);

/*
 * V2V / V2E / W2W rays and their two-pass sampling (Sec. 3.5.1-3.5.2), FP64.
 * Ray r of `family` is the segment from a to b: V2V joins two vertices from independent
 * bit streams (an end equal to the start becomes its antipode); V2E runs from a vertex to
 * the midpoint of an edge (vertex bits, one free coordinate at the box centre); W2W runs
 * from a uniform point on the face x_i = lo_i to one on x_i = hi_i of a random axis i. All
 * draws of ray r come from Philox4x32-10 blocks with counter (block, r, family tag
 * 'V2V ' / 'V2E ' / 'W2W ', purpose), key = seed: bit b of a stream is bit b % 32 of word
 * (b / 32) % 4 of block b / 128, uniform k uses words 2 (k % 2), 2 (k % 2) + 1 of block
 * k / 2 (top 52 bits), an index below n is (word 0 of block 0) n >> 32; purposes 0 and 1
 * are the start and end streams, 2 the index.
 * Coarse pass: l at t_j = j / (n_steps - 1) (t = 1/2 for one step). Refinement: n_ref
 * points drawn with density proportional to the likelihood, piecewise constant on the
 * coarse cells (clipped to [0, 1]) and zero outside the active region l > max l - delta,
 * at the inverse CDF of (k + 1/2) / n_ref; their parameters and l.
 * ends: [2][n_rays][d] (starts, then ends); ell_coarse: [n_rays][n_steps];
 * t_ref, ell_ref: [n_rays][n_ref] (may be NULL when n_ref = 0). delta >= 0 (+inf: all
 * active). ws: sb_segments_workspace_bytes. Asynchronous.
 */
sb_status sb_segments(const sb_problem *prob, int32_t family, uint64_t seed, int32_t n_rays, int32_t n_steps,
                      double delta, int32_t n_ref, double *ends, double *ell_coarse, double *t_ref, double *ell_ref,
                      void *ws, size_t ws_bytes, void *stream);

/*
 * Evidence with ChiSao (Sec. 3.5.5 between discovery and the Laplace stage):
 * sb_discover, then sb_chisao from the n_starts starts, then sb_laplace over EVERY
 * final sample (stuck or not, all eligible). The stick rule keeps only peaks within
 * log 10 of the highest, while the evidence needs every component a sample reached,
 * so the Laplace stage is not limited to the stuck peaks. Outputs as sb_evidence.
 * ws: sb_chisao_workspace_bytes. Asynchronous and capturable; the status word
 * collects what every stage records (sb_check).
 */
sb_status sb_evidence_chisao(const sb_problem *prob, const sb_config *cfg, const sb_chisao_config *cc, double *logZ,
                             double *modes, double *logZk, int32_t cap, int32_t *n_modes, void *ws, size_t ws_bytes,
                             void *stream);

/*
 * sb_evidence_batched with ChiSao: every problem is solved as sb_evidence_chisao does
 * (discovery, the ChiSao oscillation, the Laplace stage over every final sample), on
 * the same worker streams and, in graph mode, in one CUDA graph. ws:
 * sb_evidence_chisao_batched_workspace_bytes. Asynchronous.
 */
size_t sb_evidence_chisao_batched_workspace_bytes(const sb_problem *probs, int32_t P, const sb_config *cfg,
                                                  int32_t n_workers);
sb_status sb_evidence_chisao_batched(const sb_problem *probs, int32_t P, const sb_config *cfg,
                                     const sb_chisao_config *cc, double *logZ, int32_t *n_modes, int32_t n_workers,
                                     void *ws, size_t ws_bytes, void *stream);

/* sb_evidence_chisao with HOST inputs and outputs, as sb_evidence_host: copies the
 * problem arrays (host pointers in `host_prob`) into `ws`, runs discovery, ChiSao and
 * the Laplace stage over every final sample, and copies log Z, the mode count, the
 * modes and their log Z_k back (host pointers; modes / logZk may be NULL). ws must hold
 * sb_evidence_chisao_host_workspace_bytes. Synchronises `stream`. */
size_t sb_evidence_chisao_host_workspace_bytes(const sb_problem *host_prob, const sb_config *cfg);
sb_status sb_evidence_chisao_host(const sb_problem *host_prob, const sb_config *cfg, const sb_chisao_config *cc,
                                  double *logZ, double *modes, double *logZk, int32_t cap, int32_t *n_modes,
                                  void *ws, size_t ws_bytes, void *stream);

/* Counters of the last sb_chisao / sb_evidence_chisao call on this workspace
 * (synchronises `stream`): out[0] l evaluations at ray samples (discovery, when run
 * through sb_evidence_chisao, and the reseeding rays), out[1] l + grad evaluations
 * of the L-BFGS convergence phases, out[2] l + grad evaluations of the
 * anti-convergence steps, out[3] modes kept by the Laplace stage of
 * sb_evidence_chisao. out: host int64[4]. */
sb_status sb_chisao_stats(const sb_problem *prob, const sb_config *cfg, void *ws, size_t ws_bytes, int64_t *out,
                          void *stream);

/* Bytes of device scratch sb_ray_loglik_quad needs (form 0 FP64, 1 FP32, 2 BF16 and
 * 3 TF32 tensor-core split products); 0 for an invalid form or problem. */
size_t sb_ray_loglik_quad_workspace_bytes(const sb_problem *prob, int32_t form, int32_t n_rays);

/*
 * Sunburst ray likelihoods from three scalars per (ray, component) (Sec. 3.5.1-3.5.2,
 * a restructuring of the coarse pass): along x(t) = c + tau u_r, tau = ((j + 1) / n_steps)
 * t_exit,r, z_k = z_k(c) + tau L_k^T u_r, so |z_k|^2 = q0_k + 2 tau q1_rk + tau^2 q2_rk and
 * ell[r][j] = LSE_k (a_k - |z_k|^2 / 2) needs one triangular GEMM of the directions by each
 * L_k instead of one per sample. form 0: FP64 GEMM; form 1: FP32 SIMT GEMM (u and L_k
 * rounded to FP32, FP32 accumulation); forms 2 and 3: the tensor-core GEMM sb_discover
 * runs at BF16 / TF32 (u and L_k each split into a high part and the rounded remainder,
 * w = u_hi L_hi + u_lo L_hi + u_hi L_lo with FP32 accumulation, about FP32 accuracy).
 * The scalars are combined in FP64 in every form. u: [n_rays][d] device (unit
 * directions); ell: [n_rays][n_steps]. ws: sb_ray_loglik_quad_workspace_bytes.
 * Asynchronous. SB_ERR_INVALID_ARG for a form outside 0..3, n_rays < 1 or n_steps < 1;
 * SB_ERR_UNSUPPORTED for forms 2, 3 on a device without tcgen05.
 */
sb_status sb_ray_loglik_quad(const sb_problem *prob, int32_t form, const double *u, int32_t n_rays, int32_t n_steps,
                             double *ell, void *ws, size_t ws_bytes, void *stream);

/* Bytes of device scratch sb_ray_loglik_origins needs (form 2 BF16, 3 TF32); 0 for
 * another form or an invalid problem. */
size_t sb_ray_loglik_origins_workspace_bytes(const sb_problem *prob, int32_t form, int32_t n_rays);

/*
 * Ray likelihoods from per-ray origins, the rays ChiSao's reseeding casts (Sec. 3.5.5:
 * Repulse Monkey rays from unconverged samples, Golden Rooster rays from the peaks):
 * along x(t) = o_r + tau u_r, tau = ((j + 1) / n_steps) t_exit,r with t_exit,r the
 * distance from o_r along u_r to the box surface,
 *     z_k(x) = z_k(o_r) + tau L_k^T u_r,  |z_k|^2 = q0_rk + 2 tau q1_rk + tau^2 q2_rk,
 * with z_k(o_r) = o_r L_k - mu_k L_k from a tensor-core GEMM of the origins and
 * L_k^T u_r from one of the directions (operands split into high and low parts at
 * BF16 (form 2) or TF32 (form 3), FP32 accumulation; z_k(o_r) kept in FP32), the
 * scalars combined in FP64 and ell[r][j] = LSE_k (a_k - |z_k|^2 / 2).
 * o, u: [n_rays][d] device (origins inside the box, unit directions); ell:
 * [n_rays][n_steps] device; texit: [n_rays] device or NULL. ws:
 * sb_ray_loglik_origins_workspace_bytes. Asynchronous. SB_ERR_INVALID_ARG for another
 * form, n_rays < 1 or n_steps < 1; SB_ERR_UNSUPPORTED on a device without tcgen05.
 */
sb_status sb_ray_loglik_origins(const sb_problem *prob, int32_t form, const double *o, const double *u,
                                int32_t n_rays, int32_t n_steps, double *ell, double *texit, void *ws,
                                size_t ws_bytes, void *stream);

/* Bytes of device scratch sb_precheck needs. */
size_t sb_precheck_workspace_bytes(const sb_problem *prob);

/*
 * Preprocessing probe (Sec. 3.4): s_i = |l(c + Delta_i e_i) - l(c)| + |l(c - Delta_i e_i) - l(c)|
 * with c the box centre and Delta_i = (hi_i - lo_i) / 2; a coordinate is flat when
 * s_i < eps_flat median(s), soft when not flat and s_i < eps_soft max(s), else active
 * (median and max over the finite s_i; the median of an even count is the mean of the
 * two middle values; a non-finite s_i is active). The marginal log-integral of the
 * flagged coordinates is sum over flat log(2 Delta_i) + sum over soft
 * [1/2 log 2 pi + log(Delta_i / sqrt(s_i))], and their log-volume sum log(2 Delta_i): the
 * evidence of the full problem is that of the problem over the active coordinates (the
 * flagged ones held at c) plus log_int minus log_vol. The l differences are formed from
 * z_k(c) and the rows of L_k, without subtracting two l values.
 * s: [d]; cls: int8 [d] (0 active, 1 flat, 2 soft); log_int, log_vol: device scalars;
 * n_active: int32 device scalar. eps_flat, eps_soft >= 0 (defaults 1e-6, 1e-3). d <= 1024.
 * ws: sb_precheck_workspace_bytes. Asynchronous.
 */
sb_status sb_precheck(const sb_problem *prob, double eps_flat, double eps_soft, double *s, int8_t *cls,
                      double *log_int, double *log_vol, int32_t *n_active, void *ws, size_t ws_bytes, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* SB_H */
