/*
 * sb_oracle.c -- plain FP64 CPU oracle for the SunBURST evidence hot path.
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the
 * benchmark's CPU-baseline leg, never by the product path. It shares no code
 * with the CUDA implementation. Everything is double precision, plain loops,
 * no BLAS, no blocking or reordering beyond the definitions it follows.
 *
 * Paper passages followed (arXiv 2601.19957):
 *   evidence with a uniform box prior ........ Sec. 3.2 (problem statement), App. A.1
 *   sunburst rays from the prior centre ...... Sec. 3.5.1; coarse pass Sec. 3.5.2
 *   ray local maxima ......................... Sec. 4.1 (sign change of the ray gradient)
 *   L-BFGS two-loop recursion ................ App. A.5; batched refinement Sec. 3.6.2
 *   L-infinity deduplication ................. Sec. 3.5.4, App. A.7
 *   saddle / gradient filters ................ Sec. 3.6.4
 *   Laplace per mode ......................... Sec. 3.7.1, Eq. (laplace-evidence) Sec. 4.2, App. A.3
 *   Cholesky log-determinant (whitening) ..... App. A.8
 *   log-sum-exp over modes ................... Sec. 3.7.3, App. A.10
 *   ChiSao oscillation ....................... Sec. 3.5.5, Algorithm 1 (CarryTiger)
 *   preprocessing probe and marginal terms ... Sec. 3.4 and its Algorithm
 *   central-difference derivatives ........... App. A.4
 *   rotation detection ....................... Sec. 3.7.2, App. A.6
 *   V2V / V2E / W2W rays, two-pass sampling .. Sec. 3.5.1-3.5.2
 * Every function is pinned by tests/test_oracle_*.py to closed forms, library
 * routines, brute force or hand-worked cases.
 * Where the paper is silent (line search, tolerances, tie-breaks, ray grid) the
 * readings are stated next to the code that takes them.
 */
#include "sb_oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_LOG_2PI 1.8378770664093454836
#define ORC_TWO_PI 6.283185307179586477

static int nthreads_of(const orc_config *c) { return (c && c->n_threads > 0) ? c->n_threads : 1; }

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11). */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* A uniform double strictly inside (0, 1) from the top 52 bits of a 64-bit word. */
static double orc_unit(uint32_t hi, uint32_t lo) {
    uint64_t a = ((uint64_t)hi << 32) | (uint64_t)lo;
    return ((double)(a >> 12) + 0.5) * (1.0 / 4503599627370496.0); /* 2^-52 */
}

/*
 * Ray r, coordinate pair p: Philox block with counter (p, r, 'RAYS', 0) and
 * key (seed lo, seed hi); two uniforms -> two standard normals (Box-Muller).
 * The direction is the normal vector scaled to unit length, i.e. uniform on
 * S^{d-1} (Sec. 3.5.1).
 */
void orc_ray_directions(int d, int n_rays, uint64_t seed, double *u) {
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    const int npairs = (d + 1) / 2;
    for (int r = 0; r < n_rays; ++r) {
        double *ur = u + (size_t)r * d;
        for (int p = 0; p < npairs; ++p) {
            uint32_t ctr[4] = {(uint32_t)p, (uint32_t)r, 0x52415953u, 0u};
            uint32_t o[4];
            orc_philox4x32_10(ctr, key, o);
            double u1 = orc_unit(o[0], o[1]);
            double u2 = orc_unit(o[2], o[3]);
            double rad = sqrt(-2.0 * log(u1));
            double th = ORC_TWO_PI * u2;
            ur[2 * p] = rad * cos(th);
            if (2 * p + 1 < d) ur[2 * p + 1] = rad * sin(th);
        }
        double nrm2 = 0.0;
        for (int i = 0; i < d; ++i) nrm2 += ur[i] * ur[i];
        double nrm = sqrt(nrm2);
        for (int i = 0; i < d; ++i) ur[i] = ur[i] / nrm;
    }
}

/* ------------------------------------------------------------------------ */
/* Log-likelihood, gradient and negative Hessian (notation in the header).   */
/* ------------------------------------------------------------------------ */
double orc_loglik(const orc_problem *p, const double *x, double *grad, double *hneg) {
    const int d = p->d, K = p->K;
    double *z = (double *)malloc(sizeof(double) * (size_t)K * d);
    double *e = (double *)malloc(sizeof(double) * (size_t)K);
    for (int k = 0; k < K; ++k) {
        const double *Lk = p->L + (size_t)k * d * d;
        const double *mk = p->mu + (size_t)k * d;
        double a = p->log_w[k] - 0.5 * (double)d * ORC_LOG_2PI;
        for (int i = 0; i < d; ++i) a += log(Lk[(size_t)i * d + i]);
        double q = 0.0;
        for (int j = 0; j < d; ++j) {
            double zj = 0.0;
            for (int i = j; i < d; ++i) zj += (x[i] - mk[i]) * Lk[(size_t)i * d + j];
            z[(size_t)k * d + j] = zj;
            q += zj * zj;
        }
        e[k] = a - 0.5 * q;
    }
    /* log-sum-exp over components, App. A.10 */
    double emax = -INFINITY;
    for (int k = 0; k < K; ++k)
        if (e[k] > emax) emax = e[k];
    double ssum = 0.0;
    for (int k = 0; k < K; ++k) ssum += exp(e[k] - emax);
    double ell = emax + log(ssum);

    if (grad || hneg) {
        double *r = (double *)malloc(sizeof(double) * (size_t)K);
        double *gk = (double *)malloc(sizeof(double) * (size_t)K * d);
        for (int k = 0; k < K; ++k) r[k] = exp(e[k] - emax) / ssum;
        /* g_k = grad e_k = -L_k z_k */
        for (int k = 0; k < K; ++k) {
            const double *Lk = p->L + (size_t)k * d * d;
            for (int i = 0; i < d; ++i) {
                double s = 0.0;
                for (int j = 0; j <= i; ++j) s += Lk[(size_t)i * d + j] * z[(size_t)k * d + j];
                gk[(size_t)k * d + i] = -s;
            }
        }
        double *gbar = (double *)calloc((size_t)d, sizeof(double));
        for (int k = 0; k < K; ++k)
            for (int i = 0; i < d; ++i) gbar[i] += r[k] * gk[(size_t)k * d + i];
        if (grad)
            for (int i = 0; i < d; ++i) grad[i] = gbar[i];
        if (hneg) {
            /* -hess l = sum_k r_k P_k - sum_k r_k g_k g_k^T + gbar gbar^T */
            for (int i = 0; i < d; ++i)
                for (int i2 = 0; i2 < d; ++i2) {
                    double h = gbar[i] * gbar[i2];
                    for (int k = 0; k < K; ++k) {
                        const double *Lk = p->L + (size_t)k * d * d;
                        int jmax = i < i2 ? i : i2;
                        double pk = 0.0;
                        for (int j = 0; j <= jmax; ++j) pk += Lk[(size_t)i * d + j] * Lk[(size_t)i2 * d + j];
                        h += r[k] * (pk - gk[(size_t)k * d + i] * gk[(size_t)k * d + i2]);
                    }
                    hneg[(size_t)i * d + i2] = h;
                }
        }
        free(gbar);
        free(gk);
        free(r);
    }
    free(e);
    free(z);
    return ell;
}

/* ------------------------------------------------------------------------ */
/* Coarse pass along rays (Sec. 3.5.2).                                      */
/* Reading: t_j = (j+1)/n_steps, j = 0..n_steps-1, from p_start = c (centre)  */
/* to p_end = c + t_exit u, t_exit = min_i half_i / |u_i| (the box surface). */
/* ------------------------------------------------------------------------ */
static void ray_point(const orc_problem *p, const double *ur, double t_exit, int j, int n_steps, double *x) {
    double s = ((double)(j + 1) / (double)n_steps) * t_exit;
    for (int i = 0; i < p->d; ++i) {
        double c = 0.5 * (p->lo[i] + p->hi[i]);
        x[i] = c + s * ur[i];
    }
}

static double ray_exit(const orc_problem *p, const double *ur) {
    double t = INFINITY;
    for (int i = 0; i < p->d; ++i) {
        double au = fabs(ur[i]);
        if (au > 0.0) {
            double half = 0.5 * (p->hi[i] - p->lo[i]);
            double ti = half / au;
            if (ti < t) t = ti;
        }
    }
    return t;
}

void orc_ray_loglik(const orc_problem *p, const orc_config *c, double *u, double *t_exit, double *ell) {
    const int d = p->d;
    orc_ray_directions(d, c->n_rays, c->seed, u);
    for (int r = 0; r < c->n_rays; ++r) t_exit[r] = ray_exit(p, u + (size_t)r * d);
#pragma omp parallel for num_threads(nthreads_of(c)) schedule(dynamic, 4)
    for (int r = 0; r < c->n_rays; ++r) {
        double *x = (double *)malloc(sizeof(double) * (size_t)d);
        for (int j = 0; j < c->n_steps; ++j) {
            ray_point(p, u + (size_t)r * d, t_exit[r], j, c->n_steps, x);
            ell[(size_t)r * c->n_steps + j] = orc_loglik(p, x, NULL, NULL);
        }
        free(x);
    }
}

/* ------------------------------------------------------------------------ */
/* Start selection ("top ray samples", Sec. 3.5.4; local maxima, Sec. 4.1).  */
/* Key, ascending: tier (0 = discrete local maximum along its ray:           */
/* l_j > l_{j-1} and l_j >= l_{j+1}, missing neighbours = -inf; 1 otherwise), */
/* rank of l_j inside its ray (descending, ties -> lower j), -l_j, flat index. */
/* The first n_starts keys are taken and returned in ascending flat index.   */
/* ------------------------------------------------------------------------ */
typedef struct {
    int tier, rank;
    double ell;
    int64_t flat;
} orc_key;

static int key_cmp(const void *a, const void *b) {
    const orc_key *x = (const orc_key *)a, *y = (const orc_key *)b;
    if (x->tier != y->tier) return x->tier < y->tier ? -1 : 1;
    if (x->rank != y->rank) return x->rank < y->rank ? -1 : 1;
    if (x->ell != y->ell) return x->ell > y->ell ? -1 : 1;
    if (x->flat != y->flat) return x->flat < y->flat ? -1 : 1;
    return 0;
}

static int i64_cmp(const void *a, const void *b) {
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

int orc_select_starts(const orc_config *c, const double *ell, int64_t *idx) {
    const int R = c->n_rays, S = c->n_steps;
    const int64_t total = (int64_t)R * S;
    orc_key *keys = (orc_key *)malloc(sizeof(orc_key) * (size_t)total);
    for (int r = 0; r < R; ++r) {
        const double *lr = ell + (size_t)r * S;
        for (int j = 0; j < S; ++j) {
            double left = j > 0 ? lr[j - 1] : -INFINITY;
            double right = j + 1 < S ? lr[j + 1] : -INFINITY;
            int tier = (lr[j] > left && lr[j] >= right) ? 0 : 1;
            int rank = 0;
            for (int j2 = 0; j2 < S; ++j2)
                if (lr[j2] > lr[j] || (lr[j2] == lr[j] && j2 < j)) ++rank;
            orc_key *kk = &keys[(size_t)r * S + j];
            kk->tier = tier;
            kk->rank = rank;
            kk->ell = lr[j];
            kk->flat = (int64_t)r * S + j;
        }
    }
    qsort(keys, (size_t)total, sizeof(orc_key), key_cmp);
    int n = c->n_starts < total ? c->n_starts : (int)total;
    for (int s = 0; s < n; ++s) idx[s] = keys[s].flat;
    qsort(idx, (size_t)n, sizeof(int64_t), i64_cmp);
    free(keys);
    return n;
}

int orc_discover(const orc_problem *p, const orc_config *c, double *starts, double *ell_starts) {
    const int d = p->d;
    const int64_t total = (int64_t)c->n_rays * c->n_steps;
    double *u = (double *)malloc(sizeof(double) * (size_t)c->n_rays * d);
    double *te = (double *)malloc(sizeof(double) * (size_t)c->n_rays);
    double *ell = (double *)malloc(sizeof(double) * (size_t)total);
    int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)(c->n_starts > 0 ? c->n_starts : 1));
    orc_ray_loglik(p, c, u, te, ell);
    int n = orc_select_starts(c, ell, idx);
    for (int s = 0; s < n; ++s) {
        int r = (int)(idx[s] / c->n_steps), j = (int)(idx[s] % c->n_steps);
        ray_point(p, u + (size_t)r * d, te[r], j, c->n_steps, starts + (size_t)s * d);
        ell_starts[s] = ell[idx[s]];
    }
    free(idx);
    free(ell);
    free(te);
    free(u);
    return n;
}

/* ------------------------------------------------------------------------ */
/* L-BFGS (App. A.5) minimising f = -l, with Armijo backtracking.            */
/* ------------------------------------------------------------------------ */
static double dot(int d, const double *a, const double *b) {
    double s = 0.0;
    for (int i = 0; i < d; ++i) s += a[i] * b[i];
    return s;
}

void orc_two_loop(int d, int count, const double *S, const double *Y, const double *rho, const double *q_in,
                  double *r) {
    double *q = (double *)malloc(sizeof(double) * (size_t)d);
    double *alpha = (double *)malloc(sizeof(double) * (size_t)(count > 0 ? count : 1));
    memcpy(q, q_in, sizeof(double) * (size_t)d);
    /* first loop: newest to oldest */
    for (int i = count - 1; i >= 0; --i) {
        alpha[i] = rho[i] * dot(d, S + (size_t)i * d, q);
        for (int t = 0; t < d; ++t) q[t] -= alpha[i] * Y[(size_t)i * d + t];
    }
    /* H0 = gamma I with gamma = s^T y / y^T y of the newest pair */
    double gamma = 1.0;
    if (count > 0) {
        const double *sn = S + (size_t)(count - 1) * d, *yn = Y + (size_t)(count - 1) * d;
        gamma = dot(d, sn, yn) / dot(d, yn, yn);
    }
    for (int t = 0; t < d; ++t) r[t] = gamma * q[t];
    /* second loop: oldest to newest */
    for (int i = 0; i < count; ++i) {
        double beta = rho[i] * dot(d, Y + (size_t)i * d, r);
        for (int t = 0; t < d; ++t) r[t] += S[(size_t)i * d + t] * (alpha[i] - beta);
    }
    free(alpha);
    free(q);
}

static int all_finite(int d, const double *v) {
    for (int i = 0; i < d; ++i)
        if (!isfinite(v[i])) return 0;
    return 1;
}

static double max_abs(int d, const double *v) {
    double m = 0.0;
    for (int i = 0; i < d; ++i)
        if (fabs(v[i]) > m) m = fabs(v[i]);
    return m;
}

/*
 * One walker. Readings (the paper names L-BFGS but no line search or stop rule):
 *  - first step and after a history reset: p = -grad f / |grad f|_2 (H0 = I/|g|);
 *  - later: p = -two_loop(grad f), gamma from the newest pair;
 *  - if grad f . p >= 0 the history is cleared and steepest descent is used;
 *  - Armijo: alpha = 1, 1 + max_backtracks trials, alpha *= backtrack, accept
 *    f(x + alpha p) <= f + c1 alpha grad f . p (non-finite trials rejected);
 *  - if no trial is accepted with a non-empty history, clear it and retry once;
 *    a second failure (or a failure with an empty history) is STALLED;
 *  - the pair (s, y) is stored only if s^T y > 1e-10 |s|_2 |y|_2 (ring of m);
 *  - CONVERGED when |grad l|_inf <= gtol (1 + |l|); STALLED after two
 *    consecutive accepted steps with no decrease of f; MAXITER after max_iter
 *    accepted steps.
 */
static void lbfgs_one(const orc_problem *p, const orc_config *c, const double *x0, double *x_out, double *ell_out,
                      int8_t *status_out, int32_t *iters_out, int64_t *evals_out) {
    const int d = p->d, m = c->m;
    double *x = (double *)malloc(sizeof(double) * (size_t)d);
    double *g = (double *)malloc(sizeof(double) * (size_t)d);
    double *gt = (double *)malloc(sizeof(double) * (size_t)d);
    double *xt = (double *)malloc(sizeof(double) * (size_t)d);
    double *pdir = (double *)malloc(sizeof(double) * (size_t)d);
    double *S = (double *)malloc(sizeof(double) * (size_t)m * d);
    double *Y = (double *)malloc(sizeof(double) * (size_t)m * d);
    double *rho = (double *)malloc(sizeof(double) * (size_t)m);
    double *ring_s = (double *)malloc(sizeof(double) * (size_t)m * d);
    double *ring_y = (double *)malloc(sizeof(double) * (size_t)m * d);
    double *ring_rho = (double *)malloc(sizeof(double) * (size_t)m);
    int count = 0, head = 0; /* head = slot of the oldest pair */
    int64_t evals = 0;
    int it = 0, flat = 0;
    int8_t status = ORC_RUNNING;

    memcpy(x, x0, sizeof(double) * (size_t)d);
    double f = -orc_loglik(p, x, g, NULL);
    for (int i = 0; i < d; ++i) g[i] = -g[i];
    ++evals;
    if (!isfinite(f) || !all_finite(d, g)) status = ORC_NONFINITE;

    while (status == ORC_RUNNING) {
        if (max_abs(d, g) <= c->gtol * (1.0 + fabs(f))) {
            status = ORC_CONVERGED;
            break;
        }
        if (flat >= 2) {
            status = ORC_STALLED;
            break;
        }
        if (it >= c->max_iter) {
            status = ORC_MAXITER;
            break;
        }
        int accepted = 0;
        double ft = 0.0;
        for (int attempt = 0; attempt < 2 && !accepted; ++attempt) {
            if (count == 0) {
                double gn = sqrt(dot(d, g, g));
                for (int i = 0; i < d; ++i) pdir[i] = -g[i] / gn;
            } else {
                /* unroll the ring, oldest first, for the two-loop recursion */
                for (int i = 0; i < count; ++i) {
                    int slot = (head + i) % m;
                    memcpy(S + (size_t)i * d, ring_s + (size_t)slot * d, sizeof(double) * (size_t)d);
                    memcpy(Y + (size_t)i * d, ring_y + (size_t)slot * d, sizeof(double) * (size_t)d);
                    rho[i] = ring_rho[slot];
                }
                orc_two_loop(d, count, S, Y, rho, g, pdir);
                for (int i = 0; i < d; ++i) pdir[i] = -pdir[i];
            }
            double dphi = dot(d, g, pdir);
            if (!(dphi < 0.0)) {
                count = 0;
                head = 0;
                double gn = sqrt(dot(d, g, g));
                for (int i = 0; i < d; ++i) pdir[i] = -g[i] / gn;
                dphi = dot(d, g, pdir);
            }
            double alpha = 1.0;
            for (int bt = 0; bt <= c->max_backtracks; ++bt) {
                for (int i = 0; i < d; ++i) xt[i] = x[i] + alpha * pdir[i];
                ft = -orc_loglik(p, xt, gt, NULL);
                for (int i = 0; i < d; ++i) gt[i] = -gt[i];
                ++evals;
                if (isfinite(ft) && all_finite(d, gt) && ft <= f + c->armijo_c1 * alpha * dphi) {
                    accepted = 1;
                    break;
                }
                alpha *= c->backtrack;
            }
            if (!accepted) {
                if (count == 0) break;
                count = 0;
                head = 0;
            }
        }
        if (!accepted) {
            status = ORC_STALLED;
            break;
        }
        /* curvature pair */
        double *snew = xt; /* reuse buffers: s = xt - x, y = gt - g */
        double ss = 0.0, yy = 0.0, sy = 0.0;
        for (int i = 0; i < d; ++i) {
            double si = snew[i] - x[i];
            double yi = gt[i] - g[i];
            ss += si * si;
            yy += yi * yi;
            sy += si * yi;
        }
        if (sy > 1e-10 * sqrt(ss) * sqrt(yy)) {
            int slot;
            if (count < m) {
                slot = (head + count) % m;
                ++count;
            } else {
                slot = head;
                head = (head + 1) % m;
            }
            for (int i = 0; i < d; ++i) {
                ring_s[(size_t)slot * d + i] = xt[i] - x[i];
                ring_y[(size_t)slot * d + i] = gt[i] - g[i];
            }
            ring_rho[slot] = 1.0 / sy;
        }
        flat = (ft >= f) ? flat + 1 : 0;
        memcpy(x, xt, sizeof(double) * (size_t)d);
        memcpy(g, gt, sizeof(double) * (size_t)d);
        f = ft;
        ++it;
    }
    memcpy(x_out, x, sizeof(double) * (size_t)d);
    *ell_out = -f;
    *status_out = status;
    if (iters_out) *iters_out = it;
    if (evals_out) *evals_out = evals;
    free(ring_rho);
    free(ring_y);
    free(ring_s);
    free(rho);
    free(Y);
    free(S);
    free(pdir);
    free(xt);
    free(gt);
    free(g);
    free(x);
}

void orc_lbfgs(const orc_problem *p, const orc_config *c, const double *x0, int n, double *x_out, double *ell_out,
               int8_t *status_out, int32_t *iters_out, int64_t *evals_out) {
    const int d = p->d;
    int64_t *ev = (int64_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
#pragma omp parallel for num_threads(nthreads_of(c)) schedule(dynamic, 1)
    for (int w = 0; w < n; ++w)
        lbfgs_one(p, c, x0 + (size_t)w * d, x_out + (size_t)w * d, ell_out + w, status_out + w,
                  iters_out ? iters_out + w : NULL, ev + w);
    if (evals_out) {
        int64_t tot = 0;
        for (int w = 0; w < n; ++w) tot += ev[w];
        *evals_out = tot;
    }
    free(ev);
}

/* ------------------------------------------------------------------------ */
/* Cholesky-Banachiewicz, row by row (App. A.8: H = L L^T).                  */
/* ------------------------------------------------------------------------ */
int orc_cholesky(int d, const double *A, double *C) {
    memset(C, 0, sizeof(double) * (size_t)d * d);
    for (int i = 0; i < d; ++i) {
        for (int j = 0; j <= i; ++j) {
            double s = A[(size_t)i * d + j];
            for (int k = 0; k < j; ++k) s -= C[(size_t)i * d + k] * C[(size_t)j * d + k];
            if (i == j) {
                if (!(s > 0.0)) return -1;
                C[(size_t)i * d + i] = sqrt(s);
            } else {
                C[(size_t)i * d + j] = s / C[(size_t)j * d + j];
            }
        }
    }
    return 0;
}

/* Solve (C C^T) v = b: forward then backward substitution. */
static void chol_solve(int d, const double *C, const double *b, double *v) {
    double *y = (double *)malloc(sizeof(double) * (size_t)d);
    for (int i = 0; i < d; ++i) {
        double s = b[i];
        for (int k = 0; k < i; ++k) s -= C[(size_t)i * d + k] * y[k];
        y[i] = s / C[(size_t)i * d + i];
    }
    for (int i = d - 1; i >= 0; --i) {
        double s = y[i];
        for (int k = i + 1; k < d; ++k) s -= C[(size_t)k * d + i] * v[k];
        v[i] = s / C[(size_t)i * d + i];
    }
    free(y);
}

static double linf_dist(int d, const double *a, const double *b) {
    double m = 0.0;
    for (int i = 0; i < d; ++i) {
        double t = fabs(a[i] - b[i]);
        if (t > m) m = t;
    }
    return m;
}

typedef struct {
    double ell;
    int idx;
} orc_rank;

static int rank_cmp(const void *a, const void *b) {
    const orc_rank *x = (const orc_rank *)a, *y = (const orc_rank *)b;
    if (x->ell != y->ell) return x->ell > y->ell ? -1 : 1;
    return x->idx < y->idx ? -1 : (x->idx > y->idx ? 1 : 0);
}

/*
 * Greedy L-infinity deduplication (Sec. 3.5.4, App. A.7): in order of
 * decreasing l (ties -> lower index) the best unassigned point becomes a
 * representative and every unassigned point within tau joins it. Writes the
 * representatives, in that order, to reps; returns their number.
 */
static int greedy_dedup(int d, const double *X, const orc_rank *order, int n, double tau, int *reps) {
    char *assigned = (char *)calloc((size_t)(n > 0 ? n : 1), 1);
    int nr = 0;
    for (int a = 0; a < n; ++a) {
        if (assigned[a]) continue;
        assigned[a] = 1;
        reps[nr++] = a;
        const double *xa = X + (size_t)order[a].idx * d;
        for (int b = a + 1; b < n; ++b)
            if (!assigned[b] && linf_dist(d, xa, X + (size_t)order[b].idx * d) <= tau) assigned[b] = 1;
    }
    free(assigned);
    return nr;
}

/*
 * Laplace stage. Readings:
 *  - candidates: walkers with finite l and status other than NONFINITE;
 *    coarse dedup with tau_c = dedup_coarse * max_i (hi_i - lo_i); at most
 *    cand_cap representatives (highest l first) go on;
 *  - FP64 Newton polish: up to newton_steps steps x <- x + t H^{-1} grad l
 *    with H = -hess l via Cholesky; t = 1 is taken at once when the model
 *    increase g.delta/2 <= 1e-10 (1 + |l|) (the descent test is rounding noise
 *    there), otherwise t is halved (<= 30 times) until l does not decrease;
 *  - filters (Sec. 3.6.4, strengthened): keep if Cholesky of H succeeds at the
 *    final point (positive definite), |grad l|_inf <= eps_grad (1 + |l|), and
 *    lo <= x <= hi (the prior contains the mode, Sec. 3.2);
 *  - final dedup with tau_f = dedup_tol * max_i (hi_i - lo_i), highest l kept;
 *  - log Z_k = l(x*) + (d/2) log 2pi - sum_i log C_ii with H = C C^T
 *    (Sec. 3.7.1 with App. A.8); log Z = LSE_k log Z_k - log V (Sec. 3.2,
 *    Sec. 3.7.3, App. A.10). No modes: log Z = -inf.
 */
int orc_laplace(const orc_problem *p, const orc_config *c, const double *x, const double *ell, const int8_t *status,
                int n, double *modes, double *logZk, double *ell_modes, int cap, int *n_modes, double *logZ) {
    const int d = p->d;
    double wmax = 0.0, logV = 0.0;
    for (int i = 0; i < d; ++i) {
        double w = p->hi[i] - p->lo[i];
        if (w > wmax) wmax = w;
        logV += log(w);
    }
    orc_rank *order = (orc_rank *)malloc(sizeof(orc_rank) * (size_t)(n > 0 ? n : 1));
    int ne = 0;
    for (int w = 0; w < n; ++w) {
        if (!isfinite(ell[w])) continue;
        if (status && status[w] == ORC_NONFINITE) continue;
        order[ne].ell = ell[w];
        order[ne].idx = w;
        ++ne;
    }
    qsort(order, (size_t)ne, sizeof(orc_rank), rank_cmp);
    int *reps = (int *)malloc(sizeof(int) * (size_t)(ne > 0 ? ne : 1));
    int nc = greedy_dedup(d, x, order, ne, c->dedup_coarse * wmax, reps);
    if (nc > c->cand_cap) nc = c->cand_cap;

    double *cx = (double *)malloc(sizeof(double) * (size_t)(nc > 0 ? nc : 1) * d);
    double *cl = (double *)malloc(sizeof(double) * (size_t)(nc > 0 ? nc : 1));
    double *czk = (double *)malloc(sizeof(double) * (size_t)(nc > 0 ? nc : 1));
    char *keep = (char *)calloc((size_t)(nc > 0 ? nc : 1), 1);

#pragma omp parallel for num_threads(nthreads_of(c)) schedule(dynamic, 1)
    for (int ci = 0; ci < nc; ++ci) {
        double *xc = cx + (size_t)ci * d;
        double *g = (double *)malloc(sizeof(double) * (size_t)d);
        double *H = (double *)malloc(sizeof(double) * (size_t)d * d);
        double *C = (double *)malloc(sizeof(double) * (size_t)d * d);
        double *delta = (double *)malloc(sizeof(double) * (size_t)d);
        double *xn = (double *)malloc(sizeof(double) * (size_t)d);
        memcpy(xc, x + (size_t)order[reps[ci]].idx * d, sizeof(double) * (size_t)d);
        double l = orc_loglik(p, xc, g, H);
        int ok = (orc_cholesky(d, H, C) == 0);
        for (int s = 0; s < c->newton_steps && ok; ++s) {
            chol_solve(d, C, g, delta);
            double t = 1.0;
            int acc = 0;
            /* inside the quadratic-convergence regime (model increase g.delta/2 at
               the rounding level of l) the descent test is noise: take the full step */
            if (0.5 * dot(d, g, delta) <= 1e-10 * (1.0 + fabs(l))) {
                for (int i = 0; i < d; ++i) xn[i] = xc[i] + t * delta[i];
                acc = 1;
            }
            for (int h = 0; h < 30 && !acc; ++h) {
                for (int i = 0; i < d; ++i) xn[i] = xc[i] + t * delta[i];
                double ln = orc_loglik(p, xn, NULL, NULL);
                if (ln >= l) {
                    acc = 1;
                    break;
                }
                t *= 0.5;
            }
            if (!acc) break;
            memcpy(xc, xn, sizeof(double) * (size_t)d);
            l = orc_loglik(p, xc, g, H);
            ok = (orc_cholesky(d, H, C) == 0);
        }
        int inside = 1;
        for (int i = 0; i < d; ++i)
            if (!(xc[i] >= p->lo[i] && xc[i] <= p->hi[i])) inside = 0;
        keep[ci] = (char)(ok && isfinite(l) && max_abs(d, g) <= c->eps_grad * (1.0 + fabs(l)) && inside);
        cl[ci] = l;
        if (ok) {
            double ld = 0.0;
            for (int i = 0; i < d; ++i) ld += log(C[(size_t)i * d + i]);
            czk[ci] = l + 0.5 * (double)d * ORC_LOG_2PI - ld;
        } else {
            czk[ci] = NAN;
        }
        free(xn);
        free(delta);
        free(C);
        free(H);
        free(g);
    }

    /* final dedup among the kept candidates, highest polished l first */
    orc_rank *ord2 = (orc_rank *)malloc(sizeof(orc_rank) * (size_t)(nc > 0 ? nc : 1));
    int nk = 0;
    for (int ci = 0; ci < nc; ++ci)
        if (keep[ci]) {
            ord2[nk].ell = cl[ci];
            ord2[nk].idx = ci;
            ++nk;
        }
    qsort(ord2, (size_t)nk, sizeof(orc_rank), rank_cmp);
    int *reps2 = (int *)malloc(sizeof(int) * (size_t)(nk > 0 ? nk : 1));
    int nm = greedy_dedup(d, cx, ord2, nk, c->dedup_tol * wmax, reps2);

    double zmax = -INFINITY;
    for (int t = 0; t < nm; ++t) {
        int ci = ord2[reps2[t]].idx;
        if (czk[ci] > zmax) zmax = czk[ci];
        if (t < cap) {
            if (modes) memcpy(modes + (size_t)t * d, cx + (size_t)ci * d, sizeof(double) * (size_t)d);
            if (logZk) logZk[t] = czk[ci];
            if (ell_modes) ell_modes[t] = cl[ci];
        }
    }
    double lz = -INFINITY;
    if (nm > 0) {
        double ssum = 0.0;
        for (int t = 0; t < nm; ++t) ssum += exp(czk[ord2[reps2[t]].idx] - zmax);
        lz = zmax + log(ssum) - logV;
    }
    if (logZ) *logZ = lz;
    if (n_modes) *n_modes = nm;
    free(reps2);
    free(ord2);
    free(keep);
    free(czk);
    free(cl);
    free(cx);
    free(reps);
    free(order);
    return nm;
}

int orc_evidence(const orc_problem *p, const orc_config *c, double *modes, double *logZk, int cap, int *n_modes,
                 double *logZ) {
    const int d = p->d;
    int ns = c->n_starts;
    double *starts = (double *)malloc(sizeof(double) * (size_t)(ns > 0 ? ns : 1) * d);
    double *ls = (double *)malloc(sizeof(double) * (size_t)(ns > 0 ? ns : 1));
    int n = orc_discover(p, c, starts, ls);
    double *xo = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * d);
    double *lo = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    int8_t *st = (int8_t *)malloc((size_t)(n > 0 ? n : 1));
    orc_lbfgs(p, c, starts, n, xo, lo, st, NULL, NULL);
    int nm = orc_laplace(p, c, xo, lo, st, n, modes, logZk, NULL, cap, n_modes, logZ);
    free(st);
    free(lo);
    free(xo);
    free(ls);
    free(starts);
    return nm;
}

/* ------------------------------------------------------------------------ */
/* ChiSao oscillation around the refinement (Sec. 3.5.5, Algorithm 1).        */
/* Readings where the paper is silent:                                        */
/*  - an oscillation's convergence phase is L-BFGS from the current positions */
/*    with an empty history, capped at conv_iters accepted steps;             */
/*  - a sample is converged when |grad l|_inf <= eps_grad (1 + |l|) (the     */
/*    scaled form of the Laplace filter) and sticks when also l >= l_max +    */
/*    log 0.1 (l_max over all finite samples); "unconverged" samples are the  */
/*    finite ones that are not converged; with conv_from_status, converged is */
/*    the refinement's CONVERGED / STALLED state instead (the reading for a   */
/*    refinement whose gradients are too coarse for the FP64 test);           */
/*  - deduplication runs over the stuck samples with the coarse radius        */
/*    (greedy, l descending, ties to the lower index); the stuck samples that */
/*    are not representatives are the K_lost duplicates;                      */
/*  - Repulse Monkey (>= min_unconverged unconverged samples): lost sample   */
/*    l (index order) shoots a ray from the (l mod n)-th unconverged sample   */
/*    in a Philox-normal direction (counter (pair, l, osc, 'RPMK')) to        */
/*    the box boundary and moves to the best of n_steps samples on it;        */
/*  - Golden Rooster (fewer such samples): lost sample l goes to peak         */
/*    p = l mod n_peaks (representatives by decreasing l) along direction     */
/*    c = (l / n_peaks) / 2, sign + for even l / n_peaks and - for odd;       */
/*    direction c is column c mod G of orthonormal group c / G of that peak,  */
/*    G = min(d, 64) (the paper fixes no group size; at most d directions are */
/*    mutually orthogonal, and groups of at most 64 keep a QR at O(d G^2));   */
/*    a group is the Q of a QR (modified Gram-Schmidt) of G Philox-normal     */
/*    vectors, counter (pair, group G + column, osc << 16 | p, 'GRST'); on    */
/*    the ray it                                                              */
/*    moves to the best sample beyond the first valley (the first sample      */
/*    after which l rises), or to the exit sample when l never rises; it      */
/*    stays off once an oscillation that used it ends with no more peaks than */
/*    before;                                                                 */
/*  - ray origins are clamped to the box; ray samples at t_j = (j+1)/n t_exit;*/
/*  - anti-convergence: every finite sample that is not stuck takes           */
/*    anti_steps steps v <- momentum v - alpha grad l, x <- x + v (descent on */
/*    l, so away from the peak it sits near), v = 0 at the start, clamped to  */
/*    the box after each step; alpha is a fixed step size (no value given in  */
/*    the paper);                                                             */
/*  - Hands Like Clouds is not applied (out of scope); the last oscillation   */
/*    skips reseeding and anti-convergence.                                   */
/* ------------------------------------------------------------------------ */
static void box_clamp(const orc_problem *p, double *x) {
    for (int i = 0; i < p->d; ++i) x[i] = x[i] < p->lo[i] ? p->lo[i] : (x[i] > p->hi[i] ? p->hi[i] : x[i]);
}

/* d standard normals from Philox blocks with counter (pair, w1, w2, tag). */
static void philox_normals(int d, uint64_t seed, uint32_t w1, uint32_t w2, uint32_t tag, double *z) {
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int q = 0; q < (d + 1) / 2; ++q) {
        uint32_t ctr[4] = {(uint32_t)q, w1, w2, tag};
        uint32_t o[4];
        orc_philox4x32_10(ctr, key, o);
        double u1 = orc_unit(o[0], o[1]);
        double u2 = orc_unit(o[2], o[3]);
        double rad = sqrt(-2.0 * log(u1));
        double th = ORC_TWO_PI * u2;
        z[2 * q] = rad * cos(th);
        if (2 * q + 1 < d) z[2 * q + 1] = rad * sin(th);
    }
}

void orc_chisao_anticonverge(const orc_problem *p, double *x, int n, int steps, double momentum, double alpha) {
    const int d = p->d;
    double *g = (double *)malloc(sizeof(double) * (size_t)d);
    double *v = (double *)malloc(sizeof(double) * (size_t)d);
    for (int s = 0; s < n; ++s) {
        double *xs = x + (size_t)s * d;
        for (int i = 0; i < d; ++i) v[i] = 0.0;
        for (int t = 0; t < steps; ++t) {
            orc_loglik(p, xs, g, NULL);
            for (int i = 0; i < d; ++i) {
                v[i] = momentum * v[i] - alpha * g[i];
                xs[i] = xs[i] + v[i];
            }
            box_clamp(p, xs);
        }
    }
    free(v);
    free(g);
}

void orc_chisao_directions(int d, int r, uint64_t seed, int osc, int peak, int basis, double *Q) {
    const int G = d < 64 ? d : 64; /* directions per orthonormal group */
    if (r > G) r = G;
    /* columns j = 0..r-1 of Q (d x r, column j at Q[j*d..]): modified Gram-Schmidt */
    for (int j = 0; j < r; ++j) {
        double *qj = Q + (size_t)j * d;
        philox_normals(d, seed, (uint32_t)basis * (uint32_t)G + (uint32_t)j, ((uint32_t)osc << 16) | (uint32_t)peak,
                       0x47525354u, qj);
        for (int k = 0; k < j; ++k) {
            const double *qk = Q + (size_t)k * d;
            double dot = 0.0;
            for (int i = 0; i < d; ++i) dot += qk[i] * qj[i];
            for (int i = 0; i < d; ++i) qj[i] -= dot * qk[i];
        }
        double nrm = 0.0;
        for (int i = 0; i < d; ++i) nrm += qj[i] * qj[i];
        nrm = sqrt(nrm);
        for (int i = 0; i < d; ++i) qj[i] /= nrm;
    }
}

int orc_chisao_ray_best(const orc_problem *p, const double *origin, const double *dir, int n_steps, int past_valley,
                        double *x_out, double *ell_out) {
    const int d = p->d;
    double *o = (double *)malloc(sizeof(double) * (size_t)d);
    double *xt = (double *)malloc(sizeof(double) * (size_t)d);
    double *ell = (double *)malloc(sizeof(double) * (size_t)(n_steps > 0 ? n_steps : 1));
    memcpy(o, origin, sizeof(double) * (size_t)d);
    box_clamp(p, o);
    double t_exit = INFINITY;
    for (int i = 0; i < d; ++i) {
        if (dir[i] > 0.0) {
            double t = (p->hi[i] - o[i]) / dir[i];
            if (t < t_exit) t_exit = t;
        } else if (dir[i] < 0.0) {
            double t = (p->lo[i] - o[i]) / dir[i];
            if (t < t_exit) t_exit = t;
        }
    }
    if (!(t_exit < INFINITY)) t_exit = 0.0;
    for (int j = 0; j < n_steps; ++j) {
        const double t = ((double)(j + 1) / (double)n_steps) * t_exit;
        for (int i = 0; i < d; ++i) xt[i] = o[i] + t * dir[i];
        ell[j] = orc_loglik(p, xt, NULL, NULL);
    }
    int j0 = 0;
    if (past_valley) {
        /* first sample after which l rises; none: the exit sample */
        j0 = -1;
        for (int j = 0; j + 1 < n_steps; ++j)
            if (ell[j + 1] > ell[j]) {
                j0 = j + 1;
                break;
            }
        if (j0 < 0) j0 = n_steps - 1;
    }
    int best = j0;
    for (int j = j0 + 1; j < n_steps; ++j)
        if (ell[j] > ell[best]) best = j;
    const double t = ((double)(best + 1) / (double)n_steps) * t_exit;
    for (int i = 0; i < d; ++i) x_out[i] = o[i] + t * dir[i];
    if (ell_out) *ell_out = ell[best];
    free(ell);
    free(xt);
    free(o);
    return best;
}

int orc_chisao(const orc_problem *p, const orc_config *c, const orc_chisao_config *cc, const double *x0, int n,
               double *x_out, double *ell_out, int8_t *stuck_out) {
    const int d = p->d;
    double wmax = 0.0;
    for (int i = 0; i < d; ++i)
        if (p->hi[i] - p->lo[i] > wmax) wmax = p->hi[i] - p->lo[i];
    orc_config cl = *c;
    cl.max_iter = cc->conv_iters;
    double *x = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * d);
    double *xn = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * d);
    double *ell = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    int8_t *st = (int8_t *)malloc((size_t)(n > 0 ? n : 1));
    int8_t *stuck = (int8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    int8_t *lost = (int8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    int8_t *conv = (int8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    orc_rank *order = (orc_rank *)malloc(sizeof(orc_rank) * (size_t)(n > 0 ? n : 1));
    int *reps = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    int *peaks = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    double *dir = (double *)malloc(sizeof(double) * (size_t)d);
    memcpy(x, x0, sizeof(double) * (size_t)n * d);
    int gr_on = 1, gr_used_prev = 0, peaks_prev = -1, n_peaks = 0;
    for (int osc = 0; osc < cc->n_osc; ++osc) {
        /* convergence phase: all samples released, L-BFGS from where they are */
        orc_lbfgs(p, &cl, x, n, xn, ell, st, NULL, NULL);
        memcpy(x, xn, sizeof(double) * (size_t)n * d);
        /* stick detection */
        double lmax = -INFINITY;
        for (int s = 0; s < n; ++s)
            if (isfinite(ell[s]) && ell[s] > lmax) lmax = ell[s];
        int ns = 0;
        for (int s = 0; s < n; ++s) {
            conv[s] = 0;
            if (isfinite(ell[s])) {
                if (cc->conv_from_status) {
                    conv[s] = (int8_t)(st[s] == ORC_CONVERGED || st[s] == ORC_STALLED);
                } else {
                    const double l = orc_loglik(p, x + (size_t)s * d, dir, NULL);
                    conv[s] = (int8_t)(max_abs(d, dir) <= c->eps_grad * (1.0 + fabs(l)));
                }
            }
            stuck[s] = (int8_t)(conv[s] && ell[s] >= lmax + log(0.1));
            lost[s] = 0;
            if (stuck[s]) {
                order[ns].ell = ell[s];
                order[ns].idx = s;
                ++ns;
            }
        }
        /* deduplication of the stuck samples: non-representatives are lost */
        qsort(order, (size_t)ns, sizeof(orc_rank), rank_cmp);
        n_peaks = greedy_dedup(d, x, order, ns, c->dedup_coarse * wmax, reps);
        for (int a = 0; a < ns; ++a) lost[order[a].idx] = 1;
        for (int r = 0; r < n_peaks; ++r) {
            peaks[r] = order[reps[r]].idx;
            lost[peaks[r]] = 0;
        }
        for (int s = 0; s < n; ++s)
            if (lost[s]) stuck[s] = 0;
        if (gr_used_prev && n_peaks <= peaks_prev) gr_on = 0;
        gr_used_prev = 0;
        peaks_prev = n_peaks;
        if (osc == cc->n_osc - 1) break;
        /* reseeding of the lost samples */
        int n_free = 0;
        for (int s = 0; s < n; ++s)
            if (!conv[s] && isfinite(ell[s])) ++n_free;
        int l_ord = 0;
        for (int s = 0; s < n; ++s) {
            if (!lost[s]) continue;
            if (n_free > 0 && n_free >= cc->min_unconverged) {
                int which = l_ord % n_free, o = -1;
                for (int q = 0; q < n; ++q)
                    if (!conv[q] && isfinite(ell[q]) && which-- == 0) {
                        o = q;
                        break;
                    }
                philox_normals(d, c->seed, (uint32_t)l_ord, (uint32_t)osc, 0x52504D4Bu, dir);
                double nrm = 0.0;
                for (int i = 0; i < d; ++i) nrm += dir[i] * dir[i];
                nrm = sqrt(nrm);
                for (int i = 0; i < d; ++i) dir[i] /= nrm;
                orc_chisao_ray_best(p, x + (size_t)o * d, dir, c->n_steps, 0, x + (size_t)s * d, NULL);
            } else if (gr_on && n_peaks > 0) {
                const int pk = l_ord % n_peaks, k = l_ord / n_peaks, cdir = k / 2;
                const int G = d < 64 ? d : 64;
                const int basis = cdir / G, col = cdir % G;
                const double sgn = (k % 2 == 0) ? 1.0 : -1.0;
                double *Q = (double *)malloc(sizeof(double) * (size_t)(col + 1) * d);
                orc_chisao_directions(d, col + 1, c->seed, osc, pk, basis, Q);
                for (int i = 0; i < d; ++i) dir[i] = sgn * Q[(size_t)col * d + i];
                free(Q);
                orc_chisao_ray_best(p, x + (size_t)peaks[pk] * d, dir, c->n_steps, 1, x + (size_t)s * d, NULL);
                gr_used_prev = 1;
            }
            ++l_ord;
        }
        /* anti-convergence of every sample that is not stuck */
        for (int s = 0; s < n; ++s)
            if (!stuck[s] && st[s] != ORC_NONFINITE)
                orc_chisao_anticonverge(p, x + (size_t)s * d, 1, cc->anti_steps, cc->momentum, cc->anti_alpha);
    }
    memcpy(x_out, x, sizeof(double) * (size_t)n * d);
    if (ell_out) memcpy(ell_out, ell, sizeof(double) * (size_t)n);
    if (stuck_out) memcpy(stuck_out, stuck, (size_t)n);
    free(dir);
    free(peaks);
    free(reps);
    free(order);
    free(conv);
    free(lost);
    free(stuck);
    free(st);
    free(ell);
    free(xn);
    free(x);
    return n_peaks;
}

/* ------------------------------------------------------------------------ */
/* Preprocessing: dimensional pathology detection (Sec. 3.4, its Algorithm).  */
/* 2d + 1 evaluations: l at the box centre c and at c +- Delta_i e_i, with    */
/* Delta_i = (hi_i - lo_i) / 2; sensitivity s_i = |l(c + Delta_i e_i) - l(c)| */
/* + |l(c - Delta_i e_i) - l(c)|. Flat: s_i < eps_flat median(s); soft:       */
/* s_i < eps_soft max(s) and not flat; the rest is active. Readings:          */
/*  - median of an even count is the mean of the two middle values; median    */
/*    and max run over the finite s_i, and a non-finite s_i is active;        */
/*  - the marginal integrals: a flat coordinate integrates a constant over    */
/*    [lo_i, hi_i], log(2 Delta_i) (the paper prints log Delta_i); a soft     */
/*    one a Gaussian of width sigma_i = Delta_i / sqrt(s_i), 1/2 log 2 pi +   */
/*    log sigma_i; their sum is *log_int, and *log_vol is the flagged         */
/*    coordinates' share of log V, sum log(2 Delta_i), so that the evidence   */
/*    of the full problem is that of the active problem (l with the flagged   */
/*    coordinates held at c, prior over the active box) + *log_int -          */
/*    *log_vol.                                                               */
/* ------------------------------------------------------------------------ */
static int dbl_cmp(const void *a, const void *b) {
    const double x = *(const double *)a, y = *(const double *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

int orc_precheck(const orc_problem *p, double eps_flat, double eps_soft, double *s_out, int8_t *cls_out,
                 double *log_int, double *log_vol) {
    const int d = p->d;
    double *c = (double *)malloc(sizeof(double) * (size_t)d);
    double *x = (double *)malloc(sizeof(double) * (size_t)d);
    double *fin = (double *)malloc(sizeof(double) * (size_t)d);
    for (int i = 0; i < d; ++i) c[i] = 0.5 * (p->lo[i] + p->hi[i]);
    const double l0 = orc_loglik(p, c, NULL, NULL);
    int nf = 0;
    for (int i = 0; i < d; ++i) {
        const double delta = 0.5 * (p->hi[i] - p->lo[i]);
        memcpy(x, c, sizeof(double) * (size_t)d);
        x[i] = c[i] + delta;
        const double lp = orc_loglik(p, x, NULL, NULL);
        x[i] = c[i] - delta;
        const double lm = orc_loglik(p, x, NULL, NULL);
        s_out[i] = fabs(lp - l0) + fabs(lm - l0);
        if (isfinite(s_out[i])) fin[nf++] = s_out[i];
    }
    double med = 0.0, smax = 0.0;
    if (nf > 0) {
        qsort(fin, (size_t)nf, sizeof(double), dbl_cmp);
        med = (nf % 2) ? fin[nf / 2] : 0.5 * (fin[nf / 2 - 1] + fin[nf / 2]);
        smax = fin[nf - 1];
    }
    int n_active = 0;
    double li = 0.0, lv = 0.0;
    for (int i = 0; i < d; ++i) {
        const double delta = 0.5 * (p->hi[i] - p->lo[i]);
        int8_t cl = 0;
        if (isfinite(s_out[i])) {
            if (s_out[i] < eps_flat * med)
                cl = 1;
            else if (s_out[i] < eps_soft * smax)
                cl = 2;
        }
        cls_out[i] = cl;
        if (cl == 0) {
            ++n_active;
        } else {
            lv += log(2.0 * delta);
            li += (cl == 1) ? log(2.0 * delta) : 0.5 * log(ORC_TWO_PI) + log(delta / sqrt(s_out[i]));
        }
    }
    if (log_int) *log_int = li;
    if (log_vol) *log_vol = lv;
    free(fin);
    free(x);
    free(c);
    return n_active;
}

/* ------------------------------------------------------------------------ */
/* Black-box derivatives and rotation detection (App. A.4, Sec. 3.7.2).       */
/* Central differences of l with step eps along the axes; the Hessians are of */
/* l itself (negative definite at a maximum), as printed. Readings:           */
/*  - the full Hessian takes its diagonal from the 2d + 1 axis evaluations    */
/*    and each off-diagonal pair i < j from four evaluations at              */
/*    x +- eps e_i +- eps e_j, mirrored to j, i (2 d^2 + 1 evaluations in     */
/*    all);                                                                   */
/*  - the uniform-correlation probe takes v^T H v from the second difference  */
/*    of l along v = (1, ..., 1) / sqrt(d) (the two evaluations x +- eps v)   */
/*    and a = mean H_ii from the diagonal second differences;                 */
/*  - the perpendicular step fraction whitens a step and the gradient at its  */
/*    start by w_i = sqrt(-H_ii): dtheta~ = w dtheta, g~ = grad l / w (the    */
/*    gradient of l in the whitened coordinates), and f_perp is the part of   */
/*    dtheta~ orthogonal to g~, relative to |dtheta~|; it is 0 for a zero     */
/*    step or gradient and NaN when some H_ii >= 0.                           */
/* ------------------------------------------------------------------------ */
static double loglik_shift2(const orc_problem *p, const double *x, double *xs, int i, double ai, int j, double aj) {
    memcpy(xs, x, sizeof(double) * (size_t)p->d);
    if (i >= 0) xs[i] = x[i] + ai;
    if (j >= 0) xs[j] = xs[j] + aj;
    return orc_loglik(p, xs, NULL, NULL);
}

void orc_fd_grad(const orc_problem *p, const double *x, double eps, double *g) {
    double *xs = (double *)malloc(sizeof(double) * (size_t)p->d);
    for (int i = 0; i < p->d; ++i) {
        const double fp = loglik_shift2(p, x, xs, i, eps, -1, 0.0);
        const double fm = loglik_shift2(p, x, xs, i, -eps, -1, 0.0);
        g[i] = (fp - fm) / (2.0 * eps);
    }
    free(xs);
}

void orc_fd_hess_diag(const orc_problem *p, const double *x, double eps, double *hdiag) {
    double *xs = (double *)malloc(sizeof(double) * (size_t)p->d);
    const double f0 = orc_loglik(p, x, NULL, NULL);
    for (int i = 0; i < p->d; ++i) {
        const double fp = loglik_shift2(p, x, xs, i, eps, -1, 0.0);
        const double fm = loglik_shift2(p, x, xs, i, -eps, -1, 0.0);
        hdiag[i] = (fp - 2.0 * f0 + fm) / (eps * eps);
    }
    free(xs);
}

void orc_fd_hess_full(const orc_problem *p, const double *x, double eps, double *H) {
    const int d = p->d;
    double *xs = (double *)malloc(sizeof(double) * (size_t)d);
    double *hd = (double *)malloc(sizeof(double) * (size_t)d);
    orc_fd_hess_diag(p, x, eps, hd);
    for (int i = 0; i < d; ++i) {
        H[(size_t)i * d + i] = hd[i];
        for (int j = i + 1; j < d; ++j) {
            const double fpp = loglik_shift2(p, x, xs, i, eps, j, eps);
            const double fpm = loglik_shift2(p, x, xs, i, eps, j, -eps);
            const double fmp = loglik_shift2(p, x, xs, i, -eps, j, eps);
            const double fmm = loglik_shift2(p, x, xs, i, -eps, j, -eps);
            const double h = (fpp - fpm - fmp + fmm) / (4.0 * eps * eps);
            H[(size_t)i * d + j] = h;
            H[(size_t)j * d + i] = h;
        }
    }
    free(hd);
    free(xs);
}

double orc_uniform_corr_probe(const orc_problem *p, const double *x, double eps, const double *hdiag) {
    const int d = p->d;
    if (d < 2) return 0.0;
    double *xs = (double *)malloc(sizeof(double) * (size_t)d);
    const double f0 = orc_loglik(p, x, NULL, NULL);
    const double vi = 1.0 / sqrt((double)d);
    for (int i = 0; i < d; ++i) xs[i] = x[i] + eps * vi;
    const double fp = orc_loglik(p, xs, NULL, NULL);
    for (int i = 0; i < d; ++i) xs[i] = x[i] - eps * vi;
    const double fm = orc_loglik(p, xs, NULL, NULL);
    const double vhv = (fp - 2.0 * f0 + fm) / (eps * eps);
    double a = 0.0;
    for (int i = 0; i < d; ++i) a += hdiag[i];
    a /= (double)d;
    free(xs);
    return (vhv - a) / (double)(d - 1);
}

double orc_perp_fraction(int d, const double *dtheta, const double *grad, const double *hdiag) {
    double ss = 0.0, gg = 0.0, sg = 0.0;
    for (int i = 0; i < d; ++i) {
        if (!(hdiag[i] < 0.0)) return NAN;
        const double w = sqrt(-hdiag[i]);
        const double st = w * dtheta[i], gt = grad[i] / w;
        ss += st * st;
        gg += gt * gt;
        sg += st * gt;
    }
    if (ss == 0.0 || gg == 0.0) return 0.0;
    /* dtheta~_perp = dtheta~ - (dtheta~ . g~ / |g~|^2) g~, formed explicitly */
    const double c = sg / gg;
    double pp = 0.0;
    for (int i = 0; i < d; ++i) {
        const double w = sqrt(-hdiag[i]);
        const double q = w * dtheta[i] - c * (grad[i] / w);
        pp += q * q;
    }
    return sqrt(pp / ss);
}

/* ------------------------------------------------------------------------ */
/* The other ray families (Sec. 3.5.1) and the two-pass sampling along a ray  */
/* (Sec. 3.5.2). Readings where the paper is silent:                          */
/*  - every random draw of ray r of a family comes from Philox blocks with    */
/*    counter (q, r, family tag, purpose), key = seed; bit b of a stream is   */
/*    bit b % 32 of word (b / 32) % 4 of block q = b / 128; uniform k of a    */
/*    stream is orc_unit of words 2 (k % 2), 2 (k % 2) + 1 of block k / 2;    */
/*    an index below n is (word 0 of block 0 of its stream) * n >> 32;        */
/*  - V2V: start and end vertex from independent bit streams (purposes 0,     */
/*    1): coordinate i is hi_i when its bit is 1, else lo_i; an end equal to  */
/*    the start becomes the antipode;                                         */
/*  - V2E: start vertex (purpose 0); the end is the midpoint of an edge:      */
/*    vertex bits (purpose 1) with one free coordinate j (index, purpose 2)   */
/*    set to the box centre;                                                  */
/*  - W2W: axis i (index, purpose 2); start on the face x_i = lo_i, end on    */
/*    x_i = hi_i, every other coordinate uniform in [lo, hi] (purposes 0, 1); */
/*  - coarse pass: n samples at t_j = j / (n - 1) of the segment (t = 1/2     */
/*    for n = 1); the active region is {j : l_j > max_j l_j - delta};        */
/*  - refinement pass: density proportional to the likelihood, piecewise      */
/*    constant on the coarse cells [t_j - h/2, t_j + h/2] clipped to [0, 1]   */
/*    (h = 1/(n - 1)), weight exp(l_j - max l) times the cell length on       */
/*    active cells and 0 elsewhere; n_ref points at the inverse CDF of the    */
/*    midpoints u_k = (k + 1/2) / n_ref, linear inside a cell.                */
/* ------------------------------------------------------------------------ */
enum { ORC_TAG_V2V = 0x56325620u, ORC_TAG_V2E = 0x56324520u, ORC_TAG_W2W = 0x57325720u };

static uint32_t stream_word(uint64_t seed, uint32_t r, uint32_t tag, uint32_t purpose, uint32_t q, int w) {
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t ctr[4] = {q, r, tag, purpose};
    uint32_t o[4];
    orc_philox4x32_10(ctr, key, o);
    return o[w];
}
static int stream_bit(uint64_t seed, uint32_t r, uint32_t tag, uint32_t purpose, int b) {
    return (int)((stream_word(seed, r, tag, purpose, (uint32_t)(b / 128), (b / 32) % 4) >> (b % 32)) & 1u);
}
static double stream_unit(uint64_t seed, uint32_t r, uint32_t tag, uint32_t purpose, int k) {
    const uint32_t q = (uint32_t)(k / 2);
    const int w = 2 * (k % 2);
    return orc_unit(stream_word(seed, r, tag, purpose, q, w), stream_word(seed, r, tag, purpose, q, w + 1));
}
static int stream_index(uint64_t seed, uint32_t r, uint32_t tag, uint32_t purpose, int n) {
    return (int)(((uint64_t)stream_word(seed, r, tag, purpose, 0, 0) * (uint64_t)n) >> 32);
}

int orc_ray_segment(const orc_problem *p, int family, uint64_t seed, int r, double *start, double *end) {
    const int d = p->d;
    if (family == ORC_RAY_V2V || family == ORC_RAY_V2E) {
        const uint32_t tag = family == ORC_RAY_V2V ? ORC_TAG_V2V : ORC_TAG_V2E;
        int same = 1;
        for (int i = 0; i < d; ++i) {
            const int bs = stream_bit(seed, (uint32_t)r, tag, 0, i);
            const int be = stream_bit(seed, (uint32_t)r, tag, 1, i);
            start[i] = bs ? p->hi[i] : p->lo[i];
            end[i] = be ? p->hi[i] : p->lo[i];
            same &= (bs == be);
        }
        if (family == ORC_RAY_V2V) {
            if (same)
                for (int i = 0; i < d; ++i) end[i] = start[i] == p->hi[i] ? p->lo[i] : p->hi[i];
        } else {
            const int j = stream_index(seed, (uint32_t)r, tag, 2, d);
            end[j] = 0.5 * (p->lo[j] + p->hi[j]);
        }
        return 0;
    }
    if (family == ORC_RAY_W2W) {
        const int ax = stream_index(seed, (uint32_t)r, ORC_TAG_W2W, 2, d);
        for (int i = 0; i < d; ++i) {
            const double w = p->hi[i] - p->lo[i];
            start[i] = p->lo[i] + stream_unit(seed, (uint32_t)r, ORC_TAG_W2W, 0, i) * w;
            end[i] = p->lo[i] + stream_unit(seed, (uint32_t)r, ORC_TAG_W2W, 1, i) * w;
        }
        start[ax] = p->lo[ax];
        end[ax] = p->hi[ax];
        return 0;
    }
    return -1;
}

void orc_ray_two_pass(const orc_problem *p, const double *start, const double *end, int n, double delta, int n_ref,
                      double *ell_coarse, double *t_ref, double *ell_ref) {
    const int d = p->d;
    double *x = (double *)malloc(sizeof(double) * (size_t)d);
    double *cdf = (double *)malloc(sizeof(double) * (size_t)(n + 1));
    double lmax = -INFINITY;
    for (int j = 0; j < n; ++j) {
        const double t = n > 1 ? (double)j / (double)(n - 1) : 0.5;
        for (int i = 0; i < d; ++i) x[i] = start[i] + t * (end[i] - start[i]);
        ell_coarse[j] = orc_loglik(p, x, NULL, NULL);
        if (ell_coarse[j] > lmax) lmax = ell_coarse[j];
    }
    const double h = n > 1 ? 1.0 / (double)(n - 1) : 1.0;
    cdf[0] = 0.0;
    for (int j = 0; j < n; ++j) {
        const double tc = n > 1 ? (double)j / (double)(n - 1) : 0.5;
        double a = tc - 0.5 * h, b = tc + 0.5 * h;
        if (a < 0.0) a = 0.0;
        if (b > 1.0) b = 1.0;
        const double w = (ell_coarse[j] > lmax - delta) ? exp(ell_coarse[j] - lmax) * (b - a) : 0.0;
        cdf[j + 1] = cdf[j] + w;
    }
    for (int k = 0; k < n_ref; ++k) {
        const double u = ((double)k + 0.5) / (double)n_ref * cdf[n];
        int j = 0;
        while (j < n - 1 && cdf[j + 1] <= u) ++j; /* cdf[j] <= u < cdf[j + 1]: never an empty cell */
        const double tc = n > 1 ? (double)j / (double)(n - 1) : 0.5;
        double a = tc - 0.5 * h, b = tc + 0.5 * h;
        if (a < 0.0) a = 0.0;
        if (b > 1.0) b = 1.0;
        const double cw = cdf[j + 1] - cdf[j];
        const double fr = cw > 0.0 ? (u - cdf[j]) / cw : 0.5;
        const double t = a + fr * (b - a);
        t_ref[k] = t;
        for (int i = 0; i < d; ++i) x[i] = start[i] + t * (end[i] - start[i]);
        ell_ref[k] = orc_loglik(p, x, NULL, NULL);
    }
    free(cdf);
    free(x);
}
