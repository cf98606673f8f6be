// precheck.cu -- preprocessing: dimensional pathology detection (Sec. 3.4).
//
// The probe needs l at the box centre c and at c +- Delta_i e_i for every i
// (2d + 1 points). Each probe point moves one coordinate, so with
// z_k = L_k^T (x - mu_k):
//     z_k(c + t e_i) = z_k(c) + t L_k[i, :]^T,
//     e_k(c + t e_i) - e_k(c) = -t (z_k(c) . L_k[i, :]) - t^2 |L_k[i, :]|^2 / 2,
// and l(c + t e_i) - l(c) = LSE_k (e_k(c) - l(c) + that change). The whole
// probe is one GEMV per component (z_k(c)) and a dot product and a squared
// norm per row of L_k: O(K d^2) work, two streaming reads of the L_k, and the
// l differences come out without the cancellation of subtracting two l values
// (for one component the difference is the quadratic above exactly).
//
// Then one CTA sorts the finite sensitivities (bitonic, d <= 1024) for the
// median, takes the maximum, classifies (flat: s < eps_flat median; soft:
// s < eps_soft max and not flat) and sums the marginal terms in index order:
// log(2 Delta_i) for a flat coordinate, 1/2 log 2 pi + log(Delta_i / sqrt(s_i))
// for a soft one, and the flagged coordinates' log-volume sum log(2 Delta_i).
#include "sb_precheck.cuh"

namespace sb {

namespace {

constexpr int PRE_RC = 64;  // rows of L_k per partial of z_k(c)

// part[k][chunk][j] = sum over rows i of the chunk (i >= j) of L_k[i][j] (c_i - mu_k,i)
__global__ void __launch_bounds__(256) k_pre_z0_part(int d, const double *L, const double *mu, const double *c,
                                                     double *part) {
    const int chunk = blockIdx.x, k = blockIdx.y, nch = gridDim.x;
    const int i0 = chunk * PRE_RC, i1 = min(d, i0 + PRE_RC);
    const double *Lk = L + (size_t)k * d * d;
    const double *mk = mu + (size_t)k * d;
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
        double acc = 0.0;
        for (int i = max(i0, j); i < i1; ++i) acc += Lk[(size_t)i * d + j] * (c[i] - mk[i]);
        part[((size_t)k * nch + chunk) * d + j] = acc;
    }
}

// z0[k][j] = sum of the partials (chunk order); e0[k] = a_k - |z0_k|^2 / 2
__global__ void __launch_bounds__(256) k_pre_z0_fin(int d, int nch, const double *part, const double *a, double *z0,
                                                    double *e0) {
    __shared__ double sh[256 / 32];
    const int k = blockIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double ss = 0.0;
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
        double z = 0.0;
        for (int q = 0; q < nch; ++q) z += part[((size_t)k * nch + q) * d + j];
        z0[(size_t)k * d + j] = z;
        ss += z * z;
    }
    ss = warp_sum(ss);
    if (lane == 0) sh[wid] = ss;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 256 / 32; ++w) t += sh[w];
        e0[k] = a[k] - 0.5 * t;
    }
}

// warp per (k, i): dot[k][i] = z0_k . L_k[i, :], nrm[k][i] = |L_k[i, :]|^2 (j <= i)
__global__ void __launch_bounds__(256) k_pre_rows(int d, const double *L, const double *z0, double *dot, double *nrm) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * 8 + (threadIdx.x >> 5), k = blockIdx.y;
    if (i >= d) return;
    const double *row = L + ((size_t)k * d + i) * d;
    const double *zk = z0 + (size_t)k * d;
    double sd = 0.0, sn = 0.0;
    for (int j = lane; j <= i; j += 32) {
        const double v = row[j];
        sd += v * zk[j];
        sn += v * v;
    }
    sd = warp_sum(sd);
    sn = warp_sum(sn);
    if (lane == 0) {
        dot[(size_t)k * d + i] = sd;
        nrm[(size_t)k * d + i] = sn;
    }
}

// l(c + t e_i) - l(c) for t = +-Delta_i, and s_i = |up| + |down|
__global__ void __launch_bounds__(256) k_pre_sens(int d, int K, const double *e0, const double *dot,
                                                  const double *nrm, const double *half, double *s) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d) return;
    double m0 = -INFINITY;
    for (int k = 0; k < K; ++k) m0 = fmax(m0, e0[k]);
    double s0 = 0.0;
    for (int k = 0; k < K; ++k) s0 += exp(e0[k] - m0);
    const double l0 = m0 + log(s0);
    const double t = half[i];
    double out = 0.0;
    for (int sgn = 0; sgn < 2; ++sgn) {
        const double tt = sgn ? -t : t;
        double m = -INFINITY;
        for (int k = 0; k < K; ++k) {
            const double v = (e0[k] - l0) - tt * dot[(size_t)k * d + i] - 0.5 * tt * tt * nrm[(size_t)k * d + i];
            m = fmax(m, v);
        }
        double acc = 0.0;
        for (int k = 0; k < K; ++k) {
            const double v = (e0[k] - l0) - tt * dot[(size_t)k * d + i] - 0.5 * tt * tt * nrm[(size_t)k * d + i];
            acc += exp(v - m);
        }
        out += fabs(m + log(acc));
    }
    s[i] = out;
}

constexpr int PRE_SORT = 1024;  // >= kMaxD

__global__ void __launch_bounds__(PRE_SORT) k_pre_classify(int d, const double *s, const double *half,
                                                          double eps_flat, double eps_soft, int8_t *cls,
                                                          double *log_int, double *log_vol, int32_t *n_active) {
    __shared__ double v[PRE_SORT];
    __shared__ double term_i[PRE_SORT], term_v[PRE_SORT];
    __shared__ int s_nf;
    const int t = threadIdx.x;
    const double st = t < d ? s[t] : INFINITY;
    v[t] = isfinite(st) ? st : INFINITY;
    if (t == 0) s_nf = 0;
    __syncthreads();
    if (t < d && isfinite(st)) atomicAdd(&s_nf, 1);
    // bitonic sort, ascending (non-finite and padding as +inf at the end)
    for (int size = 2; size <= PRE_SORT; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            __syncthreads();
            const int p = t ^ stride;
            if (p > t) {
                const bool up = (t & size) == 0;
                const double a = v[t], b = v[p];
                if ((a > b) == up) {
                    v[t] = b;
                    v[p] = a;
                }
            }
        }
    }
    __syncthreads();
    const int nf = s_nf;
    double med = 0.0, smax = 0.0;
    if (nf > 0) {
        med = (nf & 1) ? v[nf / 2] : 0.5 * (v[nf / 2 - 1] + v[nf / 2]);
        smax = v[nf - 1];
    }
    term_i[t] = 0.0;
    term_v[t] = 0.0;
    if (t < d) {
        int8_t cl = 0;
        if (isfinite(st)) {
            if (st < eps_flat * med)
                cl = 1;
            else if (st < eps_soft * smax)
                cl = 2;
        }
        cls[t] = cl;
        if (cl != 0) {
            const double w = log(2.0 * half[t]);
            term_v[t] = w;
            term_i[t] = cl == 1 ? w : 0.5 * SB_LOG_2PI + log(half[t] / sqrt(st));
        }
    }
    __syncthreads();
    if (t == 0) {
        double li = 0.0, lv = 0.0;
        int na = 0;
        for (int i = 0; i < d; ++i) {
            li += term_i[i];
            lv += term_v[i];
            na += cls[i] == 0;
        }
        *log_int = li;
        *log_vol = lv;
        *n_active = na;
    }
}

}  // namespace

size_t precheck_scratch_elems(int d, int K) {
    const int nch = (d + PRE_RC - 1) / PRE_RC;
    return (size_t)K * nch * d + 3 * (size_t)K * d + (size_t)K;
}

void launch_precheck(const ProbView &pv, double eps_flat, double eps_soft, double *scratch, double *s, int8_t *cls,
                     double *log_int, double *log_vol, int32_t *n_active, cudaStream_t st) {
    const int d = pv.d, K = pv.K;
    const int nch = (d + PRE_RC - 1) / PRE_RC;
    double *part = scratch;
    double *z0 = part + (size_t)K * nch * d;
    double *dot = z0 + (size_t)K * d;
    double *nrm = dot + (size_t)K * d;
    double *e0 = nrm + (size_t)K * d;
    note_launch();
    k_pre_z0_part<<<dim3(nch, K), 256, 0, st>>>(d, pv.L, pv.mu, pv.c, part);
    note_launch();
    k_pre_z0_fin<<<K, 256, 0, st>>>(d, nch, part, pv.a, z0, e0);
    note_launch();
    k_pre_rows<<<dim3((d + 7) / 8, K), 256, 0, st>>>(d, pv.L, z0, dot, nrm);
    note_launch();
    k_pre_sens<<<(d + 255) / 256, 256, 0, st>>>(d, K, e0, dot, nrm, pv.half, s);
    note_launch();
    k_pre_classify<<<1, PRE_SORT, 0, st>>>(d, s, pv.half, eps_flat, eps_soft, cls, log_int, log_vol, n_active);
}

}  // namespace sb
