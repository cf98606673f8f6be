// chisao.cu -- kernels of the ChiSao oscillation (Sec. 3.5.5, Algorithm 1)
// around the batched refinement: the stick test, the ordered sample lists,
// the reseeding rays of Repulse Monkey (from unconverged samples, random
// directions) and Golden Rooster (from the peaks, orthonormal directions),
// the best sample along each ray, and the momentum anti-convergence step.
//
// The refinement, the likelihood evaluations and the L-infinity dedup are the
// hot path's own kernels; the host loop in sb_capi.cu chains them. Everything
// here is FP64 with explicitly rounded products and sums where an update
// formula is applied, and the random directions come from Philox4x32-10 with
// the seed as key (counters (pair, l, oscillation, 'RPMK') for Repulse Monkey,
// (pair, group G + column, oscillation << 16 | peak, 'GRST') for Golden
// Rooster, in orthonormal groups of G = min(d, 64) directions), two uniforms
// per block, two normals by Box-Muller.
#include <mutex>

#include "sb_chisao.cuh"

namespace sb {

namespace {

constexpr double kLogTenth = -2.302585092994045684;  // log 0.1, rounded to double
constexpr uint32_t kTagRm = 0x52504D4Bu;             // 'RPMK'
constexpr uint32_t kTagGr = 0x47525354u;             // 'GRST'

// Device-side oscillation state (int32 slots of the workspace).
constexpr int kCsGrOn = 0, kCsGrUsed = 1, kCsPeaksPrev = 2, kCsBranch = 3, kCsJobs = 4;
constexpr int kBranchNone = 0, kBranchRm = 1, kBranchGr = 2;

// Golden Rooster directions come in orthonormal groups of min(d, 64).
__host__ __device__ __forceinline__ int cs_group(int d) { return d < 64 ? d : 64; }

__device__ __forceinline__ double clamp_box(double x, double lo, double hi) {
    return x < lo ? lo : (x > hi ? hi : x);
}

// Two standard normals from one Philox block (Box-Muller on 52-bit uniforms).
__device__ __forceinline__ void normal_pair(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                            uint32_t k1, double &z0, double &z1) {
    uint32_t c[4] = {c0, c1, c2, c3};
    philox4x32_10(c, k0, k1);
    const double u1 = unit_from_words(c[0], c[1]);
    const double u2 = unit_from_words(c[2], c[3]);
    const double rad = sqrt(mul_rn(-2.0, log(u1)));
    const double th = mul_rn(SB_TWO_PI, u2);
    z0 = mul_rn(rad, cos(th));
    z1 = mul_rn(rad, sin(th));
}

// The same two normals in FP32 for the mixed path (the same Philox block; uniforms from
// the top 24 bits of each 64-bit pair, FP32 transcendentals, as its sunburst directions).
__device__ __forceinline__ void normal_pair_f32(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                                uint32_t k1, float &z0, float &z1) {
    uint32_t c[4] = {c0, c1, c2, c3};
    philox4x32_10(c, k0, k1);
    const float u1 = ((float)(c[0] >> 8) + 0.5f) * (1.0f / 16777216.0f);
    const float u2 = ((float)(c[2] >> 8) + 0.5f) * (1.0f / 16777216.0f);
    const float rad = sqrtf(-2.0f * logf(u1));
    float sn, cs;
    sincospif(2.0f * u2, &sn, &cs);
    z0 = rad * cs;
    z1 = rad * sn;
}

// Distance from o along u to the box boundary (whole warp; 0 when u = 0): the minimum
// over u_i != 0 of (hi_i - o_i) / u_i or (lo_i - o_i) / u_i, each rounded to nearest in
// FP64. Only candidates are divided in FP64: FP32 quotients (relative error below
// 2^-21 for magnitudes in [1e-30, 1e30]) bound the smallest, and a coordinate is divided
// when its estimate lies within 2^-18 of that bound, or when its numerator and u_i are
// outside that range or of opposite signs (an origin outside the box). The FP64
// quotient is monotone in the exact one, so the result is the plain minimum.
__device__ double exit_length(int lane, int d, const double *o, const double *u, const double *lo, const double *hi) {
    auto est_of = [&](int i, double &num) -> float {  // -1: always a candidate
        const double ui = u[i];
        num = ui > 0.0 ? sub_rn(hi[i], o[i]) : sub_rn(lo[i], o[i]);
        if (num == 0.0) return 0.f;  // exact
        if ((num > 0.0) != (ui > 0.0)) return -1.f;
        return exit_estimate(fabs(ui), fabs(num));
    };
    float est = INFINITY;
    for (int i = lane; i < d; i += 32) {
        if (u[i] == 0.0) continue;
        double num;
        const float e = est_of(i, num);
        if (e >= 0.f) est = fminf(est, e);
    }
    const float thr = warp_min(est) * (1.0f + 0x1p-18f);
    double t = INFINITY;
    for (int i = lane; i < d; i += 32) {
        const double ui = u[i];
        if (!(ui > 0.0 || ui < 0.0)) continue;
        double num;
        const float e = est_of(i, num);
        if (e >= 0.f && e > thr) continue;
        t = fmin(t, div_rn(num, ui));
    }
    t = warp_min(t);
    return t < INFINITY ? t : 0.0;
}

__global__ void __launch_bounds__(256) k_cs_conv(int n, int d, const double *G, const double *ell, double eps,
                                                 uint8_t *conv) {
    const int lane = threadIdx.x & 31;
    const int s = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    if (s >= n) return;
    const double *g = G + (size_t)s * d;
    double m = 0.0;
    for (int i = lane; i < d; i += 32) m = fmax(m, fabs(g[i]));
    m = warp_max(m);
    if (lane == 0) {
        const double l = ell[s];
        conv[s] = (uint8_t)(isfinite(l) && m <= mul_rn(eps, add_rn(1.0, fabs(l))));
    }
}

__global__ void __launch_bounds__(256) k_cs_conv_status(int n, const int8_t *status, const double *ell,
                                                        uint8_t *conv) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int st = status[s];
    conv[s] = (uint8_t)(isfinite(ell[s]) && (st == SB_WALKER_CONVERGED || st == SB_WALKER_STALLED));
}

constexpr int CS_CTA = 1024;  // single-CTA list kernels

__global__ void __launch_bounds__(CS_CTA) k_cs_stick(int n, const double *ell, const uint8_t *conv,
                                                    uint8_t *stuck) {
    __shared__ double s_m[CS_CTA / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    double m = -INFINITY;
    for (int s = threadIdx.x; s < n; s += CS_CTA) {
        const double l = ell[s];
        if (isfinite(l)) m = fmax(m, l);
    }
    m = warp_max(m);
    if (lane == 0) s_m[wid] = m;
    __syncthreads();
    if (wid == 0) {
        double v = s_m[lane];
        v = warp_max(v);
        if (lane == 0) s_m[0] = v;
    }
    __syncthreads();
    const double thr = add_rn(s_m[0], kLogTenth);
    for (int s = threadIdx.x; s < n; s += CS_CTA) stuck[s] = (uint8_t)(conv[s] && ell[s] >= thr);
}

__global__ void __launch_bounds__(CS_CTA) k_cs_split(int n, const int32_t *reps, const int32_t *n_reps,
                                                    uint8_t *stuck, uint8_t *lost) {
    for (int s = threadIdx.x; s < n; s += CS_CTA) lost[s] = stuck[s];
    __syncthreads();
    const int nr = *n_reps;
    for (int r = threadIdx.x; r < nr && r < n; r += CS_CTA) lost[reps[r]] = 0;
    __syncthreads();
    for (int s = threadIdx.x; s < n; s += CS_CTA) stuck[s] = (uint8_t)(stuck[s] && !lost[s]);
}

__global__ void __launch_bounds__(CS_CTA) k_cs_lists(int n, const uint8_t *lost, const uint8_t *conv,
                                                    const uint8_t *stuck, const int8_t *status, const double *ell,
                                                    int32_t *lost_list, int32_t *unconv_list, int32_t *moving_list,
                                                    int32_t *cnt) {
    __shared__ int s_w[3][CS_CTA / 32];
    __shared__ int s_base[3];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x < 3) s_base[threadIdx.x] = 0;
    __syncthreads();
    const unsigned below = (1u << lane) - 1u;
    for (int b0 = 0; b0 < n; b0 += CS_CTA) {
        const int s = b0 + threadIdx.x;
        bool p0 = false, p1 = false, p2 = false;
        if (s < n) {
            p0 = lost[s] != 0;
            p1 = !conv[s] && isfinite(ell[s]);
            p2 = !stuck[s] && status[s] != SB_WALKER_NONFINITE;
        }
        const unsigned m0 = __ballot_sync(0xffffffffu, p0);
        const unsigned m1 = __ballot_sync(0xffffffffu, p1);
        const unsigned m2 = __ballot_sync(0xffffffffu, p2);
        if (lane == 0) {
            s_w[0][wid] = __popc(m0);
            s_w[1][wid] = __popc(m1);
            s_w[2][wid] = __popc(m2);
        }
        __syncthreads();
        int o0 = s_base[0], o1 = s_base[1], o2 = s_base[2];
        for (int w = 0; w < wid; ++w) {
            o0 += s_w[0][w];
            o1 += s_w[1][w];
            o2 += s_w[2][w];
        }
        if (p0) lost_list[o0 + __popc(m0 & below)] = s;
        if (p1) unconv_list[o1 + __popc(m1 & below)] = s;
        if (p2) moving_list[o2 + __popc(m2 & below)] = s;
        __syncthreads();
        if (threadIdx.x < 3) {
            int t = 0;
            for (int w = 0; w < CS_CTA / 32; ++w) t += s_w[threadIdx.x][w];
            s_base[threadIdx.x] += t;
        }
        __syncthreads();
    }
    if (threadIdx.x < 3) cnt[threadIdx.x] = s_base[threadIdx.x];
}

__global__ void __launch_bounds__(256) k_cs_rm_rays(int d, uint32_t k0, uint32_t k1, int osc,
                                                    const int32_t *unconv_list, const int32_t *cnt,
                                                    const int32_t *state, const double *X, const double *lo,
                                                    const double *hi, double *O, double *U, double *texit) {
    const int lane = threadIdx.x & 31;
    const int l = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    if (state[kCsBranch] != kBranchRm || l >= cnt[0]) return;
    const int n_unconv = cnt[1];
    const double *src = X + (size_t)unconv_list[l % n_unconv] * d;
    double *o = O + (size_t)l * d;
    double *u = U + (size_t)l * d;
    for (int i = lane; i < d; i += 32) o[i] = clamp_box(src[i], lo[i], hi[i]);
    double ss = 0.0;
    for (int q = lane; q < (d + 1) / 2; q += 32) {
        double z0, z1;
        normal_pair((uint32_t)q, (uint32_t)l, (uint32_t)osc, kTagRm, k0, k1, z0, z1);
        u[2 * q] = z0;
        ss += z0 * z0;
        if (2 * q + 1 < d) {
            u[2 * q + 1] = z1;
            ss += z1 * z1;
        }
    }
    const double nrm = sqrt(warp_sum(ss));
    __syncwarp();
    for (int i = lane; i < d; i += 32) u[i] = div_rn(u[i], nrm);
    __syncwarp();
    const double t = exit_length(lane, d, o, u, lo, hi);
    if (lane == 0) texit[l] = t;
}

constexpr int CS_BASIS = 256;
// Golden Rooster groups as the Q of a Cholesky QR, twice (CholeskyQR2): the Gram
// matrix of the columns over row tiles, its Cholesky factor L (R = L^T), R^-1 by
// back substitution, then A <- A R^-1; the second pass restores orthogonality to
// working precision (Gaussian columns are well conditioned: cond ~ (sqrt d + sqrt G) /
// (sqrt d - sqrt G)). The Q of a QR with positive diag(R) is unique, so this is the
// Q Gram-Schmidt gives, up to rounding.
constexpr int CS_QR_MAXC = 64;                                          // columns of a group (cs_group)
constexpr int CS_QR_TILE = 64;                                          // rows per tile
constexpr int CS_QR_LD = CS_QR_MAXC + 1;                                // row stride of the shared arrays
constexpr int CS_QR_PER_T = (CS_QR_MAXC * (CS_QR_MAXC + 1) / 2 + CS_BASIS - 1) / CS_BASIS;  // Gram entries a thread
template <typename T>
constexpr size_t cs_qr_smem() {
    return sizeof(T) * (size_t)(CS_QR_TILE + 2 * CS_QR_MAXC) * CS_QR_LD;
}

// One orthonormal group per CTA: the Q factor of the Philox normals (CholeskyQR2, as
// above), in arithmetic T: FP64 on the FP64 path; FP32 (normals included) on the mixed
// path, whose rays are formed in FP32 anyway and on whose GB300 FP64 units the d G^2 QR
// would be the slowest step of a reseeding. Q stays FP64 in memory.
template <typename T>
__global__ void __launch_bounds__(CS_BASIS) k_cs_bases(int d, uint32_t k0, uint32_t k1, int osc, const int32_t *job_pk,
                                                       const int32_t *job_b, const int32_t *job_cols,
                                                       const int64_t *job_off, const int32_t *state, double *Q) {
    // [CS_QR_TILE][CS_QR_LD] rows of the job's columns, the Gram matrix / its Cholesky
    // factor, and the inverse of R = L^T, each CS_QR_LD wide
    extern __shared__ __align__(16) unsigned char cs_qr_smem[];
    T *tile = reinterpret_cast<T *>(cs_qr_smem);
    T *Lm = tile + CS_QR_TILE * CS_QR_LD;
    T *Ri = Lm + CS_QR_MAXC * CS_QR_LD;
    const int j = blockIdx.x;
    if (state[kCsBranch] != kBranchGr || j >= state[kCsJobs]) return;
    const int pk = job_pk[j], b = job_b[j], n = job_cols[j];
    double *Qj = Q + job_off[j];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int npairs = (d + 1) / 2;
    const int G = cs_group(d);
    for (int idx = threadIdx.x; idx < n * npairs; idx += CS_BASIS) {
        const int c = idx / npairs, q = idx - c * npairs;
        T z0, z1;
        if (sizeof(T) == sizeof(double)) {
            double a0, a1;
            normal_pair((uint32_t)q, (uint32_t)(b * G + c), ((uint32_t)osc << 16) | (uint32_t)pk, kTagGr, k0, k1, a0,
                        a1);
            z0 = (T)a0;
            z1 = (T)a1;
        } else {
            float a0, a1;
            normal_pair_f32((uint32_t)q, (uint32_t)(b * G + c), ((uint32_t)osc << 16) | (uint32_t)pk, kTagGr, k0, k1,
                            a0, a1);
            z0 = (T)a0;
            z1 = (T)a1;
        }
        Qj[(size_t)c * d + 2 * q] = (double)z0;
        if (2 * q + 1 < d) Qj[(size_t)c * d + 2 * q + 1] = (double)z1;
    }
    __syncthreads();
    const int ne = n * (n + 1) / 2;  // Gram entries (k <= l)
    // thread t owns entries t, t + CS_BASIS, ... of the upper triangle (row-major
    // order): entry (ek, el), or ek = -1
    int ek[CS_QR_PER_T], el[CS_QR_PER_T];
#pragma unroll
    for (int q = 0; q < CS_QR_PER_T; ++q) {
        const int e = threadIdx.x + q * CS_BASIS;
        int k = 0, rem = e;  // row k of the upper triangle holds n - k entries
        while (k < n && rem >= n - k) {
            rem -= n - k;
            ++k;
        }
        ek[q] = e < ne ? k : -1;
        el[q] = k + rem;
    }
    for (int pass = 0; pass < 2; ++pass) {
        // Gram matrix A^T A over tiles of CS_QR_TILE rows
        T acc[CS_QR_PER_T];
#pragma unroll
        for (int q = 0; q < CS_QR_PER_T; ++q) acc[q] = 0;
        for (int i0 = 0; i0 < d; i0 += CS_QR_TILE) {
            const int rows = d - i0 < CS_QR_TILE ? d - i0 : CS_QR_TILE;
            for (int e = threadIdx.x; e < CS_QR_TILE * n; e += CS_BASIS) {
                const int c = e / CS_QR_TILE, r = e - c * CS_QR_TILE;
                tile[r * CS_QR_LD + c] = r < rows ? (T)Qj[(size_t)c * d + i0 + r] : (T)0;
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < CS_QR_PER_T; ++q) {
                if (ek[q] >= 0) {
                    const int k = ek[q], l = el[q];
                    T s = 0;
                    for (int r = 0; r < rows; ++r) s += tile[r * CS_QR_LD + k] * tile[r * CS_QR_LD + l];
                    acc[q] += s;
                }
            }
            __syncthreads();
        }
#pragma unroll
        for (int q = 0; q < CS_QR_PER_T; ++q)
            if (ek[q] >= 0) Lm[el[q] * CS_QR_LD + ek[q]] = acc[q];  // lower triangle: Lm[l][k] = (A^T A)_kl
        __syncthreads();
        // Cholesky A^T A = L L^T (one warp, column by column; rows i = lane, lane + 32)
        if (wid == 0) {
            for (int c = 0; c < n; ++c) {
                T s = 0;
                for (int p = lane; p < c; p += 32) s += Lm[c * CS_QR_LD + p] * Lm[c * CS_QR_LD + p];
                s = warp_sum(s);
                const T dcc = sqrt(Lm[c * CS_QR_LD + c] - s);
                for (int i = c + 1 + lane; i < n; i += 32) {
                    T t = Lm[i * CS_QR_LD + c];
                    for (int p = 0; p < c; ++p) t -= Lm[i * CS_QR_LD + p] * Lm[c * CS_QR_LD + p];
                    Lm[i * CS_QR_LD + c] = div_rn(t, dcc);
                }
                __syncwarp();
                if (lane == 0) Lm[c * CS_QR_LD + c] = dcc;
                __syncwarp();
            }
        }
        __syncthreads();
        // Ri = R^-1 for R = L^T (upper): column c by back substitution, one thread each
        for (int c = threadIdx.x; c < n; c += CS_BASIS) {
            Ri[c * CS_QR_LD + c] = div_rn((T)1, Lm[c * CS_QR_LD + c]);
            for (int i = c - 1; i >= 0; --i) {
                T t = 0;
                for (int p = i + 1; p <= c; ++p) t += Lm[p * CS_QR_LD + i] * Ri[p * CS_QR_LD + c];  // R_ip = L_pi
                Ri[i * CS_QR_LD + c] = div_rn(-t, Lm[i * CS_QR_LD + i]);
            }
        }
        __syncthreads();
        // A <- A R^-1, tile by tile (the tile is read from HBM before it is overwritten)
        for (int i0 = 0; i0 < d; i0 += CS_QR_TILE) {
            const int rows = d - i0 < CS_QR_TILE ? d - i0 : CS_QR_TILE;
            for (int e = threadIdx.x; e < CS_QR_TILE * n; e += CS_BASIS) {
                const int c = e / CS_QR_TILE, r = e - c * CS_QR_TILE;
                tile[r * CS_QR_LD + c] = r < rows ? (T)Qj[(size_t)c * d + i0 + r] : (T)0;
            }
            __syncthreads();
            for (int e = threadIdx.x; e < CS_QR_TILE * n; e += CS_BASIS) {
                const int c = e / CS_QR_TILE, r = e - c * CS_QR_TILE;
                if (r >= rows) continue;
                T t = 0;
                for (int p = 0; p <= c; ++p) t += tile[r * CS_QR_LD + p] * Ri[p * CS_QR_LD + c];
                Qj[(size_t)c * d + i0 + r] = (double)t;
            }
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(256) k_cs_gr_rays(int d, const int32_t *n_peaks_dev, const int32_t *reps,
                                                    const double *X, const double *lo, const double *hi,
                                                    const int32_t *job_start, const int64_t *job_off, const double *Q,
                                                    const int32_t *cnt, const int32_t *state, double *O, double *U,
                                                    double *texit) {
    const int lane = threadIdx.x & 31;
    const int l = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    if (state[kCsBranch] != kBranchGr || l >= cnt[0]) return;
    const int n_peaks = *n_peaks_dev;
    const int pk = l % n_peaks, k = l / n_peaks, cdir = k >> 1;
    const int G = cs_group(d);
    const int b = cdir / G, col = cdir - b * G;
    const double sgn = (k & 1) ? -1.0 : 1.0;
    const double *q = Q + job_off[job_start[pk] + b] + (size_t)col * d;
    const double *src = X + (size_t)reps[pk] * d;
    double *o = O + (size_t)l * d;
    double *u = U + (size_t)l * d;
    for (int i = lane; i < d; i += 32) {
        o[i] = clamp_box(src[i], lo[i], hi[i]);
        u[i] = sgn * q[i];
    }
    __syncwarp();
    const double t = exit_length(lane, d, o, u, lo, hi);
    if (lane == 0) texit[l] = t;
}

__global__ void __launch_bounds__(256) k_cs_ray_points(int l0, int n_steps, int d, const double *O,
                                                       const double *U, const double *texit, const int32_t *rows,
                                                       double *P) {
    const int64_t total = (int64_t)(*rows) * d;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = idx / d;
        const int i = (int)(idx - row * d);
        const int l = l0 + (int)(row / n_steps), j = (int)(row % n_steps);
        const double t = mul_rn(div_rn((double)(j + 1), (double)n_steps), texit[l]);
        P[idx] = add_rn(O[(size_t)l * d + i], mul_rn(t, U[(size_t)l * d + i]));
    }
}

__global__ void __launch_bounds__(256) k_cs_ray_pick(int l0, int n_steps, int d, const int32_t *rows,
                                                     const int32_t *state, const double *ellp,
                                                     const int32_t *lost_list, const double *O, const double *U,
                                                     const double *texit, double *X) {
    const int lane = threadIdx.x & 31;
    const int r = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    if (r >= *rows / n_steps) return;
    const int past_valley = state[kCsBranch] == kBranchGr;
    const int l = l0 + r;
    const double *e = ellp + (size_t)r * n_steps;
    int best = 0;
    if (lane == 0) {
        int j0 = 0;
        if (past_valley) {
            // past the first valley: the first sample after which l rises; none: the exit sample
            j0 = -1;
            for (int j = 0; j + 1 < n_steps; ++j)
                if (e[j + 1] > e[j]) {
                    j0 = j + 1;
                    break;
                }
            if (j0 < 0) j0 = n_steps - 1;
        }
        best = j0;
        for (int j = j0 + 1; j < n_steps; ++j)
            if (e[j] > e[best]) best = j;
    }
    best = __shfl_sync(0xffffffffu, best, 0);
    const double t = mul_rn(div_rn((double)(best + 1), (double)n_steps), texit[l]);
    double *x = X + (size_t)lost_list[l] * d;
    for (int i = lane; i < d; i += 32) x[i] = add_rn(O[(size_t)l * d + i], mul_rn(t, U[(size_t)l * d + i]));
}

__global__ void __launch_bounds__(256) k_cs_momentum(int n, int d, const int32_t *moving_list,
                                                     const int32_t *n_moving, double m, double alpha,
                                                     const double *G, double *V, double *X, const double *lo,
                                                     const double *hi) {
    const int lane = threadIdx.x & 31;
    const int e = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    if (e >= n || e >= *n_moving) return;
    const size_t base = (size_t)moving_list[e] * d;
    for (int i = lane; i < d; i += 32) {
        const double v = sub_rn(mul_rn(m, V[base + i]), mul_rn(alpha, G[base + i]));
        V[base + i] = v;
        X[base + i] = clamp_box(add_rn(X[base + i], v), lo[i], hi[i]);
    }
}

__global__ void k_cs_stat_add(int64_t *dst, const int64_t *src, int64_t v) {
    if (threadIdx.x == 0) *dst += (src ? *src : 0) + v;
}

__global__ void k_cs_stat_add32(int64_t *dst, const int32_t *src, int64_t mult) {
    if (threadIdx.x == 0) *dst += (int64_t)(*src) * mult;
}

__global__ void k_cs_state_init(int32_t *state) {
    if (threadIdx.x == 0) {
        state[kCsGrOn] = 1;
        state[kCsGrUsed] = 0;
        state[kCsPeaksPrev] = -1;
        state[kCsBranch] = kBranchNone;
        state[kCsJobs] = 0;
    }
}

// After the stick test and its dedup: Golden Rooster stays off for good once an
// oscillation that used it ends with no more peaks than the one before.
__global__ void k_cs_osc_state(const int32_t *n_peaks, int32_t *state) {
    if (threadIdx.x != 0) return;
    const int peaks = *n_peaks;
    if (state[kCsGrUsed] && peaks <= state[kCsPeaksPrev]) state[kCsGrOn] = 0;
    state[kCsGrUsed] = 0;
    state[kCsPeaksPrev] = peaks;
}

// The reseeding branch from the sample lists (cnt: lost, unconverged, moving): Repulse
// Monkey with enough unconverged samples, else Golden Rooster while it is on and there
// are peaks, else none. For Golden Rooster, the groups of orthonormal directions: lost
// sample l uses direction c = (l / n_peaks) / 2 of peak l mod n_peaks, column c mod G of
// group c / G (G = min(d, 64)); every group a peak needs is one job, its columns only as
// far as used. The ray samples the branch evaluates go to stats[0].
__global__ void k_cs_branch(const int32_t *cnt, const int32_t *n_peaks_dev, int min_unconv, int d, int n_steps,
                            int32_t *state, int32_t *job_start, int32_t *job_pk, int32_t *job_b, int32_t *job_cols,
                            int64_t *job_off, int64_t *stats) {
    if (threadIdx.x != 0) return;
    const int n_lost = cnt[0], n_unconv = cnt[1], n_peaks = *n_peaks_dev;
    int br = kBranchNone;
    if (n_lost > 0 && n_unconv >= min_unconv)
        br = kBranchRm;
    else if (n_lost > 0 && state[kCsGrOn] && n_peaks > 0)
        br = kBranchGr;
    state[kCsBranch] = br;
    if (br != kBranchNone) stats[0] += (int64_t)n_lost * n_steps;
    if (br != kBranchGr) return;
    state[kCsGrUsed] = 1;
    const int G = cs_group(d);
    int nj = 0;
    int64_t off = 0;
    for (int p = 0; p < n_peaks; ++p) {
        job_start[p] = nj;
        const int count = n_lost > p ? (n_lost - p + n_peaks - 1) / n_peaks : 0;
        if (count == 0) continue;
        const int cmax = (count - 1) / 2;
        for (int b = 0; b <= cmax / G; ++b) {
            const int cols = b < cmax / G ? G : cmax - b * G + 1;
            job_pk[nj] = p;
            job_b[nj] = b;
            job_cols[nj] = cols;
            job_off[nj] = off;
            off += (int64_t)cols * d;
            ++nj;
        }
    }
    job_start[n_peaks] = nj;
    state[kCsJobs] = nj;
}

// Rows (ray samples) of the reseeding chunk of lost samples l0 .. l0 + lc - 1.
__global__ void k_cs_chunk_rows(const int32_t *cnt, const int32_t *state, int l0, int lc, int n_steps,
                                int32_t *rows) {
    if (threadIdx.x != 0) return;
    int nl = state[kCsBranch] != kBranchNone ? cnt[0] - l0 : 0;
    nl = nl < 0 ? 0 : (nl > lc ? lc : nl);
    *rows = nl * n_steps;
}

// The momentum step of the mixed path in FP32 (warp per moving sample): GT holds
// grad f = -grad l of the tensor-core evaluation, so v <- m v + alpha GT,
// x <- clamp(x + v); dist[s] bounds the distance the sample moved (the next
// evaluation's component skip reads it; clamping only shortens the move).
__global__ void __launch_bounds__(256) k_cs_momentum_f32(int n, int d, const int32_t *moving_list,
                                                         const int32_t *n_moving, float m, float alpha,
                                                         const float *GT, float *V, float *X, const double *lo,
                                                         const double *hi, float *dist) {
    const int lane = threadIdx.x & 31;
    const int e = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    if (e >= n || e >= *n_moving) return;
    const int smp = moving_list[e];
    const size_t base = (size_t)smp * d;
    float mv = 0.f;
    auto step = [&](float vo, float g, float x0, double l, double h, float &vn, float &x1) {
        vn = fmaf(m, vo, alpha * g);
        x1 = fminf(fmaxf(x0 + vn, (float)l), (float)h);
        const float dx = x1 - x0;
        mv = fmaf(dx, dx, mv);
    };
    // 16-byte accesses: rows start at multiples of d floats; lo and hi (the caller's
    // arrays) only when they are 16-byte aligned
    if ((d & 3) == 0 && ((reinterpret_cast<uintptr_t>(lo) | reinterpret_cast<uintptr_t>(hi)) & 15) == 0) {
        const float4 *G4 = reinterpret_cast<const float4 *>(GT + base);
        float4 *V4 = reinterpret_cast<float4 *>(V + base);
        float4 *X4 = reinterpret_cast<float4 *>(X + base);
        for (int q = lane; q < d / 4; q += 32) {
            const float4 g = G4[q], vo = V4[q], x0 = X4[q];
            const double2 l01 = reinterpret_cast<const double2 *>(lo)[2 * q];
            const double2 l23 = reinterpret_cast<const double2 *>(lo)[2 * q + 1];
            const double2 h01 = reinterpret_cast<const double2 *>(hi)[2 * q];
            const double2 h23 = reinterpret_cast<const double2 *>(hi)[2 * q + 1];
            float4 vn, x1;
            step(vo.x, g.x, x0.x, l01.x, h01.x, vn.x, x1.x);
            step(vo.y, g.y, x0.y, l01.y, h01.y, vn.y, x1.y);
            step(vo.z, g.z, x0.z, l23.x, h23.x, vn.z, x1.z);
            step(vo.w, g.w, x0.w, l23.y, h23.y, vn.w, x1.w);
            V4[q] = vn;
            X4[q] = x1;
        }
    } else {
        for (int i = lane; i < d; i += 32) {
            float vn, x1;
            step(V[base + i], GT[base + i], X[base + i], lo[i], hi[i], vn, x1);
            V[base + i] = vn;
            X[base + i] = x1;
        }
    }
    mv = warp_sum(mv);
    if (lane == 0) dist[smp] = __fsqrt_ru(mv) * 1.0001f;
}

// X[s] = (double) X32[s] for the moving samples (the others keep their FP64 positions).
__global__ void __launch_bounds__(256) k_cs_scatter_moving(int n, int d, const int32_t *moving_list,
                                                           const int32_t *n_moving, const float *X32, double *X) {
    const int lane = threadIdx.x & 31;
    const int e = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    if (e >= n || e >= *n_moving) return;
    const size_t base = (size_t)moving_list[e] * d;
    for (int i = lane; i < d; i += 32) X[base + i] = (double)X32[base + i];
}

inline unsigned warp_grid(int64_t warps) { return (unsigned)((warps * 32 + 255) / 256); }

}  // namespace

void launch_cs_stat_add(int64_t *dst, const int64_t *src, int64_t v, cudaStream_t s) {
    note_launch();
    k_cs_stat_add<<<1, 32, 0, s>>>(dst, src, v);
}

void launch_cs_conv(int n, int d, const double *G, const double *ell, double eps, uint8_t *conv, cudaStream_t s) {
    if (n <= 0) return;
    note_launch();
    k_cs_conv<<<warp_grid(n), 256, 0, s>>>(n, d, G, ell, eps, conv);
}

void launch_cs_conv_status(int n, const int8_t *status, const double *ell, uint8_t *conv, cudaStream_t s) {
    if (n <= 0) return;
    note_launch();
    k_cs_conv_status<<<(n + 255) / 256, 256, 0, s>>>(n, status, ell, conv);
}

void launch_cs_stick(int n, const double *ell, const uint8_t *conv, uint8_t *stuck, cudaStream_t s) {
    note_launch();
    k_cs_stick<<<1, CS_CTA, 0, s>>>(n, ell, conv, stuck);
}

void launch_cs_split(int n, const int32_t *reps, const int32_t *n_reps, uint8_t *stuck, uint8_t *lost,
                     cudaStream_t s) {
    note_launch();
    k_cs_split<<<1, CS_CTA, 0, s>>>(n, reps, n_reps, stuck, lost);
}

void launch_cs_lists(int n, const uint8_t *lost, const uint8_t *conv, const uint8_t *stuck, const int8_t *status,
                     const double *ell, int32_t *lost_list, int32_t *unconv_list, int32_t *moving_list, int32_t *cnt,
                     cudaStream_t s) {
    note_launch();
    k_cs_lists<<<1, CS_CTA, 0, s>>>(n, lost, conv, stuck, status, ell, lost_list, unconv_list, moving_list, cnt);
}

__global__ void __launch_bounds__(256) k_cs_exit(int n, int d, const double *O, const double *U, const double *lo,
                                                 const double *hi, double *texit) {
    const int lane = threadIdx.x & 31;
    const int l = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    if (l >= n) return;
    const double t = exit_length(lane, d, O + (size_t)l * d, U + (size_t)l * d, lo, hi);
    if (lane == 0) texit[l] = t;
}

void launch_cs_exit(int n, int d, const double *O, const double *U, const double *lo, const double *hi, double *texit,
                    cudaStream_t s) {
    if (n <= 0) return;
    note_launch();
    k_cs_exit<<<warp_grid(n), 256, 0, s>>>(n, d, O, U, lo, hi, texit);
}

void launch_cs_rm_rays(int n, int d, uint64_t seed, int osc, const int32_t *unconv_list, const int32_t *cnt,
                       const int32_t *state, const double *X, const double *lo, const double *hi, double *O, double *U,
                       double *texit, cudaStream_t s) {
    if (n <= 0) return;
    note_launch();
    k_cs_rm_rays<<<warp_grid(n), 256, 0, s>>>(d, (uint32_t)seed, (uint32_t)(seed >> 32), osc, unconv_list, cnt, state,
                                              X, lo, hi, O, U, texit);
}

void launch_cs_bases(int max_jobs, int d, uint64_t seed, int osc, const int32_t *job_pk, const int32_t *job_b,
                     const int32_t *job_cols, const int64_t *job_off, const int32_t *state, double *Q, bool fp32,
                     cudaStream_t s) {
    if (max_jobs <= 0) return;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(k_cs_bases<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cs_qr_smem<float>());
        cudaFuncSetAttribute(k_cs_bases<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cs_qr_smem<double>());
    });
    note_launch();
    if (fp32)
        k_cs_bases<float><<<max_jobs, CS_BASIS, cs_qr_smem<float>(), s>>>(
            d, (uint32_t)seed, (uint32_t)(seed >> 32), osc, job_pk, job_b, job_cols, job_off, state, Q);
    else
        k_cs_bases<double><<<max_jobs, CS_BASIS, cs_qr_smem<double>(), s>>>(
            d, (uint32_t)seed, (uint32_t)(seed >> 32), osc, job_pk, job_b, job_cols, job_off, state, Q);
}

void launch_cs_gr_rays(int n, int d, const int32_t *n_peaks, const int32_t *reps, const double *X, const double *lo,
                       const double *hi, const int32_t *job_start, const int64_t *job_off, const double *Q,
                       const int32_t *cnt, const int32_t *state, double *O, double *U, double *texit,
                       cudaStream_t s) {
    if (n <= 0) return;
    note_launch();
    k_cs_gr_rays<<<warp_grid(n), 256, 0, s>>>(d, n_peaks, reps, X, lo, hi, job_start, job_off, Q, cnt, state, O, U,
                                              texit);
}

void launch_cs_ray_points(int l0, int lc, int n_steps, int d, const double *O, const double *U, const double *texit,
                          const int32_t *rows, double *P, cudaStream_t s) {
    if (lc <= 0) return;
    const int64_t total = (int64_t)lc * n_steps * d;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    note_launch();
    k_cs_ray_points<<<(unsigned)blocks, 256, 0, s>>>(l0, n_steps, d, O, U, texit, rows, P);
}

void launch_cs_ray_pick(int l0, int lc, int n_steps, int d, const int32_t *rows, const int32_t *state,
                        const double *ellp, const int32_t *lost_list, const double *O, const double *U,
                        const double *texit, double *X, cudaStream_t s) {
    if (lc <= 0) return;
    note_launch();
    k_cs_ray_pick<<<warp_grid(lc), 256, 0, s>>>(l0, n_steps, d, rows, state, ellp, lost_list, O, U, texit, X);
}

void launch_cs_momentum_f32(int n, int d, const int32_t *moving_list, const int32_t *n_moving, double momentum,
                            double alpha, const float *GT, float *V, float *X, const double *lo, const double *hi,
                            float *dist, cudaStream_t s) {
    if (n <= 0) return;
    note_launch();
    k_cs_momentum_f32<<<warp_grid(n), 256, 0, s>>>(n, d, moving_list, n_moving, (float)momentum, (float)alpha, GT, V,
                                                   X, lo, hi, dist);
}

void launch_cs_scatter_moving(int n, int d, const int32_t *moving_list, const int32_t *n_moving, const float *X32,
                              double *X, cudaStream_t s) {
    if (n <= 0) return;
    note_launch();
    k_cs_scatter_moving<<<warp_grid(n), 256, 0, s>>>(n, d, moving_list, n_moving, X32, X);
}

void launch_cs_state_init(int32_t *state, cudaStream_t s) {
    note_launch();
    k_cs_state_init<<<1, 32, 0, s>>>(state);
}

void launch_cs_osc_state(const int32_t *n_peaks, int32_t *state, cudaStream_t s) {
    note_launch();
    k_cs_osc_state<<<1, 32, 0, s>>>(n_peaks, state);
}

void launch_cs_branch(const int32_t *cnt, const int32_t *n_peaks, int min_unconv, int d, int n_steps, int32_t *state,
                      int32_t *job_start, int32_t *job_pk, int32_t *job_b, int32_t *job_cols, int64_t *job_off,
                      int64_t *stats, cudaStream_t s) {
    note_launch();
    k_cs_branch<<<1, 32, 0, s>>>(cnt, n_peaks, min_unconv, d, n_steps, state, job_start, job_pk, job_b, job_cols,
                                 job_off, stats);
}

void launch_cs_chunk_rows(const int32_t *cnt, const int32_t *state, int l0, int lc, int n_steps, int32_t *rows,
                          cudaStream_t s) {
    note_launch();
    k_cs_chunk_rows<<<1, 32, 0, s>>>(cnt, state, l0, lc, n_steps, rows);
}

void launch_cs_stat_add32(int64_t *dst, const int32_t *src, int64_t mult, cudaStream_t s) {
    note_launch();
    k_cs_stat_add32<<<1, 32, 0, s>>>(dst, src, mult);
}

void launch_cs_momentum(int n, int d, const int32_t *moving_list, const int32_t *n_moving, double momentum,
                        double alpha, const double *G, double *V, double *X, const double *lo, const double *hi,
                        cudaStream_t s) {
    if (n <= 0) return;
    note_launch();
    k_cs_momentum<<<warp_grid(n), 256, 0, s>>>(n, d, moving_list, n_moving, momentum, alpha, G, V, X, lo, hi);
}

}  // namespace sb
