// laplace.cu -- FP64 Laplace stage: dedup, Newton polish, filters, log Z.
//
//  * coarse / final deduplication: greedy L-infinity merging in order of
//    decreasing l, ties to the lower index (Sec. 3.5.4, App. A.7); one CTA,
//    each round an argmax over the unassigned points and an early-exit
//    L-infinity test of every unassigned point against the new representative;
//  * Hessian H = -hess l = sum_k r_k P_k - sum_k r_k g_k g_k^T + gbar gbar^T,
//    with P_k = L_k L_k^T precomputed once and g_k = -L_k z_k (the analytic
//    form of the finite-difference Hessian of Sec. 3.7.2 / App. A.4.3);
//    components with r_k == 0 contribute exactly nothing and are skipped;
//  * batched blocked Cholesky H = C C^T (right-looking, 32x32 blocks:
//    diagonal factor, panel triangular solve, trailing update), which also
//    serves as the positive-definiteness (saddle) filter of Sec. 3.6.4;
//  * Newton polish x <- x + t H^{-1} grad l: t = 1 at once when the model
//    increase g^T delta / 2 <= 1e-10 (1 + |l|) (there the descent test is
//    rounding noise), otherwise t halved until l does not drop;
//  * log Z_k = l(x*) + (d/2) log 2pi - sum_i log C_ii (Sec. 3.7.1 with the
//    whitening identity of App. A.8) and log Z = LSE_k log Z_k - log V
//    (Sec. 3.7.3, App. A.10, Sec. 3.2).
#include <vector>

#include "sb_graph.cuh"
#include "sb_laplace.cuh"

namespace sb {

namespace {

constexpr int NB = 32;  // Cholesky block

// ------------------------------------------------------------------ dedup
// Greedy rounds over a grid of co-resident CTAs (cooperative launch). CTA b
// owns points [b*per, (b+1)*per) and their `assigned` flags. Each round:
//   1. every CTA reduces its unassigned points to (max l, lowest index) and
//      publishes it in the round's partial slot (two slots, alternating);
//   2. one grid barrier;
//   3. every CTA reduces the partials itself (same order, same result), so
//      all know the representative without a second barrier; the owner marks
//      it, CTA 0 records it;
//   4. every CTA tests its unassigned points against the representative,
//      one warp per point: coalesced 32-coordinate slices, leaving at the
//      first coordinate farther than tau (a warp vote).
// A slot is rewritten two rounds later, after every CTA has passed the
// barrier of the round in between, so it is never overwritten while read.
// The barrier wait is bounded: on timeout the CTA flags SB_DEV_TIMEOUT and
// leaves; every other CTA then times out at its next barrier.
constexpr int DD_THREADS = 256;
constexpr long long kBarrierSpins = 1ll << 22;

__device__ bool grid_barrier(uint32_t *bar, uint32_t n_blocks, int32_t *err) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile uint32_t *gen = bar + 1;
        const uint32_t g = *gen;
        __threadfence();
        int ok = 1;
        if (atomicAdd(bar, 1u) == n_blocks - 1) {
            bar[0] = 0;
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            long long it = 0;
            while (*gen == g) {
                if (++it > kBarrierSpins) {
                    ok = 0;
                    atomicOr(err, SB_DEV_TIMEOUT);
                    break;
                }
                if (it > 4096) __nanosleep(128);  // spin first: most waits are a few microseconds
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// (l, index) order of the greedy: larger l first, ties to the lower index; index < 0 is "none".
__device__ __forceinline__ bool dd_better(double l, int i, double bl, int bi) {
    return i >= 0 && (bi < 0 || l > bl || (l == bl && i < bi));
}

__global__ void __launch_bounds__(DD_THREADS) k_dedup(int n, int d, const double *X, const double *ell,
                                                      const int8_t *status, const uint8_t *keep_in, double tau_scale,
                                                      const double *wmax, int cap, int32_t *reps, int32_t *n_reps,
                                                      uint8_t *assigned, double *part_l, int32_t *part_i,
                                                      uint32_t *bar, int32_t *err) {
    extern __shared__ double s_xb[];  // [d] the round's representative
    __shared__ double s_l[DD_THREADS / 32];
    __shared__ int s_i[DD_THREADS / 32];
    __shared__ int s_best;
    const int G = gridDim.x;
    const int per = (n + G - 1) / G;
    const int w0 = blockIdx.x * per, w1 = min(n, w0 + per);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const double tau = tau_scale * wmax[0];
    for (int w = w0 + threadIdx.x; w < w1; w += DD_THREADS) {
        bool el = isfinite(ell[w]);
        if (status && status[w] == SB_WALKER_NONFINITE) el = false;
        if (keep_in && !keep_in[w]) el = false;
        assigned[w] = el ? 0 : 1;
    }
    __syncthreads();
    int count = 0;
    for (int round = 0;; ++round) {
        // 1. this CTA's best unassigned point
        double bl = -INFINITY;
        int bi = -1;
        for (int w = w0 + threadIdx.x; w < w1; w += DD_THREADS) {
            if (assigned[w]) continue;
            const double l = ell[w];
            if (bi < 0 || l > bl) {  // strided ascending: the first seen has the lower index
                bl = l;
                bi = w;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double ol = __shfl_xor_sync(0xffffffffu, bl, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (dd_better(ol, oi, bl, bi)) {
                bl = ol;
                bi = oi;
            }
        }
        if (lane == 0) {
            s_l[wid] = bl;
            s_i[wid] = bi;
        }
        __syncthreads();
        const int slot = (round & 1) * G;
        if (threadIdx.x == 0) {
            double b = -INFINITY;
            int ib = -1;
            for (int q = 0; q < DD_THREADS / 32; ++q)
                if (dd_better(s_l[q], s_i[q], b, ib)) {
                    b = s_l[q];
                    ib = s_i[q];
                }
            part_l[slot + blockIdx.x] = b;
            part_i[slot + blockIdx.x] = ib;
        }
        // 2.
        if (!grid_barrier(bar, (uint32_t)G, err)) break;
        // 3. the global best from the partials (read past L1: written by other CTAs)
        bl = -INFINITY;
        bi = -1;
        for (int q = threadIdx.x; q < G; q += DD_THREADS) {
            const double l = __ldcg(part_l + slot + q);
            const int i = __ldcg(part_i + slot + q);
            if (dd_better(l, i, bl, bi)) {
                bl = l;
                bi = i;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double ol = __shfl_xor_sync(0xffffffffu, bl, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (dd_better(ol, oi, bl, bi)) {
                bl = ol;
                bi = oi;
            }
        }
        __syncthreads();  // s_l / s_i of step 1 fully consumed
        if (lane == 0) {
            s_l[wid] = bl;
            s_i[wid] = bi;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double b = -INFINITY;
            int ib = -1;
            for (int q = 0; q < DD_THREADS / 32; ++q)
                if (dd_better(s_l[q], s_i[q], b, ib)) {
                    b = s_l[q];
                    ib = s_i[q];
                }
            s_best = ib;
            if (ib >= 0) {
                if (ib >= w0 && ib < w1) assigned[ib] = 1;
                if (blockIdx.x == 0 && count < cap) reps[count] = ib;
            }
        }
        __syncthreads();
        const int best = s_best;
        if (best < 0) break;
        ++count;
        if (count >= cap) break;
        // 4. L-infinity test of this CTA's unassigned points against the representative
        const double *xb = X + (size_t)best * d;
        for (int i = threadIdx.x; i < d; i += DD_THREADS) s_xb[i] = xb[i];
        __syncthreads();
        for (int w = w0 + wid; w < w1; w += DD_THREADS / 32) {
            if (assigned[w]) continue;
            const double *xw = X + (size_t)w * d;
            bool within = true;
            for (int i0 = 0; i0 < d; i0 += 32) {
                const int i = i0 + lane;
                const bool far = i < d && fabs(xw[i] - s_xb[i]) > tau;
                if (__any_sync(0xffffffffu, far)) {
                    within = false;
                    break;
                }
            }
            if (within && lane == 0) assigned[w] = 1;
        }
        __syncthreads();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *n_reps = count < cap ? count : cap;
}

__global__ void __launch_bounds__(256) k_gather_rows(int d, const double *X, const int32_t *idx, const int32_t *n_idx,
                                                     double *out, const double *ell, double *ell_out) {
    const int c = blockIdx.x;
    if (c >= *n_idx) return;
    const int w = idx[c];
    for (int i = threadIdx.x; i < d; i += blockDim.x) out[(size_t)c * d + i] = X[(size_t)w * d + i];
    if (threadIdx.x == 0 && ell_out) ell_out[c] = ell[w];
}

// ------------------------------------------------------------------ P_k = L_k L_k^T
// 32 x 32 output tiles (lower ones, mirrored on store), 256 threads with 2 x 2
// outputs each: small tiles keep the deep tiles near the diagonal short, which
// bounds the FP64 critical path when only a few components are formed.
constexpr int PT = 32;
__global__ void __launch_bounds__(256) k_precision(int d, const double *L, double *P, const int32_t *need) {
    const int k = blockIdx.z, i0 = blockIdx.y * PT, j0 = blockIdx.x * PT;
    if (j0 > i0) return;
    if (need && !need[k]) return;
    const double *Lk = L + (size_t)k * d * d;
    __shared__ double As[16][PT + 1], Bs[16][PT + 1];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    double acc[2][2] = {};
    const int jmax = min(d, j0 + PT);  // P_ij = sum_{l <= min(i,j)} L_il L_jl
    for (int l0 = 0; l0 < jmax; l0 += 16) {
        for (int e = tid; e < 16 * PT; e += 256) {
            const int r = e >> 4, kk = e & 15, l = l0 + kk;
            const int i = i0 + r, j = j0 + r;
            As[kk][r] = (i < d && l < d && l <= i) ? Lk[(size_t)i * d + l] : 0.0;
            Bs[kk][r] = (j < d && l < d && l <= j) ? Lk[(size_t)j * d + l] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            const double a0 = As[kk][ty], a1 = As[kk][ty + 16];
            const double b0 = Bs[kk][tx], b1 = Bs[kk][tx + 16];
            acc[0][0] = fma(a0, b0, acc[0][0]);
            acc[0][1] = fma(a0, b1, acc[0][1]);
            acc[1][0] = fma(a1, b0, acc[1][0]);
            acc[1][1] = fma(a1, b1, acc[1][1]);
        }
        __syncthreads();
    }
    double *Pk = P + (size_t)k * d * d;
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int i = i0 + ty + 16 * r, j = j0 + tx + 16 * c;
            if (i < d && j < d) {
                Pk[(size_t)i * d + j] = acc[r][c];
                Pk[(size_t)j * d + i] = acc[r][c];
            }
        }
}

// Components whose P_k the Hessians are about to read: r_ck != 0 at some live
// candidate whose responsibilities are not one-hot, and P_k not formed yet (the
// Hessian skips r == 0 terms and copies L_k at one-hot candidates, so the other
// P_k are never read). Marks them formed.
__global__ void k_precision_need(int K, const double *R, const int32_t *n_c, const int32_t *onehot, int32_t *done,
                                 int32_t *need) {
    const int k = threadIdx.x;
    if (k >= K) return;
    bool any = false;
    for (int c = 0; c < *n_c; ++c) any = any || (R[(size_t)c * K + k] != 0.0 && !(onehot && onehot[c] >= 0));
    const bool nk = any && !done[k];
    need[k] = nk ? 1 : 0;
    if (nk) done[k] = 1;
}

// ------------------------------------------------------------------ per-component gradients
// GK[c][k][i] = -sum_{j<=i} L_k[i][j] z_ck[j]  (zero when r_ck == 0). Grid (candidate,
// component, row slice): the rows of one product are spread over kGradSlices CTAs.
constexpr int kGradSlices = 16;
__global__ void __launch_bounds__(256) k_comp_grads(int d, int K, const double *L, const double *Z, const double *R,
                                                    const int32_t *n_c, double *GK) {
    const int c = blockIdx.x, k = blockIdx.y;
    if (c >= *n_c) return;
    const int per = (d + kGradSlices - 1) / kGradSlices;
    const int i_lo = blockIdx.z * per, i_hi = min(d, i_lo + per);
    const double r = R[(size_t)c * K + k];
    double *g = GK + ((size_t)c * K + k) * d;
    if (r == 0.0) {
        for (int i = i_lo + threadIdx.x; i < i_hi; i += blockDim.x) g[i] = 0.0;
        return;
    }
    extern __shared__ double zs[];
    const double *z = Z + ((size_t)c * K + k) * d;
    for (int i = threadIdx.x; i < i_hi; i += blockDim.x) zs[i] = z[i];
    __syncthreads();
    const double *Lk = L + (size_t)k * d * d;
    // one warp per output row: coalesced reads of L_k rows
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int i = i_lo + wid; i < i_hi; i += nw) {
        double s = 0.0;
        for (int j = lane; j <= i; j += 32) s += Lk[(size_t)i * d + j] * zs[j];
        s = warp_sum(s);
        if (lane == 0) g[i] = -s;
    }
}

// onehot[c] = k when candidate c's FP64 responsibilities are exactly r_ck = 1 and 0 for
// every other component, else -1. There H = sum_k r_k (P_k - g_k g_k^T) + gbar gbar^T
// with gbar = g_k is exactly P_k = L_k L_k^T, whose Cholesky factor is L_k itself.
__global__ void k_onehot(int K, const double *R, const int32_t *n_c, int cap, int32_t *onehot) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cap) return;
    int k1 = -1;
    bool ok = c < *n_c;
    for (int k = 0; ok && k < K; ++k) {
        const double r = R[(size_t)c * K + k];
        if (r == 1.0 && k1 < 0)
            k1 = k;
        else if (r != 0.0)
            ok = false;
    }
    onehot[c] = ok ? k1 : -1;
}

// H[c][i][i2] = gbar_i gbar_i2 + sum_k r_k (P_k[i][i2] - g_ki g_ki2); at a one-hot
// candidate the lower triangle of its factor L_k instead (the blocked Cholesky skips it)
__global__ void __launch_bounds__(256) k_hessian(int d, int K, const double *P, const double *GK, const double *R,
                                                 const double *gbar, const int32_t *n_c, const int32_t *onehot,
                                                 const double *L, double *H, int32_t *info) {
    const int c = blockIdx.y;
    if (c >= *n_c) return;
    // a fresh factorisation of this candidate follows (candidates past the count keep
    // their factor and its success flag)
    if (blockIdx.x == 0 && threadIdx.x == 0) info[c] = 0;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)d * d) return;
    const int i = (int)(e / d), i2 = (int)(e % d);
    if (onehot && onehot[c] >= 0) {
        H[(size_t)c * d * d + e] = i2 <= i ? L[(size_t)onehot[c] * d * d + e] : 0.0;
        return;
    }
    const double *gb = gbar + (size_t)c * d;
    double h = gb[i] * gb[i2];
    for (int k = 0; k < K; ++k) {
        const double r = R[(size_t)c * K + k];
        if (r == 0.0) continue;
        const double *gk = GK + ((size_t)c * K + k) * d;
        h += r * (P[(size_t)k * d * d + e] - gk[i] * gk[i2]);
    }
    H[(size_t)c * d * d + e] = h;
}

// ------------------------------------------------------------------ blocked Cholesky
// Right-looking, NB x NB blocks, every live candidate of a batch at once, in one
// cooperative launch: for each block step kb, (A) the diagonal block of every
// candidate, (B) its panel blocks below, (C) the trailing blocks, with a bounded grid
// barrier after each phase (a launch per phase and step waited on the previous one's
// launch latency: 96 dependent launches per factorisation at d = 1024). Blocks written
// by one CTA are read by others after a barrier, so every read of H bypasses L1.
//
// Diagonal block factor, 256 threads, one barrier per column. Step j updates the
// trailing lower triangle with the unscaled pivot column, a_ik -= a_ij a_kj / a_jj
// (= L_ij L_kj), every thread taking 1 / a_jj itself; column j is final after
// step j (later steps touch only columns > j), so the columns are scaled by
// 1 / sqrt(a_jj) once at the end. A pivot <= 0 (not positive definite) sets the
// candidate's info flag (read by every CTA after the next barrier).
constexpr int CF_THREADS = 256;
__device__ void potrf_block(int d, int kb, double *A, int32_t *info_c) {
    __shared__ double a[NB][NB + 1];
    const int o = kb * NB;
    for (int e = threadIdx.x; e < NB * NB; e += CF_THREADS) {
        const int i = e / NB, j = e % NB;
        a[i][j] = (o + i < d && o + j < d) ? __ldcg(&A[(size_t)(o + i) * d + o + j])
                                           : (i == j ? 1.0 : 0.0);  // identity padding
    }
    __syncthreads();
    bool bad = false;
    for (int j = 0; j < NB; ++j) {
        const double p = a[j][j];
        if (!(p > 0.0)) {
            bad = true;
            break;
        }
        const double ip = 1.0 / p;
        const int m = NB - 1 - j;
        for (int e = threadIdx.x; e < m * (m + 1) / 2; e += CF_THREADS) {
            // e -> (ii >= kk) in the packed lower triangle of the trailing block
            int ii = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
            while (ii * (ii + 1) / 2 > e) --ii;
            while ((ii + 1) * (ii + 2) / 2 <= e) ++ii;
            const int kk = e - ii * (ii + 1) / 2;
            const int i = j + 1 + ii, k = j + 1 + kk;
            a[i][k] -= a[i][j] * a[k][j] * ip;
        }
        __syncthreads();
    }
    if (bad) {
        if (threadIdx.x == 0) *info_c = 1;
        __syncthreads();
        return;
    }
    for (int e = threadIdx.x; e < NB * NB; e += CF_THREADS) {
        const int i = e / NB, j = e % NB;
        if (o + i < d && o + j < d && j <= i) {
            const double r = rsqrt(a[j][j]);
            A[(size_t)(o + i) * d + o + j] = i == j ? a[j][j] * r : a[i][j] * r;
        }
    }
    __syncthreads();  // the shared block is free for the next item
}

// Panel: A[ib][kb] <- A[ib][kb] L_kk^{-T}. Threads 0..127: thread (r, part) holds row r's
// columns part, part + 4, ... in registers; per column j the owner scales by
// 1 / L_jj (reciprocals taken once, in parallel) and publishes it, then every
// thread updates its later columns. One barrier per column (every thread of the
// CTA takes part in them); the FP64 updates are spread over four warps.
constexpr int TRSM_THREADS = 128;
__device__ void trsm_block(int d, int kb, int ib, double *A) {
    __shared__ double l[NB][NB + 1];
    __shared__ double xs[NB][NB + 1];
    __shared__ double inv[NB];
    const int o = kb * NB;
    for (int e = threadIdx.x; e < NB * NB; e += CF_THREADS) {
        const int i = e / NB, j = e % NB;
        l[i][j] = (o + i < d && o + j < d) ? __ldcg(&A[(size_t)(o + i) * d + o + j]) : (i == j ? 1.0 : 0.0);
    }
    __syncthreads();
    const bool act = threadIdx.x < TRSM_THREADS;
    if (threadIdx.x < NB) inv[threadIdx.x] = 1.0 / l[threadIdx.x][threadIdx.x];
    const int r = threadIdx.x & (NB - 1), part = (threadIdx.x >> 5) & 3;
    const int row = ib * NB + r;
    double x[NB / 4];
#pragma unroll
    for (int q = 0; q < NB / 4; ++q) {
        const int j = part + 4 * q;
        x[q] = (act && row < d && o + j < d) ? __ldcg(&A[(size_t)row * d + o + j]) : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        if (act && part == (j & 3)) {
            x[j >> 2] *= inv[j];
            xs[r][j] = x[j >> 2];
        }
        __syncthreads();
        const double xj = xs[r][j];
#pragma unroll
        for (int q = 0; q < NB / 4; ++q)
            if (part + 4 * q > j) x[q] -= xj * l[part + 4 * q][j];
    }
    if (act) {
#pragma unroll
        for (int q = 0; q < NB / 4; ++q) {
            const int j = part + 4 * q;
            if (row < d && o + j < d) A[(size_t)row * d + o + j] = x[q];
        }
    }
    __syncthreads();  // the shared blocks are free for the next item
}

// Trailing update A[ib][jb] -= A[ib][kb] A[jb][kb]^T for kb < jb <= ib.
__device__ void syrk_block(int d, int kb, int ib, int jb, double *A) {
    __shared__ double pa[NB][NB + 1], pb[NB][NB + 1];
    const int o = kb * NB;
    for (int e = threadIdx.x; e < NB * NB; e += CF_THREADS) {
        const int r = e / NB, q = e % NB;
        const int ia = ib * NB + r, ja = jb * NB + r, col = o + q;
        pa[r][q] = (ia < d && col < d) ? __ldcg(&A[(size_t)ia * d + col]) : 0.0;
        pb[r][q] = (ja < d && col < d) ? __ldcg(&A[(size_t)ja * d + col]) : 0.0;
    }
    __syncthreads();
    const int tx = threadIdx.x % NB, ty = threadIdx.x / NB;  // ty 0..7
#pragma unroll
    for (int rr = 0; rr < NB / 8; ++rr) {
        const int r = ty + 8 * rr;
        const int i = ib * NB + r, j = jb * NB + tx;
        if (i >= d || j >= d || j > i) continue;
        double s = 0.0;
#pragma unroll
        for (int q = 0; q < NB; ++q) s += pa[r][q] * pb[tx][q];
        A[(size_t)i * d + j] = __ldcg(&A[(size_t)i * d + j]) - s;
    }
    __syncthreads();  // the shared blocks are free for the next item
}

// Whether candidate c is factored here: live, not failed, and not one-hot (a one-hot
// candidate's factor is L_k, copied in place by k_hessian). info[c] is read after a
// grid barrier, so every CTA sees the same value.
__device__ __forceinline__ bool chol_live(int c, const int32_t *onehot, const int32_t *info) {
    return !(onehot && onehot[c] >= 0) && *reinterpret_cast<const volatile int32_t *>(&info[c]) == 0;
}

__global__ void __launch_bounds__(CF_THREADS) k_chol_coop(int d, double *H, const int32_t *n_c,
                                                         const int32_t *onehot, int32_t *info, uint32_t *bar,
                                                         int32_t *err) {
    // the candidate count is the same value in every CTA, so all CTAs reach every barrier
    const int nc = *n_c;
    const int nblk = (d + NB - 1) / NB;
    for (int kb = 0; kb < nblk; ++kb) {
        for (int c = blockIdx.x; c < nc; c += gridDim.x)
            if (chol_live(c, onehot, info)) potrf_block(d, kb, H + (size_t)c * d * d, info + c);
        if (!grid_barrier(bar, gridDim.x, err)) return;
        const int rest = nblk - kb - 1;
        if (rest == 0) break;
        for (int it = blockIdx.x; it < nc * rest; it += gridDim.x) {
            const int c = it / rest;
            if (chol_live(c, onehot, info)) trsm_block(d, kb, kb + 1 + it % rest, H + (size_t)c * d * d);
        }
        if (!grid_barrier(bar, gridDim.x, err)) return;
        const int tri = rest * (rest + 1) / 2;  // trailing blocks (ii >= jj) per candidate
        for (int it = blockIdx.x; it < nc * tri; it += gridDim.x) {
            const int c = it / tri, e = it - c * tri;
            if (!chol_live(c, onehot, info)) continue;
            int ii = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
            while (ii * (ii + 1) / 2 > e) --ii;
            while ((ii + 1) * (ii + 2) / 2 <= e) ++ii;
            const int jj = e - ii * (ii + 1) / 2;
            syrk_block(d, kb, kb + 1 + ii, kb + 1 + jj, H + (size_t)c * d * d);
        }
        if (!grid_barrier(bar, gridDim.x, err)) return;
    }
}

// Solve (C C^T) delta = g for each candidate still polishing and the model
// increase g^T delta / 2 (cooperative launch, one bounded grid barrier per 32-row
// block and direction). The grid is split into slots of Gc CTAs (Gc from the
// candidate count on the device, 1 to 16); slot j serves candidates j, j + slots,
// ... in turn, and CTA q of a slot owns the row blocks J with J % Gc == q of each.
// Forward (C y = g): in step I the owner of block I (already updated by every
// earlier step, by itself) solves the diagonal block and publishes y_I; after the
// barrier every owner subtracts C_JI y_I from its blocks J > I. The owner of block
// I + 1 has then finished block I + 1's last update before it solves it in step
// I + 1, so one barrier per step suffices. Backward (C^T delta = y) mirrors it
// with (C^T)_JI = (C_IJ)^T for J < I. The right-hand side lives in delta[c]
// (global, read past L1 after barriers).
constexpr int CS_THREADS = 256;
__global__ void __launch_bounds__(CS_THREADS) k_chol_solve_coop(int d, const double *H, const double *g,
                                                                const int32_t *n_c, const int32_t *info,
                                                                const uint8_t *active, double *delta, double *pred,
                                                                uint32_t *bar, int32_t *err) {
    __shared__ double Dg[32][33];
    __shared__ double dinv[32];
    __shared__ double xs[32];
    __shared__ double part[8];
    __shared__ double red[8][33];
    // the candidate count is the same value in every CTA, so either all CTAs leave
    // here or all reach every grid barrier
    const int ncand = *n_c;
    if (ncand <= 0) return;
    int Gc = (int)gridDim.x / ncand;
    Gc = Gc < 1 ? 1 : (Gc > 16 ? 16 : Gc);
    const int slots = (int)gridDim.x / Gc;
    const int slot = blockIdx.x / Gc, q = blockIdx.x % Gc;
    const int c0 = slot < slots ? slot : ncand;  // CTAs past the last whole slot serve nothing
    const int nb = (d + 31) / 32;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    auto live = [&](int c) { return !info[c] && active[c]; };
    for (int c = c0; c < ncand; c += slots) {
        if (!live(c)) continue;
        double *y = delta + (size_t)c * d;
        for (int J = q; J < nb; J += Gc)
            for (int i = J * 32 + (int)threadIdx.x; i < min(d, J * 32 + 32); i += CS_THREADS)
                y[i] = g[(size_t)c * d + i];
    }
    __syncthreads();
    // the owner's diagonal solve of block I of candidate c (lower: forward; upper: with C^T)
    auto diag = [&](int c, int I, bool upper) {
        const double *C = H + (size_t)c * d * d;
        double *y = delta + (size_t)c * d;
        const int r0 = I * 32, rows = min(32, d - r0);
        for (int e = threadIdx.x; e < 32 * 32; e += CS_THREADS) {
            const int i = e / 32, j = e % 32;
            Dg[i][j] = (i < rows && j < rows) ? C[(size_t)(r0 + i) * d + r0 + j] : (i == j ? 1.0 : 0.0);
        }
        __syncthreads();
        if (threadIdx.x < 32) dinv[threadIdx.x] = 1.0 / Dg[threadIdx.x][threadIdx.x];
        __syncthreads();
        if (wid == 0) {
            double v = lane < rows ? __ldcg(y + r0 + lane) : 0.0;
            if (!upper) {
                for (int i = 0; i < 32; ++i) {
                    const double yi = __shfl_sync(0xffffffffu, v, i) * dinv[i];
                    if (lane == i) v = yi;
                    if (lane > i) v -= Dg[lane][i] * yi;
                }
            } else {
                for (int i = 31; i >= 0; --i) {
                    const double xi = __shfl_sync(0xffffffffu, v, i) * dinv[i];
                    if (lane == i) v = xi;
                    if (lane < i) v -= Dg[i][lane] * xi;
                }
            }
            if (lane < rows) y[r0 + lane] = v;
        }
        __threadfence();
        __syncthreads();
    };
    // forward
    for (int I = 0; I < nb; ++I) {
        if (I % Gc == q)
            for (int c = c0; c < ncand; c += slots)
                if (live(c)) diag(c, I, false);
        if (!grid_barrier(bar, gridDim.x, err)) return;
        const int r0 = I * 32, rows = min(32, d - r0);
        for (int c = c0; c < ncand; c += slots) {
            if (!live(c)) continue;
            const double *C = H + (size_t)c * d * d;
            double *y = delta + (size_t)c * d;
            if (threadIdx.x < 32) xs[threadIdx.x] = threadIdx.x < rows ? __ldcg(y + r0 + threadIdx.x) : 0.0;
            __syncthreads();
            // y_J -= C_JI y_I for owned J > I: warp per output row
            for (int J = I + 1; J < nb; ++J) {
                if (J % Gc != q) continue;
                const int j0 = J * 32, jr = min(32, d - j0);
                for (int rr = wid; rr < jr; rr += CS_THREADS / 32) {
                    const double a = lane < rows ? C[(size_t)(j0 + rr) * d + r0 + lane] * xs[lane] : 0.0;
                    const double sum = warp_sum(a);
                    if (lane == 0) y[j0 + rr] -= sum;
                }
            }
            __syncthreads();
        }
    }
    // backward
    for (int I = nb - 1; I >= 0; --I) {
        if (I % Gc == q)
            for (int c = c0; c < ncand; c += slots)
                if (live(c)) diag(c, I, true);
        if (!grid_barrier(bar, gridDim.x, err)) return;
        const int r0 = I * 32, rows = min(32, d - r0);
        for (int c = c0; c < ncand; c += slots) {
            if (!live(c)) continue;
            const double *C = H + (size_t)c * d * d;
            double *y = delta + (size_t)c * d;
            if (threadIdx.x < 32) xs[threadIdx.x] = threadIdx.x < rows ? __ldcg(y + r0 + threadIdx.x) : 0.0;
            __syncthreads();
            // y_J -= (C_IJ)^T x_I for owned J < I: thread per output column j (coalesced rows of C)
            for (int J = 0; J < I; ++J) {
                if (J % Gc != q) continue;
                const int j0 = J * 32;
                // 8 warps split the 32 rows of block I; lane = column j
                double a = 0.0;
                for (int i = wid; i < rows; i += CS_THREADS / 32) a += C[(size_t)(r0 + i) * d + j0 + lane] * xs[i];
                red[wid][lane] = a;
                __syncthreads();
                if (wid == 0) {
                    double t = 0.0;
                    for (int w = 0; w < CS_THREADS / 32; ++w) t += red[w][lane];
                    y[j0 + lane] -= t;
                }
                __syncthreads();
            }
        }
    }
    if (!grid_barrier(bar, gridDim.x, err)) return;
    // model increase of l along the Newton step: g^T delta / 2 (first CTA of the slot)
    if (q != 0) return;
    for (int c = c0; c < ncand; c += slots) {
        if (!live(c)) continue;
        const double *y = delta + (size_t)c * d;
        double gd = 0.0;
        for (int i = threadIdx.x; i < d; i += CS_THREADS) gd += g[(size_t)c * d + i] * __ldcg(y + i);
        gd = warp_sum(gd);
        if (lane == 0) part[wid] = gd;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < CS_THREADS / 32; ++w) t += part[w];
            pred[c] = 0.5 * t;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ Newton line search
// mode 0: start (t = 1, trial = x + delta, searching = active & Cholesky ok).
//   A candidate whose Newton step is already below kNewtonXtol (1 + |x|_inf) in
//   max norm has converged: it stays where it is (its H factor is the one at
//   that point) and stops polishing; the others are counted in *n_live.
// mode 1: decide on the evaluated trial (accept if l_t >= l, else halve)
constexpr double kNewtonXtol = 1e-11;
__global__ void __launch_bounds__(256) k_newton_ls(int d, int mode, const int32_t *n_c, const int32_t *info,
                                                   uint8_t *active, uint8_t *searching, int32_t *halvings, double *t,
                                                   double *XC, double *LC, const double *delta, double *XN,
                                                   const double *LN, const double *pred, int32_t *n_live) {
    const int c = blockIdx.x;
    if (c >= *n_c) return;
    __shared__ int s_act;
    __shared__ double s_mx[2][8];
    bool small = false;
    if (mode == 0) {  // max |delta| and max |x| of the candidate
        double md = 0.0, mx = 0.0;
        for (int i = threadIdx.x; i < d; i += blockDim.x) {
            md = fmax(md, fabs(delta[(size_t)c * d + i]));
            mx = fmax(mx, fabs(XC[(size_t)c * d + i]));
        }
        md = warp_max(md);
        mx = warp_max(mx);
        if ((threadIdx.x & 31) == 0) {
            s_mx[0][threadIdx.x >> 5] = md;
            s_mx[1][threadIdx.x >> 5] = mx;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int q = 1; q < 8; ++q) {
                md = fmax(md, s_mx[0][q]);
                mx = fmax(mx, s_mx[1][q]);
            }
            small = md <= kNewtonXtol * (1.0 + mx);
        }
    }
    if (threadIdx.x == 0) {
        int act = 0;
        if (mode == 0) {
            const int s = active[c] && !info[c] && !small;
            if (!s) active[c] = 0;
            halvings[c] = 0;
            t[c] = 1.0;
            if (s) atomicAdd(n_live, 1);
            if (s && pred[c] <= 1e-10 * (1.0 + fabs(LC[c]))) {
                // quadratic-convergence regime: the descent test is rounding noise, take t = 1
                searching[c] = 0;
                act = 3;
            } else {
                searching[c] = (uint8_t)s;
                act = s ? 2 : 0;  // 2: write the trial
            }
        } else if (searching[c]) {
            if (LN[c] >= LC[c]) {
                searching[c] = 0;
                LC[c] = LN[c];
                act = 1;  // 1: accept
            } else if (halvings[c] + 1 >= 30) {
                searching[c] = 0;
                active[c] = 0;  // no acceptable step: stop polishing this candidate
            } else {
                ++halvings[c];
                t[c] *= 0.5;
                act = 2;
            }
        }
        s_act = act;
    }
    __syncthreads();
    const int act = s_act;
    if (act == 1) {
        for (int i = threadIdx.x; i < d; i += blockDim.x) XC[(size_t)c * d + i] = XN[(size_t)c * d + i];
    } else if (act == 3) {
        for (int i = threadIdx.x; i < d; i += blockDim.x)
            XC[(size_t)c * d + i] = add_rn(XC[(size_t)c * d + i], mul_rn(1.0, delta[(size_t)c * d + i]));
    } else if (act == 2) {
        const double tc = t[c];
        for (int i = threadIdx.x; i < d; i += blockDim.x)
            XN[(size_t)c * d + i] = add_rn(XC[(size_t)c * d + i], mul_rn(tc, delta[(size_t)c * d + i]));
    }
}

// Halvings 1..kHalvings-1 evaluated as one batch: the first acceptable
// halving is the one a sequential search would stop at.
__global__ void __launch_bounds__(256) k_ls_batch_setup(int d, const int32_t *n_c, const uint8_t *searching,
                                                        const double *XC, const double *delta, double *XN2,
                                                        int32_t *rows2, int32_t *n_rows2) {
    const int c = blockIdx.x;
    if (c >= *n_c || !searching[c]) return;
    __shared__ int base;
    if (threadIdx.x == 0) base = atomicAdd(n_rows2, kHalvings - 1);
    __syncthreads();
    double t = 1.0;
    for (int h = 1; h < kHalvings; ++h) {
        t *= 0.5;
        const size_t row = (size_t)c * (kHalvings - 1) + (h - 1);
        for (int i = threadIdx.x; i < d; i += blockDim.x)
            XN2[row * d + i] = add_rn(XC[(size_t)c * d + i], mul_rn(t, delta[(size_t)c * d + i]));
        if (threadIdx.x == 0) rows2[base + h - 1] = (int32_t)row;
    }
}

__global__ void __launch_bounds__(256) k_ls_batch_decide(int d, const int32_t *n_c, uint8_t *searching,
                                                         uint8_t *active, double *XC, double *LC, const double *XN2,
                                                         const double *LN2) {
    const int c = blockIdx.x;
    if (c >= *n_c || !searching[c]) return;
    __shared__ int hsel;
    if (threadIdx.x == 0) {
        int hs = -1;
        for (int h = 1; h < kHalvings; ++h)
            if (LN2[(size_t)c * (kHalvings - 1) + h - 1] >= LC[c]) {
                hs = h;
                break;
            }
        hsel = hs;
    }
    __syncthreads();
    const int h = hsel;
    if (h < 0) {
        if (threadIdx.x == 0) {
            searching[c] = 0;
            active[c] = 0;
        }
        return;
    }
    const size_t row = (size_t)c * (kHalvings - 1) + (h - 1);
    for (int i = threadIdx.x; i < d; i += blockDim.x) XC[(size_t)c * d + i] = XN2[row * d + i];
    __syncthreads();
    if (threadIdx.x == 0) {
        LC[c] = LN2[row];
        searching[c] = 0;
    }
}

// ------------------------------------------------------------------ filters and log Z_k
__global__ void __launch_bounds__(256) k_cand_stats(int d, const double *XC, const double *LC, const double *GC,
                                                    const double *H, const int32_t *info, const double *lo,
                                                    const double *hi, double eps_grad, const int32_t *n_c,
                                                    uint8_t *keep, double *logZk) {
    const int c = blockIdx.x;
    if (c >= *n_c) return;
    __shared__ double s_gm[32], s_ld[32];
    __shared__ int s_in[32];
    double gm = 0.0, ld = 0.0;
    int inside = 1;
    const bool ok = info[c] == 0;
    for (int i = threadIdx.x; i < d; i += blockDim.x) {
        gm = fmax(gm, fabs(GC[(size_t)c * d + i]));
        const double x = XC[(size_t)c * d + i];
        if (!(x >= lo[i] && x <= hi[i])) inside = 0;
        if (ok) ld += log(H[(size_t)c * d * d + (size_t)i * d + i]);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    gm = warp_max(gm);
    ld = warp_sum(ld);
    inside = __all_sync(0xffffffffu, inside);
    if (lane == 0) {
        s_gm[wid] = gm;
        s_ld[wid] = ld;
        s_in[wid] = inside;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double g = 0.0, l = 0.0;
        int in = 1;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
            g = fmax(g, s_gm[q]);
            l += s_ld[q];
            in &= s_in[q];
        }
        const double ell = LC[c];
        keep[c] = (uint8_t)(ok && isfinite(ell) && g <= eps_grad * (1.0 + fabs(ell)) && in);
        logZk[c] = ok ? (ell + 0.5 * (double)d * SB_LOG_2PI) - l : NAN;
    }
}

// Final dedup of the kept candidates, outputs in order of decreasing l, LSE - log V.
__global__ void __launch_bounds__(1024) k_laplace_final(int d, const double *XC, const double *LC,
                                                        const double *logZk_c, const int32_t *n_c,
                                                        const int32_t *reps, const int32_t *n_reps, const double *logV,
                                                        int cap, double *modes, double *logZk, double *ell_modes,
                                                        int32_t *n_modes, double *logZ, int32_t *dev_status) {
    const int nm = *n_reps;
    for (int t = 0; t < nm && t < cap; ++t) {
        const int c = reps[t];
        for (int i = threadIdx.x; i < d; i += blockDim.x) modes[(size_t)t * d + i] = XC[(size_t)c * d + i];
        if (threadIdx.x == 0) {
            logZk[t] = logZk_c[c];
            if (ell_modes) ell_modes[t] = LC[c];
        }
    }
    if (threadIdx.x == 0) {
        double zmax = -INFINITY;
        for (int t = 0; t < nm; ++t) zmax = fmax(zmax, logZk_c[reps[t]]);
        double lz = -INFINITY;
        if (nm > 0) {
            double s = 0.0;
            for (int t = 0; t < nm; ++t) s += exp(logZk_c[reps[t]] - zmax);
            lz = zmax + log(s) - logV[0];
        } else {
            atomicOr(dev_status, SB_DEV_NO_MODES);
        }
        *logZ = lz;
        *n_modes = nm;
    }
}

}  // namespace

void launch_dedup(int n, int d, const double *X, const double *ell, const int8_t *status, const uint8_t *keep,
                  double tau_scale, const double *wmax, int cap, int32_t *reps, int32_t *n_reps, uint8_t *assigned,
                  const DedupScratch &sc, cudaStream_t s) {
    // one CTA per 128 points up to one per SM (kept small so that concurrent
    // solves on other streams can still be co-resident)
    static const int sms = [] {  // thread-safe one-time query (batched solves use several host threads)
        int dev = 0, n = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        return n > 0 ? n : 1;
    }();
    int G = (n + 127) / 128;
    if (G > sms) G = sms;
    if (G > kDedupMaxGrid) G = kDedupMaxGrid;
    if (G < 1) G = 1;
    cudaMemsetAsync(sc.bar, 0, 2 * sizeof(uint32_t), s);
    void *args[] = {&n, &d, &X, &ell, &status, &keep, &tau_scale, &wmax, &cap, &reps, &n_reps, &assigned,
                    const_cast<double **>(&sc.part_l), const_cast<int32_t **>(&sc.part_i),
                    const_cast<uint32_t **>(&sc.bar), const_cast<int32_t **>(&sc.err)};
    note_launch();
    cudaLaunchCooperativeKernel((const void *)k_dedup, dim3(G), dim3(DD_THREADS), args, sizeof(double) * d, s);
}

void launch_gather_rows(int d, int cap, const double *X, const int32_t *idx, const int32_t *n_idx, double *out,
                        const double *ell, double *ell_out, cudaStream_t s) {
    note_launch();
    k_gather_rows<<<cap, 256, 0, s>>>(d, X, idx, n_idx, out, ell, ell_out);
}

void launch_precision(int d, int K, const double *L, double *P, cudaStream_t s) {
    dim3 g((d + PT - 1) / PT, (d + PT - 1) / PT, K);
    note_launch();
    k_precision<<<g, 256, 0, s>>>(d, L, P, nullptr);
}

void launch_onehot(int K, const double *R, const int32_t *n_c, int cap, int32_t *onehot, cudaStream_t s) {
    note_launch();
    k_onehot<<<(cap + 127) / 128, 128, 0, s>>>(K, R, n_c, cap, onehot);
}

void launch_precision_needed(int d, int K, const double *L, const double *R, const int32_t *n_c, int32_t *done,
                             int32_t *need, double *P, cudaStream_t s, const int32_t *onehot) {
    note_launch();
    k_precision_need<<<1, kMaxK, 0, s>>>(K, R, n_c, onehot, done, need);
    dim3 g((d + PT - 1) / PT, (d + PT - 1) / PT, K);
    note_launch();
    k_precision<<<g, 256, 0, s>>>(d, L, P, need);
}

// Condition of the blocked factorisation: some live candidate is not one-hot.
__global__ void k_chol_needed(cudaGraphConditionalHandle h, const int32_t *n_c, const int32_t *onehot) {
    __shared__ int any;
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    const int nc = *n_c;
    for (int c = threadIdx.x; c < nc; c += blockDim.x)
        if (onehot[c] < 0) any = 1;
    __syncthreads();
    if (threadIdx.x == 0) cudaGraphSetConditional(h, any ? 1u : 0u);
}

int laplace_sms();

void launch_hessian_chol(int d, int K, int cap, const double *L, const double *P, const double *Z, const double *R,
                         const double *gbar, const int32_t *n_c, double *GK, double *H, int32_t *info,
                         uint32_t *bar, int32_t *err, cudaStream_t s, const int32_t *onehot) {
    note_launch();
    k_comp_grads<<<dim3(cap, K, kGradSlices), 256, sizeof(double) * d, s>>>(d, K, L, Z, R, n_c, GK);
    const int64_t dd = (int64_t)d * d;
    note_launch();
    k_hessian<<<dim3((unsigned)((dd + 255) / 256), cap), 256, 0, s>>>(d, K, P, GK, R, gbar, n_c, onehot, L, H,
                                                                        info);
    auto factor = [&](cudaStream_t fs) {
        ProfScope prof(PROF_CHOLESKY, fs);
        // one CTA per SM (a cooperative grid must be co-resident), no more than the
        // largest phase's items
        const int nblk = (d + NB - 1) / NB;
        const long long items = (long long)cap * (nblk - 1) * nblk / 2;
        int G = laplace_sms();
        if (items < G) G = (int)(items > 0 ? items : 1);
        cudaMemsetAsync(bar, 0, 2 * sizeof(uint32_t), fs);
        void *args[] = {&d, &H, &n_c, &onehot, &info, &bar, &err};
        note_launch();
        cudaLaunchCooperativeKernel((const void *)k_chol_coop, dim3(G), dim3(CF_THREADS), args, 0, fs);
    };
    // in a graph, the factorisation is the body of an IF node that runs only when some
    // live candidate is not one-hot (its launches would otherwise all be idle CTAs)
    if (onehot && stream_capturing(s)) {
        const sb_status st = capture_if(
            s,
            [&](cudaStream_t cs, cudaGraphConditionalHandle h) {
                note_launch();
                k_chol_needed<<<1, 256, 0, cs>>>(h, n_c, onehot);
            },
            factor);
        if (st == SB_OK) return;
        // the node could not be added: factor unconditionally (a capture left broken by
        // the failure reports it when it ends)
    } else if (onehot && !stream_capturing(s)) {
        // eager mode (host reads allowed): the same decision on the host, so that an
        // all-one-hot candidate set launches no idle factorisation kernels either
        int32_t nc = 0;
        std::vector<int32_t> oh((size_t)cap);
        if (cudaMemcpyAsync(&nc, n_c, sizeof(int32_t), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
            cudaMemcpyAsync(oh.data(), onehot, sizeof(int32_t) * (size_t)cap, cudaMemcpyDeviceToHost, s) ==
                cudaSuccess &&
            cudaStreamSynchronize(s) == cudaSuccess) {
            bool any = false;
            for (int c = 0; c < nc && c < cap; ++c) any = any || oh[(size_t)c] < 0;
            if (!any) return;
        }
    }
    factor(s);
}

int laplace_sms() {
    static const int n = [] {  // thread-safe one-time query
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        return v > 0 ? v : 1;
    }();
    return n;
}

void launch_chol_solve_coop(int d, int cap, const double *H, const double *g, const int32_t *n_c, const int32_t *info,
                            const uint8_t *active, double *delta, double *pred, uint32_t *bar, int32_t *err,
                            cudaStream_t s) {
    // one CTA per SM at most (a cooperative grid must be co-resident), up to 16 per
    // candidate of the cap; the kernel divides them among the live candidates
    int G = laplace_sms();
    if (G > 16 * cap) G = 16 * cap;
    cudaMemsetAsync(bar, 0, 2 * sizeof(uint32_t), s);
    void *args[] = {&d, &H, &g, &n_c, &info, &active, &delta, &pred, &bar, &err};
    note_launch();
    cudaLaunchCooperativeKernel((const void *)k_chol_solve_coop, dim3(G), dim3(CS_THREADS), args, 0, s);
}

__global__ void k_set_eff(int32_t *n_eff, const int32_t *n_reps, const int32_t *n_live) {
    if (threadIdx.x == 0) *n_eff = (!n_live || *n_live > 0) ? *n_reps : 0;
}

void launch_set_eff(int32_t *n_eff, const int32_t *n_reps, const int32_t *n_live, cudaStream_t s) {
    note_launch();
    k_set_eff<<<1, 32, 0, s>>>(n_eff, n_reps, n_live);
}

void launch_newton_ls(int d, int cap, int mode, const int32_t *n_c, const int32_t *info, uint8_t *active,
                      uint8_t *searching, int32_t *halvings, double *t, double *XC, double *LC, const double *delta,
                      double *XN, const double *LN, const double *pred, int32_t *n_live, cudaStream_t s) {
    note_launch();
    k_newton_ls<<<cap, 256, 0, s>>>(d, mode, n_c, info, active, searching, halvings, t, XC, LC, delta, XN, LN,
                                    pred, n_live);
}

void launch_ls_batch_setup(int d, int cap, const int32_t *n_c, const uint8_t *searching, const double *XC,
                           const double *delta, double *XN2, int32_t *rows2, int32_t *n_rows2, cudaStream_t s) {
    cudaMemsetAsync(n_rows2, 0, sizeof(int32_t), s);
    note_launch();
    k_ls_batch_setup<<<cap, 256, 0, s>>>(d, n_c, searching, XC, delta, XN2, rows2, n_rows2);
}

void launch_ls_batch_decide(int d, int cap, const int32_t *n_c, uint8_t *searching, uint8_t *active, double *XC,
                            double *LC, const double *XN2, const double *LN2, cudaStream_t s) {
    note_launch();
    k_ls_batch_decide<<<cap, 256, 0, s>>>(d, n_c, searching, active, XC, LC, XN2, LN2);
}

void launch_cand_stats(int d, int cap, const double *XC, const double *LC, const double *GC, const double *H,
                       const int32_t *info, const double *lo, const double *hi, double eps_grad, const int32_t *n_c,
                       uint8_t *keep, double *logZk, cudaStream_t s) {
    note_launch();
    k_cand_stats<<<cap, 256, 0, s>>>(d, XC, LC, GC, H, info, lo, hi, eps_grad, n_c, keep, logZk);
}

void launch_laplace_final(int d, const double *XC, const double *LC, const double *logZk_c, const int32_t *n_c,
                          const int32_t *reps, const int32_t *n_reps, const double *logV, int cap, double *modes,
                          double *logZk, double *ell_modes, int32_t *n_modes, double *logZ, int32_t *dev_status,
                          cudaStream_t s) {
    note_launch();
    k_laplace_final<<<1, 1024, 0, s>>>(d, XC, LC, logZk_c, n_c, reps, n_reps, logV, cap, modes, logZk, ell_modes,
                                       n_modes, logZ, dev_status);
}

}  // namespace sb
