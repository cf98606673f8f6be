// segments.cu -- the other ray families (Sec. 3.5.1) and the two-pass sampling
// along a ray (Sec. 3.5.2), FP64.
//
// Families: V2V joins two vertices drawn from independent bit streams (an end
// equal to the start becomes its antipode); V2E runs from a vertex to the
// midpoint of an edge (vertex bits, one free coordinate at the box centre);
// W2W runs from a uniform point on the face x_i = lo_i to one on x_i = hi_i
// of a random axis i. Ray r of a family draws from Philox4x32-10 blocks with
// counter (block, r, family tag, purpose) and the seed as key: bit b of a
// stream is bit b % 32 of word (b / 32) % 4 of block b / 128; uniform k is
// built from words 2 (k % 2), 2 (k % 2) + 1 of block k / 2; an index below n
// is (word 0 of block 0) * n >> 32.
//
// Along a segment x(t) = a + t (b - a) every component's z is affine in t,
// z_k(t) = z_k(a) + t (z_k(b) - z_k(a)), so |z_k(t)|^2 = q0 + 2 t q1 + t^2 q2
// with q0 = |z_k(a)|^2, q1 = z_k(a).w, q2 = |w|^2, w = z_k(b) - z_k(a). One
// z GEMM over the 2 n_rays end points gives every coarse and refined sample's
// l from three scalars per (ray, component) instead of a GEMM row per sample.
//
// Coarse pass: t_j = j / (n - 1) (t = 1/2 for n = 1); the active region is
// l_j > max l - delta; the refinement density is piecewise constant on the
// coarse cells [t_j - h/2, t_j + h/2] clipped to [0, 1], proportional to
// exp(l_j - max l) on active cells; n_ref points at the inverse CDF of the
// midpoints (k + 1/2) / n_ref, linear inside a cell.
#include "sb_segments.cuh"

namespace sb {

namespace {

constexpr uint32_t kTagV2V = 0x56325620u, kTagV2E = 0x56324520u, kTagW2W = 0x57325720u;

__device__ __forceinline__ uint32_t seg_word(uint32_t k0, uint32_t k1, uint32_t r, uint32_t tag, uint32_t purpose,
                                             uint32_t q, int w) {
    uint32_t c[4] = {q, r, tag, purpose};
    philox4x32_10(c, k0, k1);
    return c[w];
}

__device__ __forceinline__ int seg_bit(uint32_t k0, uint32_t k1, uint32_t r, uint32_t tag, uint32_t purpose, int b) {
    return (int)((seg_word(k0, k1, r, tag, purpose, (uint32_t)(b / 128), (b / 32) % 4) >> (b % 32)) & 1u);
}

__device__ __forceinline__ int seg_index(uint32_t k0, uint32_t k1, uint32_t r, uint32_t tag, uint32_t purpose, int n) {
    return (int)(((uint64_t)seg_word(k0, k1, r, tag, purpose, 0, 0) * (uint64_t)n) >> 32);
}

__device__ __forceinline__ double seg_unit(uint32_t k0, uint32_t k1, uint32_t r, uint32_t tag, uint32_t purpose,
                                           int k) {
    uint32_t c[4] = {(uint32_t)(k / 2), r, tag, purpose};
    philox4x32_10(c, k0, k1);
    const int w = 2 * (k % 2);
    return unit_from_words(c[w], c[w + 1]);
}

// warp per ray: start and end points
__global__ void __launch_bounds__(256) k_seg_ends(int family, int n_rays, int d, uint32_t k0, uint32_t k1,
                                                  const double *lo, const double *hi, double *A, double *B) {
    const int lane = threadIdx.x & 31;
    const int r = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    if (r >= n_rays) return;
    double *a = A + (size_t)r * d;
    double *b = B + (size_t)r * d;
    if (family == SB_RAY_W2W) {
        const int ax = seg_index(k0, k1, (uint32_t)r, kTagW2W, 2, d);
        for (int i = lane; i < d; i += 32) {
            const double w = sub_rn(hi[i], lo[i]);
            a[i] = i == ax ? lo[i] : add_rn(lo[i], mul_rn(seg_unit(k0, k1, (uint32_t)r, kTagW2W, 0, i), w));
            b[i] = i == ax ? hi[i] : add_rn(lo[i], mul_rn(seg_unit(k0, k1, (uint32_t)r, kTagW2W, 1, i), w));
        }
        return;
    }
    const uint32_t tag = family == SB_RAY_V2V ? kTagV2V : kTagV2E;
    int same = 1;
    for (int i = lane; i < d; i += 32) {
        const int bs = seg_bit(k0, k1, (uint32_t)r, tag, 0, i);
        const int be = seg_bit(k0, k1, (uint32_t)r, tag, 1, i);
        a[i] = bs ? hi[i] : lo[i];
        b[i] = be ? hi[i] : lo[i];
        same &= (bs == be);
    }
    same = __all_sync(0xffffffffu, same);
    if (family == SB_RAY_V2V) {
        if (same) {
            __syncwarp();
            for (int i = lane; i < d; i += 32) b[i] = a[i] == hi[i] ? lo[i] : hi[i];
        }
    } else {
        const int j = seg_index(k0, k1, (uint32_t)r, tag, 2, d);
        __syncwarp();
        if (lane == 0) b[j] = 0.5 * (lo[j] + hi[j]);
    }
}

// warp per (ray, component): q = (|z_a|^2, z_a . w, |w|^2), w = z_b - z_a
__global__ void __launch_bounds__(256) k_seg_q(int n_rays, int d, int K, const double *Z, double *Q) {
    const int lane = threadIdx.x & 31;
    const int e = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    if (e >= n_rays * K) return;
    const int r = e / K, k = e - r * K;
    const double *za = Z + ((size_t)r * K + k) * d;
    const double *zb = Z + ((size_t)(n_rays + r) * K + k) * d;
    double q0 = 0.0, q1 = 0.0, q2 = 0.0;
    for (int j = lane; j < d; j += 32) {
        const double x = za[j], w = zb[j] - za[j];
        q0 += x * x;
        q1 += x * w;
        q2 += w * w;
    }
    q0 = warp_sum(q0);
    q1 = warp_sum(q1);
    q2 = warp_sum(q2);
    if (lane == 0) {
        Q[(size_t)e * 3 + 0] = q0;
        Q[(size_t)e * 3 + 1] = q1;
        Q[(size_t)e * 3 + 2] = q2;
    }
}

__device__ double seg_ell(int K, const double *a, const double *q, double t) {
    double m = -INFINITY;
    for (int k = 0; k < K; ++k) {
        const double zz = q[3 * k] + 2.0 * t * q[3 * k + 1] + t * t * q[3 * k + 2];
        m = fmax(m, a[k] - 0.5 * zz);
    }
    double s = 0.0;
    for (int k = 0; k < K; ++k) {
        const double zz = q[3 * k] + 2.0 * t * q[3 * k + 1] + t * t * q[3 * k + 2];
        s += exp(a[k] - 0.5 * zz - m);
    }
    return m + log(s);
}

__device__ __forceinline__ double coarse_t(int j, int n) { return n > 1 ? (double)j / (double)(n - 1) : 0.5; }

__global__ void __launch_bounds__(256) k_seg_coarse(int n_rays, int n, int K, const double *a, const double *Q,
                                                    double *ell) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)n_rays * n) return;
    const int r = (int)(e / n), j = (int)(e - (int64_t)r * n);
    ell[e] = seg_ell(K, a, Q + (size_t)r * K * 3, coarse_t(j, n));
}

// thread per ray: the refinement pass (cdf scratch [n_rays][n + 1])
__global__ void __launch_bounds__(128) k_seg_refine(int n_rays, int n, int n_ref, int K, double delta, const double *a,
                                                    const double *Q, const double *ell, double *cdf_all,
                                                    double *t_ref, double *ell_ref) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rays) return;
    const double *l = ell + (size_t)r * n;
    double *cdf = cdf_all + (size_t)r * (n + 1);
    double lmax = -INFINITY;
    for (int j = 0; j < n; ++j) lmax = fmax(lmax, l[j]);
    const double h = n > 1 ? 1.0 / (double)(n - 1) : 1.0;
    cdf[0] = 0.0;
    for (int j = 0; j < n; ++j) {
        const double tc = coarse_t(j, n);
        const double lo = fmax(tc - 0.5 * h, 0.0), hi = fmin(tc + 0.5 * h, 1.0);
        const double w = l[j] > lmax - delta ? exp(l[j] - lmax) * (hi - lo) : 0.0;
        cdf[j + 1] = cdf[j] + w;
    }
    const double total = cdf[n];
    int j = 0;
    for (int k = 0; k < n_ref; ++k) {
        const double u = ((double)k + 0.5) / (double)n_ref * total;
        while (j < n - 1 && cdf[j + 1] <= u) ++j;  // u grows with k: the cell index never goes back
        const double tc = coarse_t(j, n);
        const double lo = fmax(tc - 0.5 * h, 0.0), hi = fmin(tc + 0.5 * h, 1.0);
        const double cw = cdf[j + 1] - cdf[j];
        const double fr = cw > 0.0 ? (u - cdf[j]) / cw : 0.5;
        const double t = lo + fr * (hi - lo);
        t_ref[(size_t)r * n_ref + k] = t;
        ell_ref[(size_t)r * n_ref + k] = seg_ell(K, a, Q + (size_t)r * K * 3, t);
    }
}

inline unsigned warp_blocks(int64_t warps) { return (unsigned)((warps * 32 + 255) / 256); }

}  // namespace

size_t segments_scratch_elems(int n_rays, int n_steps, int d, int K) {
    const size_t rows = 2 * (size_t)n_rays;
    return rows * K * d + lik_f64_qpart_elems(d, K, (int)rows) + (size_t)n_rays * K * 3 + (size_t)n_rays * (n_steps + 1);
}

void launch_segments(const ProbView &pv, int family, uint64_t seed, int n_rays, int n_steps, double delta, int n_ref,
                     double *scratch, double *ends, double *ell_coarse, double *t_ref, double *ell_ref,
                     cudaStream_t s) {
    const int d = pv.d, K = pv.K;
    const size_t rows = 2 * (size_t)n_rays;
    double *Z = scratch;
    double *qpart = Z + rows * K * d;
    double *Q = qpart + lik_f64_qpart_elems(d, K, (int)rows);
    double *cdf = Q + (size_t)n_rays * K * 3;
    double *A = ends, *B = ends + (size_t)n_rays * d;
    note_launch();
    k_seg_ends<<<warp_blocks(n_rays), 256, 0, s>>>(family, n_rays, d, (uint32_t)seed, (uint32_t)(seed >> 32), pv.lo,
                                                   pv.hi, A, B);
    LikF64Args a{};
    a.d = d;
    a.K = K;
    a.mu = pv.mu;
    a.L = pv.L;
    a.a = pv.a;
    a.c = pv.c;
    a.X = ends;  // rows 0 .. n_rays - 1: starts; n_rays .. 2 n_rays - 1: ends
    a.n_rows = (int)rows;
    a.qpart = qpart;
    a.Z = Z;
    a.out_by_walker = 0;
    launch_lik_f64_z(a, s);
    note_launch();
    k_seg_q<<<warp_blocks((int64_t)n_rays * K), 256, 0, s>>>(n_rays, d, K, Z, Q);
    note_launch();
    k_seg_coarse<<<(unsigned)(((int64_t)n_rays * n_steps + 255) / 256), 256, 0, s>>>(n_rays, n_steps, K, pv.a, Q,
                                                                                    ell_coarse);
    if (n_ref > 0) {
        note_launch();
        k_seg_refine<<<(n_rays + 127) / 128, 128, 0, s>>>(n_rays, n_steps, n_ref, K, delta, pv.a, Q, ell_coarse, cdf,
                                                          t_ref, ell_ref);
    }
}

}  // namespace sb
