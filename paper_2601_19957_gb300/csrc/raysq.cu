// raysq.cu -- sunburst ray likelihoods from three scalars per (ray, component).
//
// Along ray r, x(t) = c + tau u_r with tau = t t_exit,r, and for every
// component z_k(x(t)) = z_k(c) + tau w_rk with w_rk = L_k^T u_r, so
//     |z_k(x(t))|^2 = q0_k + 2 tau q1_rk + tau^2 q2_rk,
//     q0_k = |z_k(c)|^2, q1_rk = z_k(c) . w_rk, q2_rk = |w_rk|^2,
// and l at every sample of the ray is LSE_k (a_k - |z_k|^2 / 2). One
// triangular GEMM of the directions by each L_k (n_rays K d(d+1)/2
// multiply-adds) replaces one per sample (n_steps times more). The scalars
// are combined in FP64. Two forms of the GEMM:
//   FP64: the batched z GEMM over the rows c and c + u_r (w = z(c + u) - z(c));
//   FP32: a SIMT triangular GEMM of u_r (rounded to FP32) by L_k (rounded to
//         FP32) with FP32 accumulation, whose epilogue reduces z_k(c) . w and
//         |w|^2 over each 128-column tile (the partials are summed in FP64).
// The terms are large and cancel near a mode (|z(c)|^2 ~ 1e5 at d = 1024), so
// the FP32 form's error is ~1e-7 of them: sub-nat at such samples.
#include "sb_raysq.cuh"

namespace sb {

namespace {

constexpr int QB_M = 128, QB_N = 128, QB_K = 8;

// t_exit of each ray from the centre (warp per ray): min_i half_i / |u_i|
__global__ void __launch_bounds__(256) k_rq_texit(int n_rays, int d, const double *u, const double *half,
                                                  double *texit) {
    const int lane = threadIdx.x & 31;
    const int r = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    if (r >= n_rays) return;
    const double t = warp_exit_min(lane, d, u + (size_t)r * d, half);
    if (lane == 0) texit[r] = t;
}

// rows 0 = c, 1 + r = c + u_r (FP64 form)
__global__ void __launch_bounds__(256) k_rq_rows(int n_rays, int d, const double *c, const double *u, double *X) {
    const int64_t total = (int64_t)(n_rays + 1) * d;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = e / d;
        const int i = (int)(e - row * d);
        X[e] = row == 0 ? c[i] : add_rn(c[i], u[(row - 1) * d + i]);
    }
}

// FP64 form: q1, q2 from z(c + u_r) - z(c) (warp per (ray, component)); q0 from z(c)
__global__ void __launch_bounds__(256) k_rq_q64(int n_rays, int d, int K, const double *Z, double *q0, double *q1,
                                                double *q2) {
    const int lane = threadIdx.x & 31;
    const int e = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    if (e >= n_rays * K) return;
    const int r = e / K, k = e - r * K;
    const double *zc = Z + (size_t)k * d;
    const double *zu = Z + ((size_t)(1 + r) * K + k) * d;
    double a = 0.0, b = 0.0, s0 = 0.0;
    for (int j = lane; j < d; j += 32) {
        const double w = zu[j] - zc[j];
        a += zc[j] * w;
        b += w * w;
        s0 += zc[j] * zc[j];
    }
    a = warp_sum(a);
    b = warp_sum(b);
    s0 = warp_sum(s0);
    if (lane == 0) {
        q1[e] = a;
        q2[e] = b;
        if (r == 0) q0[k] = s0;
    }
}

__global__ void __launch_bounds__(256) k_rq_to_f32(int64_t n, const double *a, float *b) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        b[e] = (float)a[e];
}

// FP32 form: per (128 rays, 128 columns j, component k) tile, w[r][j] = sum_{i >= j} L_k[i][j] u_r[i]
// (8 x 8 outputs per thread, rows ty + 16 a, columns tx + 16 b), then partials of z_k(c) . w and
// |w|^2 over the tile's columns.
__global__ void __launch_bounds__(256) k_rq_gemm_f32(int n_rays, int d, int K, const float *Uf, const float *Lf,
                                                     const double *zc, float *p1, float *p2) {
    const int r0 = blockIdx.x * QB_M;
    const int jt = blockIdx.y, j0 = jt * QB_N, k = blockIdx.z;
    const int nJT = (d + QB_N - 1) / QB_N;
    __shared__ float As[QB_K][QB_M + 4];
    __shared__ float Bs[QB_K][QB_N];
    __shared__ float Zc[QB_N];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const float *Lk = Lf + (size_t)k * d * d;
    if (tid < QB_N) Zc[tid] = j0 + tid < d ? (float)zc[(size_t)k * d + j0 + tid] : 0.0f;
    float acc[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = 0.0f;
    for (int i0 = (j0 / QB_K) * QB_K; i0 < d; i0 += QB_K) {
        // A: 128 rays x 8 i (u), B: 8 i x 128 j (L_k rows i, columns j; zero above the diagonal)
        for (int e = tid; e < QB_M * QB_K; e += 256) {
            const int rr = e / QB_K, ii = e - rr * QB_K;
            const int r = r0 + rr, i = i0 + ii;
            As[ii][rr] = (r < n_rays && i < d) ? Uf[(size_t)r * d + i] : 0.0f;
        }
        for (int e = tid; e < QB_K * QB_N; e += 256) {
            const int ii = e / QB_N, jj = e - ii * QB_N;
            const int i = i0 + ii, j = j0 + jj;
            Bs[ii][jj] = (i < d && j < d && j <= i) ? Lk[(size_t)i * d + j] : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < QB_K; ++kk) {
            float av[8], bv[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) av[q] = As[kk][ty + 16 * q];
#pragma unroll
            for (int q = 0; q < 8; ++q) bv[q] = Bs[kk][tx + 16 * q];
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        const int r = r0 + ty + 16 * a;
        float s1 = 0.0f, s2 = 0.0f;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            const int jj = tx + 16 * b;
            s1 = fmaf(Zc[jj], acc[a][b], s1);
            s2 = fmaf(acc[a][b], acc[a][b], s2);
        }
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
            s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        }
        if (tx == 0 && r < n_rays) {
            p1[((size_t)r * K + k) * nJT + jt] = s1;
            p2[((size_t)r * K + k) * nJT + jt] = s2;
        }
    }
}

// FP32 form: sum the tile partials in FP64; q0 from z(c) in FP64
__global__ void __launch_bounds__(256) k_rq_qsum(int n_rays, int d, int K, const float *p1, const float *p2,
                                                 const double *zc, double *q0, double *q1, double *q2) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int nJT = (d + QB_N - 1) / QB_N;
    if (e < K) {
        double s = 0.0;
        for (int j = 0; j < d; ++j) s += zc[(size_t)e * d + j] * zc[(size_t)e * d + j];
        q0[e] = s;
    }
    if (e >= n_rays * K) return;
    double a = 0.0, b = 0.0;
    for (int t = 0; t < nJT; ++t) {
        a += (double)p1[(size_t)e * nJT + t];
        b += (double)p2[(size_t)e * nJT + t];
    }
    q1[e] = a;
    q2[e] = b;
}

// l at sample j of ray r: tau = ((j + 1) / n_steps) t_exit,r
__global__ void __launch_bounds__(256) k_rq_ell(int n_rays, int n_steps, int K, const double *a, const double *q0,
                                                const double *q1, const double *q2, const double *texit, double *ell) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)n_rays * n_steps) return;
    const int r = (int)(e / n_steps), j = (int)(e - (int64_t)r * n_steps);
    const double tau = mul_rn(div_rn((double)(j + 1), (double)n_steps), texit[r]);
    double m = -INFINITY;
    for (int k = 0; k < K; ++k) {
        const double zz = q0[k] + 2.0 * tau * q1[(size_t)r * K + k] + tau * tau * q2[(size_t)r * K + k];
        m = fmax(m, a[k] - 0.5 * zz);
    }
    double s = 0.0;
    for (int k = 0; k < K; ++k) {
        const double zz = q0[k] + 2.0 * tau * q1[(size_t)r * K + k] + tau * tau * q2[(size_t)r * K + k];
        s += exp(a[k] - 0.5 * zz - m);
    }
    ell[e] = m + log(s);
}

inline unsigned grid_for(int64_t n, int64_t cap = 65535) {
    int64_t b = (n + 255) / 256;
    return (unsigned)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace

size_t rayq_scratch_elems(int n_rays, int d, int K, int form) {
    size_t e = (size_t)n_rays + (size_t)K + 2 * (size_t)n_rays * K;  // texit, q0, q1, q2
    if (form == 0) {
        const size_t rows = (size_t)n_rays + 1;
        e += rows * d + rows * K * d + lik_f64_qpart_elems(d, K, (int)rows);  // X, Z, qpart
    } else {
        const int nJT = (d + QB_N - 1) / QB_N;
        e += (size_t)K * d;  // z(c)
        e += ((size_t)n_rays * d + (size_t)K * d * d + 2 * (size_t)n_rays * K * nJT + 1) / 2;  // floats
        e += lik_f64_qpart_elems(d, K, 1) + 4;  // + alignment slack of the qpart block
    }
    return e;
}

void launch_ray_texit(const ProbView &pv, const double *u, int n_rays, double *texit, cudaStream_t s) {
    note_launch();
    k_rq_texit<<<(unsigned)(((int64_t)n_rays * 32 + 255) / 256), 256, 0, s>>>(n_rays, pv.d, u, pv.half, texit);
}

void launch_ray_loglik_quad(const ProbView &pv, int form, const double *u, int n_rays, int n_steps, double *scratch,
                            double *ell, cudaStream_t s) {
    const int d = pv.d, K = pv.K;
    double *texit = scratch;
    double *q0 = texit + n_rays;
    double *q1 = q0 + K;
    double *q2 = q1 + (size_t)n_rays * K;
    double *rest = q2 + (size_t)n_rays * K;
    note_launch();
    k_rq_texit<<<(unsigned)(((int64_t)n_rays * 32 + 255) / 256), 256, 0, s>>>(n_rays, d, u, pv.half, texit);
    LikF64Args la{};
    la.d = d;
    la.K = K;
    la.mu = pv.mu;
    la.L = pv.L;
    la.a = pv.a;
    la.c = pv.c;
    la.out_by_walker = 0;
    if (form == 0) {
        const int rows = n_rays + 1;
        double *X = rest;
        double *Z = X + (size_t)rows * d;
        double *qpart = Z + (size_t)rows * K * d;
        note_launch();
        k_rq_rows<<<grid_for((int64_t)rows * d), 256, 0, s>>>(n_rays, d, pv.c, u, X);
        la.X = X;
        la.n_rows = rows;
        la.Z = Z;
        la.qpart = qpart;
        launch_lik_f64_z(la, s);
        note_launch();
        k_rq_q64<<<(unsigned)(((int64_t)n_rays * K * 32 + 255) / 256), 256, 0, s>>>(n_rays, d, K, Z, q0, q1, q2);
    } else {
        const int nJT = (d + QB_N - 1) / QB_N;
        double *zc = rest;
        float *Uf = (float *)(zc + (size_t)K * d);
        float *Lf = Uf + (size_t)n_rays * d;
        float *p1 = Lf + (size_t)K * d * d;
        float *p2 = p1 + (size_t)n_rays * K * nJT;
        double *qpart = (double *)(((uintptr_t)(p2 + (size_t)n_rays * K * nJT) + 15) & ~(uintptr_t)15);
        // z_k(c) in FP64 (one row)
        la.X = pv.c;
        la.n_rows = 1;
        la.Z = zc;
        la.qpart = qpart;
        launch_lik_f64_z(la, s);
        note_launch();
        k_rq_to_f32<<<grid_for((int64_t)n_rays * d), 256, 0, s>>>((int64_t)n_rays * d, u, Uf);
        note_launch();
        k_rq_to_f32<<<grid_for((int64_t)K * d * d), 256, 0, s>>>((int64_t)K * d * d, pv.L, Lf);
        note_launch();
        k_rq_gemm_f32<<<dim3((n_rays + QB_M - 1) / QB_M, nJT, K), 256, 0, s>>>(n_rays, d, K, Uf, Lf, zc, p1, p2);
        note_launch();
        k_rq_qsum<<<(unsigned)(((int64_t)n_rays * K + 255) / 256 > 0 ? ((int64_t)n_rays * K + 255) / 256 : 1), 256, 0,
                    s>>>(n_rays, d, K, p1, p2, zc, q0, q1, q2);
    }
    note_launch();
    k_rq_ell<<<(unsigned)(((int64_t)n_rays * n_steps + 255) / 256), 256, 0, s>>>(n_rays, n_steps, K, pv.a, q0, q1, q2,
                                                                                texit, ell);
}

}  // namespace sb
