// lik_f64.cu -- FP64 batched log-likelihood and gradient on CUDA cores.
//
// For a batch of points x_n (gathered walker rows, or ray samples generated on
// the fly) and components k:
//   z_nk = L_k^T (x_n - mu_k)                      (a triangular GEMM per k)
//   e_nk = a_k - |z_nk|^2 / 2,  l_n = LSE_k e_nk,  r_nk = softmax_k e_nk
//   grad l_n = -sum_k r_nk L_k z_nk                 (a second triangular GEMM)
// The Gaussian-mixture likelihood is the paper's problem statement (Sec. 3.2);
// the analytic gradient replaces its finite differences (App. A.4.1).
//
// Tiling: 64 points x 64 output coordinates per CTA, reduction chunks of 16,
// 256 threads with a 4x4 register tile each. Only the triangle that L_k
// occupies is visited: the z GEMM for output column block [j0, j0+64) reads
// rows i >= j0 of L_k; the gradient GEMM for output block [i0, i0+64) reads
// columns j < i0 + 64. FP64 throughput bounds this path; it exists as the
// exact reference path and the plain-FP64 comparator of the tensor-core path.
#include "sb_internal.cuh"

namespace sb {

namespace {
constexpr int BM = 64, BN = 64, BK = 16;

enum { SRC_GATHER = 0, SRC_RAYS = 1 };

__device__ __forceinline__ int rows_of(const LikF64Args &a) { return a.n_rows_dev ? *a.n_rows_dev : a.n_rows; }

template <int SRC, bool STORE_Z>
__global__ void __launch_bounds__(256) k_zgemm_f64(LikF64Args a) {
    const int n_rows = rows_of(a);
    const int n0 = blockIdx.x * BM;
    if (n0 >= n_rows) return;
    const int jt = blockIdx.y, j0 = jt * BN, k = blockIdx.z;
    const int d = a.d, K = a.K, nJT = (d + BN - 1) / BN;
    const double *Lk = a.L + (size_t)k * d * d;
    const double *mk = a.mu + (size_t)k * d;

    __shared__ double As[BK][BM + 1];
    __shared__ double Bs[BK][BN];
    __shared__ const double *s_src[BM];
    __shared__ double s_scale[BM];
    __shared__ int s_out[BM];

    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    if (tid < BM) {
        const int n = n0 + tid;
        const bool valid = n < n_rows;
        if (SRC == SRC_GATHER) {
            const int w = valid ? (a.rows ? a.rows[n] : n) : 0;
            s_src[tid] = a.X + (size_t)w * d;
            s_out[tid] = valid ? (a.out_by_walker ? w : n) : -1;
            s_scale[tid] = 0.0;
        } else {
            const int64_t flat = a.flat0 + n;
            const int r = valid ? (int)(flat / a.n_steps) : 0;
            const int j = valid ? (int)(flat % a.n_steps) : 0;
            s_src[tid] = a.u + (size_t)r * d;
            // t_j * t_exit with t_j = (j+1)/n_steps (ray grid reading, Sec. 3.5.2)
            s_scale[tid] = valid ? mul_rn(div_rn((double)(j + 1), (double)a.n_steps), a.texit[r]) : 0.0;
            s_out[tid] = valid ? n : -1;
        }
    }
    __syncthreads();

    double acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = 0.0;

    for (int i0 = (j0 / BK) * BK; i0 < d; i0 += BK) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + 256 * q;
            const int row = e >> 4, kk = e & 15, i = i0 + kk;
            double v = 0.0;
            if (s_out[row] >= 0 && i < d) {
                double x;
                if (SRC == SRC_GATHER) {
                    x = s_src[row][i];
                } else {
                    x = add_rn(a.c[i], mul_rn(s_scale[row], s_src[row][i]));
                }
                v = sub_rn(x, mk[i]);
            }
            As[kk][row] = v;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int e = tid + 256 * q;
            const int kk = e >> 6, col = e & 63, i = i0 + kk, j = j0 + col;
            Bs[kk][col] = (i < d && j < d && j <= i) ? Lk[(size_t)i * d + j] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            double av[4], bv[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) av[r] = As[kk][ty + 16 * r];
#pragma unroll
            for (int c = 0; c < 4; ++c) bv[c] = Bs[kk][tx + 16 * c];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = fma(av[r], bv[c], acc[r][c]);
        }
        __syncthreads();
    }

#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int row = ty + 16 * r;
        const int out = s_out[row];
        double q = 0.0;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int j = j0 + tx + 16 * c;
            if (j < d) q += acc[r][c] * acc[r][c];
        }
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
        if (out >= 0) {
            if (tx == 0) a.qpart[((size_t)out * K + k) * nJT + jt] = q;
            if (STORE_Z) {
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const int j = j0 + tx + 16 * c;
                    if (j < d) a.Z[((size_t)out * K + k) * d + j] = acc[r][c];
                }
            }
        }
    }
}

// Per point: l = LSE_k (a_k - q_k/2) and the responsibilities r_k.
__global__ void __launch_bounds__(256) k_lse_f64(LikF64Args a) {
    const int n_rows = rows_of(a);
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= n_rows) return;
    const int K = a.K, nJT = (a.d + BN - 1) / BN;
    const int out = a.out_by_walker ? (a.rows ? a.rows[n] : n) : n;
    double e[kMaxK];
    double emax = -INFINITY;
    for (int k = 0; k < K; ++k) {
        const double *qp = a.qpart + ((size_t)out * K + k) * nJT;
        double q = 0.0;
        for (int t = 0; t < nJT; ++t) q += qp[t];
        e[k] = a.a[k] - 0.5 * q;
        emax = fmax(emax, e[k]);
    }
    double ssum = 0.0;
    for (int k = 0; k < K; ++k) ssum += exp(e[k] - emax);
    const double ell = emax + log(ssum);
    a.ell[out] = a.ell_sign * ell;
    if (a.R)
        for (int k = 0; k < K; ++k) a.R[(size_t)out * K + k] = exp(e[k] - emax) / ssum;
}

// grad: out[n][i] = sign * sum_k sum_{j<=i} r_nk z_nk[j] L_k[i][j]  (= -sign * grad l)
__global__ void __launch_bounds__(256) k_ggemm_f64(LikF64Args a) {
    const int n_rows = rows_of(a);
    const int n0 = blockIdx.x * BM;
    if (n0 >= n_rows) return;
    const int i0 = blockIdx.y * BN;
    const int d = a.d, K = a.K;

    __shared__ double As[BK][BM + 1];
    __shared__ double Bs[BK][BN + 1];
    __shared__ int s_out[BM];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    if (tid < BM) {
        const int n = n0 + tid;
        s_out[tid] = n < n_rows ? (a.out_by_walker ? (a.rows ? a.rows[n] : n) : n) : -1;
    }
    __syncthreads();

    double acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = 0.0;

    const int jmax = min(d, i0 + BN);
    for (int k = 0; k < K; ++k) {
        const double *Lk = a.L + (size_t)k * d * d;
        for (int j0 = 0; j0 < jmax; j0 += BK) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int e = tid + 256 * q;
                const int row = e >> 4, kk = e & 15, j = j0 + kk;
                const int out = s_out[row];
                double v = 0.0;
                if (out >= 0 && j < d) v = a.R[(size_t)out * K + k] * a.Z[((size_t)out * K + k) * d + j];
                As[kk][row] = v;
            }
            {
                // 64 columns (rows i of L_k) x 16 j: each thread loads 4 consecutive j of one row
                const int col = tid >> 2, kq = (tid & 3) * 4;
                const int i = i0 + col;
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int j = j0 + kq + t;
                    Bs[kq + t][col] = (i < d && j < d && j <= i) ? Lk[(size_t)i * d + j] : 0.0;
                }
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < BK; ++kk) {
                double av[4], bv[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) av[r] = As[kk][ty + 16 * r];
#pragma unroll
                for (int c = 0; c < 4; ++c) bv[c] = Bs[kk][tx + 16 * c];
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[r][c] = fma(av[r], bv[c], acc[r][c]);
            }
            __syncthreads();
        }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int out = s_out[ty + 16 * r];
        if (out < 0) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int i = i0 + tx + 16 * c;
            if (i < d) a.G[(size_t)out * d + i] = a.grad_sign * acc[r][c];
        }
    }
}
}  // namespace

size_t lik_f64_qpart_elems(int d, int K, int rows) { return (size_t)rows * K * ((d + BN - 1) / BN); }

void launch_lik_f64_rays(const LikF64Args &a, cudaStream_t s) {
    if (a.n_rows <= 0) return;
    dim3 g((a.n_rows + BM - 1) / BM, (a.d + BN - 1) / BN, a.K);
    {
        ProfScope prof(PROF_F64_Z, s);
        note_launch();
        k_zgemm_f64<SRC_RAYS, false><<<g, 256, 0, s>>>(a);
    }
    note_launch();
    k_lse_f64<<<(a.n_rows + 255) / 256, 256, 0, s>>>(a);
}

void launch_lik_f64_points(const LikF64Args &a, bool want_grad, cudaStream_t s) {
    if (a.n_rows <= 0) return;
    dim3 g((a.n_rows + BM - 1) / BM, (a.d + BN - 1) / BN, a.K);
    if (want_grad) {
        {
            ProfScope prof(PROF_F64_Z, s);
            note_launch();
            k_zgemm_f64<SRC_GATHER, true><<<g, 256, 0, s>>>(a);
        }
        note_launch();
        k_lse_f64<<<(a.n_rows + 255) / 256, 256, 0, s>>>(a);
        dim3 g2((a.n_rows + BM - 1) / BM, (a.d + BN - 1) / BN);
        {
            ProfScope prof(PROF_F64_GRAD, s);
            note_launch();
            k_ggemm_f64<<<g2, 256, 0, s>>>(a);
        }
    } else {
        {
            ProfScope prof(PROF_F64_Z, s);
            note_launch();
            k_zgemm_f64<SRC_GATHER, false><<<g, 256, 0, s>>>(a);
        }
        note_launch();
        k_lse_f64<<<(a.n_rows + 255) / 256, 256, 0, s>>>(a);
    }
}

}  // namespace sb
