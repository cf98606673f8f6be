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
// ------------------------------------------------------------------ few points (GEMV shape)
// For a handful of points (the Laplace stage's candidates) a 64-row GEMM tile
// does 64 rows of FP64 work for each real row. These kernels spread the work
// over (column block, component, point block) instead, with the same outputs,
// layouts and a fixed summation order.
constexpr int FEW_CB = 8;  // points per CTA

// z_k[j] for the 64 columns j of one tile, one component and CB points: thread
// (column, row group of 4) accumulates rows i = i0 + rg, i0 + rg + 4, ... of
// L_k (coalesced row segments), then the four row groups are summed in a
// fixed order.
struct FewZShared {
    double dl[FEW_CB][64];  // delta = x - mu_k for 64 rows i of the current chunk
    double part[4][FEW_CB][64];
    double red[FEW_CB][2];
    int s_src[FEW_CB], s_out[FEW_CB];
};

template <int CB>
__device__ __forceinline__ void few_z_body(const LikF64Args &a, int jt, int k, int c0, FewZShared &sm) {
    const int d = a.d, K = a.K, nJT = (d + 63) / 64, j0 = jt * 64;
    const int tx = threadIdx.x & 63, rg = threadIdx.x >> 6;
    auto &dl = sm.dl;
    auto &part = sm.part;
    auto &red = sm.red;
    auto &s_src = sm.s_src;
    auto &s_out = sm.s_out;
    if (threadIdx.x < CB) {
        const int n = c0 + threadIdx.x;
        const int w = a.rows ? a.rows[n] : n;
        s_src[threadIdx.x] = w;
        s_out[threadIdx.x] = a.out_by_walker ? w : n;
    }
    __syncthreads();
    const double *Lk = a.L + (size_t)k * d * d;
    const double *mk = a.mu + (size_t)k * d;
    const int j = j0 + tx;
    double acc[CB];
#pragma unroll
    for (int c = 0; c < CB; ++c) acc[c] = 0.0;
    for (int i0 = j0; i0 < d; i0 += 64) {
        for (int e = threadIdx.x; e < CB * 64; e += 256) {
            const int c = e >> 6, ii = e & 63, i = i0 + ii;
            dl[c][ii] = i < d ? sub_rn(a.X[(size_t)s_src[c] * d + i], mk[i]) : 0.0;
        }
        __syncthreads();
        const int imax = min(64, d - i0);
        for (int ii = rg; ii < imax; ii += 4) {
            const int ig = i0 + ii;
            const double l = (j < d && j <= ig) ? Lk[(size_t)ig * d + j] : 0.0;
#pragma unroll
            for (int c = 0; c < CB; ++c) acc[c] = fma(dl[c][ii], l, acc[c]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int c = 0; c < CB; ++c) part[rg][c][tx] = acc[c];
    __syncthreads();
    if (rg == 0) {
        // |z|^2 over the 64 columns: warp shuffles, then the two warps through shared memory
#pragma unroll
        for (int c = 0; c < CB; ++c) {
            const double z = ((part[0][c][tx] + part[1][c][tx]) + part[2][c][tx]) + part[3][c][tx];
            acc[c] = z;
            double q = (j < d) ? z * z : 0.0;
            q = warp_sum(q);
            if ((tx & 31) == 0) red[c][tx >> 5] = q;
        }
        asm volatile("bar.sync 1, 64;" ::: "memory");  // the two warps of row group 0
        if (tx < CB) a.qpart[((size_t)s_out[tx] * K + k) * nJT + jt] = red[tx][0] + red[tx][1];
        if (a.Z && j < d)
#pragma unroll
            for (int c = 0; c < CB; ++c) a.Z[((size_t)s_out[c] * K + k) * d + j] = acc[c];
    }
}

__global__ void __launch_bounds__(256) k_few_z(LikF64Args a) {
    __shared__ FewZShared sm;
    const int n_rows = rows_of(a);
    const int c0 = blockIdx.z * FEW_CB;
    if (c0 >= n_rows) return;
    switch (min(FEW_CB, n_rows - c0)) {  // the live point count of this CTA (device-side)
        case 1: few_z_body<1>(a, blockIdx.x, blockIdx.y, c0, sm); break;
        case 2: few_z_body<2>(a, blockIdx.x, blockIdx.y, c0, sm); break;
        case 3: few_z_body<3>(a, blockIdx.x, blockIdx.y, c0, sm); break;
        case 4: few_z_body<4>(a, blockIdx.x, blockIdx.y, c0, sm); break;
        case 5: few_z_body<5>(a, blockIdx.x, blockIdx.y, c0, sm); break;
        case 6: few_z_body<6>(a, blockIdx.x, blockIdx.y, c0, sm); break;
        case 7: few_z_body<7>(a, blockIdx.x, blockIdx.y, c0, sm); break;
        default: few_z_body<8>(a, blockIdx.x, blockIdx.y, c0, sm); break;
    }
}

// grad: out[n][i] = sign * sum_k sum_{j<=i} r_nk z_nk[j] L_k[i][j]; warp per row i,
// CB points; components with r == 0 at every point of the CTA are skipped.
template <int CB>
__device__ __forceinline__ void few_g_body(const LikF64Args &a, int c0, int *s_out) {
    const int d = a.d, K = a.K;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int i = blockIdx.x * 8 + wid;
    if (threadIdx.x < CB) {
        const int n = c0 + threadIdx.x;
        s_out[threadIdx.x] = a.out_by_walker ? (a.rows ? a.rows[n] : n) : n;
    }
    __syncthreads();
    if (i >= d) return;
    double acc[CB];
#pragma unroll
    for (int c = 0; c < CB; ++c) acc[c] = 0.0;
    for (int k = 0; k < K; ++k) {
        double rk[CB];
        const double *zk[CB];
        bool any = false;
#pragma unroll
        for (int c = 0; c < CB; ++c) {
            const int o = s_out[c];
            rk[c] = a.R[(size_t)o * K + k];
            zk[c] = a.Z + ((size_t)o * K + k) * d;
            any = any || rk[c] != 0.0;
        }
        if (!any) continue;
        const double *Lrow = a.L + (size_t)k * d * d + (size_t)i * d;
        for (int j = lane; j <= i; j += 32) {
            const double l = Lrow[j];
#pragma unroll
            for (int c = 0; c < CB; ++c) acc[c] = fma(rk[c] * zk[c][j], l, acc[c]);
        }
    }
#pragma unroll
    for (int c = 0; c < CB; ++c) {
        const double v = warp_sum(acc[c]);
        if (lane == 0) a.G[(size_t)s_out[c] * d + i] = a.grad_sign * v;
    }
}

__global__ void __launch_bounds__(256) k_few_g(LikF64Args a) {
    __shared__ int s_out[FEW_CB];
    const int n_rows = rows_of(a);
    const int c0 = blockIdx.y * FEW_CB;
    if (c0 >= n_rows) return;
    switch (min(FEW_CB, n_rows - c0)) {
        case 1: few_g_body<1>(a, c0, s_out); break;
        case 2: few_g_body<2>(a, c0, s_out); break;
        case 3: few_g_body<3>(a, c0, s_out); break;
        case 4: few_g_body<4>(a, c0, s_out); break;
        case 5: few_g_body<5>(a, c0, s_out); break;
        case 6: few_g_body<6>(a, c0, s_out); break;
        case 7: few_g_body<7>(a, c0, s_out); break;
        default: few_g_body<8>(a, c0, s_out); break;
    }
}

}  // namespace

size_t lik_f64_qpart_elems(int d, int K, int rows) { return (size_t)rows * K * ((d + BN - 1) / BN); }

void launch_lik_f64_z(const LikF64Args &a, cudaStream_t s) {
    if (a.n_rows <= 0) return;
    dim3 g((a.n_rows + BM - 1) / BM, (a.d + BN - 1) / BN, a.K);
    ProfScope prof(PROF_F64_Z, s);
    note_launch();
    k_zgemm_f64<SRC_GATHER, true><<<g, 256, 0, s>>>(a);
}

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

namespace sb {
void launch_lik_f64_few(const LikF64Args &a, bool want_grad, cudaStream_t s) {
    if (a.n_rows <= 0) return;
    const int nJT = (a.d + 63) / 64;
    const int cb = (a.n_rows + 7) / 8;
    {
        ProfScope prof(PROF_F64_Z, s);
        note_launch();
        k_few_z<<<dim3(nJT, a.K, cb), 256, 0, s>>>(a);
    }
    note_launch();
    k_lse_f64<<<(a.n_rows + 255) / 256, 256, 0, s>>>(a);
    if (want_grad) {
        ProfScope prof(PROF_F64_GRAD, s);
        note_launch();
        k_few_g<<<dim3((a.d + 7) / 8, cb), 256, 0, s>>>(a);
    }
}
}  // namespace sb
