// adjoint.cu -- FP64 adjoint of log Z with respect to the component means and
// precision Cholesky factors (mu_k, L_k), for torch.autograd.
//
// log Z = LSE_m log Z_m - log V with log Z_m = l(x*_m) + (d/2) log 2pi - 1/2 log det H_m
// (Sec. 3.7.1, App. A.3, A.8) and x*_m a stationary point of l. With
// pi_m = softmax_m log Z_m and W = H^-1 at x*:
//
//   d log Z_m / d phi = d/dphi [ l - 1/2 log det H - 1/2 v^T grad l ]   (x = x*, v held fixed)
//   v = W t,  t = grad_x log det H = (tr(W dH/dx_i))_i
//
// The last term is the implicit shift of the mode, dx*/dphi = W d(grad l)/dphi,
// which moves log det H (l itself is stationary). Reverse-mode through the
// mixture pieces at x (delta_k = x - mu_k, z_k = L_k^T delta_k, r = softmax(e),
// g_k = -L_k z_k, gbar = sum r_k g_k, H = sum_k r_k (P_k - g_k g_k^T) + gbar gbar^T):
//
//   c       = -W gbar - v/2
//   beta_k  = -1/2 [tr(W P_k) - g_k^T W g_k] + c^T g_k
//   eps_k   = r_k + r_k (beta_k - sum_j r_j beta_j)                       (adjoint of e_k)
//   gam_k   = r_k (W g_k + c)                                             (adjoint of g_k)
//   dmu_k   = -eps_k g_k + P_k gam_k
//   dL_k    = lower[ eps_k (diag(1/L_ii) - delta_k z_k^T) - gam_k z_k^T - delta_k (L_k^T gam_k)^T - r_k W L_k ]
//
// and t from the same reverse pass applied to log det H alone:
//   beta'_k = tr(W P_k) - g_k^T W g_k + 2 gbar^T W g_k,  eps'_k = r_k (beta'_k - sum_j r_j beta'_j)
//   gam'_k  = 2 r_k W (gbar - g_k),  t = sum_k (eps'_k g_k - P_k gam'_k).
// tr(W P_k) = <W L_k, L_k>_F. Components with r_k == 0 contribute exactly zero
// and are skipped. H is recomputed at every mode (not stored by the forward),
// factored H = C C^T, and W is applied through triangular solves: W B =
// C^-T (C^-1 B) for the d right-hand sides of L_k and for vectors. At a one-hot
// mode (r_k = 1, the other r exactly 0) H = P_k and C = L_k, so W L_k = L_k^-T:
// tr(W P_k) = d and lower[W L_k] = diag(1 / L_ii), with no d x d solve. Products
// with P_k are formed as L_k (L_k^T v); P_k itself is built only for the Hessian
// of a mode that is not one-hot.
#include "sb_adjoint.cuh"

namespace sb {

namespace {

constexpr int TB = 32;  // triangular-solve row block

// ------------------------------------------------------------------ blocked TRSM, row-major B [d][n]
// Right-looking: once row block I of X is solved, every later row block J takes
// its update B_J -= A_JI X_I in one launch over (J, 64-column tile), so a launch
// has up to (row blocks left) x n / 64 CTAs. Lower (X = C^-1 B): A_JI = C_JI for
// J > I. Upper (X = C^-T B, row blocks in reverse): A_JI = (C_IJ)^T for J < I.
__global__ void __launch_bounds__(256) k_trsm_right(int d, int n, int I, bool upper, const double *C, double *B) {
    const int c0 = blockIdx.x * 64;
    const int J = upper ? (int)blockIdx.y : I + 1 + (int)blockIdx.y;
    const int rJ = J * TB, rI = I * TB;
    __shared__ double As[TB][TB + 1];
    __shared__ double Xs[TB][64 + 1];
    const int tid = threadIdx.x, tc = tid & 63, tr = tid >> 6;  // 4 row groups x 64 columns
    for (int e = tid; e < TB * TB; e += 256) {
        const int i = e / TB, k = e % TB;
        const int gi = rJ + i, gk = rI + k;
        double v = 0.0;
        if (gi < d && gk < d) v = upper ? C[(size_t)gk * d + gi] : C[(size_t)gi * d + gk];
        As[i][k] = v;
    }
    for (int e = tid; e < TB * 64; e += 256) {
        const int k = e / 64, c = e % 64;
        const int gk = rI + k, gc = c0 + c;
        Xs[k][c] = (gk < d && gc < n) ? B[(size_t)gk * n + gc] : 0.0;
    }
    __syncthreads();
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int k = 0; k < TB; ++k) {
        const double x = Xs[k][tc];
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[q] = fma(As[tr + 4 * q][k], x, acc[q]);
    }
    const int gc = c0 + tc;
    if (gc < n)
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int gi = rJ + tr + 4 * q;
            if (gi < d) B[(size_t)gi * n + gc] -= acc[q];
        }
}

// Diagonal block solve for 32 columns per CTA: the 32 x 32 block of B is staged
// in shared memory, each warp solves four columns with lanes over rows (one
// shuffle per unknown, multiplication by the diagonal's reciprocals).
__global__ void __launch_bounds__(256) k_trsm_diag(int d, int n, int I, bool upper, const double *C, double *B) {
    __shared__ double Cs[TB][TB + 1];
    __shared__ double Bs[TB][TB + 1];
    __shared__ double inv[TB];
    const int r0 = I * TB, c0 = blockIdx.x * TB;
    const int rows = min(TB, d - r0);
    for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) {
        const int i = e / TB, k = e % TB;
        const int gi = r0 + i, gk = r0 + k;
        double v = (i == k) ? 1.0 : 0.0;
        if (gi < d && gk < d) v = upper ? C[(size_t)gk * d + gi] : C[(size_t)gi * d + gk];
        Cs[i][k] = v;
        Bs[i][k] = (i < rows && c0 + k < n) ? B[(size_t)(r0 + i) * n + c0 + k] : 0.0;
    }
    __syncthreads();
    if (threadIdx.x < TB) inv[threadIdx.x] = 1.0 / Cs[threadIdx.x][threadIdx.x];
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int col = wid; col < TB; col += (int)(blockDim.x >> 5)) {
        double b = Bs[lane][col];
        if (!upper) {
            for (int i = 0; i < TB; ++i) {
                const double xi = __shfl_sync(0xffffffffu, b, i) * inv[i];
                if (lane == i) b = xi;
                else if (lane > i) b -= Cs[lane][i] * xi;
            }
        } else {
            for (int i = TB - 1; i >= 0; --i) {
                const double xi = __shfl_sync(0xffffffffu, b, i) * inv[i];
                if (lane == i) b = xi;
                else if (lane < i) b -= Cs[lane][i] * xi;
            }
        }
        Bs[lane][col] = b;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < TB * TB; e += blockDim.x) {
        const int i = e / TB, k = e % TB;
        if (i < rows && c0 + k < n) B[(size_t)(r0 + i) * n + c0 + k] = Bs[i][k];
    }
}

// W B = C^-T C^-1 B in place (B row-major [d][n]).
void apply_W(int d, int n, const double *C, double *B, cudaStream_t s) {
    const int nb = (d + TB - 1) / TB;
    const int gc = (n + 63) / 64, gd = (n + TB - 1) / TB;
    for (int I = 0; I < nb; ++I) {
        note_launch();
        k_trsm_diag<<<gd, 256, 0, s>>>(d, n, I, false, C, B);
        if (I < nb - 1) {
            note_launch();
            k_trsm_right<<<dim3(gc, nb - 1 - I), 256, 0, s>>>(d, n, I, false, C, B);
        }
    }
    for (int I = nb - 1; I >= 0; --I) {
        note_launch();
        k_trsm_diag<<<gd, 256, 0, s>>>(d, n, I, true, C, B);
        if (I > 0) {
            note_launch();
            k_trsm_right<<<dim3(gc, I), 256, 0, s>>>(d, n, I, true, C, B);
        }
    }
}

// ------------------------------------------------------------------ per-mode vector algebra
// Column vectors for the right-hand-side block V [d][nv] (row-major, so W acts on columns):
// columns 0..K-1 = g_k (active only, else 0), K = gbar.
__global__ void k_pack_rhs(int d, int K, const double *GK, const double *gbar, const double *R, double *V) {
    const int nv = K + 1;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < d * nv; e += gridDim.x * blockDim.x) {
        const int i = e / nv, c = e % nv;
        double v;
        if (c < K)
            v = R[c] != 0.0 ? GK[(size_t)c * d + i] : 0.0;
        else
            v = gbar[i];
        V[e] = v;
    }
}

// copy L_k (lower, zero above) into M [d][d]
__global__ void k_copy_lower(int d, const double *Lk, double *M) {
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < (size_t)d * d;
         e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / d), j = (int)(e % d);
        M[e] = j <= i ? Lk[e] : 0.0;
    }
}

template <typename T>
__device__ T block_sum256(T v, T *sh) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    T t = 0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += sh[q];
    __syncthreads();
    return t;
}

// tr(W P_k) = <W L_k, L_k>_F over the lower triangle (W L_k in M).
__global__ void __launch_bounds__(256) k_trace_WP(int d, const double *M, const double *Lk, double *out) {
    __shared__ double sh[8];
    double s = 0.0;
    for (size_t e = threadIdx.x; e < (size_t)d * d; e += blockDim.x) {
        const int i = (int)(e / d), j = (int)(e % d);
        if (j <= i) s += M[e] * Lk[e];
    }
    s = block_sum256(s, sh);
    if (threadIdx.x == 0) *out = s;
}

// One CTA: given WV (W applied to [g_0..g_{K-1}, gbar]) and tr(W P_k), form t (stage 0),
// or with Wt known form c, eps, gam (stage 1). Vectors of length d in global scratch.
__global__ void __launch_bounds__(256) k_adj_stage(int stage, int d, int K, const double *R, const double *GK,
                                                   const double *gbar, const double *WV, const double *trWP,
                                                   const double *PY, const double *Wt, double *t_out, double *eps,
                                                   double *gam, double *cvec) {
    __shared__ double sh[8];
    __shared__ double s_beta[kMaxK];
    const int nv = K + 1;
    // per active component: dot products g_k^T W g_k, gbar^T W g_k, c^T g_k
    for (int k = 0; k < K; ++k) {
        const double r = R[k];
        if (r == 0.0) {
            if (threadIdx.x == 0) s_beta[k] = 0.0;
            continue;
        }
        double a1 = 0.0, a2 = 0.0;
        for (int i = threadIdx.x; i < d; i += blockDim.x) {
            const double gk = GK[(size_t)k * d + i];
            const double wgk = WV[(size_t)i * nv + k];
            a1 += gk * wgk;                     // g_k^T W g_k
            if (stage == 0)
                a2 += gbar[i] * wgk;            // gbar^T W g_k
            else
                a2 += (-WV[(size_t)i * nv + K] - 0.5 * Wt[i]) * gk;  // c^T g_k
        }
        a1 = block_sum256(a1, sh);
        a2 = block_sum256(a2, sh);
        if (threadIdx.x == 0)
            s_beta[k] = stage == 0 ? (trWP[k] - a1 + 2.0 * a2) : (-0.5 * (trWP[k] - a1) + a2);
    }
    __syncthreads();
    double sb = 0.0;
    for (int k = 0; k < K; ++k) sb += R[k] * s_beta[k];
    if (stage == 0) {
        // t = sum_k eps'_k g_k - P_k gam'_k,  gam'_k = 2 r_k W (gbar - g_k)
        for (int i = threadIdx.x; i < d; i += blockDim.x) {
            double ti = 0.0;
            for (int k = 0; k < K; ++k) {
                const double r = R[k];
                if (r == 0.0) continue;
                const double e1 = r * (s_beta[k] - sb);
                ti += e1 * GK[(size_t)k * d + i];
                // (P_k gam'_k)_i = 2 r (P_k (W gbar - W g_k))_i, formed apart (PY)
                ti -= 2.0 * r * PY[(size_t)k * d + i];
            }
            t_out[i] = ti;
        }
    } else {
        if (threadIdx.x < K) {
            const int k = threadIdx.x;
            eps[k] = R[k] == 0.0 ? 0.0 : R[k] + R[k] * (s_beta[k] - sb);
        }
        for (int i = threadIdx.x; i < d; i += blockDim.x) {
            const double c = -WV[(size_t)i * nv + K] - 0.5 * Wt[i];
            cvec[i] = c;
            for (int k = 0; k < K; ++k) gam[(size_t)k * d + i] = R[k] == 0.0 ? 0.0 : R[k] * (WV[(size_t)i * nv + k] + c);
        }
    }
}

// dmu_k += pi (-eps_k g_k + P_k gam_k) for one component, P_k gam_k given (y).
__global__ void __launch_bounds__(256) k_adj_dmu(int d, int k, double pi, const double *eps, const double *GK,
                                                 const double *y, double *dmu) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= d) return;
    dmu[(size_t)k * d + i] += pi * (-eps[k] * GK[(size_t)k * d + i] + y[i]);
}

// v = W gbar - W g_k (columns K and k of WV [d][K + 1]).
__global__ void __launch_bounds__(256) k_adj_wdiff(int d, int K, int k, const double *WV, double *v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < d) v[i] = WV[(size_t)i * (K + 1) + K] - WV[(size_t)i * (K + 1) + k];
}

// y = L_k u (lower triangular), a warp per row: y_i = sum_{j <= i} L[i][j] u_j.
__global__ void __launch_bounds__(256) k_adj_Lu(int d, const double *Lk, const double *u, double *y) {
    const int lane = threadIdx.x & 31;
    const int i = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
    if (i >= d) return;
    double s = 0.0;
    for (int j = lane; j <= i; j += 32) s += Lk[(size_t)i * d + j] * u[j];
    s = warp_sum(s);
    if (lane == 0) y[i] = s;
}

// L^T gam for component k (u[j] = sum_i L[i][j] gam[i]).
__global__ void __launch_bounds__(256) k_adj_Ltg(int d, const double *Lk, const double *g, double *u) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= d) return;
    double s = 0.0;
    for (int i = j; i < d; ++i) s += Lk[(size_t)i * d + j] * g[i];
    u[j] = s;
}

// dL_k += pi lower[ eps (diag(1/L) - delta z^T) - gam z^T - delta u^T - r M ],  M = W L_k, u = L^T gam.
// M null: the one-hot case W = (L_k L_k^T)^-1, where W L_k = L_k^-T, whose lower
// triangle is diag(1 / L_ii).
__global__ void __launch_bounds__(256) k_adj_dL(int d, double pi, double r, double eps, const double *Lk,
                                                const double *x, const double *mu, const double *z, const double *gam,
                                                const double *u, const double *M, double *dL) {
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < (size_t)d * d;
         e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / d), j = (int)(e % d);
        if (j > i) continue;
        const double di = x[i] - mu[i];
        const double wl = M ? M[e] : (i == j ? 1.0 / Lk[e] : 0.0);
        double v = -eps * di * z[j] - gam[i] * z[j] - di * u[j] - r * wl;
        if (i == j) v += eps / Lk[e];
        dL[e] += pi * v;
    }
}

__global__ void k_set_f64(double *p, double v) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *p = v;
}

__global__ void k_softmax_pi(int n, const double *logZk, double g, double *pi) {
    if (threadIdx.x != 0) return;
    double mx = -INFINITY;
    for (int i = 0; i < n; ++i) mx = fmax(mx, logZk[i]);
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += exp(logZk[i] - mx);
    for (int i = 0; i < n; ++i) pi[i] = g * exp(logZk[i] - mx) / s;
}

}  // namespace

void adjoint_carve(Carver &cv, AdjWs &w, int d, int K) {
    const int nJT = (d + 63) / 64;
    w.P = cv.take<double>((size_t)K * d * d);
    w.H = cv.take<double>((size_t)d * d);
    w.M = cv.take<double>((size_t)K * d * d);
    w.Z = cv.take<double>((size_t)K * d);
    w.R = cv.take<double>((size_t)K);
    w.qpart = cv.take<double>((size_t)K * nJT);
    w.gbar = cv.take<double>(d);
    w.ell = cv.take<double>(1);
    w.GK = cv.take<double>((size_t)K * d);
    w.V = cv.take<double>((size_t)d * (K + 1));
    w.T = cv.take<double>(d);
    w.cvec = cv.take<double>(d);
    w.eps = cv.take<double>(K);
    w.gam = cv.take<double>((size_t)K * d);
    w.u = cv.take<double>(d);
    w.trWP = cv.take<double>(K);
    w.PY = cv.take<double>((size_t)K * d);
    w.y = cv.take<double>(d);
    w.pi = cv.take<double>(kMaxAdjModes);
    w.info = cv.take<int32_t>(1);
    w.one = cv.take<int32_t>(1);
    w.onehot = cv.take<int32_t>(1);
    w.bar = cv.take<uint32_t>(2);
}

sb_status adjoint_run(const ProbView &pv, const AdjWs &w, const double *modes, const double *logZk, int n_modes,
                      double grad_logZ, double *dmu, double *dL, cudaStream_t s) {
    const int d = pv.d, K = pv.K;
    if (n_modes < 1 || n_modes > kMaxAdjModes) return SB_ERR_INVALID_ARG;
    SB_CUDA_TRY(cudaMemsetAsync(dmu, 0, sizeof(double) * K * d, s));
    SB_CUDA_TRY(cudaMemsetAsync(dL, 0, sizeof(double) * (size_t)K * d * d, s));
    const int32_t one = 1;
    SB_CUDA_TRY(cudaMemcpyAsync(w.one, &one, sizeof(int32_t), cudaMemcpyHostToDevice, s));
    note_launch();
    k_softmax_pi<<<1, 32, 0, s>>>(n_modes, logZk, grad_logZ, w.pi);
    // P_k = L_k L_k^T is formed only for the Hessian at a mode that is not one-hot;
    // every product with P_k below is L_k (L_k^T v)
    bool p_ready = false;
    std::vector<double> pis(n_modes), Rh(K), epsh(K);
    SB_CUDA_TRY(cudaMemcpyAsync(pis.data(), w.pi, sizeof(double) * n_modes, cudaMemcpyDeviceToHost, s));
    SB_CUDA_TRY(cudaStreamSynchronize(s));
    for (int mo = 0; mo < n_modes; ++mo) {
        const double *x = modes + (size_t)mo * d;
        // l, grad l, z_k, r_k at x (FP64 likelihood kernels), then g_k, H and H = C C^T
        LikF64Args la{};
        la.d = d;
        la.K = K;
        la.mu = pv.mu;
        la.L = pv.L;
        la.a = pv.a;
        la.X = x;
        la.n_rows = 1;
        la.qpart = w.qpart;
        la.Z = w.Z;
        la.R = w.R;
        la.ell = w.ell;
        la.ell_sign = 1.0;
        la.G = w.gbar;
        la.grad_sign = -1.0;
        la.out_by_walker = 0;
        launch_lik_f64_few(la, true, s);
        SB_CUDA_TRY(cudaMemcpyAsync(Rh.data(), w.R, sizeof(double) * K, cudaMemcpyDeviceToHost, s));
        SB_CUDA_TRY(cudaStreamSynchronize(s));
        // at a one-hot mode (r_k = 1, every other r exactly 0) H = P_k, whose factor is
        // L_k: copied, not assembled and factored (as in the Laplace stage)
        int oh = -1, nz = 0;
        for (int k = 0; k < K; ++k)
            if (Rh[k] != 0.0) {
                ++nz;
                oh = Rh[k] == 1.0 ? k : -2;
            }
        if (nz != 1 || oh < 0) oh = -1;
        if (oh < 0 && !p_ready) {
            launch_precision(d, K, pv.L, w.P, s);
            p_ready = true;
        }
        launch_onehot(K, w.R, w.one, 1, w.onehot, s);
        launch_hessian_chol(d, K, 1, pv.L, w.P, w.Z, w.R, w.gbar, w.one, w.GK, w.H, w.info, w.bar, pv.status, s,
                            w.onehot);
        // W [g_0 .. g_{K-1}, gbar]
        note_launch();
        k_pack_rhs<<<(d * (K + 1) + 255) / 256, 256, 0, s>>>(d, K, w.GK, w.gbar, w.R, w.V);
        apply_W(d, K + 1, w.H, w.V, s);
        // W L_k and tr(W P_k) = <W L_k, L_k>_F for the components with r_k > 0. At a
        // one-hot mode the factor is L_k, so W L_k = L_k^-T and tr(W P_k) = d exactly:
        // no d x d solve
        for (int k = 0; k < K; ++k) {
            if (Rh[k] == 0.0) continue;
            if (k == oh) {
                note_launch();
                k_set_f64<<<1, 32, 0, s>>>(w.trWP + k, (double)d);
                continue;
            }
            double *Mk = w.M + (size_t)k * d * d;
            note_launch();
            k_copy_lower<<<1184, 256, 0, s>>>(d, pv.L + (size_t)k * d * d, Mk);
            apply_W(d, d, w.H, Mk, s);
            note_launch();
            k_trace_WP<<<1, 256, 0, s>>>(d, Mk, pv.L + (size_t)k * d * d, w.trWP + k);
        }
        // P_k (W gbar - W g_k) for the components with r_k > 0
        for (int k = 0; k < K; ++k) {
            if (Rh[k] == 0.0) continue;
            const double *Lk = pv.L + (size_t)k * d * d;
            note_launch();
            k_adj_wdiff<<<(d + 255) / 256, 256, 0, s>>>(d, K, k, w.V, w.y);
            note_launch();
            k_adj_Ltg<<<(d + 255) / 256, 256, 0, s>>>(d, Lk, w.y, w.u);
            note_launch();
            k_adj_Lu<<<(d * 32 + 255) / 256, 256, 0, s>>>(d, Lk, w.u, w.PY + (size_t)k * d);
        }
        // t = grad_x log det H, then v = W t (in place)
        note_launch();
        k_adj_stage<<<1, 256, 0, s>>>(0, d, K, w.R, w.GK, w.gbar, w.V, w.trWP, w.PY, nullptr, w.T, nullptr, nullptr,
                                      nullptr);
        apply_W(d, 1, w.H, w.T, s);
        // c, eps_k, gam_k
        note_launch();
        k_adj_stage<<<1, 256, 0, s>>>(1, d, K, w.R, w.GK, w.gbar, w.V, w.trWP, w.PY, w.T, nullptr, w.eps, w.gam,
                                      w.cvec);
        SB_CUDA_TRY(cudaMemcpyAsync(epsh.data(), w.eps, sizeof(double) * K, cudaMemcpyDeviceToHost, s));
        SB_CUDA_TRY(cudaStreamSynchronize(s));
        for (int k = 0; k < K; ++k) {
            if (Rh[k] == 0.0) continue;
            const double *Lk = pv.L + (size_t)k * d * d;
            // u = L_k^T gam_k, then P_k gam_k = L_k u for dmu_k
            note_launch();
            k_adj_Ltg<<<(d + 255) / 256, 256, 0, s>>>(d, Lk, w.gam + (size_t)k * d, w.u);
            note_launch();
            k_adj_Lu<<<(d * 32 + 255) / 256, 256, 0, s>>>(d, Lk, w.u, w.y);
            note_launch();
            k_adj_dmu<<<(d + 255) / 256, 256, 0, s>>>(d, k, pis[mo], w.eps, w.GK, w.y, dmu);
            note_launch();
            k_adj_dL<<<1184, 256, 0, s>>>(d, pis[mo], Rh[k], epsh[k], Lk, x, pv.mu + (size_t)k * d,
                                          w.Z + (size_t)k * d, w.gam + (size_t)k * d, w.u,
                                          k == oh ? nullptr : w.M + (size_t)k * d * d, dL + (size_t)k * d * d);
        }
    }
    SB_CUDA_TRY(cudaGetLastError());
    return SB_OK;
}

}  // namespace sb
