// lbfgs_cta.cu -- FP32 batched L-BFGS step, one CTA per walker (mixed-precision path).
//
// Same state machine as the warp-per-walker kernel (Armijo backtracking,
// history reset and one retry, curvature skip, CONVERGED / STALLED / MAXITER;
// Sec. 3.6.2, App. A.5), but the direction p = -H_k grad f is formed through
// the compact representation of the L-BFGS inverse Hessian (Byrd, Nocedal &
// Schnabel, Math. Prog. 63, 1994, Thm. 2.2):
//
//   H_k = gamma I + [S  gamma Y] [ R^-T (D + gamma Y^T Y) R^-1   -R^-T ] [ S^T       ]
//                               [ -R^-1                          0     ] [ gamma Y^T ]
//
// with S, Y the stored pairs (oldest first), R_ij = s_i^T y_j (i <= j),
// D = diag(s_i^T y_i), gamma = s^T y / y^T y of the newest pair. It is the
// same matrix the two-loop recursion applies (App. A.5), so the direction is
// identical in exact arithmetic; what changes is the data flow. The two-loop
// walks the pairs with a serial dependency (each alpha_i needs the q left by
// the previous pair), so a walker waits on one memory latency per pair. Here
// one pass computes all inner products S^T g, Y^T g and the new pair's row and
// column of S^T Y and Y^T Y at once (all loads independent), an m x m
// triangular solve gives the coefficients, and a second pass forms
// p = -gamma g - S a + gamma Y w. The m x m matrices S^T Y and Y^T Y live per
// walker in HBM and are updated incrementally, so the history S, Y is read
// twice per iteration (the second read mostly from L2) and never re-walked.
//
// Layout: thread t of the CTA owns coordinates 4t..4t+3 (float4, d <= 1024).
#include "sb_lbfgs.cuh"

namespace sb {

namespace {

constexpr int CTA = 256;
constexpr int NW = CTA / 32;

// Sum of NV per-thread values over the CTA (sh holds NW * NV floats); every thread gets the totals.
template <int NV>
__device__ __forceinline__ void block_sum(float (&v)[NV], float *sh) {
    static_assert(NV <= 20, "block_sum scratch holds 20 values per warp");
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < NV; ++j) v[j] = warp_sum(v[j]);
    if (lane == 0)
#pragma unroll
        for (int j = 0; j < NV; ++j) sh[wid * NV + j] = v[j];
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        float t = 0.f;
#pragma unroll
        for (int q = 0; q < NW; ++q) t += sh[q * NV + j];
        v[j] = t;
    }
    __syncthreads();
}

__device__ __forceinline__ float block_max(float v, float *sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_max(v);
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    float t = sh[0];
#pragma unroll
    for (int q = 1; q < NW; ++q) t = fmaxf(t, sh[q]);
    __syncthreads();
    return t;
}

// Vector accesses need 16-byte aligned rows: d % 4 == 0 (rows start at multiples of d).
__device__ __forceinline__ float4 ld4(const float *p, int i0, int d) {
    if (((d & 3) == 0) && i0 + 3 < d) return *reinterpret_cast<const float4 *>(p + i0);
    float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i0 + 0 < d) r.x = p[i0 + 0];
    if (i0 + 1 < d) r.y = p[i0 + 1];
    if (i0 + 2 < d) r.z = p[i0 + 2];
    if (i0 + 3 < d) r.w = p[i0 + 3];
    return r;
}
__device__ __forceinline__ void st4(float *p, int i0, int d, float4 v) {
    if (((d & 3) == 0) && i0 + 3 < d) {
        *reinterpret_cast<float4 *>(p + i0) = v;
        return;
    }
    if (i0 + 0 < d) p[i0 + 0] = v.x;
    if (i0 + 1 < d) p[i0 + 1] = v.y;
    if (i0 + 2 < d) p[i0 + 2] = v.z;
    if (i0 + 3 < d) p[i0 + 3] = v.w;
}
__device__ __forceinline__ float dot4(float4 a, float4 b) { return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w; }
__device__ __forceinline__ float4 axpy4(float a, float4 x, float4 y) {
    return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
}

struct Shared {
    float red[NW * 20];  // block_sum scratch: up to 20 values per warp
    float u1[kMaxM], u2[kMaxM], nsy[kMaxM], nys[kMaxM], nyy[kMaxM];
    float ca[kMaxM], cw[kMaxM], tv[kMaxM];
    float R[kMaxM * kMaxM];   // S^T Y in logical (oldest-first) order
    float YY[kMaxM * kMaxM];  // Y^T Y in logical order
    float gamma;
    int slot_of[kMaxM];
};

// Direction for walker state st (count pairs from ring slot head). When
// new_slot >= 0 the pair in that slot was stored this iteration and the new
// row/column of S^T Y, Y^T Y is computed in the same pass. Writes P and the
// unit trial X + P; updates st.dphi / alpha / bt and possibly resets history.
__device__ void direction(const LbfgsArgs<float> &a, int w, WalkerState<float> &st, int new_slot, float4 g4,
                          float4 x4, float4 s_new, float4 y_new, float *MSY, float *MYY, Shared &sh) {
    const int d = a.d, m = a.m, i0 = 4 * threadIdx.x;
    const int count = st.count;
    float4 p4;
    if (count > 0) {
        const float *S = a.S + (size_t)w * m * d;
        const float *Y = a.Y + (size_t)w * m * d;
        if (threadIdx.x < count) sh.slot_of[threadIdx.x] = (st.head + threadIdx.x) % m;
        __syncthreads();
        // pass 1: inner products, four pairs per block reduction
        for (int i = 0; i < count; i += 4) {
            float v[20];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float4 s4 = make_float4(0.f, 0.f, 0.f, 0.f), y4 = s4;
                if (i + q < count) {
                    const int slot = sh.slot_of[i + q];
                    s4 = ld4(S + (size_t)slot * d, i0, d);
                    y4 = ld4(Y + (size_t)slot * d, i0, d);
                }
                v[5 * q + 0] = dot4(s4, g4);
                v[5 * q + 1] = dot4(y4, g4);
                v[5 * q + 2] = dot4(s4, y_new);
                v[5 * q + 3] = dot4(s_new, y4);
                v[5 * q + 4] = dot4(y4, y_new);
            }
            block_sum<20>(v, sh.red);
            if (threadIdx.x < 4 && i + (int)threadIdx.x < count) {
                const int q = threadIdx.x;
                sh.u1[i + q] = v[5 * q + 0];
                sh.u2[i + q] = v[5 * q + 1];
                sh.nsy[i + q] = v[5 * q + 2];
                sh.nys[i + q] = v[5 * q + 3];
                sh.nyy[i + q] = v[5 * q + 4];
            }
        }
        __syncthreads();
        // incremental update of S^T Y and Y^T Y for the new pair (slot-indexed, m x m)
        float *msy = MSY + (size_t)w * m * m;
        float *myy = MYY + (size_t)w * m * m;
        if (new_slot >= 0 && threadIdx.x < count) {
            const int so = sh.slot_of[threadIdx.x];
            msy[(size_t)so * m + new_slot] = sh.nsy[threadIdx.x];  // s_i . y_new
            msy[(size_t)new_slot * m + so] = sh.nys[threadIdx.x];  // s_new . y_i
            myy[(size_t)so * m + new_slot] = sh.nyy[threadIdx.x];
            myy[(size_t)new_slot * m + so] = sh.nyy[threadIdx.x];
        }
        __syncthreads();
        // stage both matrices in logical order
        for (int e = threadIdx.x; e < count * count; e += CTA) {
            const int i = e / count, j = e % count;
            const int si = sh.slot_of[i], sj = sh.slot_of[j];
            sh.R[i * kMaxM + j] = msy[(size_t)si * m + sj];
            sh.YY[i * kMaxM + j] = myy[(size_t)si * m + sj];
        }
        __syncthreads();
        const int c = count;
        const int lane = threadIdx.x & 31;
        if (threadIdx.x < 32) {
            // w = R^-1 u1, R upper (R_ij = s_i . y_j, i <= j): back substitution, lanes over j
            for (int i = c - 1; i >= 0; --i) {
                float part = 0.f;
                for (int j = i + 1 + lane; j < c; j += 32) part += sh.R[i * kMaxM + j] * sh.cw[j];
                part = warp_sum(part);
                if (lane == 0) sh.cw[i] = (sh.u1[i] - part) / sh.R[i * kMaxM + i];
                __syncwarp();
            }
            if (lane == 0) sh.gamma = sh.R[(c - 1) * kMaxM + (c - 1)] / sh.YY[(c - 1) * kMaxM + (c - 1)];
            __syncwarp();
            const float gam = sh.gamma;
            // tv = D w + gamma Y^T Y w - gamma Y^T g   (lanes over i)
            for (int i = lane; i < c; i += 32) {
                float yyw = 0.f;
                for (int j = 0; j < c; ++j) yyw += sh.YY[i * kMaxM + j] * sh.cw[j];
                sh.tv[i] = sh.R[i * kMaxM + i] * sh.cw[i] + gam * yyw - gam * sh.u2[i];
            }
            __syncwarp();
            // a = R^-T tv: forward substitution, lanes over j
            for (int i = 0; i < c; ++i) {
                float part = 0.f;
                for (int j = lane; j < i; j += 32) part += sh.R[j * kMaxM + i] * sh.ca[j];
                part = warp_sum(part);
                if (lane == 0) sh.ca[i] = (sh.tv[i] - part) / sh.R[i * kMaxM + i];
                __syncwarp();
            }
        }
        __syncthreads();
    // pass 2: p = -gamma g - S a + gamma Y w (four pairs' loads in flight per step)
        const float gam = sh.gamma;
        p4 = make_float4(-gam * g4.x, -gam * g4.y, -gam * g4.z, -gam * g4.w);
        for (int i = 0; i < count; i += 4) {
            float4 s4[4], y4[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                s4[q] = y4[q] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (i + q < count) {
                    const int slot = sh.slot_of[i + q];
                    s4[q] = ld4(S + (size_t)slot * d, i0, d);
                    y4[q] = ld4(Y + (size_t)slot * d, i0, d);
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (i + q < count) {
                    p4 = axpy4(-sh.ca[i + q], s4[q], p4);
                    p4 = axpy4(gam * sh.cw[i + q], y4[q], p4);
                }
        }
    }
    float dp[1];
    if (count > 0) {
        dp[0] = dot4(g4, p4);
        block_sum<1>(dp, sh.red);
    }
    if (count == 0 || !(dp[0] < 0.f)) {
        st.count = 0;
        st.head = 0;
        float gg[1] = {dot4(g4, g4)};
        block_sum<1>(gg, sh.red);
        const float gn = sqrtf(gg[0]);
        p4 = make_float4(-g4.x / gn, -g4.y / gn, -g4.z / gn, -g4.w / gn);
        dp[0] = dot4(g4, p4);
        block_sum<1>(dp, sh.red);
    }
    st.dphi = dp[0];
    st.alpha = 1.f;
    st.bt = 0;
    st4(a.P + (size_t)w * d, i0, d, p4);
    st4(a.XT + (size_t)w * d, i0, d, make_float4(x4.x + p4.x, x4.y + p4.y, x4.z + p4.z, x4.w + p4.w));
}

__global__ void __launch_bounds__(CTA) k_lbfgs_cta(LbfgsArgs<float> a, float *MSY, float *MYY) {
    __shared__ Shared sh;
    __shared__ WalkerState<float> s_st;
    const int d = a.d, m = a.m, i0 = 4 * threadIdx.x;
    const int n_act = *a.n_act;
    for (int n = blockIdx.x; n < n_act; n += gridDim.x) {
        const int w = a.act[n];
        if (threadIdx.x == 0) s_st = a.st[w];
        __syncthreads();
        WalkerState<float> st = s_st;
        __syncthreads();
        const float ft = a.FT[w];
        float *X = a.X + (size_t)w * d;
        float *G = a.G + (size_t)w * d;
        const float *XT = a.XT + (size_t)w * d;
        const float *GT = a.GT + (size_t)w * d;
        float4 x4 = ld4(X, i0, d), g4 = ld4(G, i0, d);
        const float4 xt4 = ld4(XT, i0, d), gt4 = ld4(GT, i0, d);
        float fin[1] = {(isfinite(gt4.x) && isfinite(gt4.y) && isfinite(gt4.z) && isfinite(gt4.w)) ? 0.f : 1.f};
        block_sum<1>(fin, sh.red);
        const bool finite = isfinite(ft) && fin[0] == 0.f;
        bool newiter = false;
        int new_slot = -1;
        float4 s_new = make_float4(0.f, 0.f, 0.f, 0.f), y_new = s_new;
        if (st.phase == 0) {
            x4 = xt4;
            g4 = gt4;
            st4(X, i0, d, x4);
            st4(G, i0, d, g4);
            st.f = ft;
            st.phase = 1;
            if (!finite)
                st.status = SB_WALKER_NONFINITE;
            else
                newiter = true;
        } else if (finite && ft <= st.f + (a.c1 * st.alpha) * st.dphi) {
            const float4 s4 = make_float4(xt4.x - x4.x, xt4.y - x4.y, xt4.z - x4.z, xt4.w - x4.w);
            const float4 y4 = make_float4(gt4.x - g4.x, gt4.y - g4.y, gt4.z - g4.z, gt4.w - g4.w);
            float r3[3] = {dot4(s4, s4), dot4(y4, y4), dot4(s4, y4)};
            block_sum<3>(r3, sh.red);
            if (r3[2] > 1e-10f * sqrtf(r3[0]) * sqrtf(r3[1])) {
                int slot;
                if (st.count < m) {
                    slot = (st.head + st.count) % m;
                    ++st.count;
                } else {
                    slot = st.head;
                    st.head = (st.head + 1) % m;
                }
                st4(a.S + ((size_t)w * m + slot) * d, i0, d, s4);
                st4(a.Y + ((size_t)w * m + slot) * d, i0, d, y4);
                if (threadIdx.x == 0) a.rho[(size_t)w * m + slot] = 1.f / r3[2];
                new_slot = slot;
                s_new = s4;
                y_new = y4;
            }
            st.flat = (ft >= st.f) ? st.flat + 1 : 0;
            x4 = xt4;
            g4 = gt4;
            st4(X, i0, d, x4);
            st4(G, i0, d, g4);
            st.f = ft;
            ++st.it;
            newiter = true;
        } else {
            ++st.bt;
            if (st.bt <= a.max_backtracks) {
                st.alpha *= a.backtrack;
                const float4 p4 = ld4(a.P + (size_t)w * d, i0, d);
                st4(a.XT + (size_t)w * d, i0, d,
                    make_float4(fmaf(st.alpha, p4.x, x4.x), fmaf(st.alpha, p4.y, x4.y), fmaf(st.alpha, p4.z, x4.z),
                                fmaf(st.alpha, p4.w, x4.w)));
            } else if (st.count > 0 && st.attempt == 0) {
                st.count = 0;
                st.head = 0;
                st.attempt = 1;
                direction(a, w, st, -1, g4, x4, s_new, y_new, MSY, MYY, sh);
            } else {
                st.status = SB_WALKER_STALLED;
            }
        }
        if (newiter) {
            const float gm = block_max(fmaxf(fmaxf(fabsf(g4.x), fabsf(g4.y)), fmaxf(fabsf(g4.z), fabsf(g4.w))), sh.red);
            if (gm <= a.gtol * (1.f + fabsf(st.f))) {
                st.status = SB_WALKER_CONVERGED;
            } else if (st.flat >= 2) {
                st.status = SB_WALKER_STALLED;
            } else if (st.it >= a.max_iter) {
                st.status = SB_WALKER_MAXITER;
            } else {
                st.attempt = 0;
                direction(a, w, st, new_slot, g4, x4, s_new, y_new, MSY, MYY, sh);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) a.st[w] = st;
        __syncthreads();
    }
}

}  // namespace

void launch_lbfgs_step_cta(const LbfgsArgs<float> &a, int n, float *MSY, float *MYY, int num_sms, cudaStream_t s) {
    ProfScope prof(PROF_LBFGS_STEP, s);
    int grid = num_sms * 4;
    if (grid > n) grid = n > 0 ? n : 1;
    note_launch();
    k_lbfgs_cta<<<grid, CTA, 0, s>>>(a, MSY, MYY);
}

}  // namespace sb
