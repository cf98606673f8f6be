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
// History storage is FP32 or bf16 (the BF16-likelihood path stores bf16 pairs:
// half the bytes of the stream that bounds this kernel).
//
// Layout: thread t of the CTA owns coordinates 4t..4t+3 (float4, d <= 1024).
#include <cuda_bf16.h>
#include <stdlib.h>

#include "sb_lbfgs.cuh"

namespace sb {

namespace {

constexpr int CTA = 256;
constexpr int NW = CTA / 32;

// Sum of NV per-thread values over the CTA (sh holds NW * NV floats); every thread gets the totals.
// One barrier: callers alternate between two scratch buffers, so a buffer is
// never rewritten before every thread has read it (the next call's barrier
// orders it).
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

// History storage: FP32, or bf16 (half the bytes of the dominant stream). Inner
// products and S^T Y / Y^T Y are formed from the stored (rounded) vectors, so the
// step applies the exact L-BFGS matrix of the stored pairs.
__device__ __forceinline__ float4 ldh4(const float *p, int i0, int d) { return ld4(p, i0, d); }
__device__ __forceinline__ float4 ldh4(const __nv_bfloat16 *p, int i0, int d) {
    if (((d & 3) == 0) && i0 + 3 < d) {
        const uint2 u = *reinterpret_cast<const uint2 *>(p + i0);
        const __nv_bfloat162 a = *reinterpret_cast<const __nv_bfloat162 *>(&u.x);
        const __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162 *>(&u.y);
        return make_float4(__low2float(a), __high2float(a), __low2float(b), __high2float(b));
    }
    float4 r = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i0 + 0 < d) r.x = __bfloat162float(p[i0 + 0]);
    if (i0 + 1 < d) r.y = __bfloat162float(p[i0 + 1]);
    if (i0 + 2 < d) r.z = __bfloat162float(p[i0 + 2]);
    if (i0 + 3 < d) r.w = __bfloat162float(p[i0 + 3]);
    return r;
}
__device__ __forceinline__ void sth4(float *p, int i0, int d, float4 v) { st4(p, i0, d, v); }
__device__ __forceinline__ void sth4(__nv_bfloat16 *p, int i0, int d, float4 v) {
    if (((d & 3) == 0) && i0 + 3 < d) {
        __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
        uint2 u;
        u.x = *reinterpret_cast<uint32_t *>(&a);
        u.y = *reinterpret_cast<uint32_t *>(&b);
        *reinterpret_cast<uint2 *>(p + i0) = u;
        return;
    }
    if (i0 + 0 < d) p[i0 + 0] = __float2bfloat16_rn(v.x);
    if (i0 + 1 < d) p[i0 + 1] = __float2bfloat16_rn(v.y);
    if (i0 + 2 < d) p[i0 + 2] = __float2bfloat16_rn(v.z);
    if (i0 + 3 < d) p[i0 + 3] = __float2bfloat16_rn(v.w);
}
// The value a stored vector reads back as.
__device__ __forceinline__ float4 stored(float4 v, const float *) { return v; }
__device__ __forceinline__ float4 stored(float4 v, const __nv_bfloat16 *) {
    return make_float4(__bfloat162float(__float2bfloat16_rn(v.x)), __bfloat162float(__float2bfloat16_rn(v.y)),
                       __bfloat162float(__float2bfloat16_rn(v.z)), __bfloat162float(__float2bfloat16_rn(v.w)));
}

constexpr int LD = kMaxM + 1;  // padded row stride of the m x m matrices: rows and columns both conflict-free

struct Shared {
    float red2[2][NW * 32];  // reduction scratch, used alternately (see block_sum)
    float u1[kMaxM], u2[kMaxM], nsy[kMaxM], nys[kMaxM], nyy[kMaxM];
    float ca[kMaxM], cw[kMaxM], dinv[kMaxM];
    float R[kMaxM * LD];   // S^T Y in logical (oldest-first) order
    float YY[kMaxM * LD];  // Y^T Y in logical order
    float gamma;
    int slot_of[kMaxM];
};

// Reduce 32 per-lane values over the warp with 31 shuffles (recursive halving:
// at each level a lane keeps one half of its values and adds its partner's
// copy of that half). Lane j returns the warp total of value j.
__device__ __forceinline__ float warp_transpose_sum(float (&v)[32]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int j = 0; j < o; ++j) {
            const float send = up ? v[j] : v[j + o];
            const float keep = up ? v[j + o] : v[j];
            v[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    return v[0];
}

// Sums over the CTA of NV <= 32 per-thread values; thread t < NV returns total
// t (the others return garbage). One barrier, alternating scratch as block_sum.
template <int NV>
__device__ __forceinline__ float block_sum_scatter(const float (&in)[NV], float *sh) {
    float v[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = j < NV ? in[j] : 0.f;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    sh[wid * 32 + lane] = warp_transpose_sum(v);
    __syncthreads();
    float t = 0.f;
    if (threadIdx.x < NV)
#pragma unroll
        for (int q = 0; q < NW; ++q) t += sh[q * 32 + threadIdx.x];
    return t;
}

// NV sums and one maximum over the CTA with a single barrier; every thread gets all.
template <int NV>
__device__ __forceinline__ void block_sum_max(float (&v)[NV], float &mx, float *sh) {
    static_assert(NV + 1 <= 32, "scratch holds 32 values per warp");
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < NV; ++j) v[j] = warp_sum(v[j]);
    mx = warp_max(mx);
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < NV; ++j) sh[wid * 32 + j] = v[j];
        sh[wid * 32 + NV] = mx;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        float t = 0.f;
#pragma unroll
        for (int q = 0; q < NW; ++q) t += sh[q * 32 + j];
        v[j] = t;
    }
    float m = sh[NV];
#pragma unroll
    for (int q = 1; q < NW; ++q) m = fmaxf(m, sh[q * 32 + NV]);
    mx = m;
}

// Direction for walker state st (count pairs from ring slot head). When
// new_slot >= 0 the pair in that slot was stored this iteration (it is the
// newest, logical index count - 1) and the new row/column of S^T Y, Y^T Y is
// computed in the same pass. Writes P and the unit trial X + P; updates
// st.dphi / alpha / bt and possibly resets history. Returns the algorithmic
// bytes it moved.
template <typename HT>
__device__ uint64_t direction(const LbfgsArgs<float> &a, int w, WalkerState<float> &st, int new_slot, float4 g4,
                              float4 x4, float4 s_new, float4 y_new, float *MSY, float *MYY, Shared &sh, int &par) {
    const int d = a.d, m = a.m, i0 = 4 * threadIdx.x;
    const int count = st.count;
    uint64_t bytes = 0;
    float4 p4;
    if (count > 0) {
        const HT *S = reinterpret_cast<const HT *>(a.S) + (size_t)w * m * d;
        const HT *Y = reinterpret_cast<const HT *>(a.Y) + (size_t)w * m * d;
        if (threadIdx.x < count) sh.slot_of[threadIdx.x] = (st.head + threadIdx.x) % m;
        __syncthreads();
        // pass 1: inner products, four pairs per reduction; the loads of the next
        // group are issued before the current group is reduced
        float4 s4[4], y4[4];
        auto load_group = [&](int i) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                s4[q] = y4[q] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (i + q < count) {
                    const int slot = sh.slot_of[i + q];
                    s4[q] = ldh4(S + (size_t)slot * d, i0, d);
                    y4[q] = ldh4(Y + (size_t)slot * d, i0, d);
                }
            }
        };
        load_group(0);
        for (int i = 0; i < count; i += 4) {
            float v[20];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                v[q] = dot4(s4[q], g4);            // u1 = S^T g
                v[4 + q] = dot4(y4[q], g4);        // u2 = Y^T g
                v[8 + q] = dot4(s4[q], y_new);     // s_i . y_new
                v[12 + q] = dot4(s_new, y4[q]);    // s_new . y_i
                v[16 + q] = dot4(y4[q], y_new);    // y_i . y_new
            }
            if (i + 4 < count) load_group(i + 4);
            const float t = block_sum_scatter<20>(v, sh.red2[par++ & 1]);
            if (threadIdx.x < 20) {
                const int q = threadIdx.x & 3, k = threadIdx.x >> 2;
                if (i + q < count) {
                    float *dst = k == 0 ? sh.u1 : k == 1 ? sh.u2 : k == 2 ? sh.nsy : k == 3 ? sh.nys : sh.nyy;
                    dst[i + q] = t;
                }
            }
        }
        __syncthreads();
        // S^T Y and Y^T Y in logical order: the new pair's row and column from
        // this pass, the rest from the per-walker copies (slot-indexed, m x m),
        // which receive the new row and column at the same time
        float *msy = MSY + (size_t)w * m * m;
        float *myy = MYY + (size_t)w * m * m;
        const int cn = new_slot >= 0 ? count - 1 : -1;  // logical index of the new pair
        for (int e = threadIdx.x; e < count * count; e += CTA) {
            const int i = e / count, j = e % count;
            const int si = sh.slot_of[i], sj = sh.slot_of[j];
            float r, yy;
            if (j == cn) {
                r = sh.nsy[i];
                yy = sh.nyy[i];
            } else if (i == cn) {
                r = sh.nys[j];
                yy = sh.nyy[j];
            } else {
                r = msy[(size_t)si * m + sj];
                yy = myy[(size_t)si * m + sj];
            }
            if (i == cn || j == cn) {
                msy[(size_t)si * m + sj] = r;
                myy[(size_t)si * m + sj] = yy;
            }
            sh.R[i * LD + j] = r;
            sh.YY[i * LD + j] = yy;
        }
        bytes += (uint64_t)count * count * 8 + (cn >= 0 ? (uint64_t)(2 * count - 1) * 8 : 0);
        // pass 2's first two pairs are fetched before the solve (they do not depend on it)
        float4 cs[2], cy[2], ns[2], ny[2];
        auto load_pair2 = [&](int i, float4(&ps)[2], float4(&py)[2]) {
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                ps[q] = py[q] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (i + q < count) {
                    const int slot = sh.slot_of[i + q];
                    ps[q] = ldh4(S + (size_t)slot * d, i0, d);
                    py[q] = ldh4(Y + (size_t)slot * d, i0, d);
                }
            }
        };
        load_pair2(0, cs, cy);
        __syncthreads();
        const int c = count;
        const int lane = threadIdx.x & 31;
        if (threadIdx.x < 32) {
            // Column-oriented substitutions: lane j holds the running right-hand
            // side of rows j and j + 32; each step broadcasts one solved unknown.
            for (int i = lane; i < c; i += 32) sh.dinv[i] = 1.f / sh.R[i * LD + i];
            __syncwarp();
            // w = R^-1 u1, R upper (R_ij = s_i . y_j for i <= j)
            float acc0 = lane < c ? sh.u1[lane] : 0.f, acc1 = lane + 32 < c ? sh.u1[lane + 32] : 0.f;
            for (int i = c - 1; i >= 0; --i) {
                const float wi = __shfl_sync(0xffffffffu, i < 32 ? acc0 : acc1, i & 31) * sh.dinv[i];
                if (lane == 0) sh.cw[i] = wi;
                if (lane < i) acc0 -= sh.R[lane * LD + i] * wi;
                if (lane + 32 < i) acc1 -= sh.R[(lane + 32) * LD + i] * wi;
            }
            __syncwarp();
            const float gam = sh.R[(c - 1) * LD + (c - 1)] / sh.YY[(c - 1) * LD + (c - 1)];
            if (lane == 0) sh.gamma = gam;
            // tv = D w + gamma Y^T Y w - gamma Y^T g   (lane i: rows i, i + 32)
            float tv0 = 0.f, tv1 = 0.f;
            if (lane < c) {
                float yyw = 0.f;
                for (int j = 0; j < c; ++j) yyw += sh.YY[lane * LD + j] * sh.cw[j];
                tv0 = sh.R[lane * LD + lane] * sh.cw[lane] + gam * yyw - gam * sh.u2[lane];
            }
            if (lane + 32 < c) {
                const int i = lane + 32;
                float yyw = 0.f;
                for (int j = 0; j < c; ++j) yyw += sh.YY[i * LD + j] * sh.cw[j];
                tv1 = sh.R[i * LD + i] * sh.cw[i] + gam * yyw - gam * sh.u2[i];
            }
            // a = R^-T tv (R^T lower)
            for (int i = 0; i < c; ++i) {
                const float ai = __shfl_sync(0xffffffffu, i < 32 ? tv0 : tv1, i & 31) * sh.dinv[i];
                if (lane == 0) sh.ca[i] = ai;
                if (lane > i && lane < c) tv0 -= sh.R[i * LD + lane] * ai;
                if (lane + 32 > i && lane + 32 < c) tv1 -= sh.R[i * LD + lane + 32] * ai;
            }
        }
        __syncthreads();
        // pass 2: p = -gamma g - S a + gamma Y w, two pairs consumed while the next two load
        const float gam = sh.gamma;
        p4 = make_float4(-gam * g4.x, -gam * g4.y, -gam * g4.z, -gam * g4.w);
        for (int i = 0; i < count; i += 2) {
            if (i + 2 < count) load_pair2(i + 2, ns, ny);
#pragma unroll
            for (int q = 0; q < 2; ++q)
                if (i + q < count) {
                    p4 = axpy4(-sh.ca[i + q], cs[q], p4);
                    p4 = axpy4(gam * sh.cw[i + q], cy[q], p4);
                }
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                cs[q] = ns[q];
                cy[q] = ny[q];
            }
        }
        // the two-loop recursion's history traffic: each pair read in both passes
        bytes += (uint64_t)4 * count * d * sizeof(HT);
    }
    float dp[1];
    if (count > 0) {
        dp[0] = dot4(g4, p4);
        block_sum<1>(dp, sh.red2[par++ & 1]);
    }
    if (count == 0 || !(dp[0] < 0.f)) {
        st.count = 0;
        st.head = 0;
        float gg[1] = {dot4(g4, g4)};
        block_sum<1>(gg, sh.red2[par++ & 1]);
        const float gn = sqrtf(gg[0]);
        p4 = make_float4(-g4.x / gn, -g4.y / gn, -g4.z / gn, -g4.w / gn);
        dp[0] = dot4(g4, p4);
        block_sum<1>(dp, sh.red2[par++ & 1]);
    }
    st.dphi = dp[0];
    st.alpha = 1.f;
    st.bt = 0;
    st4(a.P + (size_t)w * d, i0, d, p4);
    st4(a.XT + (size_t)w * d, i0, d, make_float4(x4.x + p4.x, x4.y + p4.y, x4.z + p4.z, x4.w + p4.w));
    return bytes + (uint64_t)8 * d;
}

// Algorithmic bytes of the L-BFGS step launches (added only while counting is on).
__device__ unsigned long long g_lbfgs_bytes;

template <typename HT, int MINB>
__global__ void __launch_bounds__(CTA, MINB) k_lbfgs_cta(LbfgsArgs<float> a, float *MSY, float *MYY, int count_bytes) {
    __shared__ Shared sh;
    const int d = a.d, m = a.m, i0 = 4 * threadIdx.x;
    const int n_act = *a.n_act;
    int par = 0;  // alternation of the reduction scratch (identical in every thread)
    uint64_t bytes = 0;
    for (int n = blockIdx.x; n < n_act; n += gridDim.x) {
        const int w = a.act[n];
        WalkerState<float> st = a.st[w];  // same address in every thread: one broadcast load
        const float ft = a.FT[w];
        float *X = a.X + (size_t)w * d;
        float *G = a.G + (size_t)w * d;
        const float *XT = a.XT + (size_t)w * d;
        const float *GT = a.GT + (size_t)w * d;
        float4 x4 = ld4(X, i0, d), g4 = ld4(G, i0, d);
        const float4 xt4 = ld4(XT, i0, d), gt4 = ld4(GT, i0, d);
        bytes += (uint64_t)16 * d + 4 + 2 * sizeof(WalkerState<float>);
        // finiteness of the trial gradient, the candidate pair's inner products and
        // max |grad| at the trial, all in one reduction
        const HT *tag = nullptr;
        const float4 s4 = stored(make_float4(xt4.x - x4.x, xt4.y - x4.y, xt4.z - x4.z, xt4.w - x4.w), tag);
        const float4 y4 = stored(make_float4(gt4.x - g4.x, gt4.y - g4.y, gt4.z - g4.z, gt4.w - g4.w), tag);
        float r4[4] = {(isfinite(gt4.x) && isfinite(gt4.y) && isfinite(gt4.z) && isfinite(gt4.w)) ? 0.f : 1.f,
                       dot4(s4, s4), dot4(y4, y4), dot4(s4, y4)};
        float gm = fmaxf(fmaxf(fabsf(gt4.x), fabsf(gt4.y)), fmaxf(fabsf(gt4.z), fabsf(gt4.w)));
        block_sum_max<4>(r4, gm, sh.red2[par++ & 1]);
        const bool finite = isfinite(ft) && r4[0] == 0.f;
        bool newiter = false;
        int new_slot = -1;
        float4 s_new = make_float4(0.f, 0.f, 0.f, 0.f), y_new = s_new;
        if (st.phase == 0) {
            x4 = xt4;
            g4 = gt4;
            st4(X, i0, d, x4);
            st4(G, i0, d, g4);
            bytes += (uint64_t)8 * d;
            st.f = ft;
            st.phase = 1;
            if (!finite)
                st.status = SB_WALKER_NONFINITE;
            else
                newiter = true;
        } else if (finite && ft <= st.f + (a.c1 * st.alpha) * st.dphi) {
            if (r4[3] > 1e-10f * sqrtf(r4[1]) * sqrtf(r4[2])) {
                int slot;
                if (st.count < m) {
                    slot = (st.head + st.count) % m;
                    ++st.count;
                } else {
                    slot = st.head;
                    st.head = (st.head + 1) % m;
                }
                sth4(reinterpret_cast<HT *>(a.S) + ((size_t)w * m + slot) * d, i0, d, s4);
                sth4(reinterpret_cast<HT *>(a.Y) + ((size_t)w * m + slot) * d, i0, d, y4);
                if (threadIdx.x == 0) a.rho[(size_t)w * m + slot] = 1.f / r4[3];
                bytes += (uint64_t)2 * d * sizeof(HT) + 4;
                new_slot = slot;
                s_new = s4;
                y_new = y4;
            }
            st.flat = (ft >= st.f) ? st.flat + 1 : 0;
            x4 = xt4;
            g4 = gt4;
            st4(X, i0, d, x4);
            st4(G, i0, d, g4);
            bytes += (uint64_t)8 * d;
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
                bytes += (uint64_t)8 * d;
            } else if (st.count > 0 && st.attempt == 0) {
                st.count = 0;
                st.head = 0;
                st.attempt = 1;
                bytes += direction<HT>(a, w, st, -1, g4, x4, s_new, y_new, MSY, MYY, sh, par);
            } else {
                st.status = SB_WALKER_STALLED;
            }
        }
        if (newiter) {
            if (gm <= a.gtol * (1.f + fabsf(st.f))) {
                st.status = SB_WALKER_CONVERGED;
            } else if (st.flat >= 2) {
                st.status = SB_WALKER_STALLED;
            } else if (st.it >= a.max_iter) {
                st.status = SB_WALKER_MAXITER;
            } else {
                st.attempt = 0;
                bytes += direction<HT>(a, w, st, new_slot, g4, x4, s_new, y_new, MSY, MYY, sh, par);
            }
        }
        if (threadIdx.x == 0) a.st[w] = st;
        __syncthreads();  // shared scratch (slot_of, m x m matrices) is reused by the next walker
    }
    if (count_bytes && threadIdx.x == 0 && bytes) atomicAdd(&g_lbfgs_bytes, (unsigned long long)bytes);
}

}  // namespace

void launch_lbfgs_step_cta(const LbfgsArgs<float> &a, int n, float *MSY, float *MYY, int num_sms, bool bf16_history,
                           cudaStream_t s) {
    ProfScope prof(PROF_LBFGS_STEP, s);
    const int count_bytes = prof_enabled() ? 1 : 0;
    static const int minb = [] {
        const char *e = getenv("SB_LBFGS_MINB");
        return (e && atoi(e) == 3) ? 3 : 2;
    }();
    int grid = num_sms * minb;
    if (grid > n) grid = n > 0 ? n : 1;
    note_launch();
    if (minb == 3) {
        if (bf16_history)
            k_lbfgs_cta<__nv_bfloat16, 3><<<grid, CTA, 0, s>>>(a, MSY, MYY, count_bytes);
        else
            k_lbfgs_cta<float, 3><<<grid, CTA, 0, s>>>(a, MSY, MYY, count_bytes);
    } else {
        if (bf16_history)
            k_lbfgs_cta<__nv_bfloat16, 2><<<grid, CTA, 0, s>>>(a, MSY, MYY, count_bytes);
        else
            k_lbfgs_cta<float, 2><<<grid, CTA, 0, s>>>(a, MSY, MYY, count_bytes);
    }
}

double lbfgs_bytes_take() {
    unsigned long long v = 0, z = 0;
    if (cudaDeviceSynchronize() != cudaSuccess) return -1.0;
    if (cudaMemcpyFromSymbol(&v, g_lbfgs_bytes, sizeof(v)) != cudaSuccess) return -1.0;
    if (cudaMemcpyToSymbol(g_lbfgs_bytes, &z, sizeof(z)) != cudaSuccess) return -1.0;
    return (double)v;
}

}  // namespace sb
