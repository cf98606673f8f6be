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
// the previous pair). Here one pass computes all inner products S^T g, Y^T g
// and the new pair's row and column of S^T Y and Y^T Y at once (independent
// loads, several pairs in flight), an m x m triangular solve gives the
// coefficients, and a second pass forms p = -gamma g - S a + gamma Y w. The
// m x m matrices S^T Y and Y^T Y live per walker in HBM and are updated
// incrementally, so the history S, Y is read twice per iteration (the second
// read mostly from L2) and never re-walked.
//
// A walker's step is a chain of dependent phases (reductions, the m x m
// solve), so the SM is kept busy by several walkers at once: CT threads per
// walker, thread t owning the float4 groups at coordinates 4 (t + q CT),
// q < VPT = 1024 / (4 CT).
#include <cuda_bf16.h>

#include "sb_lbfgs.cuh"

namespace sb {

namespace {

template <int CT>
struct Cfg {
    static constexpr int NW = CT / 32;            // warps per walker
    static constexpr int VPT = kMaxD / (4 * CT);  // float4 groups per thread
    static constexpr int PG = CT >= 256 ? 4 : 2;  // pairs per pass-1 reduction
    static constexpr int MINB = CT >= 256 ? 2 : 4; // CTAs per SM
    static constexpr int DEPTH = CT >= 256 ? 2 : 3; // pair groups in flight (cp.async ring)
    // ring bytes: DEPTH groups x PG pairs x (s, y) x VPT float4 per thread
    static constexpr int RING_F4 = DEPTH * PG * 2 * VPT * CT;
};
constexpr int kCT = 128;  // threads per walker used by the solver

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
__device__ __forceinline__ float4 zero4() { return make_float4(0.f, 0.f, 0.f, 0.f); }

// Per-thread asynchronous copies global -> shared (16 bytes, L2 only). A thread
// only ever reads back the chunks it copied itself, so completing its own
// groups (cp.async.wait_group) is all the synchronisation the ring needs.
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async4(float *dst, const float *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
// History storage of the stored pairs: FP32, or bf16 (half the bytes of the
// stream that bounds the step). Inner products and S^T Y / Y^T Y are formed
// from the stored (rounded) vectors, so the direction applies the exact
// L-BFGS matrix of the pairs as stored.
__device__ __forceinline__ float4 round_bf16(float4 v) {
    return make_float4(__bfloat162float(__float2bfloat16_rn(v.x)), __bfloat162float(__float2bfloat16_rn(v.y)),
                       __bfloat162float(__float2bfloat16_rn(v.z)), __bfloat162float(__float2bfloat16_rn(v.w)));
}
__device__ __forceinline__ uint32_t pack2(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}
__device__ __forceinline__ float4 unpack4(uint32_t lo, uint32_t hi) {
    const __nv_bfloat162 a = *reinterpret_cast<const __nv_bfloat162 *>(&lo);
    const __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162 *>(&hi);
    return make_float4(__low2float(a), __high2float(a), __low2float(b), __high2float(b));
}

template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// A vector of d coordinates as this thread's VPT float4 groups. Mapping M = 0
// (FP32 pairs): group q of thread t holds coordinates 4 (t + q CT) .. +3, so one
// 16-byte access instruction of a warp covers a contiguous 512-byte stretch.
// M = 1 (bf16 pairs): thread t holds the 4 VPT consecutive coordinates from
// 4 VPT t, so its share of a bf16 row is one 16-byte chunk and a warp's copy
// instruction covers 512 contiguous bytes.
template <int CT, int M>
struct Vec {
    float4 v[Cfg<CT>::VPT];
    __device__ __forceinline__ static int i0(int q) {
        return M ? 4 * (Cfg<CT>::VPT * (int)threadIdx.x + q) : 4 * ((int)threadIdx.x + q * CT);
    }
    __device__ __forceinline__ void load(const float *p, int d) {
#pragma unroll
        for (int q = 0; q < Cfg<CT>::VPT; ++q) v[q] = ld4(p, i0(q), d);
    }
    __device__ __forceinline__ void store(float *p, int d) const {
#pragma unroll
        for (int q = 0; q < Cfg<CT>::VPT; ++q) st4(p, i0(q), d, v[q]);
    }
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int q = 0; q < Cfg<CT>::VPT; ++q) v[q] = zero4();
    }
};
template <int CT, int M>
__device__ __forceinline__ float dotv(const Vec<CT, M> &a, const Vec<CT, M> &b) {
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < Cfg<CT>::VPT; ++q) s += dot4(a.v[q], b.v[q]);
    return s;
}
// y += c x
template <int CT, int M>
__device__ __forceinline__ void axpyv(float c, const Vec<CT, M> &x, Vec<CT, M> &y) {
#pragma unroll
    for (int q = 0; q < Cfg<CT>::VPT; ++q) y.v[q] = axpy4(c, x.v[q], y.v[q]);
}
// a + c b
template <int CT, int M>
__device__ __forceinline__ Vec<CT, M> lincomb(const Vec<CT, M> &a, float c, const Vec<CT, M> &b) {
    Vec<CT, M> r;
#pragma unroll
    for (int q = 0; q < Cfg<CT>::VPT; ++q) r.v[q] = axpy4(c, b.v[q], a.v[q]);
    return r;
}
template <int CT, int M>
__device__ __forceinline__ Vec<CT, M> subv(const Vec<CT, M> &a, const Vec<CT, M> &b) {
    Vec<CT, M> r;
#pragma unroll
    for (int q = 0; q < Cfg<CT>::VPT; ++q)
        r.v[q] = make_float4(a.v[q].x - b.v[q].x, a.v[q].y - b.v[q].y, a.v[q].z - b.v[q].z, a.v[q].w - b.v[q].w);
    return r;
}
template <int CT, int M>
__device__ __forceinline__ bool finitev(const Vec<CT, M> &a) {
    bool f = true;
#pragma unroll
    for (int q = 0; q < Cfg<CT>::VPT; ++q)
        f = f && isfinite(a.v[q].x) && isfinite(a.v[q].y) && isfinite(a.v[q].z) && isfinite(a.v[q].w);
    return f;
}
template <int CT, int M>
__device__ __forceinline__ float absmaxv(const Vec<CT, M> &a) {
    float m = 0.f;
#pragma unroll
    for (int q = 0; q < Cfg<CT>::VPT; ++q)
        m = fmaxf(m, fmaxf(fmaxf(fabsf(a.v[q].x), fabsf(a.v[q].y)), fmaxf(fabsf(a.v[q].z), fabsf(a.v[q].w))));
    return m;
}

// Sum of NV per-thread values over the CTA; every thread gets the totals.
// One barrier: callers alternate between two scratch buffers, so a buffer is
// never rewritten before every thread has read it (the next call's barrier
// orders it).
template <int CT, int NV>
__device__ __forceinline__ void block_sum(float (&v)[NV], float *sh) {
    static_assert(NV <= 32, "block_sum scratch holds 32 values per warp");
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
        for (int q = 0; q < Cfg<CT>::NW; ++q) t += sh[q * NV + j];
        v[j] = t;
    }
}

// Reduce 16 per-lane values over the warp with 16 shuffles (recursive halving
// within each half-warp: at each level a lane keeps one half of its values and
// adds its partner's copy of that half; then one exchange between the halves).
// Lanes j and j + 16 return the warp total of value j.
__device__ __forceinline__ float warp_transpose_sum16(float (&v)[16]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 8; o >= 1; o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int j = 0; j < o; ++j) {
            const float send = up ? v[j] : v[j + o];
            const float keep = up ? v[j + o] : v[j];
            v[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 16);
}

// NV sums and one maximum over the CTA with a single barrier; every thread gets all.
template <int CT, int NV>
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
        for (int q = 0; q < Cfg<CT>::NW; ++q) t += sh[q * 32 + j];
        v[j] = t;
    }
    float m = sh[NV];
#pragma unroll
    for (int q = 1; q < Cfg<CT>::NW; ++q) m = fmaxf(m, sh[q * 32 + NV]);
    mx = m;
}

// Odd row stride of the m x m matrices: their rows and their columns are both
// free of shared-memory bank conflicts.
__host__ __device__ __forceinline__ int mm_ld(int m) { return (m & 1) ? m + 2 : m + 1; }
// Floats of the dynamic area after the ring: S^T Y and Y^T Y, which also hold
// pass 1's per-warp partial sums before they are staged.
template <int CT>
__host__ __device__ __forceinline__ int mm_floats(int m) {
    const int mats = 2 * m * mm_ld(m);
    const int p1 = (m + Cfg<CT>::PG - 1) / Cfg<CT>::PG * Cfg<CT>::NW * 5 * Cfg<CT>::PG;
    return mats > p1 ? mats : p1;
}

template <int CT>
struct Shared {
    float red2[2][Cfg<CT>::NW * 32];  // reduction scratch, used alternately (see block_sum)
    float u1[kMaxM], u2[kMaxM], nsy[kMaxM], nys[kMaxM], nyy[kMaxM];
    float ca[kMaxM], cw[kMaxM], dinv[kMaxM];
    float gamma;
    int slot_of[kMaxM];
    // dynamic shared memory: the pair ring, then S^T Y and Y^T Y (logical order, stride ld)
    float4 *ring;
    float *R, *YY;
    int ld;
};

// S^T Y and Y^T Y of the walker in logical order: the new pair's row and column
// (logical cn, or -1) from pass 1, the rest from the per-walker slot-indexed
// copies, which receive the new row and column at the same time. Returns bytes moved.
template <int CT>
__device__ __forceinline__ uint64_t stage_mm(Shared<CT> &sh, float *msy, float *myy, int count, int m, int cn) {
    for (int e = threadIdx.x; e < count * count; e += CT) {
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
        sh.R[i * sh.ld + j] = r;
        sh.YY[i * sh.ld + j] = yy;
    }
    return (uint64_t)count * count * 8 + (cn >= 0 ? (uint64_t)(2 * count - 1) * 8 : 0);
}

// Warp that runs the m x m solve: CTAs are dealt to SMs round-robin, so the
// CTAs co-resident on one SM have consecutive values of blockIdx / (grid / MINB).
template <int CT>
__device__ __forceinline__ int solver_warp() {
    const int per = max(1, (int)gridDim.x / Cfg<CT>::MINB);
    return (int)(blockIdx.x / per) % Cfg<CT>::NW;
}

// The m x m part (one warp): w = R^-1 u1, gamma, tv = D w + gamma Y^T Y w -
// gamma Y^T g, a = R^-T tv. Column-oriented substitutions: lane j holds the
// running right-hand side of rows j and j + 32; each step broadcasts one
// solved unknown. Results in sh.cw, sh.ca, sh.gamma.
template <int CT>
__device__ __forceinline__ void solve_mm(Shared<CT> &sh, int c) {
    const int lane = threadIdx.x & 31;
    const int LD = sh.ld;
    const float *R = sh.R, *YY = sh.YY;
    for (int i = lane; i < c; i += 32) sh.dinv[i] = 1.f / R[i * LD + i];
    __syncwarp();
    float acc0 = lane < c ? sh.u1[lane] : 0.f, acc1 = lane + 32 < c ? sh.u1[lane + 32] : 0.f;
    for (int i = c - 1; i >= 0; --i) {
        const float wi = __shfl_sync(0xffffffffu, i < 32 ? acc0 : acc1, i & 31) * sh.dinv[i];
        if (lane == 0) sh.cw[i] = wi;
        if (lane < i) acc0 -= R[lane * LD + i] * wi;
        if (lane + 32 < i) acc1 -= R[(lane + 32) * LD + i] * wi;
    }
    __syncwarp();
    const float gam = R[(c - 1) * LD + (c - 1)] / YY[(c - 1) * LD + (c - 1)];
    if (lane == 0) sh.gamma = gam;
    float tv0 = 0.f, tv1 = 0.f;
    if (lane < c) {
        float yyw = 0.f;
        for (int j = 0; j < c; ++j) yyw += YY[lane * LD + j] * sh.cw[j];
        tv0 = R[lane * LD + lane] * sh.cw[lane] + gam * yyw - gam * sh.u2[lane];
    }
    if (lane + 32 < c) {
        const int i = lane + 32;
        float yyw = 0.f;
        for (int j = 0; j < c; ++j) yyw += YY[i * sh.ld + j] * sh.cw[j];
        tv1 = R[i * LD + i] * sh.cw[i] + gam * yyw - gam * sh.u2[i];
    }
    for (int i = 0; i < c; ++i) {
        const float ai = __shfl_sync(0xffffffffu, i < 32 ? tv0 : tv1, i & 31) * sh.dinv[i];
        if (lane == 0) sh.ca[i] = ai;
        if (lane > i && lane < c) tv0 -= R[i * LD + lane] * ai;
        if (lane + 32 > i && lane + 32 < c) tv1 -= R[i * LD + lane + 32] * ai;
    }
}

// Stores this thread's coordinates of a history vector (already rounded to HT).
template <int CT, int M, typename HT>
__device__ __forceinline__ void store_hist(const Vec<CT, M> &v, HT *row, int d) {
    if (sizeof(HT) == 4) {
        v.store(reinterpret_cast<float *>(row), d);
    } else {  // mapping 1: 8 consecutive coordinates, one 16-byte chunk
        const int e0 = Vec<CT, M>::i0(0);
        if ((d & 7) == 0 && e0 + 7 < d) {
            *reinterpret_cast<uint4 *>(row + e0) = make_uint4(pack2(v.v[0].x, v.v[0].y), pack2(v.v[0].z, v.v[0].w),
                                                              pack2(v.v[1].x, v.v[1].y), pack2(v.v[1].z, v.v[1].w));
        } else {
            const float f[8] = {v.v[0].x, v.v[0].y, v.v[0].z, v.v[0].w, v.v[1].x, v.v[1].y, v.v[1].z, v.v[1].w};
            __nv_bfloat16 *r = reinterpret_cast<__nv_bfloat16 *>(row);
            for (int e = 0; e < 8 && e0 + e < d; ++e) r[e0 + e] = __float2bfloat16_rn(f[e]);
        }
    }
}

// Direction for walker state st (count pairs from ring slot head). When
// new_slot >= 0 the pair in that slot was stored this visit (it is the newest,
// logical index count - 1) and its row and column of S^T Y, Y^T Y come from the
// same pass. Writes P and the unit trial X + P; updates st.dphi / alpha / bt
// and possibly resets the history (steepest descent when p is not a descent
// direction). Returns the algorithmic bytes moved.
template <int CT, typename HT, int MAP = (sizeof(HT) == 2)>
__device__ uint64_t direction(const LbfgsArgs<float> &a, int w, WalkerState<float> &st, int new_slot,
                              const Vec<CT, MAP> &g, const Vec<CT, MAP> &x, const Vec<CT, MAP> &s_new, const Vec<CT, MAP> &y_new,
                              float *MSY, float *MYY, Shared<CT> &sh, int &par) {
    constexpr int PG = Cfg<CT>::PG;
    const int d = a.d, m = a.m;
    const int count = st.count;
    uint64_t bytes = 0;
    Vec<CT, MAP> p;
    p.zero();
    if (count > 0) {
        const HT *S = reinterpret_cast<const HT *>(a.S) + (size_t)w * m * d;
        const HT *Y = reinterpret_cast<const HT *>(a.Y) + (size_t)w * m * d;
        if (threadIdx.x < count) sh.slot_of[threadIdx.x] = (st.head + threadIdx.x) % m;
        __syncthreads();
        // Both passes stream the pairs through the shared-memory ring, DEPTH groups
        // of PG pairs in flight per thread (cp.async); pass 2's first groups are
        // issued before the m x m solve, which does not need them.
        constexpr int VPT = Cfg<CT>::VPT;
        // bf16 chunks are half the size: twice the groups in flight in the same ring
        constexpr int D = sizeof(HT) == 2 ? 2 * Cfg<CT>::DEPTH : Cfg<CT>::DEPTH;
        const int ngroups = (count + PG - 1) / PG;
        const bool vec_ok = (d & 3) == 0;
        constexpr bool BF = sizeof(HT) == 2;
        static_assert(!BF || VPT == 2, "bf16 history: two groups of 4 (8 bytes each) per thread");
        constexpr int U4 = BF ? VPT / 2 : VPT;  // 16-byte ring chunks per stored vector per thread
        auto rp = [&](int grp, int q, int v, int j) -> uint4 * {
            return reinterpret_cast<uint4 *>(sh.ring) + ((((size_t)(grp % D) * PG + q) * 2 + v) * U4 + j) * CT +
                   threadIdx.x;
        };
        // this thread's chunks of one stored vector into the ring (cp.async, or
        // plain copies for a ragged end of the row)
        auto issue_vec = [&](int grp, int q, int v, const HT *row) {
#pragma unroll
            for (int j = 0; j < U4; ++j) {
                if (BF) {
                    const int e0 = Vec<CT, MAP>::i0(0);  // 8 consecutive elements
                    if ((d & 7) == 0 && e0 + 7 < d) {
                        cp_async16(rp(grp, q, v, j), row + e0);
                    } else {
                        HT *dst = reinterpret_cast<HT *>(rp(grp, q, v, j));
                        for (int e = 0; e < 8 && e0 + e < d; ++e) dst[e] = row[e0 + e];
                    }
                } else {
                    const int i0 = Vec<CT, MAP>::i0(j);
                    if (vec_ok && i0 + 3 < d) {
                        cp_async16(rp(grp, q, v, j), row + i0);
                    } else {
                        for (int e = 0; e < 4 && i0 + e < d; ++e)
                            cp_async4(reinterpret_cast<float *>(rp(grp, q, v, j)) + e,
                                      reinterpret_cast<const float *>(row) + i0 + e);
                    }
                }
            }
        };
        auto issue = [&](int grp) {  // always commits one group (possibly empty)
            if (grp < ngroups) {
#pragma unroll
                for (int q = 0; q < PG; ++q) {
                    const int i = grp * PG + q;
                    if (i >= count) break;
                    const size_t row = (size_t)sh.slot_of[i] * d;
                    issue_vec(grp, q, 0, S + row);
                    issue_vec(grp, q, 1, Y + row);
                }
            }
            cp_async_commit();
        };
        auto fetch = [&](int grp, int q, Vec<CT, MAP> &sv, Vec<CT, MAP> &yv) {  // this thread's chunks of one pair
            if (BF) {
                const uint4 a4 = *rp(grp, q, 0, 0), b4 = *rp(grp, q, 1, 0);
                sv.v[0] = unpack4(a4.x, a4.y);
                sv.v[1] = unpack4(a4.z, a4.w);
                yv.v[0] = unpack4(b4.x, b4.y);
                yv.v[1] = unpack4(b4.z, b4.w);
            } else {
#pragma unroll
                for (int j = 0; j < VPT; ++j) {
                    const uint4 a4 = *rp(grp, q, 0, j), b4 = *rp(grp, q, 1, j);
                    sv.v[j] = make_float4(__uint_as_float(a4.x), __uint_as_float(a4.y), __uint_as_float(a4.z),
                                          __uint_as_float(a4.w));
                    yv.v[j] = make_float4(__uint_as_float(b4.x), __uint_as_float(b4.y), __uint_as_float(b4.z),
                                          __uint_as_float(b4.w));
                }
            }
#pragma unroll
            for (int j = 0; j < VPT; ++j) {
                const int i0 = Vec<CT, MAP>::i0(j);
                if (!(i0 + 3 < d)) {  // ragged tail: lanes past d hold stale data
                    if (i0 + 0 >= d) sv.v[j].x = yv.v[j].x = 0.f;
                    if (i0 + 1 >= d) sv.v[j].y = yv.v[j].y = 0.f;
                    if (i0 + 2 >= d) sv.v[j].z = yv.v[j].z = 0.f;
                    if (i0 + 3 >= d) sv.v[j].w = yv.v[j].w = 0.f;
                }
            }
        };
        // pass 1: inner products. Each warp reduces its share of a group's 5 PG
        // products over its lanes and parks the totals in shared scratch (the
        // m x m area, not staged yet); the warps' totals are summed once after the
        // pass, so the pass itself runs without CTA barriers.
        constexpr int NV = 5 * PG;
        static_assert(NV <= 16, "one half-warp transpose per group");
        float *p1 = sh.R;
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll 1
        for (int g0 = 0; g0 < D; ++g0) issue(g0);
        for (int grp = 0; grp < ngroups; ++grp) {
            cp_async_wait<D - 1>();
            const int i = grp * PG;
            float v[5 * PG];
#pragma unroll
            for (int q = 0; q < PG; ++q) {
                Vec<CT, MAP> s4, y4;
                if (i + q < count) {
                    fetch(grp, q, s4, y4);
                } else {
                    s4.zero();
                    y4.zero();
                }
                v[q] = dotv(s4, g);               // u1 = S^T g
                v[PG + q] = dotv(y4, g);          // u2 = Y^T g
                v[2 * PG + q] = dotv(s4, y_new);  // s_i . y_new
                v[3 * PG + q] = dotv(s_new, y4);  // s_new . y_i
                v[4 * PG + q] = dotv(y4, y_new);  // y_i . y_new
            }
            issue(grp + D);  // into the slot just read (this thread's reads are done)
            float v16[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) v16[j] = j < NV ? v[j] : 0.f;
            const float t = warp_transpose_sum16(v16);
            if (lane < NV) p1[(grp * Cfg<CT>::NW + wid) * NV + lane] = t;
        }
        __syncthreads();
        // warp totals -> the 5 count inner products (warps summed in order)
        for (int e = threadIdx.x; e < 5 * count; e += CT) {
            const int k = e / count, i = e % count;
            const float *src = p1 + (i / PG) * Cfg<CT>::NW * NV + k * PG + i % PG;
            float t = 0.f;
#pragma unroll
            for (int q = 0; q < Cfg<CT>::NW; ++q) t += src[q * NV];
            float *dst = k == 0 ? sh.u1 : k == 1 ? sh.u2 : k == 2 ? sh.nsy : k == 3 ? sh.nys : sh.nyy;
            dst[i] = t;
        }
#pragma unroll 1
        for (int g0 = 0; g0 < D; ++g0) issue(g0);  // pass 2's first groups
        __syncthreads();
        bytes += stage_mm<CT>(sh, MSY + (size_t)w * m * m, MYY + (size_t)w * m * m, count, m,
                              new_slot >= 0 ? count - 1 : -1);
        __syncthreads();
        // the solving warp differs between the CTAs that share an SM (their warp w
        // would otherwise all sit on the same scheduler)
        if ((int)(threadIdx.x >> 5) == solver_warp<CT>()) solve_mm<CT>(sh, count);
        __syncthreads();
        // pass 2: p = -gamma g - S a + gamma Y w
        const float gam = sh.gamma;
        p.zero();
        axpyv(-gam, g, p);
        for (int grp = 0; grp < ngroups; ++grp) {
            cp_async_wait<D - 1>();
#pragma unroll
            for (int q = 0; q < PG; ++q) {
                const int i = grp * PG + q;
                if (i < count) {
                    Vec<CT, MAP> s4, y4;
                    fetch(grp, q, s4, y4);
                    axpyv(-sh.ca[i], s4, p);
                    axpyv(gam * sh.cw[i], y4, p);
                }
            }
            issue(grp + D);
        }
        cp_async_wait<0>();  // (only empty groups remain) the ring is free for the next walker
        // the two-loop recursion's history traffic: each pair read in both passes
        bytes += (uint64_t)4 * count * d * sizeof(HT);
    }
    float dp[1];
    if (count > 0) {
        dp[0] = dotv(g, p);
        block_sum<CT, 1>(dp, sh.red2[par++ & 1]);
    }
    if (count == 0 || !(dp[0] < 0.f)) {
        st.count = 0;
        st.head = 0;
        float gg[1] = {dotv(g, g)};
        block_sum<CT, 1>(gg, sh.red2[par++ & 1]);
        const float gn = sqrtf(gg[0]);
#pragma unroll
        for (int q = 0; q < Cfg<CT>::VPT; ++q)
            p.v[q] = make_float4(-g.v[q].x / gn, -g.v[q].y / gn, -g.v[q].z / gn, -g.v[q].w / gn);
        dp[0] = dotv(g, p);
        block_sum<CT, 1>(dp, sh.red2[par++ & 1]);
    }
    st.dphi = dp[0];
    st.alpha = 1.f;
    st.bt = 0;
    p.store(a.P + (size_t)w * d, d);
    lincomb(x, 1.f, p).store(a.XT + (size_t)w * d, d);
    return bytes + (uint64_t)8 * d;
}

// Algorithmic bytes of the L-BFGS step launches (added only while counting is on).
__device__ unsigned long long g_lbfgs_bytes;

template <int CT, typename HT>
__global__ void __launch_bounds__(CT, Cfg<CT>::MINB) k_lbfgs_cta(LbfgsArgs<float> a, float *MSY, float *MYY,
                                                                int count_bytes) {
    constexpr int MAP = sizeof(HT) == 2;  // coordinate mapping (see Vec)
    __shared__ Shared<CT> sh;
    extern __shared__ __align__(16) float4 dyn[];  // [RING_F4] ring, then R, YY [m][ld]
    const int d = a.d, m = a.m;
    if (threadIdx.x == 0) {
        sh.ring = dyn;
        sh.ld = mm_ld(m);
        sh.R = reinterpret_cast<float *>(dyn + Cfg<CT>::RING_F4);
        sh.YY = sh.R + (size_t)m * sh.ld;
    }
    __syncthreads();
    const int n_act = *a.n_act;
    int par = 0;  // alternation of the reduction scratch (identical in every thread)
    uint64_t bytes = 0;
    for (int n = blockIdx.x; n < n_act; n += gridDim.x) {
        const int w = a.act[n];
        WalkerState<float> st = a.st[w];  // same address in every thread: one broadcast load
        const float ft = a.FT[w];
        float *X = a.X + (size_t)w * d;
        float *G = a.G + (size_t)w * d;
        Vec<CT, MAP> x, g, xt, gt;
        x.load(X, d);
        g.load(G, d);
        xt.load(a.XT + (size_t)w * d, d);
        gt.load(a.GT + (size_t)w * d, d);
        bytes += (uint64_t)16 * d + 4 + 2 * sizeof(WalkerState<float>);
        // finiteness of the trial gradient, the candidate pair's inner products and
        // max |grad| at the trial, all in one reduction
        Vec<CT, MAP> s4 = subv(xt, x), y4 = subv(gt, g);
        if (sizeof(HT) == 2) {  // the pair as it will be stored
#pragma unroll
            for (int q = 0; q < Cfg<CT>::VPT; ++q) {
                s4.v[q] = round_bf16(s4.v[q]);
                y4.v[q] = round_bf16(y4.v[q]);
            }
        }
        float r4[4] = {finitev(gt) ? 0.f : 1.f, dotv(s4, s4), dotv(y4, y4), dotv(s4, y4)};
        float gm = absmaxv(gt);
        block_sum_max<CT, 4>(r4, gm, sh.red2[par++ & 1]);
        const bool finite = isfinite(ft) && r4[0] == 0.f;
        bool newiter = false;
        int new_slot = -1;
        Vec<CT, MAP> s_new, y_new;
        s_new.zero();
        y_new.zero();
        if (st.phase == 0) {
            x = xt;
            g = gt;
            x.store(X, d);
            g.store(G, d);
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
                store_hist<CT, MAP, HT>(s4, reinterpret_cast<HT *>(a.S) + ((size_t)w * m + slot) * d, d);
                store_hist<CT, MAP, HT>(y4, reinterpret_cast<HT *>(a.Y) + ((size_t)w * m + slot) * d, d);
                if (threadIdx.x == 0) a.rho[(size_t)w * m + slot] = 1.f / r4[3];
                bytes += (uint64_t)2 * d * sizeof(HT) + 4;
                new_slot = slot;
                s_new = s4;
                y_new = y4;
            }
            st.flat = (ft >= st.f) ? st.flat + 1 : 0;
            x = xt;
            g = gt;
            x.store(X, d);
            g.store(G, d);
            bytes += (uint64_t)8 * d;
            st.f = ft;
            ++st.it;
            newiter = true;
        } else {
            ++st.bt;
            if (st.bt <= a.max_backtracks) {
                st.alpha *= a.backtrack;
                Vec<CT, MAP> p;
                p.load(a.P + (size_t)w * d, d);
                lincomb(x, st.alpha, p).store(a.XT + (size_t)w * d, d);
                bytes += (uint64_t)8 * d;
            } else if (st.count > 0 && st.attempt == 0) {
                st.count = 0;
                st.head = 0;
                st.attempt = 1;
                bytes += direction<CT, HT>(a, w, st, -1, g, x, s_new, y_new, MSY, MYY, sh, par);
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
                bytes += direction<CT, HT>(a, w, st, new_slot, g, x, s_new, y_new, MSY, MYY, sh, par);
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
    int grid = num_sms * Cfg<kCT>::MINB;
    if (grid > n) grid = n > 0 ? n : 1;
    const size_t dyn = (size_t)Cfg<kCT>::RING_F4 * sizeof(float4) + sizeof(float) * mm_floats<kCT>(a.m);
    static bool attr = false;
    if (!attr) {
        const size_t most = (size_t)Cfg<kCT>::RING_F4 * sizeof(float4) + sizeof(float) * mm_floats<kCT>(kMaxM);
        cudaFuncSetAttribute(k_lbfgs_cta<kCT, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most);
        cudaFuncSetAttribute(k_lbfgs_cta<kCT, __nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)most);
        attr = true;
    }
    note_launch();
    if (bf16_history)
        k_lbfgs_cta<kCT, __nv_bfloat16><<<grid, kCT, dyn, s>>>(a, MSY, MYY, count_bytes);
    else
        k_lbfgs_cta<kCT, float><<<grid, kCT, dyn, s>>>(a, MSY, MYY, count_bytes);
}

double lbfgs_bytes_take() {
    unsigned long long v = 0, z = 0;
    if (cudaDeviceSynchronize() != cudaSuccess) return -1.0;
    if (cudaMemcpyFromSymbol(&v, g_lbfgs_bytes, sizeof(v)) != cudaSuccess) return -1.0;
    if (cudaMemcpyToSymbol(g_lbfgs_bytes, &z, sizeof(z)) != cudaSuccess) return -1.0;
    return (double)v;
}

}  // namespace sb
