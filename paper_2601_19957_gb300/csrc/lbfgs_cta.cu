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
// and the new pair's column of R and row and column of Y^T Y at once
// (independent loads, several pairs in flight), m x m matrix-vector products
// with R^-1 (kept per walker, one new column per appended pair) give the
// coefficients, and a second pass forms p = -gamma g - S a + gamma Y w. R^-1,
// Y^T Y and D live per walker in HBM and are updated incrementally, so the
// history S, Y is read twice per iteration (the second read mostly from L2)
// and never re-walked. The pairs are stored in bf16, and the first pass runs
// on the tensor cores (mma.sync, the pairs as the B operand; g split into
// three bf16 terms).
//
// A walker's step is a chain of dependent phases (reductions, the m x m
// solve), so the SM is kept busy by several walkers at once: CT threads per
// walker, thread t owning the 8 consecutive coordinates from 8 t (one 16-byte
// chunk of a stored bf16 row).
#include <cuda_bf16.h>

#include <mutex>

#include "sb_lbfgs.cuh"

namespace sb {

namespace {

template <int CT>
struct Cfg {
    static constexpr int NW = CT / 32;            // warps per walker
    static constexpr int VPT = kMaxD / (4 * CT);  // float4 groups per thread
    static constexpr int MINB = 4;                // CTAs per SM
    // ring of the stored pairs: DB slots of PGB pairs (one 8-column tensor-core tile
    // of s, y vectors), each stored row up to kMaxD bf16 coordinates plus 16 bytes:
    // row r of a slot starts 16 r bytes further into the 128-byte bank window than
    // row 0, so the same 16-byte chunk of the 8 rows falls in 8 different bank groups
    static constexpr int PGB = 4;
    static constexpr int DB = 3;
    static constexpr int ROW_B = kMaxD * 2 + 16;
    static constexpr int SLOT_B = 2 * PGB * ROW_B;
    static constexpr int RING_B = DB * SLOT_B;
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

// Per-thread asynchronous copies global -> shared (16 bytes of a stored row, L2 only;
// 4 bytes of the m x m state). A thread completes its own copy groups
// (cp.async.wait_group); a warp barrier then makes them visible to the warp.
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async4(float *dst, const float *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
// The stored pairs are bf16 (half the bytes of the stream that bounds the
// step). Inner products, R and Y^T Y are formed from the stored (rounded)
// vectors, so the direction applies the exact L-BFGS matrix of the pairs as
// stored.
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

// Four 8 x 8 bf16 matrices from shared memory; lane l gives the address of row
// l % 8 of matrix l / 8 (16 bytes) and receives row l / 4, columns 2 (l % 4),
// 2 (l % 4) + 1 of each matrix.
__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void *row) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"((uint32_t)__cvta_generic_to_shared(row))
                 : "memory");
}
// D += A B for a 16 x 16 bf16 A whose rows 8..15 are zero (a0: row l / 4,
// k = 2 (l % 4) + {0, 1}; a2: the same row, k + 8), a 16 x 8 bf16 B (b0: k =
// 2 (l % 4) + {0, 1}, column l / 4; b1: k + 8) and FP32 accumulation; d0, d1
// are row l / 4, columns 2 (l % 4) + {0, 1}.
__device__ __forceinline__ void mma_rows8(float (&d)[4], uint32_t a0, uint32_t a2, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(0u), "r"(a2), "r"(0u), "r"(b0), "r"(b1));
}
// v = hi + mid + lo with each term a bf16 (the remainders are exact in FP32), so
// products with bf16 vectors accumulate to FP32 accuracy on the tensor cores.
__device__ __forceinline__ void split3_bf16(float v, float &hi, float &mid, float &lo) {
    hi = __bfloat162float(__float2bfloat16_rn(v));
    const float r = v - hi;
    mid = __bfloat162float(__float2bfloat16_rn(r));
    lo = r - mid;
}

// A vector of d coordinates as this thread's VPT float4 groups: thread t holds
// the 4 VPT consecutive coordinates from 4 VPT t, so its share of a bf16 row is
// one 16-byte chunk and a warp's copy instruction covers 512 contiguous bytes.
template <int CT>
struct Vec {
    float4 v[Cfg<CT>::VPT];
    __device__ __forceinline__ static int i0(int q) { return 4 * (Cfg<CT>::VPT * (int)threadIdx.x + q); }
    // EVEN: d % (4 VPT) == 0, so a thread holds all of its coordinates or none
    template <bool EVEN>
    __device__ __forceinline__ void load(const float *p, int d) {
        if (EVEN) {
            const bool own = i0(0) < d;
#pragma unroll
            for (int q = 0; q < Cfg<CT>::VPT; ++q)
                v[q] = own ? *reinterpret_cast<const float4 *>(p + i0(q)) : zero4();
        } else {
#pragma unroll
            for (int q = 0; q < Cfg<CT>::VPT; ++q) v[q] = ld4(p, i0(q), d);
        }
    }
    template <bool EVEN>
    __device__ __forceinline__ void store(float *p, int d) const {
        if (EVEN) {
            if (i0(0) < d)
#pragma unroll
                for (int q = 0; q < Cfg<CT>::VPT; ++q) *reinterpret_cast<float4 *>(p + i0(q)) = v[q];
        } else {
#pragma unroll
            for (int q = 0; q < Cfg<CT>::VPT; ++q) st4(p, i0(q), d, v[q]);
        }
    }
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int q = 0; q < Cfg<CT>::VPT; ++q) v[q] = zero4();
    }
};
template <int CT>
__device__ __forceinline__ float dotv(const Vec<CT> &a, const Vec<CT> &b) {
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < Cfg<CT>::VPT; ++q) s += dot4(a.v[q], b.v[q]);
    return s;
}
// y += c x
template <int CT>
__device__ __forceinline__ void axpyv(float c, const Vec<CT> &x, Vec<CT> &y) {
#pragma unroll
    for (int q = 0; q < Cfg<CT>::VPT; ++q) y.v[q] = axpy4(c, x.v[q], y.v[q]);
}
// a + c b
template <int CT>
__device__ __forceinline__ Vec<CT> lincomb(const Vec<CT> &a, float c, const Vec<CT> &b) {
    Vec<CT> r;
#pragma unroll
    for (int q = 0; q < Cfg<CT>::VPT; ++q) r.v[q] = axpy4(c, b.v[q], a.v[q]);
    return r;
}
template <int CT>
__device__ __forceinline__ Vec<CT> subv(const Vec<CT> &a, const Vec<CT> &b) {
    Vec<CT> r;
#pragma unroll
    for (int q = 0; q < Cfg<CT>::VPT; ++q)
        r.v[q] = make_float4(a.v[q].x - b.v[q].x, a.v[q].y - b.v[q].y, a.v[q].z - b.v[q].z, a.v[q].w - b.v[q].w);
    return r;
}
template <int CT>
__device__ __forceinline__ bool finitev(const Vec<CT> &a) {
    bool f = true;
#pragma unroll
    for (int q = 0; q < Cfg<CT>::VPT; ++q)
        f = f && isfinite(a.v[q].x) && isfinite(a.v[q].y) && isfinite(a.v[q].z) && isfinite(a.v[q].w);
    return f;
}
template <int CT>
__device__ __forceinline__ float absmaxv(const Vec<CT> &a) {
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

// The dynamic shared memory of the step kernel: the pair ring (Cfg RING_B bytes),
// then R^-1 and Y^T Y (logical order, stride ld), pass 1's per-warp partial sums and
// the m-vectors S^T g, Y^T g, the direction's coefficients a, w, D = diag(S^T Y) and
// the new pair's column of R. Addresses are formed from the array and m (registers),
// not kept in shared memory, so that no access waits on a pointer load.
extern __shared__ __align__(16) float4 lb_dyn[];
__device__ __forceinline__ unsigned char *ring_base() { return reinterpret_cast<unsigned char *>(lb_dyn); }

// Odd row stride of the m x m matrices: their rows and their columns are both
// free of shared-memory bank conflicts.
__host__ __device__ __forceinline__ int mm_ld(int m) { return (m & 1) ? m + 2 : m + 1; }
// Pass 1's partial sums per ring group and warp: three rows (g, y_new, s_new) x
// the group's 2 PGB vectors.
template <int CT>
__host__ __device__ __forceinline__ int p1_floats(int m) {
    return (m + Cfg<CT>::PGB - 1) / Cfg<CT>::PGB * Cfg<CT>::NW * 3 * 2 * Cfg<CT>::PGB;
}
// Floats of the dynamic area after the ring: R^-1, Y^T Y, pass 1's sums and the
// six m-vectors (u1, u2, ca, cw, dg, nr).
template <int CT>
__host__ __device__ __forceinline__ int mm_floats(int m) {
    return 2 * m * mm_ld(m) + p1_floats<CT>(m) + 6 * m;
}
template <int CT>
struct Lay {
    int m, ld;
    __device__ __forceinline__ explicit Lay(int m_) : m(m_), ld(mm_ld(m_)) {}
    __device__ __forceinline__ float *RI() const { return reinterpret_cast<float *>(ring_base() + Cfg<CT>::RING_B); }
    __device__ __forceinline__ float *YY() const { return RI() + m * ld; }
    __device__ __forceinline__ float *p1() const { return YY() + m * ld; }
    __device__ __forceinline__ float *u1() const { return p1() + p1_floats<CT>(m); }
    __device__ __forceinline__ float *u2() const { return u1() + m; }
    __device__ __forceinline__ float *ca() const { return u2() + m; }
    __device__ __forceinline__ float *cw() const { return ca() + m; }
    __device__ __forceinline__ float *dg() const { return cw() + m; }
    __device__ __forceinline__ float *nr() const { return dg() + m; }
};

template <int CT>
struct Shared {
    float red2[2][Cfg<CT>::NW * 32];  // reduction scratch, used alternately (see block_sum)
    float gamma;
    uint4 zero16;  // a zero row for the unused rows of the tensor-core operand
};

// The m x m state of a walker, slot-indexed in HBM (logical pair i sits in slot
// (head + i) mod m): R^-1, the inverse of R = upper(S^T Y) (entries i <= j), Y^T Y,
// and D_i = s_i . y_i (in rho). R^-1 is kept instead of R because the history
// changes only by appending a pair (one new column of R^-1, a triangular
// matvec) and dropping the oldest (the inverse of R's trailing block is the
// trailing block of R^-1), so the direction needs matvecs, not substitutions.
//
// Copies the walker's R^-1, Y^T Y and D into shared memory in logical order as
// 4-byte asynchronous copies (one copy group, waited for before the solve); the new
// pair's row and column (logical cn, or -1) are skipped: pass 1 supplies them.
template <int CT>
__device__ __forceinline__ void fetch_mm(const Lay<CT> &L, const float *mri, const float *myy, const float *dw,
                                         int count, int m, int head, int cn) {
    float *RI = L.RI(), *YY = L.YY(), *dg = L.dg();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int i = wid; i < count; i += Cfg<CT>::NW) {
        if (i == cn) continue;
        int si = head + i;
        if (si >= m) si -= m;
        for (int j = lane; j < count; j += 32) {
            if (j == cn) continue;
            int sj = head + j;
            if (sj >= m) sj -= m;
            if (j >= i) cp_async4(RI + i * L.ld + j, mri + (size_t)si * m + sj);
            cp_async4(YY + i * L.ld + j, myy + (size_t)si * m + sj);
        }
        if (lane == 0) cp_async4(dg + i, dw + si);
    }
}
// The new pair's part of the state from pass 1: Y^T Y's row and column (y_i .
// y_new) into shared memory and HBM, R's new column (s_i . y_new, the last entry
// being D_new) into nr and D_new into dg and HBM. R^-1's new column is
// formed by the solver. Returns the bytes of m x m state moved this visit.
template <int CT, typename P1>
__device__ __forceinline__ uint64_t new_mm(const Lay<CT> &L, float *myy, float *dw, int count, int m, int head, int cn,
                                           P1 p1sum) {
    if (cn >= 0) {
        float *YY = L.YY(), *nr = L.nr(), *dg = L.dg();
        for (int e = threadIdx.x; e < 2 * count - 1; e += CT) {
            // e < count: column cn, row e; else row cn, column e - count
            const int i = e < count ? e : cn, j = e < count ? cn : e - count;
            const float yy = p1sum(4, e < count ? i : j);
            int si = head + i, sj = head + j;
            if (si >= m) si -= m;
            if (sj >= m) sj -= m;
            myy[(size_t)si * m + sj] = yy;
            YY[i * L.ld + j] = yy;
            if (e < count) {
                const float r = p1sum(2, i);
                nr[i] = r;
                if (i == cn) {
                    dg[cn] = r;
                    dw[si] = r;
                }
            }
        }
    }
    const uint64_t c = count;
    return (c * (c + 1) / 2 + c * c + c) * 4 + (cn >= 0 ? (uint64_t)(3 * c) * 4 : 0);
}

// The m x m part, on the whole CTA, with R^-1 in shared memory: the new column
// of R^-1 when a pair was appended (logical cn; RI_i,cn = -(sum_{i<=k<cn} RI_ik
// R_k,cn) / D_cn, RI_cn,cn = 1 / D_cn, also written to HBM), then w = R^-1 u1,
// gamma = D_c-1 / (y^T y)_c-1, tv = D w + gamma Y^T Y w - gamma u2 and
// a = R^-T tv. Each entry is a dot product over G threads (strided terms, then a
// fixed-order shuffle sum), one barrier between the stages. Every thread calls
// it. Results in cw, ca and sh.gamma.
template <int CT>
__device__ __forceinline__ void solve_mm(Shared<CT> &sh, const Lay<CT> &L, int c, int cn, float *mri, int m, int head) {
    const int G = c <= CT / 4 ? 4 : (c <= CT / 2 ? 2 : 1);  // threads per entry
    const int i = (int)threadIdx.x / G, p = (int)threadIdx.x % G;
    const int LD = L.ld;
    float *RI = L.RI();
    const float *YY = L.YY();
    float *tv = L.p1();  // pass 1's partial sums are consumed before the solve
    const float *nr = L.nr(), *u1 = L.u1(), *u2 = L.u2(), *dg = L.dg();
    float *cw = L.cw(), *ca = L.ca();
    auto gsum = [&](float v) {  // every lane calls it: full-warp shuffles
        if (G >= 2) v += __shfl_xor_sync(0xffffffffu, v, 1);
        if (G >= 4) v += __shfl_xor_sync(0xffffffffu, v, 2);
        return v;
    };
    if (cn >= 0) {
        const float dn = nr[cn];
        float t = 0.f;
        if (i < cn)
            for (int k = i + p; k < cn; k += G) t += RI[i * LD + k] * nr[k];
        t = gsum(t);
        if (p == 0 && i <= cn) {
            const float v = i == cn ? 1.f / dn : -t / dn;
            RI[i * LD + cn] = v;
            int si = head + i, sc = head + cn;
            if (si >= m) si -= m;
            if (sc >= m) sc -= m;
            mri[(size_t)si * m + sc] = v;
        }
        __syncthreads();
    }
    {
        float t = 0.f;
        if (i < c)
            for (int k = i + p; k < c; k += G) t += RI[i * LD + k] * u1[k];
        t = gsum(t);
        if (p == 0 && i < c) cw[i] = t;
    }
    __syncthreads();
    const float gam = dg[c - 1] / YY[(c - 1) * LD + (c - 1)];
    if (threadIdx.x == 0) sh.gamma = gam;
    {
        float t = 0.f;
        if (i < c)
            for (int j = p; j < c; j += G) t += YY[i * LD + j] * cw[j];
        t = gsum(t);
        if (p == 0 && i < c) tv[i] = dg[i] * cw[i] + gam * t - gam * u2[i];
    }
    __syncthreads();
    {
        float t = 0.f;
        if (i < c)
            for (int k = p; k <= i; k += G) t += RI[k * LD + i] * tv[k];
        t = gsum(t);
        if (p == 0 && i < c) ca[i] = t;
    }
}

using bf16 = __nv_bfloat16;

// Stores this thread's chunk of a history row (values already bf16; coordinates past
// d are zero in the vector): 8 consecutive coordinates, one 16-byte store, for every
// chunk inside the row pitch.
template <int CT>
__device__ __forceinline__ void store_hist(const Vec<CT> &v, bf16 *row, int ldh) {
    const int e0 = Vec<CT>::i0(0);
    if (e0 >= ldh) return;
    *reinterpret_cast<uint4 *>(row + e0) = make_uint4(pack2(v.v[0].x, v.v[0].y), pack2(v.v[0].z, v.v[0].w),
                                                      pack2(v.v[1].x, v.v[1].y), pack2(v.v[1].z, v.v[1].w));
}

// The ring the stored pairs stream through (Cfg: DB slots of PGB pairs; row 2 q + v of
// a slot is vector v (0: s, 1: y) of its pair q). Each thread copies and reads its own
// 16-byte chunk of every row (cp.async); pass 1's tensor-core operands also read the
// chunks of the other lanes of the warp, after a warp barrier. Every issue commits one
// copy group (empty when there is nothing to copy), so a wait for the group issued
// D - 1 issues earlier is cp.async.wait_group D - 1.
template <int CT>
struct Ring {
    static constexpr int PG = Cfg<CT>::PGB, D = Cfg<CT>::DB;
    static_assert(Cfg<CT>::VPT == 2, "one 16-byte bf16 chunk (8 coordinates) per stored vector and thread");
    int ldh, m, head, J, cn;  // row pitch, history size, first slot, pairs in the ring, new pair (or -1)
    const bf16 *S, *Y;

    __device__ __forceinline__ unsigned char *row(int sl, int r) const {
        return ring_base() + sl * Cfg<CT>::SLOT_B + r * Cfg<CT>::ROW_B;
    }
    // this thread's chunk of row r of slot sl
    __device__ __forceinline__ uint4 *chunk(int sl, int r) const {
        return reinterpret_cast<uint4 *>(row(sl, r)) + threadIdx.x;
    }
    // Group k (logical pairs k PG .. k PG + PG - 1 below J; none for k < 0) into slot sl.
    // The visit's new pair comes from registers (s_new, y_new), not HBM.
    __device__ __forceinline__ void issue(int k, int sl, const Vec<CT> &s_new, const Vec<CT> &y_new) const {
        const int e0 = Vec<CT>::i0(0);
        if (k >= 0 && e0 < ldh) {
#pragma unroll
            for (int q = 0; q < PG; ++q) {
                const int j = k * PG + q;
                if (j >= J) break;
                if (j == cn) {
                    *chunk(sl, 2 * q) = make_uint4(pack2(s_new.v[0].x, s_new.v[0].y), pack2(s_new.v[0].z, s_new.v[0].w),
                                                   pack2(s_new.v[1].x, s_new.v[1].y), pack2(s_new.v[1].z, s_new.v[1].w));
                    *chunk(sl, 2 * q + 1) = make_uint4(pack2(y_new.v[0].x, y_new.v[0].y), pack2(y_new.v[0].z, y_new.v[0].w),
                                                       pack2(y_new.v[1].x, y_new.v[1].y), pack2(y_new.v[1].z, y_new.v[1].w));
                    continue;
                }
                int slot = head + j;
                if (slot >= m) slot -= m;
                cp_async16(chunk(sl, 2 * q), S + (size_t)slot * ldh + e0);
                cp_async16(chunk(sl, 2 * q + 1), Y + (size_t)slot * ldh + e0);
            }
        }
        cp_async_commit();
    }
    // the group issued D - 1 issues ago has landed, and is visible to the warp
    __device__ __forceinline__ void wait() const {
        cp_async_wait<D - 1>();
        __syncwarp();
    }
    // this thread's coordinates of pair q of slot sl
    __device__ __forceinline__ void fetch(int sl, int q, Vec<CT> &sv, Vec<CT> &yv) const {
        const uint4 a4 = *chunk(sl, 2 * q), b4 = *chunk(sl, 2 * q + 1);
        sv.v[0] = unpack4(a4.x, a4.y);
        sv.v[1] = unpack4(a4.z, a4.w);
        yv.v[0] = unpack4(b4.x, b4.y);
        yv.v[1] = unpack4(b4.z, b4.w);
    }
};

// Direction for walker state st (count pairs from ring slot head). When
// new_slot >= 0 the pair in that slot was stored this visit (the newest, logical
// index count - 1; s_new, y_new) and its column of R, row and column of Y^T Y
// come from the same pass. Writes P and the unit trial X + P; updates st.dphi /
// alpha / bt and possibly resets the history (steepest descent when p is not a
// descent direction). Returns the algorithmic bytes moved.
//
// Pass 1 streams the pairs oldest first; at its end the ring holds the newest
// min(groups, DB) groups, so pass 2 walks the groups newest first: those are read
// where they are, and each slot it frees is refilled with the group DB older (the
// same slot, g mod DB), the only ones read from HBM (L2) again.
template <int CT, bool EVEN>
__device__ uint64_t direction(const LbfgsArgs<float> &a, int w, WalkerState<float> &st, int new_slot,
                              const Vec<CT> &g_in, const Vec<CT> &x_in, const Vec<CT> &s_new, const Vec<CT> &y_new,
                              float *MRI, float *MYY, Shared<CT> &sh, const Lay<CT> &L, int &par) {
    using RG = Ring<CT>;
    constexpr int PG = RG::PG, D = RG::D, NW = Cfg<CT>::NW;
    const int d = a.d, m = a.m, ldh = hist_ld(d);
    const int count = st.count;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint64_t bytes = 0;
    Vec<CT> p;
    p.zero();
    // x and g are stored at X, G by the caller; they are read back after pass 1
    // instead of being held through it
    Vec<CT> g = g_in, x = x_in;
    if (count > 0) {
        const bool added = new_slot >= 0;
        const int cn = added ? count - 1 : -1;
        const RG ring{ldh, m, st.head, count, cn, reinterpret_cast<const bf16 *>(a.S) + (size_t)w * m * ldh,
                      reinterpret_cast<const bf16 *>(a.Y) + (size_t)w * m * ldh};
        const int ng = (count + PG - 1) / PG;
        float *mri_w = MRI + (size_t)w * m * m, *myy_w = MYY + (size_t)w * m * m, *dw = a.rho + (size_t)w * m;
#pragma unroll 1
        for (int k = 0; k < D - 1; ++k) ring.issue(k, k, s_new, y_new);
        float *p1 = L.p1();
        {
            // Pass 1 on the tensor cores: per warp (its 256 coordinates, 16 k-steps of
            // 16) and group (8 stored vectors s_0 y_0 .. s_3 y_3 as the columns of B),
            // D = A B with the rows of A = (g_hi, g_mid, g_lo, y_new, s_new, 0 ..) at the
            // same coordinates. The A fragments are staged once through this warp's
            // own chunks of ring slot D - 1 (free until group D - 1 is issued into it).
            {
                float hi[8], mi[8], lo[8];
                const float gv[8] = {g.v[0].x, g.v[0].y, g.v[0].z, g.v[0].w, g.v[1].x, g.v[1].y, g.v[1].z, g.v[1].w};
#pragma unroll
                for (int e = 0; e < 8; ++e) split3_bf16(gv[e], hi[e], mi[e], lo[e]);
                *ring.chunk(D - 1, 0) =
                    make_uint4(pack2(hi[0], hi[1]), pack2(hi[2], hi[3]), pack2(hi[4], hi[5]), pack2(hi[6], hi[7]));
                *ring.chunk(D - 1, 1) =
                    make_uint4(pack2(mi[0], mi[1]), pack2(mi[2], mi[3]), pack2(mi[4], mi[5]), pack2(mi[6], mi[7]));
                *ring.chunk(D - 1, 2) =
                    make_uint4(pack2(lo[0], lo[1]), pack2(lo[2], lo[3]), pack2(lo[4], lo[5]), pack2(lo[6], lo[7]));
                // s_new, y_new are bf16 values already (the pair as stored): exact
                *ring.chunk(D - 1, 3) = make_uint4(pack2(y_new.v[0].x, y_new.v[0].y), pack2(y_new.v[0].z, y_new.v[0].w),
                                                   pack2(y_new.v[1].x, y_new.v[1].y), pack2(y_new.v[1].z, y_new.v[1].w));
                *ring.chunk(D - 1, 4) = make_uint4(pack2(s_new.v[0].x, s_new.v[0].y), pack2(s_new.v[0].z, s_new.v[0].w),
                                                   pack2(s_new.v[1].x, s_new.v[1].y), pack2(s_new.v[1].z, s_new.v[1].w));
            }
            __syncwarp();
            const int mi8 = lane >> 3, ri8 = lane & 7;  // ldmatrix: matrix and row this lane addresses
            uint32_t af[16][2];                         // A fragments (a0, a2) per k-step
#pragma unroll
            for (int c = 0; c < 16; c += 2) {
                const int u = 32 * wid + 2 * (c + (mi8 >> 1)) + (mi8 & 1);  // chunk (thread) index
                const void *src = ri8 < 5 ? (const void *)(ring.row(D - 1, ri8) + 16 * u) : (const void *)&sh.zero16;
                uint32_t r[4];
                ldsm_x4(r, src);
                af[c][0] = r[0];
                af[c][1] = r[1];
                af[c + 1][0] = r[2];
                af[c + 1][1] = r[3];
            }
            int nk = (d - 256 * wid + 15) / 16;  // k-steps of this warp inside d (warp-uniform)
            nk = nk < 0 ? 0 : (nk > 16 ? 16 : nk);
            const int gid = lane >> 2, tig = lane & 3;
            __syncwarp();
            fetch_mm<CT>(L, mri_w, myy_w, dw, count, m, st.head, cn);
            ring.issue(D - 1, D - 1, s_new, y_new);
            for (int k = 0; k < ng; ++k) {
                const int sl = k % D;
                ring.wait();
                // B rows: the group's 8 stored vectors (pair n / 2, s or y); the k-steps
                // accumulate into four independent sets (k-step mod 4), summed after, so
                // that the MMAs are not one dependent chain
                float a4[4][4] = {};
#pragma unroll
                for (int c = 0; c < 16; c += 2) {
                    if (c < nk) {
                        uint32_t b[4];
                        ldsm_x4(b, ring.row(sl, ri8) + 16 * (32 * wid + 2 * (c + (mi8 >> 1)) + (mi8 & 1)));
                        mma_rows8(a4[c & 3], af[c][0], af[c][1], b[0], b[1]);
                        if (c + 1 < nk) mma_rows8(a4[(c + 1) & 3], af[c + 1][0], af[c + 1][1], b[2], b[3]);
                    }
                }
                float acc[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) acc[e] = (a4[0][e] + a4[1][e]) + (a4[2][e] + a4[3][e]);
                // g . v = (g_hi + g_mid) . v + g_lo . v from rows 0, 1, 2
                const float h0 = __shfl_down_sync(0xffffffffu, acc[0], 4);
                const float l0 = __shfl_down_sync(0xffffffffu, acc[0], 8);
                const float h1 = __shfl_down_sync(0xffffffffu, acc[1], 4);
                const float l1 = __shfl_down_sync(0xffffffffu, acc[1], 8);
                const int r = gid == 0 ? 0 : gid == 3 ? 1 : gid == 4 ? 2 : -1;
                if (r >= 0 && tig < PG) {
                    const float2 o = gid == 0 ? make_float2((acc[0] + h0) + l0, (acc[1] + h1) + l1)
                                              : make_float2(acc[0], acc[1]);
                    *reinterpret_cast<float2 *>(p1 + ((k * NW + wid) * 3 + r) * (2 * PG) + 2 * tig) = o;
                }
                __syncwarp();  // the warp has read the group before its slot is refilled
                ring.issue(k + D < ng ? k + D : -1, sl, s_new, y_new);
            }
        }
        cp_async_wait<0>();  // the m x m state
        __syncthreads();
        // product k of logical pair i (k: 0 s.g, 1 y.g, 2 s.y_new, 3 s_new.y, 4 y.y_new):
        // the warps' totals summed in warp order
        auto p1sum = [&](int k, int i) {
            // rows (g, y_new, s_new) x columns (s_q, y_q) of the group's warp totals
            constexpr int rk[5] = {0, 0, 1, 2, 1}, ck[5] = {0, 1, 0, 1, 1};
            const float *src = p1 + ((i / PG) * NW * 3 + rk[k]) * (2 * PG) + 2 * (i % PG) + ck[k];
            float t = 0.f;
#pragma unroll
            for (int q = 0; q < NW; ++q) t += src[q * 3 * 2 * PG];
            return t;
        };
        {
            float *u1 = L.u1(), *u2 = L.u2();
            for (int e = threadIdx.x; e < 2 * count; e += CT) {
                if (e < count)
                    u1[e] = p1sum(0, e);
                else
                    u2[e - count] = p1sum(1, e - count);
            }
        }
        bytes += new_mm<CT>(L, myy_w, dw, count, m, st.head, cn, p1sum);
        g.template load<EVEN>(a.G + (size_t)w * d, d);
        x.template load<EVEN>(a.X + (size_t)w * d, d);
        __syncthreads();
        solve_mm<CT>(sh, L, count, cn, mri_w, m, st.head);
        __syncthreads();
        // pass 2: p = -gamma g - S a + gamma Y w, the groups newest first
        const float gam = sh.gamma;
        p.zero();
        axpyv(-gam, g, p);
        const int r0 = ng > D ? ng - D : 0;  // groups below r0 are no longer in the ring
        const float *ca = L.ca(), *cw = L.cw();
        for (int k = ng - 1; k >= 0; --k) {
            const int sl = k % D;
            if (k < r0) ring.wait();
#pragma unroll
            for (int q = 0; q < PG; ++q) {
                const int i = k * PG + q;
                if (i < count) {
                    Vec<CT> s4, y4;
                    ring.fetch(sl, q, s4, y4);
                    axpyv(-ca[i], s4, p);
                    axpyv(gam * cw[i], y4, p);
                }
            }
            ring.issue(k - D, sl, s_new, y_new);  // this thread's own chunks, just read
        }
        cp_async_wait<0>();  // (only empty groups remain) the ring is free for the next walker
        // the two-loop recursion's history traffic: each pair read in both passes
        bytes += (uint64_t)4 * count * d * sizeof(bf16);
    }
    float dp[2];  // grad f . p and |p|^2
    if (count > 0) {
        dp[0] = dotv(g, p);
        dp[1] = dotv(p, p);
        block_sum<CT, 2>(dp, sh.red2[par++ & 1]);
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
        dp[1] = dotv(p, p);
        block_sum<CT, 2>(dp, sh.red2[par++ & 1]);
    }
    st.dphi = dp[0];
    st.pn = sqrtf(dp[1]);
    st.alpha = 1.f;
    st.bt = 0;
    p.template store<EVEN>(a.P + (size_t)w * d, d);
    lincomb(x, 1.f, p).template store<EVEN>(a.XT + (size_t)w * d, d);
    return bytes + (uint64_t)8 * d;
}

// Algorithmic bytes of the L-BFGS step launches (added only while counting is on).
__device__ unsigned long long g_lbfgs_bytes;

template <int CT, bool EVEN>
__global__ void __launch_bounds__(CT, Cfg<CT>::MINB) k_lbfgs_cta(LbfgsArgs<float> a, float *MRI, float *MYY,
                                                                int count_bytes) {
    __shared__ Shared<CT> sh;
    const int d = a.d, m = a.m, ldh = hist_ld(d);
    const Lay<CT> L(m);
    // the ring starts zeroed: chunks past the row pitch are never copied into and must
    // read as zeros where a k-step of pass 1 straddles the end of the coordinates
    for (int e = threadIdx.x; e < Cfg<CT>::RING_B / 16; e += CT) lb_dyn[e] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (threadIdx.x == 0) {
        sh.zero16 = make_uint4(0u, 0u, 0u, 0u);
    }
    __syncthreads();
    const int n_act = *a.n_act;
    int par = 0;  // alternation of the reduction scratch (identical in every thread)
    uint64_t bytes = 0;
    // the next visit's walker id is loaded one visit ahead, so a visit's first
    // loads (state, vectors) do not wait behind the active-list read
    int w_next = (int)blockIdx.x < n_act ? a.act[blockIdx.x] : 0;
    for (int n = blockIdx.x; n < n_act; n += gridDim.x) {
        const int w = w_next;
        if (n + (int)gridDim.x < n_act) w_next = a.act[n + gridDim.x];
        WalkerState<float> st = a.st[w];  // same address in every thread: one broadcast load
        const float ft = a.FT[w];
        const float alpha0 = st.alpha, pn0 = st.pn;
        float dnext = -1.f;  // bound on |new trial - this visit's trial| (see k_tc_need)
        float *X = a.X + (size_t)w * d;
        float *G = a.G + (size_t)w * d;
        Vec<CT> x, g, xt, gt;
        x.template load<EVEN>(X, d);
        g.template load<EVEN>(G, d);
        xt.template load<EVEN>(a.XT + (size_t)w * d, d);
        gt.template load<EVEN>(a.GT + (size_t)w * d, d);
        bytes += (uint64_t)16 * d + 4 + 2 * sizeof(WalkerState<float>);
        // finiteness of the trial gradient, the candidate pair's inner products and
        // max |grad| at the trial, all in one reduction
        Vec<CT> s4 = subv(xt, x), y4 = subv(gt, g);
#pragma unroll
        for (int q = 0; q < Cfg<CT>::VPT; ++q) {  // the pair as it will be stored
            s4.v[q] = round_bf16(s4.v[q]);
            y4.v[q] = round_bf16(y4.v[q]);
        }
        float r4[4] = {finitev(gt) ? 0.f : 1.f, dotv(s4, s4), dotv(y4, y4), dotv(s4, y4)};
        float gm = absmaxv(gt);
        block_sum_max<CT, 4>(r4, gm, sh.red2[par++ & 1]);
        const bool finite = isfinite(ft) && r4[0] == 0.f;
        bool newiter = false;
        int new_slot = -1;
        Vec<CT> s_new, y_new;
        s_new.zero();
        y_new.zero();
        if (st.phase == 0) {
            x = xt;
            g = gt;
            x.template store<EVEN>(X, d);
            g.template store<EVEN>(G, d);
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
                store_hist<CT>(s4, reinterpret_cast<bf16 *>(a.S) + ((size_t)w * m + slot) * ldh, ldh);
                store_hist<CT>(y4, reinterpret_cast<bf16 *>(a.Y) + ((size_t)w * m + slot) * ldh, ldh);
                bytes += (uint64_t)2 * d * sizeof(bf16);
                new_slot = slot;
                s_new = s4;
                y_new = y4;
            }
            st.flat = (ft >= st.f) ? st.flat + 1 : 0;
            x = xt;
            g = gt;
            x.template store<EVEN>(X, d);
            g.template store<EVEN>(G, d);
            bytes += (uint64_t)8 * d;
            st.f = ft;
            ++st.it;
            newiter = true;
        } else {
            ++st.bt;
            if (st.bt <= a.max_backtracks) {
                st.alpha *= a.backtrack;
                Vec<CT> p;
                p.template load<EVEN>(a.P + (size_t)w * d, d);
                lincomb(x, st.alpha, p).template store<EVEN>(a.XT + (size_t)w * d, d);
                bytes += (uint64_t)8 * d;
                dnext = (alpha0 - st.alpha) * st.pn;
            } else if (st.count > 0 && st.attempt == 0) {
                st.count = 0;
                st.head = 0;
                st.attempt = 1;
                bytes += direction<CT, EVEN>(a, w, st, -1, g, x, s_new, y_new, MRI, MYY, sh, L, par);
                dnext = st.pn + alpha0 * pn0;  // from the old trial back to x, then out
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
                bytes += direction<CT, EVEN>(a, w, st, new_slot, g, x, s_new, y_new, MRI, MYY, sh, L, par);
                dnext = st.pn;  // x is this visit's trial
            }
        }
        if (threadIdx.x == 0) {
            a.st[w] = st;
            if (a.dist && dnext >= 0.f) a.dist[w] = dnext * 1.0001f;  // margin for the rounding of |p|
        }
        // No barrier before the next walker: a thread's ring chunks are read by
        // other lanes only in pass 1, behind warp barriers, and every copy group has
        // completed. The reduction scratch alternates, and every other shared array
        // is rewritten only after the next walker's first reduction barrier.
    }
    if (count_bytes && threadIdx.x == 0 && bytes) atomicAdd(&g_lbfgs_bytes, (unsigned long long)bytes);
}

// The active list of the mixed path, compacted and grouped by each walker's dominant
// component (key[w], the component of the largest term at its latest evaluation;
// -1 goes last), keeping the list order inside a group: the evaluation round skips
// (128-row block, component) pairs no row of the block needs, and walkers of
// different basins interleaved in one block would make every block need every
// component. Skipped terms are exactly zero, so the grouping changes no result.
// Two launches over G CTAs, CTA c owning the list entries [c R, (c + 1) R), R = E x
// threads, E consecutive entries per thread (lane, then warp, then CTA order is list
// order). The first gathers every entry's walker, status and key (independent loads,
// spread over the GPU), packs (bucket, walker) into tmp and counts the buckets per
// CTA; the second reads the G x buckets count table, so CTA c knows where each
// bucket starts and how many entries of it the CTAs before c hold, ranks its entries
// per warp and places each in act. tmp decouples the two, as entries move between
// CTAs' ranges.
constexpr int kSortBuckets = kMaxK + 1;
constexpr int kCompactE = 16;        // most entries per thread
constexpr int kCkThreads = 256;      // threads per CTA
constexpr int kCkMinBlocks = 64;     // CTAs for a short list (one entry per thread up to 16384)
constexpr int kPackShift = 25;       // packed entry: bucket << 25 | walker
constexpr uint32_t kPackDrop = 0xffffffffu;  // a dropped entry (bucket field 127)
static_assert(kSortBuckets < 127, "the bucket field holds 7 bits");

__device__ __forceinline__ int warp_incl_scan(int v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Buckets present in this warp's entries (bit b for bucket b < nb).
__device__ __forceinline__ uint64_t warp_buckets(const uint32_t (&pk)[kCompactE], int E, int nb) {
    uint64_t present = 0;
#pragma unroll
    for (int e = 0; e < kCompactE; ++e) {
        const uint32_t b = pk[e] >> kPackShift;
        if (e < E && b < (uint32_t)nb) present |= 1ull << b;
    }
    return (uint64_t)__reduce_or_sync(0xffffffffu, (uint32_t)present) |
           ((uint64_t)__reduce_or_sync(0xffffffffu, (uint32_t)(present >> 32)) << 32);
}
__device__ __forceinline__ int count_bucket(const uint32_t (&pk)[kCompactE], int E, int b) {
    int cnt = 0;
#pragma unroll
    for (int e = 0; e < kCompactE; ++e) cnt += (e < E && (pk[e] >> kPackShift) == (uint32_t)b);
    return cnt;
}
// entries per thread for prev entries over G CTAs
__device__ __forceinline__ int compact_E(int prev, int G) {
    const int per = G * kCkThreads;
    return (prev + per - 1) / per;
}

// cnt: [G][nb] bucket counts, then cnt[G nb] = the list length before compaction
__global__ void __launch_bounds__(kCkThreads) k_compact_count(const WalkerState<float> *st, const int32_t *act,
                                                              const int32_t *n_act, const int32_t *key, int K,
                                                              uint32_t *tmp, int32_t *cnt) {
    __shared__ int total[kSortBuckets];
    const int prev = *n_act, G = (int)gridDim.x, nb = K + 1;
    const int E = compact_E(prev, G);
    const int lane = threadIdx.x & 31;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) total[b] = 0;
    __syncthreads();
    const int s0 = ((int)blockIdx.x * kCkThreads + (int)threadIdx.x) * E;
    int w[kCompactE];
    uint32_t pk[kCompactE];
#pragma unroll
    for (int e = 0; e < kCompactE; ++e) w[e] = (e < E && s0 + e < prev) ? act[s0 + e] : -1;
#pragma unroll
    for (int e = 0; e < kCompactE; ++e) {
        const bool run = w[e] >= 0 && st[w[e]].status == SB_WALKER_RUNNING;
        const int k = w[e] >= 0 ? key[w[e]] : -1;
        const int b = (k >= 0 && k < K) ? k : K;
        pk[e] = run ? ((uint32_t)b << kPackShift) | (uint32_t)w[e] : kPackDrop;
        if (e < E && s0 + e < prev) tmp[s0 + e] = pk[e];
    }
    for (uint64_t m = warp_buckets(pk, E, nb); m; m &= m - 1) {
        const int b = __ffsll((long long)m) - 1;
        const int sum = __reduce_add_sync(0xffffffffu, count_bucket(pk, E, b));
        if (lane == 0) atomicAdd(&total[b], sum);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nb; b += blockDim.x) cnt[(size_t)blockIdx.x * nb + b] = total[b];
    if (blockIdx.x == 0 && threadIdx.x == 0) cnt[(size_t)G * nb] = prev;
}

__global__ void __launch_bounds__(kCkThreads) k_compact_place(int32_t *act, int32_t *n_act, int64_t *n_evals, int K,
                                                              const uint32_t *tmp, const int32_t *cnt) {
    constexpr int NW = kCkThreads / 32;
    __shared__ int off[kSortBuckets];             // this CTA's first slot of each bucket
    __shared__ int wtot[NW][kSortBuckets], woff[NW][kSortBuckets];
    const int G = (int)gridDim.x, nb = K + 1, c = (int)blockIdx.x;
    const int prev = cnt[(size_t)G * nb];
    const int E = compact_E(prev, G);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (wid == 0) {
        // per bucket: all CTAs' total and the CTAs before c; then the exclusive sums of
        // the totals, 32 buckets at a time
        int carry = 0;
        for (int b0 = 0; b0 < nb; b0 += 32) {
            const int b = b0 + lane;
            int tot = 0, before = 0;
            if (b < nb)
                for (int q = 0; q < G; ++q) {
                    const int v = cnt[(size_t)q * nb + b];
                    tot += v;
                    before += q < c ? v : 0;
                }
            const int incl = warp_incl_scan(tot);
            if (b < nb) off[b] = carry + incl - tot + before;
            carry += __shfl_sync(0xffffffffu, incl, 31);
        }
        if (c == 0 && lane == 0) {
            *n_act = carry;
            if (n_evals) *n_evals += prev;
        }
    }
    const int s0 = (c * kCkThreads + (int)threadIdx.x) * E;
    uint32_t pk[kCompactE];
#pragma unroll
    for (int e = 0; e < kCompactE; ++e) pk[e] = (e < E && s0 + e < prev) ? tmp[s0 + e] : kPackDrop;
    const uint64_t wpres = warp_buckets(pk, E, nb);
    for (int b = lane; b < nb; b += 32) wtot[wid][b] = 0;
    __syncwarp();
    for (uint64_t m = wpres; m; m &= m - 1) {
        const int b = __ffsll((long long)m) - 1;
        const int incl = warp_incl_scan(count_bucket(pk, E, b));
        if (lane == 31) wtot[wid][b] = incl;
    }
    __syncthreads();
    // per bucket: the warps' offsets (a scan over the NW warps' totals)
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        int run = off[b];
        for (int q = 0; q < NW; ++q) {
            woff[q][b] = run;
            run += wtot[q][b];
        }
    }
    __syncthreads();
    for (uint64_t m = wpres; m; m &= m - 1) {
        const int b = __ffsll((long long)m) - 1;
        const int n_b = count_bucket(pk, E, b);
        int pos = woff[wid][b] + warp_incl_scan(n_b) - n_b;
#pragma unroll
        for (int e = 0; e < kCompactE; ++e)
            if (e < E && (pk[e] >> kPackShift) == (uint32_t)b) act[pos++] = (int32_t)(pk[e] & ((1u << kPackShift) - 1u));
    }
}

}  // namespace

int lbfgs_compact_blocks(int n) {
    const int per = kCkThreads * kCompactE;
    const int need = (n + per - 1) / per;
    return need > kCkMinBlocks ? need : kCkMinBlocks;
}

size_t lbfgs_compact_cnt_elems(int n) { return (size_t)lbfgs_compact_blocks(n) * kSortBuckets + 1; }

void launch_lbfgs_compact_by_key(const LbfgsArgs<float> &a, int n, int64_t *n_evals, const int32_t *key, int K,
                                 int32_t *tmp, int32_t *cnt, cudaStream_t s) {
    const int G = lbfgs_compact_blocks(n);
    note_launch();
    k_compact_count<<<G, kCkThreads, 0, s>>>(a.st, a.act, a.n_act, key, K, reinterpret_cast<uint32_t *>(tmp), cnt);
    note_launch();
    k_compact_place<<<G, kCkThreads, 0, s>>>(a.act, a.n_act, n_evals, K, reinterpret_cast<const uint32_t *>(tmp), cnt);
}

bool lbfgs_compact_by_key_fits(int n) { return n >= 0 && n < (1 << kPackShift); }

void launch_lbfgs_step_cta(const LbfgsArgs<float> &a, int n, float *MRI, float *MYY, int num_sms, cudaStream_t s) {
    ProfScope prof(PROF_LBFGS_STEP, s);
    const int count_bytes = prof_class_on(PROF_LBFGS_STEP) ? 1 : 0;
    int grid = num_sms * Cfg<kCT>::MINB;
    if (grid > n) grid = n > 0 ? n : 1;
    const size_t dyn = (size_t)Cfg<kCT>::RING_B + sizeof(float) * mm_floats<kCT>(a.m);
    static std::once_flag once;  // batched solves launch from several host threads
    std::call_once(once, [] {
        const size_t most = (size_t)Cfg<kCT>::RING_B + sizeof(float) * mm_floats<kCT>(kMaxM);
        cudaFuncSetAttribute(k_lbfgs_cta<kCT, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most);
        cudaFuncSetAttribute(k_lbfgs_cta<kCT, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most);
    });
    note_launch();
    // d a multiple of 8 (one whole 16-byte chunk per thread or none): no per-element bounds
    if (a.d % (4 * Cfg<kCT>::VPT) == 0)
        k_lbfgs_cta<kCT, true><<<grid, kCT, dyn, s>>>(a, MRI, MYY, count_bytes);
    else
        k_lbfgs_cta<kCT, false><<<grid, kCT, dyn, s>>>(a, MRI, MYY, count_bytes);
}

double lbfgs_bytes_take() {
    unsigned long long v = 0, z = 0;
    if (cudaDeviceSynchronize() != cudaSuccess) return -1.0;
    if (cudaMemcpyFromSymbol(&v, g_lbfgs_bytes, sizeof(v)) != cudaSuccess) return -1.0;
    if (cudaMemcpyToSymbol(g_lbfgs_bytes, &z, sizeof(z)) != cudaSuccess) return -1.0;
    return (double)v;
}

}  // namespace sb
