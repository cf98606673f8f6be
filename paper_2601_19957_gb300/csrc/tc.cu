// tc.cu -- mixed-precision log-likelihood and gradient on the 5th-generation
// tensor cores (tcgen05, TMEM accumulators, TMA-staged operands), sm_103a.
//
// For points x_n and components k (notation of the FP64 path):
//   GEMM1  z_nk[j]  = sum_{i>=j} (x_n - mu_k)[i] L_k[i][j]     M = points, N = j, K = i
//   LSE    l_n = LSE_k (a_k - |z_nk|^2/2), r_nk = softmax_k    (FP64 reduction of FP32 partials)
//   GEMM2  g_n[i]   = sum_k sum_{j<=i} (r_nk z_nk[j]) L_k[i][j] M = points, N = i, K = (k, j)
// g_n is grad f for f = -l (Sec. 3.2 likelihood, analytic gradient for App. A.5).
//
// Kernel anatomy (one persistent CTA per SM, 10 warps):
//   warps 0-3  build the A tile of each K chunk in shared memory: GEMM1 gathers
//              x rows (walkers through the active list, or ray samples
//              c + t u generated on the fly), subtracts mu_k in FP32 and rounds
//              to bf16 / tf32; GEMM2 scales the stored z rows by r_nk. The tile
//              is written in the 128-byte-swizzled K-major layout the MMA reads.
//   warp 4     TMA loads of the L_k tile (3-D tensor map, OOB rows zero-filled).
//   warp 5     allocates TMEM and issues tcgen05.mma (M=128, N=BN, 4 per chunk).
//   warps 6-9  drain the FP32 accumulator from TMEM (tcgen05.ld) into the
//              epilogue: |z|^2 partials and z (GEMM1), or grad f rows (GEMM2).
// Two TMEM accumulator buffers let the epilogue of one tile overlap the MMAs
// of the next. Only the triangle occupied by L_k is visited (K chunks i >= j0
// for GEMM1, j < i0 + BN for GEMM2). Every mbarrier wait is bounded: on
// timeout the CTA raises SB_DEV_TIMEOUT, drains its TMA loads and MMAs, frees
// TMEM and exits.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "sb_tc.cuh"

namespace sb {

namespace {

constexpr int BM = 128;
constexpr int ROWB = 128;  // bytes of one K chunk per row (one swizzle atom row)
constexpr int THREADS = 320;
constexpr long long kSpinLimit = 1ll << 24;

enum { MODE_ZW = 0, MODE_ZR = 1, MODE_G = 2 };

struct TcArgs {
    int d, K, ld;           // ld: row stride of X (elements)
    const int32_t *n_rows_dev;
    int n_rows_max;
    const int32_t *act;     // compact row -> walker id (null: identity)
    const float *X;         // walker points (FP32)
    const float *mu32;      // [K][d]
    const float *c32;       // [d] box centre
    const double *u;        // [n_rays][d] ray directions
    const double *texit;    // [n_rays]
    int n_steps;
    long long flat0;
    void *Z;                // [rows][K][ldz] (bf16 or fp32)
    int ldz;
    float *qpart;           // [rows][K][n_ntile]
    const float *R;         // [rows][K]
    float *G;               // [walkers][d] grad f
    int n_ntile;
    int32_t *err;
};

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
// Bounded wait: false on timeout or when another role aborted.
__device__ __forceinline__ bool bwait(uint64_t *bar, uint32_t parity, volatile int *abort_flag) {
    for (long long it = 0;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63) == 63) {
            if (*abort_flag) return false;
            if (it > kSpinLimit) {
                *abort_flag = 1;
                return false;
            }
        }
    }
}
// Warp-uniform variants for roles where all 32 lanes take part.
__device__ __forceinline__ bool warp_bwait(uint64_t *bar, uint32_t parity, volatile int *abort_flag) {
    return __all_sync(0xffffffffu, bwait(bar, parity, abort_flag) ? 1 : 0) != 0;
}
__device__ __forceinline__ bool warp_aborted(volatile int *abort_flag) {
    return __any_sync(0xffffffffu, *abort_flag != 0) != 0;
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
        "[%2];" ::"r"(smem_u32(dst)),
        "l"(map), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
        : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row groups 1024 bytes apart (SBO), descriptor version 1.
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(16u >> 4) << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor: D = F32, A/B format fmt (1 = bf16 for kind::f16,
// 2 = tf32 for kind::tf32), both K-major, N = n, M = 128.
__host__ __device__ constexpr uint32_t idesc_make(uint32_t fmt, uint32_t n) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((n >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

template <int PREC>
__device__ __forceinline__ void mma_issue(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accum) {
    if (PREC == SB_PREC_BF16) {
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum));
    } else {
        asm volatile(
            "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
            "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum));
    }
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

#define SB_TMEM_LD32(taddr, v)                                                                                     \
    asm volatile(                                                                                                  \
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,"    \
        "%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"                                         \
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),           \
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),     \
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),   \
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])    \
        : "r"(taddr));                                                                                             \
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory")

__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}

// ------------------------------------------------------------------ tile decoding
struct TileInfo {
    int mb, nt, k;     // row block, output column tile, component (GEMM1)
    int c_lo, c_hi;    // K-chunk range (GEMM1) or chunk count per component (GEMM2: c_hi)
    int nchunks;
};

template <int MODE, int BN, int KC>
__device__ __forceinline__ TileInfo decode_tile(int t, int d, int K) {
    TileInfo ti;
    const int nct = (d + BN - 1) / BN;
    if (MODE == MODE_G) {
        ti.nt = t % nct;
        ti.mb = t / nct;
        ti.k = 0;
        const int jmax = min(d, (ti.nt + 1) * BN);
        ti.c_lo = 0;
        ti.c_hi = (jmax + KC - 1) / KC;
        ti.nchunks = K * ti.c_hi;
    } else {
        ti.k = t % K;
        ti.nt = (t / K) % nct;
        ti.mb = t / (K * nct);
        ti.c_lo = (ti.nt * BN) / KC;
        ti.c_hi = (d + KC - 1) / KC;
        ti.nchunks = ti.c_hi - ti.c_lo;
    }
    return ti;
}

// ------------------------------------------------------------------ the kernel
template <int BN, int PREC, int MODE>
__global__ void __launch_bounds__(THREADS, 1) k_tc_gemm(const __grid_constant__ CUtensorMap tmapB, TcArgs a) {
    constexpr int KC = (PREC == SB_PREC_BF16) ? 64 : 32;  // elements per 128-byte chunk row
    constexpr int STAGES = (BN >= 256) ? 4 : 6;
    constexpr int A_BYTES = BM * ROWB;
    constexpr int B_BYTES = BN * ROWB;
    constexpr uint32_t IDESC = idesc_make(PREC == SB_PREC_BF16 ? 1u : 2u, BN);

    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *sA = smem;
    uint8_t *sB = smem + STAGES * A_BYTES;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sB + STAGES * B_BYTES);
    uint64_t *full_a = bars;
    uint64_t *full_b = bars + STAGES;
    uint64_t *empty = bars + 2 * STAGES;
    uint64_t *tfull = bars + 3 * STAGES;
    uint64_t *tempty = tfull + 2;
    uint64_t *drain = tempty + 2;
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(drain + 1);
    volatile int *s_abort = reinterpret_cast<volatile int *>(s_tmem + 1);
    int *s_row = const_cast<int *>(reinterpret_cast<volatile int *>(s_abort + 1));  // [BM] per-row source
    float *s_scale = reinterpret_cast<float *>(s_row + BM);                          // [BM] ray t * t_exit

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int d = a.d, K = a.K;
    const int n_rows = a.n_rows_dev ? *a.n_rows_dev : a.n_rows_max;
    const int n_mblk = (n_rows + BM - 1) / BM;
    const int nct = (d + BN - 1) / BN;
    const int n_tiles = (MODE == MODE_G) ? n_mblk * nct : n_mblk * nct * K;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full_a[s], 4);
            mbar_init(&full_b[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&tfull[s], 1);
            mbar_init(&tempty[s], 4);
        }
        mbar_init(drain, 1);
        *s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 5) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_tmem)),
                     "r"(2 * BN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *s_tmem;

    if (warp < 4) {
        // ---------------------------------------------------------- A producers
        int stage = 0;
        uint32_t phase = 0;
        const int sub = lane >> 4;          // bf16: lanes 0-15 row r, 16-31 row r+1
        const int l16 = lane & 15;
        for (int t = blockIdx.x; t < n_tiles && !warp_aborted(s_abort); t += gridDim.x) {
            const TileInfo ti = decode_tile<MODE, BN, KC>(t, d, K);
            // per-row sources of this warp's 32 rows
            {
                const int r = warp * 32 + lane;
                const int n = ti.mb * BM + r;
                int src = -1;
                float sc = 0.f;
                if (n < n_rows) {
                    if (MODE == MODE_ZW) {
                        src = a.act ? a.act[n] : n;
                    } else if (MODE == MODE_ZR) {
                        const long long flat = a.flat0 + n;
                        const int ray = (int)(flat / a.n_steps), j = (int)(flat % a.n_steps);
                        src = ray;
                        sc = (float)(((double)(j + 1) / (double)a.n_steps) * a.texit[ray]);
                    } else {
                        src = n;
                    }
                }
                s_row[r] = src;
                s_scale[r] = sc;
            }
            __syncwarp();
            for (int q = 0; q < ti.nchunks; ++q) {
                int kk, c0;
                if (MODE == MODE_G) {
                    kk = q / ti.c_hi;
                    c0 = (q % ti.c_hi) * KC;
                } else {
                    kk = ti.k;
                    c0 = (ti.c_lo + q) * KC;
                }
                if (!warp_bwait(&empty[stage], phase ^ 1, s_abort)) break;
                uint8_t *tile = sA + stage * A_BYTES;
                if (PREC == SB_PREC_BF16) {
                    // each lane: 4 consecutive columns (8 bytes of the swizzled row)
                    const int col = c0 + 4 * l16;
                    float m4[4] = {0.f, 0.f, 0.f, 0.f}, c4[4] = {0.f, 0.f, 0.f, 0.f};
                    if (MODE != MODE_G) {
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            if (col + e < d) {
                                m4[e] = a.mu32[(size_t)kk * d + col + e];
                                if (MODE == MODE_ZR) c4[e] = a.c32[col + e];
                            }
                    }
#pragma unroll 4
                    for (int rr = 0; rr < 16; ++rr) {
                        const int r = warp * 32 + 2 * rr + sub;
                        const int src = s_row[r];
                        float v[4] = {0.f, 0.f, 0.f, 0.f};
                        if (src >= 0) {
                            if (MODE == MODE_ZW) {
                                const float *xr = a.X + (size_t)src * a.ld;
                                if (((a.ld & 3) == 0) && col + 3 < d) {
                                    const float4 x4 = *reinterpret_cast<const float4 *>(xr + col);
                                    v[0] = x4.x - m4[0];
                                    v[1] = x4.y - m4[1];
                                    v[2] = x4.z - m4[2];
                                    v[3] = x4.w - m4[3];
                                } else {
#pragma unroll
                                    for (int e = 0; e < 4; ++e)
                                        if (col + e < d) v[e] = xr[col + e] - m4[e];
                                }
                            } else if (MODE == MODE_ZR) {
                                const double *ur = a.u + (size_t)src * d;
                                const float sc = s_scale[r];
#pragma unroll
                                for (int e = 0; e < 4; ++e)
                                    if (col + e < d) v[e] = (c4[e] + sc * (float)ur[col + e]) - m4[e];
                            } else {
                                const float rk = a.R[(size_t)src * K + kk];
                                if (rk != 0.f) {
                                    const __nv_bfloat16 *zr = reinterpret_cast<const __nv_bfloat16 *>(a.Z) +
                                                              ((size_t)src * K + kk) * a.ldz;
                                    if (col + 3 < a.ldz) {
                                        const uint2 z2 = *reinterpret_cast<const uint2 *>(zr + col);
                                        const __nv_bfloat162 p0 = *reinterpret_cast<const __nv_bfloat162 *>(&z2.x);
                                        const __nv_bfloat162 p1 = *reinterpret_cast<const __nv_bfloat162 *>(&z2.y);
                                        v[0] = __low2float(p0) * rk;
                                        v[1] = __high2float(p0) * rk;
                                        v[2] = __low2float(p1) * rk;
                                        v[3] = __high2float(p1) * rk;
                                    }
                                    if (col + 3 >= d) {
#pragma unroll
                                        for (int e = 0; e < 4; ++e)
                                            if (col + e >= d) v[e] = 0.f;
                                    }
                                }
                            }
                        }
                        uint2 packed;
                        packed.x = pack_bf16x2(v[0], v[1]);
                        packed.y = pack_bf16x2(v[2], v[3]);
                        const int chunk = (l16 >> 1) ^ (r & 7);
                        *reinterpret_cast<uint2 *>(tile + r * ROWB + chunk * 16 + (l16 & 1) * 8) = packed;
                    }
                } else {
                    // TF32: each lane 4 columns = one 16-byte chunk; 4 rows per warp step
                    const int l8 = lane & 7, sub4 = lane >> 3;
                    const int col = c0 + 4 * l8;
                    float m4[4] = {0.f, 0.f, 0.f, 0.f}, c4[4] = {0.f, 0.f, 0.f, 0.f};
                    if (MODE != MODE_G) {
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            if (col + e < d) {
                                m4[e] = a.mu32[(size_t)kk * d + col + e];
                                if (MODE == MODE_ZR) c4[e] = a.c32[col + e];
                            }
                    }
#pragma unroll 2
                    for (int rr = 0; rr < 8; ++rr) {
                        const int r = warp * 32 + 4 * rr + sub4;
                        const int src = s_row[r];
                        float v[4] = {0.f, 0.f, 0.f, 0.f};
                        if (src >= 0) {
                            if (MODE == MODE_ZW) {
                                const float *xr = a.X + (size_t)src * a.ld;
                                if (((a.ld & 3) == 0) && col + 3 < d) {
                                    const float4 x4 = *reinterpret_cast<const float4 *>(xr + col);
                                    v[0] = x4.x - m4[0];
                                    v[1] = x4.y - m4[1];
                                    v[2] = x4.z - m4[2];
                                    v[3] = x4.w - m4[3];
                                } else {
#pragma unroll
                                    for (int e = 0; e < 4; ++e)
                                        if (col + e < d) v[e] = xr[col + e] - m4[e];
                                }
                            } else if (MODE == MODE_ZR) {
                                const double *ur = a.u + (size_t)src * d;
                                const float sc = s_scale[r];
#pragma unroll
                                for (int e = 0; e < 4; ++e)
                                    if (col + e < d) v[e] = (c4[e] + sc * (float)ur[col + e]) - m4[e];
                            } else {
                                const float rk = a.R[(size_t)src * K + kk];
                                if (rk != 0.f) {
                                    const float *zr =
                                        reinterpret_cast<const float *>(a.Z) + ((size_t)src * K + kk) * a.ldz;
#pragma unroll
                                    for (int e = 0; e < 4; ++e)
                                        if (col + e < d) v[e] = zr[col + e] * rk;
                                }
                            }
                        }
                        float4 o;
                        o.x = to_tf32(v[0]);
                        o.y = to_tf32(v[1]);
                        o.z = to_tf32(v[2]);
                        o.w = to_tf32(v[3]);
                        const int chunk = l8 ^ (r & 7);
                        *reinterpret_cast<float4 *>(tile + r * ROWB + chunk * 16) = o;
                    }
                }
                fence_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(&full_a[stage]);
                if (++stage == STAGES) {
                    stage = 0;
                    phase ^= 1;
                }
            }
        }
    } else if (warp == 4) {
        // ---------------------------------------------------------- TMA loads of L_k tiles
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int inflight_stage[8];
            uint32_t inflight_phase[8];
            int n_inflight = 0;
            for (int t = blockIdx.x; t < n_tiles && !*s_abort; t += gridDim.x) {
                const TileInfo ti = decode_tile<MODE, BN, KC>(t, d, K);
                bool ok = true;
                for (int q = 0; q < ti.nchunks; ++q) {
                    if (!bwait(&empty[stage], phase ^ 1, s_abort)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_tx(&full_b[stage], B_BYTES);
                    if (MODE == MODE_G) {
                        const int kk = q / ti.c_hi, j0 = (q % ti.c_hi) * KC;
                        tma_load_3d(sB + stage * B_BYTES, &tmapB, &full_b[stage], j0, ti.nt * BN, kk);
                    } else {
                        tma_load_3d(sB + stage * B_BYTES, &tmapB, &full_b[stage], (ti.c_lo + q) * KC, ti.nt * BN,
                                    ti.k);
                    }
                    inflight_stage[n_inflight % 8] = stage;
                    inflight_phase[n_inflight % 8] = phase;
                    ++n_inflight;
                    if (++stage == STAGES) {
                        stage = 0;
                        phase ^= 1;
                    }
                }
                if (!ok) break;
            }
            if (*s_abort) {
                // let the copies already issued land before the CTA exits (bounded)
                const int first = n_inflight > STAGES ? n_inflight - STAGES : 0;
                for (int q = first; q < n_inflight; ++q) {
                    volatile int never = 0;
                    bwait(&full_b[inflight_stage[q % 8]], inflight_phase[q % 8], &never);
                }
            }
        }
    } else if (warp == 5) {
        // ---------------------------------------------------------- MMA issue
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int acc = 0;
            uint32_t acc_phase = 0;
            bool issued = false;
            for (int t = blockIdx.x; t < n_tiles && !*s_abort; t += gridDim.x) {
                const TileInfo ti = decode_tile<MODE, BN, KC>(t, d, K);
                if (!bwait(&tempty[acc], acc_phase ^ 1, s_abort)) break;
                tc_fence_after();
                const uint32_t dt = tmem + (uint32_t)(acc * BN);
                bool ok = true;
                for (int q = 0; q < ti.nchunks; ++q) {
                    if (!bwait(&full_a[stage], phase, s_abort) || !bwait(&full_b[stage], phase, s_abort)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t ad = sdesc_sw128(smem_u32(sA + stage * A_BYTES));
                    const uint64_t bd = sdesc_sw128(smem_u32(sB + stage * B_BYTES));
#pragma unroll
                    for (int s = 0; s < 4; ++s)
                        mma_issue<PREC>(dt, ad + (uint64_t)(2 * s), bd + (uint64_t)(2 * s), IDESC,
                                        (q > 0 || s > 0) ? 1u : 0u);
                    issued = true;
                    mma_commit(&empty[stage]);
                    if (++stage == STAGES) {
                        stage = 0;
                        phase ^= 1;
                    }
                }
                if (!ok) break;
                mma_commit(&tfull[acc]);
                if (++acc == 2) {
                    acc = 0;
                    acc_phase ^= 1;
                }
            }
            if (*s_abort && issued) {
                // wait for every MMA issued so far before TMEM is released
                mma_commit(drain);
                volatile int never = 0;
                bwait(drain, 0, &never);
            }
        }
        __syncwarp();
    } else {
        // ---------------------------------------------------------- epilogue
        const int quad = warp & 3;
        const int r = quad * 32 + lane;
        int acc = 0;
        uint32_t acc_phase = 0;
        for (int t = blockIdx.x; t < n_tiles && !warp_aborted(s_abort); t += gridDim.x) {
            const TileInfo ti = decode_tile<MODE, BN, KC>(t, d, K);
            if (!warp_bwait(&tfull[acc], acc_phase, s_abort)) break;
            tc_fence_after();
            const int n = ti.mb * BM + r;
            const bool valid = n < n_rows;
            const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(acc * BN);
            float q2 = 0.f;
#pragma unroll 1
            for (int c0 = 0; c0 < BN; c0 += 32) {
                uint32_t v[32];
                SB_TMEM_LD32(taddr + c0, v);
                const int col = ti.nt * BN + c0;
                if (MODE == MODE_G) {
                    if (valid && col < d) {
                        const int w = a.act ? a.act[n] : n;
                        float *g = a.G + (size_t)w * d + col;
                        if ((d & 3) == 0 && col + 32 <= d) {
#pragma unroll
                            for (int e = 0; e < 32; e += 4)
                                *reinterpret_cast<float4 *>(g + e) =
                                    make_float4(__uint_as_float(v[e]), __uint_as_float(v[e + 1]),
                                                __uint_as_float(v[e + 2]), __uint_as_float(v[e + 3]));
                        } else {
#pragma unroll
                            for (int e = 0; e < 32; ++e)
                                if (col + e < d) g[e] = __uint_as_float(v[e]);
                        }
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < 32; ++e) {
                        const float z = __uint_as_float(v[e]);
                        q2 = fmaf(z, z, q2);
                    }
                    if (MODE == MODE_ZW && valid && col < a.ldz) {
                        if (PREC == SB_PREC_BF16) {
                            __nv_bfloat16 *zr =
                                reinterpret_cast<__nv_bfloat16 *>(a.Z) + ((size_t)n * K + ti.k) * a.ldz + col;
#pragma unroll
                            for (int e = 0; e < 32; e += 8) {
                                if (col + e + 8 <= a.ldz) {
                                    uint4 p;
                                    p.x = pack_bf16x2(__uint_as_float(v[e]), __uint_as_float(v[e + 1]));
                                    p.y = pack_bf16x2(__uint_as_float(v[e + 2]), __uint_as_float(v[e + 3]));
                                    p.z = pack_bf16x2(__uint_as_float(v[e + 4]), __uint_as_float(v[e + 5]));
                                    p.w = pack_bf16x2(__uint_as_float(v[e + 6]), __uint_as_float(v[e + 7]));
                                    *reinterpret_cast<uint4 *>(zr + e) = p;
                                }
                            }
                        } else {
                            float *zr = reinterpret_cast<float *>(a.Z) + ((size_t)n * K + ti.k) * a.ldz + col;
#pragma unroll
                            for (int e = 0; e < 32; e += 4)
                                if (col + e + 4 <= a.ldz)
                                    *reinterpret_cast<float4 *>(zr + e) =
                                        make_float4(__uint_as_float(v[e]), __uint_as_float(v[e + 1]),
                                                    __uint_as_float(v[e + 2]), __uint_as_float(v[e + 3]));
                        }
                    }
                }
            }
            if (MODE != MODE_G && valid) a.qpart[((size_t)n * K + ti.k) * a.n_ntile + ti.nt] = q2;
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[acc]);
            if (++acc == 2) {
                acc = 0;
                acc_phase ^= 1;
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (*s_abort && threadIdx.x == 0) atomicOr(a.err, SB_DEV_TIMEOUT);
    if (warp == 5) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * BN));
    }
}

// ------------------------------------------------------------------ small kernels
// LSE over components from the FP32 |z|^2 partials, in FP64.
// mode 0: walkers (FT[act[n]] = -l, R); mode 1: ray samples (ell[flat0 + n] = l);
// mode 2: points (ell[n] = l, R).
__global__ void __launch_bounds__(256) k_tc_lse(int mode, int K, int n_ntile, const int32_t *n_rows_dev,
                                                int n_rows_max, const int32_t *act, const float *qpart,
                                                const double *a_k, float *R, float *FT, double *ell) {
    const int n_rows = n_rows_dev ? *n_rows_dev : n_rows_max;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= n_rows) return;
    double e[kMaxK];
    double emax = -INFINITY;
    for (int k = 0; k < K; ++k) {
        const float *qp = qpart + ((size_t)n * K + k) * n_ntile;
        double q = 0.0;
        for (int t = 0; t < n_ntile; ++t) q += (double)qp[t];
        e[k] = a_k[k] - 0.5 * q;
        emax = fmax(emax, e[k]);
    }
    double s = 0.0;
    for (int k = 0; k < K; ++k) s += exp(e[k] - emax);
    const double l = emax + log(s);
    if (mode == 1) {
        ell[n] = l;
        return;
    }
    for (int k = 0; k < K; ++k) R[(size_t)n * K + k] = (float)(exp(e[k] - emax) / s);
    if (mode == 0)
        FT[act ? act[n] : n] = (float)(-l);
    else
        ell[n] = l;
}

template <typename E>
__global__ void k_tc_convert_L(int d, int K, int ldp, const double *L, E *LT, E *LB) {
    const size_t tot = (size_t)K * d * ldp;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(e / ((size_t)d * ldp));
        const size_t rem = e % ((size_t)d * ldp);
        const int row = (int)(rem / ldp), col = (int)(rem % ldp);
        double lt = 0.0, lb = 0.0;
        if (col < d) {
            const double *Lk = L + (size_t)k * d * d;
            if (col >= row) lt = Lk[(size_t)col * d + row];  // LT[k][j=row][i=col] = L[i][j], i >= j
            if (col <= row) lb = Lk[(size_t)row * d + col];  // LB[k][i=row][j=col] = L[i][j], j <= i
        }
        if (sizeof(E) == 2) {
            reinterpret_cast<__nv_bfloat16 *>(LT)[e] = __double2bfloat16(lt);
            reinterpret_cast<__nv_bfloat16 *>(LB)[e] = __double2bfloat16(lb);
        } else {
            reinterpret_cast<float *>(LT)[e] = to_tf32((float)lt);
            reinterpret_cast<float *>(LB)[e] = to_tf32((float)lb);
        }
    }
}

__global__ void k_tc_convert_vec(int d, int K, const double *mu, const double *c, float *mu32, float *c32) {
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < K * d; e += gridDim.x * blockDim.x) {
        mu32[e] = (float)mu[e];
        if (e < d && c) c32[e] = (float)c[e];
    }
}

__global__ void k_tc_points_in(int n, int d, const double *x, float *X) {
    const size_t tot = (size_t)n * d;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x)
        X[e] = (float)x[e];
}

__global__ void k_tc_points_out(int n, int d, const float *G, double *grad) {
    const size_t tot = (size_t)n * d;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x)
        grad[e] = -(double)G[e];  // G holds grad f = -grad l
}

// ------------------------------------------------------------------ host side
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

int num_sms() {
    static int n = 0;
    static std::once_flag once;
    std::call_once(once, [] {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    });
    return n;
}

inline int esz(int prec) { return prec == SB_PREC_BF16 ? 2 : 4; }
inline int ldp_of(int d, int prec) { return prec == SB_PREC_BF16 ? (d + 7) / 8 * 8 : (d + 3) / 4 * 4; }
inline int bn_of(int d) { return d > 128 ? 256 : (d > 64 ? 128 : 64); }
inline int ldz_of(int d) { return (d + 63) / 64 * 64; }

// 3-D map over [K][d rows][ldp] with box (128 bytes of K, BN rows, 1).
bool make_map(CUtensorMap *m, void *base, int d, int K, int prec, int bn) {
    auto fn = encode_fn();
    if (!fn) return false;
    const int e = esz(prec);
    const int ldp = ldp_of(d, prec);
    cuuint64_t dims[3] = {(cuuint64_t)d, (cuuint64_t)d, (cuuint64_t)K};
    cuuint64_t strides[2] = {(cuuint64_t)ldp * e, (cuuint64_t)ldp * e * d};
    cuuint32_t box[3] = {(cuuint32_t)(128 / e), (cuuint32_t)bn, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    const CUtensorMapDataType dt =
        prec == SB_PREC_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    return fn(m, dt, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN, int PREC, int MODE>
constexpr int smem_bytes() {
    constexpr int STAGES = (BN >= 256) ? 4 : 6;
    return 1024 + STAGES * (BM * ROWB + BN * ROWB) + (3 * STAGES + 5) * 8 + 16 + BM * 8 + 64;
}

template <int BN, int PREC, int MODE>
void launch_gemm(const CUtensorMap &map, const TcArgs &a, cudaStream_t s) {
    constexpr int SM = smem_bytes<BN, PREC, MODE>();
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(k_tc_gemm<BN, PREC, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, SM);
    });
    const int nct = (a.d + BN - 1) / BN;
    const int mb = (a.n_rows_max + BM - 1) / BM;
    long long tiles = (long long)mb * nct * (MODE == MODE_G ? 1 : a.K);
    int grid = num_sms();
    if (tiles < grid) grid = (int)(tiles > 0 ? tiles : 1);
    ProfScope prof(MODE == MODE_ZW ? PROF_TC_Z_WALKERS : (MODE == MODE_ZR ? PROF_TC_Z_RAYS : PROF_TC_GRAD), s);
    note_launch();
    k_tc_gemm<BN, PREC, MODE><<<grid, THREADS, SM, s>>>(map, a);
}

template <int PREC, int MODE>
void launch_gemm_bn(int bn, const CUtensorMap &map, const TcArgs &a, cudaStream_t s) {
    if (bn == 256)
        launch_gemm<256, PREC, MODE>(map, a, s);
    else if (bn == 128)
        launch_gemm<128, PREC, MODE>(map, a, s);
    else
        launch_gemm<64, PREC, MODE>(map, a, s);
}

void launch_gemm_any(int prec, int mode, int bn, const CUtensorMap &map, const TcArgs &a, cudaStream_t s) {
    if (prec == SB_PREC_BF16) {
        if (mode == MODE_ZW) launch_gemm_bn<SB_PREC_BF16, MODE_ZW>(bn, map, a, s);
        else if (mode == MODE_ZR) launch_gemm_bn<SB_PREC_BF16, MODE_ZR>(bn, map, a, s);
        else launch_gemm_bn<SB_PREC_BF16, MODE_G>(bn, map, a, s);
    } else {
        if (mode == MODE_ZW) launch_gemm_bn<SB_PREC_TF32, MODE_ZW>(bn, map, a, s);
        else if (mode == MODE_ZR) launch_gemm_bn<SB_PREC_TF32, MODE_ZR>(bn, map, a, s);
        else launch_gemm_bn<SB_PREC_TF32, MODE_G>(bn, map, a, s);
    }
}

TcArgs base_args(const ProbView &pv, const TcWs &t) {
    TcArgs a{};
    a.d = pv.d;
    a.K = pv.K;
    a.mu32 = (const float *)t.p[2];
    a.c32 = (const float *)t.p[3];
    a.Z = t.p[4];
    a.ldz = ldz_of(pv.d);
    a.qpart = (float *)t.p[5];
    a.R = (const float *)t.p[6];
    a.n_ntile = (pv.d + t.bn - 1) / t.bn;
    a.err = pv.status;
    return a;
}

}  // namespace

bool tc_available(int prec) { return (prec == SB_PREC_BF16 || prec == SB_PREC_TF32) && encode_fn() != nullptr; }

// Layout: [0] LT, [1] LB, [2] mu32, [3] c32, [4] Z, [5] qpart, [6] R, [7] X32 (points), [8] G32 (points)
void carve_tc(Carver &cv, TcWs &t, int rows, int d, int K, int prec) {
    const int e = esz(prec), ldp = ldp_of(d, prec), bn = bn_of(d);
    const int nct = (d + bn - 1) / bn;
    t.rows = rows;
    t.prec = prec;
    t.bn = bn;
    t.p[0] = cv.take<uint8_t>((size_t)K * d * ldp * e);
    t.p[1] = cv.take<uint8_t>((size_t)K * d * ldp * e);
    t.p[2] = cv.take<float>((size_t)K * d);
    t.p[3] = cv.take<float>((size_t)d);
    t.p[4] = cv.take<uint8_t>((size_t)rows * K * ldz_of(d) * e);
    t.p[5] = cv.take<float>((size_t)rows * K * nct);
    t.p[6] = cv.take<float>((size_t)rows * K);
    t.p[7] = cv.take<float>((size_t)rows * d);
    t.p[8] = cv.take<float>((size_t)rows * d);
}

int tc_ray_chunk(int d, int K, int64_t total) {
    (void)d;
    (void)K;
    const int64_t b = 65536;
    return (int)(total < b ? total : b);
}

sb_status tc_prepare(const ProbView &pv, TcWs &t, cudaStream_t s) {
    const int d = pv.d, K = pv.K;
    const int ldp = ldp_of(d, t.prec);
    note_launch();
    if (t.prec == SB_PREC_BF16)
        k_tc_convert_L<uint16_t><<<1184, 256, 0, s>>>(d, K, ldp, pv.L, (uint16_t *)t.p[0], (uint16_t *)t.p[1]);
    else
        k_tc_convert_L<float><<<1184, 256, 0, s>>>(d, K, ldp, pv.L, (float *)t.p[0], (float *)t.p[1]);
    note_launch();
    k_tc_convert_vec<<<(K * d + 255) / 256, 256, 0, s>>>(d, K, pv.mu, pv.c, (float *)t.p[2], (float *)t.p[3]);
    if (!make_map(&t.mapT, t.p[0], d, K, t.prec, t.bn) || !make_map(&t.mapB, t.p[1], d, K, t.prec, t.bn))
        return SB_ERR_CUDA;
    return cudaGetLastError() == cudaSuccess ? SB_OK : SB_ERR_CUDA;
}

sb_status tc_ray_loglik(const ProbView &pv, const sb_config *c, const TcWs &t, const double *u, const double *texit,
                        double *ell_all, cudaStream_t s) {
    const int64_t total = (int64_t)c->n_rays * c->n_steps;
    for (int64_t f0 = 0; f0 < total; f0 += (int64_t)t.rows) {
        const int rows = (int)((total - f0) < (int64_t)t.rows ? (total - f0) : (int64_t)t.rows);
        TcArgs a = base_args(pv, t);
        a.n_rows_max = rows;
        a.u = u;
        a.texit = texit;
        a.n_steps = c->n_steps;
        a.flat0 = f0;
        launch_gemm_any(t.prec, MODE_ZR, t.bn, t.mapT, a, s);
        note_launch();
        k_tc_lse<<<(rows + 255) / 256, 256, 0, s>>>(1, pv.K, a.n_ntile, nullptr, rows, nullptr, a.qpart, pv.a,
                                                    nullptr, nullptr, ell_all + f0);
    }
    return cudaGetLastError() == cudaSuccess ? SB_OK : SB_ERR_CUDA;
}

void tc_eval_walkers(const ProbView &pv, const sb_config *c, const TcWs &t, const float *XT, const int32_t *act,
                     const int32_t *n_act, int n, float *FT, float *GT, cudaStream_t s) {
    (void)c;
    TcArgs a = base_args(pv, t);
    a.X = XT;
    a.ld = pv.d;
    a.act = act;
    a.n_rows_dev = n_act;
    a.n_rows_max = n;
    launch_gemm_any(t.prec, MODE_ZW, t.bn, t.mapT, a, s);
    note_launch();
    k_tc_lse<<<(n + 255) / 256, 256, 0, s>>>(0, pv.K, a.n_ntile, n_act, n, act, a.qpart, pv.a, (float *)t.p[6], FT,
                                             nullptr);
    a.G = GT;
    launch_gemm_any(t.prec, MODE_G, t.bn, t.mapB, a, s);
}

sb_status tc_loglik_points(const ProbView &pv, const sb_config *c, const TcWs &t, const double *x, int n, float *f,
                           float *g, double *ell, double *grad, cudaStream_t s) {
    (void)c;
    (void)f;
    float *X = (float *)t.p[7];
    float *G = g ? g : (float *)t.p[8];
    note_launch();
    k_tc_points_in<<<(unsigned)(((size_t)n * pv.d + 255) / 256 < 4096 ? ((size_t)n * pv.d + 255) / 256 : 4096), 256,
                     0, s>>>(n, pv.d, x, X);
    TcArgs a = base_args(pv, t);
    a.X = X;
    a.ld = pv.d;
    a.n_rows_max = n;
    launch_gemm_any(t.prec, MODE_ZW, t.bn, t.mapT, a, s);
    note_launch();
    k_tc_lse<<<(n + 255) / 256, 256, 0, s>>>(2, pv.K, a.n_ntile, nullptr, n, nullptr, a.qpart, pv.a,
                                             (float *)t.p[6], nullptr, ell);
    if (grad) {
        a.G = G;
        launch_gemm_any(t.prec, MODE_G, t.bn, t.mapB, a, s);
        note_launch();
        k_tc_points_out<<<(unsigned)(((size_t)n * pv.d + 255) / 256 < 4096 ? ((size_t)n * pv.d + 255) / 256 : 4096),
                          256, 0, s>>>(n, pv.d, G, grad);
    }
    return cudaGetLastError() == cudaSuccess ? SB_OK : SB_ERR_CUDA;
}

}  // namespace sb
