// tc.cu -- mixed-precision log-likelihood and gradient on the 5th-generation
// tensor cores (tcgen05, TMEM accumulators, TMA-staged operands), sm_103a.
//
// For points x_n and components k (notation of the FP64 path):
//   GEMM1  z_nk[j]  = sum_{i>=j} (x_n - mu_k)[i] L_k[i][j]     M = points, N = j, K = i
//   LSE    l_n = LSE_k (a_k - |z_nk|^2/2), r_nk = softmax_k    (FP64 reduction of FP32 partials)
//   GEMM2  g_n[i]   = sum_k sum_{j<=i} (r_nk z_nk[j]) L_k[i][j] M = points, N = i, K = (k, j)
// g_n is grad f for f = -l (Sec. 3.2 likelihood, analytic gradient for App. A.5).
//
// Data flow per evaluation round:
//   k_tc_need     (walker rounds) the (128-row block, component) pairs whose term
//                 can still reach l, from per-walker bounds on |z_k| and on the
//                 largest term (a skipped term is below FP32 resolution: exactly 0)
//   k_tc_center   A1[k][n][:] = round(x_n - mu_k), formed in FP32 (walkers gathered
//                 through the active list), bf16 or tf32
//   k_tc_gemm ZW  z = A1 L_k (GEMM1) for the kept pairs: |z|^2 partials, and z
//                 itself stored (bf16 / tf32) as Z[k][n][:] when the gradient is wanted
//                 (ZR: the |z|^2 partials only, for l alone)
//   k_tc_lse      l, r; flags of the (128-row block, component) pairs with r > 0,
//                 marking those whose live rows all have r = 1 exactly
//   k_tc_scale_z  Z[k][n][:] = round(r_nk z_nk) for the flagged pairs (the A
//                 operand of GEMM2; rows with r_nk = 0 become zeros), except the
//                 pairs with r = 1 throughout, where it is the identity
//   k_tc_gemm G   grad f = sum_k Z_k L_k^T rows over the flagged components (GEMM2)
// With separated modes most responsibilities are exactly 0 in FP32 (the
// exponent underflows), so the scaling pass and GEMM2 visit a fraction of the
// K components; the terms they skip are exactly zero.
// Both operands of both GEMMs reach shared memory by TMA (3-D tensor maps,
// 128-byte swizzle, out-of-range rows/columns zero-filled), so the MMA
// pipeline never waits on a gathered load. Centring before rounding keeps the
// stationary point: at x = mu_k the A operand is exactly zero.
//
// Rays (x = o + tau u) take another route, the quadratic form in tau (Q below):
//   k_tc_gemm Q   w = L_k^T u from split operands u_hi L_hi + u_lo L_hi + u_hi L_lo
//                 (about FP32 accuracy) with q1 = z_k(o) . w and q2 = |w|^2 partials;
//                 from per-ray origins a first pass stores z_k(o) = o L_k - mu_k L_k
//   k_q_ell       l at every sample from q0 + 2 tau q1 + tau^2 q2 (FP64)
//
// Kernel anatomy (one persistent CTA per SM, 6 warps): warp 0 issues the TMA
// loads of A and B for each 128-byte K chunk; warp 1 allocates TMEM and issues
// tcgen05.mma (M=128, N=BN<=256, four per chunk) with tcgen05.commit to the
// stage's empty barrier; warps 2-5 drain the FP32 accumulator with
// tcgen05.ld (one thread per row). Two TMEM accumulators let the epilogue of
// one tile overlap the MMAs of the next. Only the triangle occupied by L_k is
// visited (K chunks i >= j0 for GEMM1, j < i0 + BN for GEMM2). Every mbarrier
// wait is bounded: on timeout the CTA raises SB_DEV_TIMEOUT, lets its issued
// TMA loads and MMAs land, frees TMEM and exits.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>

#include "sb_ptx.cuh"
#include "sb_tc.cuh"

namespace sb {

namespace {

constexpr int BM = 128;
constexpr int ROWB = 128;  // bytes of one K chunk per row (one swizzle atom row)
constexpr int THREADS = 192;
constexpr int kMaxGroupList = 4096;  // store-pass groups compacted in shared memory

// MODE_ZW: GEMM1 storing z (walkers/points); MODE_ZR: GEMM1 values only (points); MODE_G: GEMM2;
// MODE_Q: GEMM1 of split operands (ray directions, the quadratic form of a sunburst ray)
enum { MODE_ZW = 0, MODE_ZR = 1, MODE_G = 2, MODE_Q = 3 };

struct TcArgs {
    int d, K;
    const int32_t *n_rows_dev;
    int n_rows_max;
    const int32_t *act;     // compact row -> walker id (null: identity)
    void *Z;                // [K][z_rows][ldz] z rows, component-major (bf16 or fp32)
    int ldz, z_rows;
    float *qpart;           // [rows][K][n_ntile]
    const float *R;         // [rows][K]
    const uint32_t *rflag;  // [row blocks][K]: 1 some row of the block has r_nk > 0; 3 every live row r_nk = 1
    const uint32_t *zmask;  // [row blocks][K]: GEMM1 |z|^2 pairs to visit (null: all; see k_tc_need)
    int prof;               // profiling class of the launch (-1: by mode)
    float *G;               // [walkers][d] grad f
    int n_ntile;
    int32_t *err;
    // MODE_Q: A = [u_hi | u_lo], B = [L_k^T hi | L_k^T lo], segments qseg elements apart;
    // the epilogue also sums qalpha[k][j] w_j (partials qpart1) beside w_j^2 (qpart),
    // qalpha rows qald >= the column tiles' span apart, zero past d
    const float *qalpha;
    float *qpart1;
    int qseg, qald;
    // MODE_Q origin pass (qzout given): z = acc + qoff[k][j] (qoff = -mu_k L_k in FP32) is
    // stored to qzout[row][k][0 .. qald) and its |z|^2 summed into qpart; qalpha_rows: the
    // alpha of a row is qalpha[row][k] (an origin pass's z) instead of qalpha[k]
    float *qzout;
    const float *qoff;
    int qalpha_rows;
};

// ------------------------------------------------------------------ PTX helpers
// Warp-uniform variants for roles where all 32 lanes take part.
__device__ __forceinline__ bool warp_bwait(uint64_t *bar, uint32_t parity, volatile int *abort_flag) {
    return __all_sync(0xffffffffu, bwait(bar, parity, abort_flag) ? 1 : 0) != 0;
}
__device__ __forceinline__ bool warp_aborted(volatile int *abort_flag) {
    return __any_sync(0xffffffffu, *abort_flag != 0) != 0;
}
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
    uint64_t kmask;    // GEMM2: components with r_nk > 0 somewhere in the row block
    bool skip;         // GEMM1 store pass: this (row block, component) is not needed
};

// Components with r_nk > 0 at some row of row block mb (all when no flags are
// given); a block with none keeps component 0 (non-finite or empty rows). One bit
// per component (K <= 64).
__device__ __forceinline__ uint64_t block_kmask(const uint32_t *rflag, int mb, int K) {
    uint64_t m = 0;
    for (int k = 0; k < K; ++k)
        if (!rflag || rflag[(size_t)mb * K + k]) m |= 1ull << k;
    return m ? m : 1ull;
}

// Component of GEMM2 chunk q: the (q / c_hi)-th set bit of the tile's mask.
__device__ __forceinline__ int chunk_component(const TileInfo &ti, int q) {
    int idx = q / ti.c_hi;
    uint64_t m = ti.kmask;
    while (idx-- > 0) m &= m - 1;
    return __ffsll((long long)m) - 1;
}

template <int MODE, int BN, int KC>
__device__ __forceinline__ TileInfo decode_tile(int t, int d, int K, const uint32_t *rflag, const int *glist,
                                                int n_mblk) {
    TileInfo ti;
    const int nct = (d + BN - 1) / BN;
    if (glist) t = glist[t / nct] * nct + t % nct;  // compacted store-pass schedule
    ti.kmask = 0;
    ti.skip = false;
    if (MODE == MODE_G) {
        // single tiles, widest K range first (column tile nct - 1 of every row
        // block, then nct - 2, ...), dealt round-robin: the costly tiles start
        // first and the short ones fill in, and small row counts still spread
        // over every SM
        ti.nt = nct - 1 - t / n_mblk;
        ti.mb = t % n_mblk;
        ti.k = 0;
        const int jmax = min(d, (ti.nt + 1) * BN);
        ti.c_lo = 0;
        ti.c_hi = (jmax + KC - 1) / KC;
        // components whose responsibility is zero at every row of the block add
        // exactly nothing to the gradient: their chunks are not visited (every
        // role reads the same flags, so the three agree on the chunk list)
        ti.kmask = block_kmask(rflag, ti.mb, K);
        ti.nchunks = __popcll(ti.kmask) * ti.c_hi;
    } else {
        // column tiles of one (row block, component) are adjacent in the schedule, so
        // CTAs that run together gather the same x rows (served from L2)
        ti.nt = t % nct;
        ti.k = (t / nct) % K;
        ti.mb = t / (K * nct);
        ti.c_lo = (ti.nt * BN) / KC;
        ti.c_hi = (d + KC - 1) / KC;
        // MODE_Q: the triangle's chunks three times, for the products lo hi, hi lo, hi hi
        ti.nchunks = (ti.c_hi - ti.c_lo) * (MODE == MODE_Q ? 3 : 1);
        // store pass (flags given): only the (block, component) pairs GEMM2 reads;
        // |z|^2 pass (mask given): only the pairs k_tc_need keeps (already the case
        // for a compacted schedule)
        if (MODE != MODE_G && rflag && !glist) ti.skip = !((block_kmask(rflag, ti.mb, K) >> ti.k) & 1ull);
    }
    return ti;
}

// Tile sequence of one CTA: groups of gsz consecutive tile indices dealt
// round-robin. GEMM1 groups are whole (row block, component) pairs — every
// column tile, whose K ranges differ (the triangle), so single tiles dealt with
// a grid that is a multiple of the tile count per group would give each CTA the
// same column tile over and over; whole groups carry equal work and reuse their
// A rows inside the CTA. GEMM2 deals single tiles in decreasing cost order
// (see decode_tile).
__device__ __forceinline__ int tile_of(int i, int nct) {
    return (blockIdx.x + (i / nct) * gridDim.x) * nct + (i % nct);
}

// ------------------------------------------------------------------ the kernel
template <int BN, int PREC, int MODE>
__global__ void __launch_bounds__(THREADS, 1) k_tc_gemm(const __grid_constant__ CUtensorMap tmapA,
                                                        const __grid_constant__ CUtensorMap tmapB, TcArgs a) {
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
    uint64_t *full = bars;
    uint64_t *empty = bars + STAGES;
    uint64_t *tfull = bars + 2 * STAGES;
    uint64_t *tempty = tfull + 2;
    uint64_t *drain = tempty + 2;
    uint32_t *s_tmem = reinterpret_cast<uint32_t *>(drain + 1);
    volatile int *s_abort = reinterpret_cast<volatile int *>(s_tmem + 1);
    int *s_wcnt = const_cast<int *>(s_abort) + 1;  // [8] per-warp counts (group compaction)
    int *s_gcount = s_wcnt + 8;
    int *s_glist = s_gcount + 1;                  // [kMaxGroupList] GEMM1 with a mask: groups to visit

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int d = a.d, K = a.K;
    const int n_rows = a.n_rows_dev ? *a.n_rows_dev : a.n_rows_max;
    const int n_mblk = (n_rows + BM - 1) / BM;
    const int nct = (d + BN - 1) / BN;
    int n_tiles = (MODE == MODE_G) ? n_mblk * nct : n_mblk * nct * K;
    // Store pass: the (row block, component) groups GEMM2 reads, compacted in
    // order, so that the round-robin deal spreads the work that remains (a
    // fixed stride over all groups would hand every CTA the same component).
    const int n_groups = n_mblk * K;
    // (row block, component) pairs to visit: GEMM2's flags for the store pass, the
    // component-skip mask for the |z|^2 pass
    const uint32_t *gmask = MODE == MODE_G ? nullptr : ((MODE == MODE_ZW && a.rflag) ? a.rflag : a.zmask);
    const bool compact = MODE != MODE_G && gmask != nullptr && n_groups <= kMaxGroupList;
    if (compact) {
        if (threadIdx.x == 0) *s_gcount = 0;
        __syncthreads();
        for (int g0 = 0; g0 < n_groups; g0 += (int)blockDim.x) {
            const int g = g0 + (int)threadIdx.x;
            const bool act = g < n_groups && ((block_kmask(gmask, g / K, K) >> (g % K)) & 1ull);
            const unsigned bal = __ballot_sync(0xffffffffu, act);
            if (lane == 0) s_wcnt[warp] = __popc(bal);
            __syncthreads();
            int off = *s_gcount;
            for (int w = 0; w < warp; ++w) off += s_wcnt[w];
            if (act) s_glist[off + __popc(bal & ((1u << lane) - 1u))] = g;
            __syncthreads();
            if (threadIdx.x == 0) {
                int tot = 0;
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += s_wcnt[w];
                *s_gcount += tot;
            }
            __syncthreads();
        }
        n_tiles = *s_gcount * nct;
    }
    const int *glist = compact ? s_glist : nullptr;
    const int gsz = (MODE == MODE_G) ? 1 : nct;  // tiles per scheduling group

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&tfull[s], 1);
            mbar_init(&tempty[s], 4);
        }
        mbar_init(drain, 1);
        *s_abort = 0;
        mbar_fence_init();
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_tmem)),
                     "r"(2 * BN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *s_tmem;

    if (warp == 0) {
        // ---------------------------------------------------------- TMA loads of A and B
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int inflight_stage[8];
            uint32_t inflight_phase[8];
            int n_inflight = 0;
            for (int it = 0, t = tile_of(0, gsz); t < n_tiles && !*s_abort; t = tile_of(++it, gsz)) {
                const TileInfo ti = decode_tile<MODE, BN, KC>(t, d, K, MODE == MODE_G ? a.rflag : gmask, glist, n_mblk);
                if (ti.skip) continue;
                bool ok = true;
                for (int q = 0; q < ti.nchunks; ++q) {
                    if (!bwait(&empty[stage], phase ^ 1, s_abort)) {
                        ok = false;
                        break;
                    }
                    mbar_arrive_tx(&full[stage], A_BYTES + B_BYTES);
                    int kk, c0, cA, kA;
                    if (MODE == MODE_G) {
                        kk = chunk_component(ti, q);
                        c0 = (q % ti.c_hi) * KC;
                        cA = c0;
                        kA = kk;
                    } else if (MODE == MODE_Q) {
                        // segment 0: u_lo L_hi, 1: u_hi L_lo, 2: u_hi L_hi (one A row per ray);
                        // the small products first, so that only the last third of the
                        // accumulation steps adds to an accumulator of full magnitude
                        const int nc = ti.c_hi - ti.c_lo, seg = q / nc;
                        kk = ti.k;
                        const int cc = (ti.c_lo + q - seg * nc) * KC;
                        cA = (seg == 0 ? a.qseg : 0) + cc;
                        c0 = (seg == 1 ? a.qseg : 0) + cc;
                        kA = 0;
                    } else {
                        kk = ti.k;
                        c0 = (ti.c_lo + q) * KC;
                        cA = c0;
                        kA = kk;
                    }
                    tma_load_3d(sA + stage * A_BYTES, &tmapA, &full[stage], cA, ti.mb * BM, kA);
                    tma_load_3d(sB + stage * B_BYTES, &tmapB, &full[stage], c0, ti.nt * BN, kk);
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
                    bwait(&full[inflight_stage[q % 8]], inflight_phase[q % 8], &never);
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---------------------------------------------------------- MMA issue
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            int acc = 0;
            uint32_t acc_phase = 0;
            bool issued = false;
            for (int it = 0, t = tile_of(0, gsz); t < n_tiles && !*s_abort; t = tile_of(++it, gsz)) {
                const TileInfo ti = decode_tile<MODE, BN, KC>(t, d, K, MODE == MODE_G ? a.rflag : gmask, glist, n_mblk);
                if (ti.skip) continue;
                if (!bwait(&tempty[acc], acc_phase ^ 1, s_abort)) break;
                tc_fence_after();
                const uint32_t dt = tmem + (uint32_t)(acc * BN);
                bool ok = true;
                for (int q = 0; q < ti.nchunks; ++q) {
                    if (!bwait(&full[stage], phase, s_abort)) {
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
        // ---------------------------------------------------------- epilogue (warps 2-5)
        const int quad = warp & 3;
        const int r = quad * 32 + lane;
        int acc = 0;
        uint32_t acc_phase = 0;
        for (int it = 0, t = tile_of(0, gsz); t < n_tiles && !warp_aborted(s_abort); t = tile_of(++it, gsz)) {
            const TileInfo ti = decode_tile<MODE, BN, KC>(t, d, K, MODE == MODE_G ? a.rflag : gmask, glist, n_mblk);
            if (ti.skip) continue;
            if (!warp_bwait(&tfull[acc], acc_phase, s_abort)) break;
            tc_fence_after();
            const int n = ti.mb * BM + r;
            const bool valid = n < n_rows;
            const int w_out = (MODE == MODE_G && valid) ? (a.act ? a.act[n] : n) : 0;
            // store pass: z is written as r_nk z_nk (GEMM2's A operand); rows past the
            // live count are written as zeros (their z rows would be stale)
            const bool scaled = MODE == MODE_ZW && a.rflag != nullptr;
            const float sc = scaled ? (valid ? a.R[(size_t)n * K + ti.k] : 0.f) : 1.f;
            const bool store_row = MODE == MODE_ZW && (valid || (scaled && n < a.z_rows));
            const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(acc * BN);
            float q2 = 0.f, q1 = 0.f;
#pragma unroll 1
            for (int c0 = 0; c0 < BN; c0 += 32) {
                uint32_t v[32];
                // MODE_Q: this chunk's alpha (one 128-byte row piece per thread when the
                // alphas are per row) is read before the accumulator, so that the two
                // latencies overlap
                float4 alv[8];
                if (MODE == MODE_Q && a.qalpha) {
                    const float4 *al4 = reinterpret_cast<const float4 *>(
                        a.qalpha + (a.qalpha_rows ? ((size_t)n * K + ti.k) : (size_t)ti.k) * a.qald + ti.nt * BN + c0);
#pragma unroll
                    for (int e = 0; e < 8; ++e) alv[e] = al4[e];
                }
                SB_TMEM_LD32(taddr + c0, v);
                const int col = ti.nt * BN + c0;
                if (MODE == MODE_G) {
                    if (valid && col < d) {
                        float *g = a.G + (size_t)w_out * d + col;
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
                    if (MODE == MODE_Q && a.qzout) {
                        // origin pass: z_k(o) = o L_k - mu_k L_k (zero past d: both terms are)
                        const float *off = a.qoff + (size_t)ti.k * a.qald + col;
#pragma unroll
                        for (int e = 0; e < 32; ++e) v[e] = __float_as_uint(__uint_as_float(v[e]) + off[e]);
                        if (valid) {
                            float *zo = a.qzout + ((size_t)n * K + ti.k) * a.qald + col;
#pragma unroll
                            for (int e = 0; e < 32; e += 4)
                                *reinterpret_cast<float4 *>(zo + e) =
                                    make_float4(__uint_as_float(v[e]), __uint_as_float(v[e + 1]),
                                                __uint_as_float(v[e + 2]), __uint_as_float(v[e + 3]));
                        }
                    }
#pragma unroll
                    for (int e = 0; e < 32; ++e) {
                        const float z = __uint_as_float(v[e]);
                        q2 = fmaf(z, z, q2);
                    }
                    if (MODE == MODE_Q && a.qalpha) {  // alv: zero past d
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            q1 = fmaf(alv[e].x, __uint_as_float(v[4 * e]), q1);
                            q1 = fmaf(alv[e].y, __uint_as_float(v[4 * e + 1]), q1);
                            q1 = fmaf(alv[e].z, __uint_as_float(v[4 * e + 2]), q1);
                            q1 = fmaf(alv[e].w, __uint_as_float(v[4 * e + 3]), q1);
                        }
                    }
                    if (store_row && col < a.ldz) {
                        if (scaled)
#pragma unroll
                            for (int e = 0; e < 32; ++e) {
                                const float y = __uint_as_float(v[e]) * sc;
                                v[e] = __float_as_uint(PREC == SB_PREC_BF16 ? y : to_tf32(y));
                            }
                        const size_t zrow = ((size_t)ti.k * a.z_rows + n) * a.ldz + col;
                        if (PREC == SB_PREC_BF16) {
                            __nv_bfloat16 *zr = reinterpret_cast<__nv_bfloat16 *>(a.Z) + zrow;
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
                            // rounded to tf32 as stored (as bf16 is by its packing), so that a
                            // pair the scaling pass skips is GEMM2's operand as it stands
                            float *zr = reinterpret_cast<float *>(a.Z) + zrow;
#pragma unroll
                            for (int e = 0; e < 32; e += 4)
                                if (col + e + 4 <= a.ldz)
                                    *reinterpret_cast<float4 *>(zr + e) =
                                        make_float4(to_tf32(__uint_as_float(v[e])), to_tf32(__uint_as_float(v[e + 1])),
                                                    to_tf32(__uint_as_float(v[e + 2])),
                                                    to_tf32(__uint_as_float(v[e + 3])));
                        }
                    }
                }
            }
            if (MODE != MODE_G && !scaled && valid) {
                a.qpart[((size_t)n * K + ti.k) * a.n_ntile + ti.nt] = q2;
                if (MODE == MODE_Q && a.qpart1) a.qpart1[((size_t)n * K + ti.k) * a.n_ntile + ti.nt] = q1;
            }
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
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * BN));
    }
}

// ------------------------------------------------------------------ small kernels
// LSE over components from the FP32 |z|^2 partials: e_k and the maximum in
// FP64, exp/log of the shifted values (in [0, 1] and [1, K]) in FP32, whose
// absolute error stays below the FP32 resolution of the outputs.
// mode 0: walkers (FT[act[n]] = -l, R); mode 1: ray samples (ell[flat0 + n] = l);
// mode 2: points (ell[n] = l, R). Modes 0 and 2 also raise rflag[block][k] when
// some row of the 128-row block has r_nk > 0 (GEMM2 and the scaling pass skip
// the other (block, component) pairs, whose terms are exactly zero).
__global__ void __launch_bounds__(128) k_tc_lse(int mode, int K, int n_ntile, const int32_t *n_rows_dev,
                                                int n_rows_max, const int32_t *act, const float *qpart,
                                                const double *a_k, float *R, float *FT, double *ell,
                                                uint32_t *rflag, const uint32_t *zmask, float *zb, int32_t *jst,
                                                float *zst) {
    const int n_rows = n_rows_dev ? *n_rows_dev : n_rows_max;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = n < n_rows;
    // components the |z|^2 pass skipped for this row block (zmask): e_k = -inf. Each
    // pass below recomputes e_k from the partials (the same sum in the same order, so
    // the same value), which keeps the terms out of a local-memory array.
    const uint64_t km = zmask ? block_kmask(zmask, n / BM, K) : ~0ull;
    auto term = [&](int k) -> double {
        if (!((km >> k) & 1ull)) return -INFINITY;
        const float *qp = qpart + ((size_t)n * K + k) * n_ntile;
        double q = 0.0;
        for (int t = 0; t < n_ntile; ++t) q += (double)qp[t];
        return a_k[k] - 0.5 * q;
    };
    double emax = -INFINITY;
    float s = 0.f;
    if (valid) {
        for (int k = 0; k < K; ++k) emax = fmax(emax, term(k));
        // bounds for the next round's skip (k_tc_need): |z_k| of the evaluated
        // components, lowered by a 1/32 margin for the GEMM's rounding, and the
        // largest term's |z|, raised by the same margin
        const int w = zb ? (act ? act[n] : n) : 0;
        int jm = -1;
        double ejm = 0.0;
        for (int k = 0; k < K; ++k) {
            const double e = term(k);
            s += __expf((float)(e - emax));
            if (zb && isfinite(e)) {
                zb[(size_t)w * K + k] = __double2float_rd(sqrt(fmax((a_k[k] - e) * 2.0, 0.0)) * (1.0 - 1.0 / 32));
                if (e == emax && jm < 0) {
                    jm = k;
                    ejm = e;
                }
            }
        }
        if (zb) {
            jst[w] = jm;
            if (jm >= 0) zst[w] = __double2float_ru(sqrt(fmax((a_k[jm] - ejm) * 2.0, 0.0)) * (1.0 + 1.0 / 32));
        }
    }
    const double l = emax + (double)__logf(s);
    if (mode == 1) {
        if (valid) ell[n] = l;
        return;
    }
    const float inv = 1.f / s;
    // One CTA is one 128-row block. Flag of (block, component k): bit 0 when some row
    // has r_nk > 0; bit 1 as well when every live row has r_nk == 1 exactly (all other
    // terms of each row underflow), where r z = z and the scaling pass is skipped.
    __shared__ unsigned long long s_any, s_one;
    if (threadIdx.x == 0) {
        s_any = 0ull;
        s_one = ~0ull;
    }
    __syncthreads();
    uint64_t any_m = 0, one_m = 0;
    for (int k = 0; k < K; ++k) {
        const float r = valid ? __expf((float)(term(k) - emax)) * inv : 0.f;
        if (valid) R[(size_t)n * K + k] = r;
        if (__any_sync(0xffffffffu, r > 0.f)) any_m |= 1ull << k;
        if (__all_sync(0xffffffffu, !valid || r == 1.f)) one_m |= 1ull << k;
    }
    if ((threadIdx.x & 31) == 0) {
        atomicOr(&s_any, (unsigned long long)any_m);
        atomicAnd(&s_one, (unsigned long long)one_m);
    }
    __syncthreads();
    if (rflag && (int)threadIdx.x < K) {
        const int k = threadIdx.x;
        const bool any = (s_any >> k) & 1ull, one = (s_one >> k) & 1ull;
        rflag[(size_t)blockIdx.x * K + k] = any ? (one ? 3u : 1u) : 0u;
    }
    if (!valid) return;
    if (mode == 0)
        FT[act ? act[n] : n] = (float)(-l);
    else
        ell[n] = l;
}

// GEMM2's A operand from the stored z: for every (128-row block, component) pair whose
// flag says some row has r_nk > 0, Z[k][n][:] = round(r_nk z_nk) (rows past the live
// count, and rows with r_nk = 0, become exact zeros), so GEMM2 adds r_nk L_k z_nk.
// Pairs whose live rows all have r_nk = 1 (flag 3) keep the stored z, which is already
// rounded: round(1 z) = z. Their rows past the live count keep stale values, which
// reach only GEMM2 output rows that are not stored (each output row depends on its
// own A row alone).
template <int PREC>
__global__ void __launch_bounds__(256) k_tc_scale_z(int K, int ldz, int z_rows, const int32_t *n_rows_dev,
                                                    int n_rows_max, const float *R, const uint32_t *rflag, void *Z) {
    const int mb = blockIdx.x, k = blockIdx.y;
    const int n_rows = n_rows_dev ? *n_rows_dev : n_rows_max;
    if (mb * BM >= n_rows || rflag[(size_t)mb * K + k] != 1u) return;
    constexpr int VE = (PREC == SB_PREC_BF16) ? 8 : 4;  // elements per 16-byte vector
    constexpr int NB = 16;                              // vectors in flight per thread
    // the block's rows are split over gridDim.z CTAs (more loads in flight per pair)
    const int rows = BM / (int)gridDim.z, row0 = (int)blockIdx.z * rows;
    const int nv = ldz / VE, tot = rows * nv;
    uint4 *Zv = reinterpret_cast<uint4 *>(Z);  // 16-byte vectors (ldz is a multiple of 64 elements)
    for (int e0 = 0; e0 < tot; e0 += NB * (int)blockDim.x) {
        // every load of the batch is issued before the first store
        uint4 w[NB];
        float r[NB];
        size_t at[NB];
        bool in[NB];
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            const int e = e0 + (int)threadIdx.x + j * (int)blockDim.x;
            const int row = row0 + e / nv, v = e % nv;
            const int n = mb * BM + row;
            in[j] = e < tot && n < z_rows;
            r[j] = (in[j] && n < n_rows) ? R[(size_t)n * K + k] : 0.f;
            at[j] = (((size_t)k * z_rows + n) * ldz) / VE + (size_t)v;
            w[j] = (in[j] && r[j] > 0.f) ? Zv[at[j]] : make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            if (!in[j]) continue;
            uint4 q = make_uint4(0u, 0u, 0u, 0u);
            if (r[j] > 0.f) {
                const uint32_t src[4] = {w[j].x, w[j].y, w[j].z, w[j].w};
                uint32_t out[4];
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    if (PREC == SB_PREC_BF16) {
                        const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&src[h]));
                        out[h] = pack_bf16x2(f.x * r[j], f.y * r[j]);
                    } else {
                        out[h] = __float_as_uint(to_tf32(__uint_as_float(src[h]) * r[j]));
                    }
                }
                q = make_uint4(out[0], out[1], out[2], out[3]);
            }
            Zv[at[j]] = q;
        }
    }
}

// Component skip of the walker rounds. e_k = a_k - |z_k|^2 / 2 with z_k = L_k^T (x - mu_k);
// a component whose e_k lies more than kSkipNats below the largest term adds exp(-110)
// < 2e-48 relative: below FP32 resolution, so the LSE's FP32 exponential and the
// responsibility r_k it yields are exactly 0 and the component changes neither l
// nor grad l. Per walker the round before leaves, for every component evaluated
// there, |z_k| lowered by a 1/32 margin (zb), and the largest term's component j
// with |z_j| raised by that margin (jst, zst); the L-BFGS step leaves an upper bound
// D on the distance from that point to the new trial (dist). With |L_k^T v| <=
// lnorm_k |v| (lnorm_k = |L_k|_F >= |L_k|_2):
//   |z_k(new)| >= zb_k - lnorm_k D   (stored back as zb_k for a skipped component),
//   e_j(new) >= a_j - (zst + lnorm_j D)^2 / 2 =: e_lb,
// and the (row block, component) pair is visited unless every row of the block has
// a_k - zb_k(new)^2 / 2 < e_lb - kSkipNats. The largest term's component is always
// visited, so the LSE's maximum is at least e_lb.
constexpr double kSkipNats = 110.0;
__global__ void __launch_bounds__(128) k_tc_need(int K, const int32_t *n_rows_dev, int n_rows_max,
                                                 const int32_t *act, const double *a_k, const float *lnorm, float *zb,
                                                 const int32_t *jst, const float *zst, const float *dist,
                                                 uint32_t *zmask) {
    const int n_rows = n_rows_dev ? *n_rows_dev : n_rows_max;
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = n < n_rows;
    const int w = valid ? (act ? act[n] : n) : 0;
    const int j = valid ? jst[w] : -1;
    const float D = valid ? dist[w] : 0.f;
    const bool bounded = j >= 0 && D >= 0.f && isfinite(D);
    double elb = 0.0;
    if (bounded) {
        const double ub = (double)__fmaf_ru(lnorm[j], D, zst[w]);
        elb = a_k[j] - 0.5 * ub * ub;
    }
    // one CTA is one 128-row block: it writes every component's word of its block
    __shared__ unsigned long long s_need;
    if (threadIdx.x == 0) s_need = 0ull;
    __syncthreads();
    uint64_t mk = 0;
    for (int k = 0; k < K; ++k) {
        bool need = valid;
        if (bounded) {
            const float b = fmaxf(__fmaf_rd(-lnorm[k], D, zb[(size_t)w * K + k]), 0.f);
            zb[(size_t)w * K + k] = b;
            need = !(a_k[k] - 0.5 * (double)b * (double)b < elb - kSkipNats);
        }
        if (__any_sync(0xffffffffu, need)) mk |= 1ull << k;
    }
    if ((threadIdx.x & 31) == 0 && mk) atomicOr(&s_need, (unsigned long long)mk);
    __syncthreads();
    if ((int)threadIdx.x < K) zmask[(size_t)blockIdx.x * K + threadIdx.x] = (uint32_t)((s_need >> threadIdx.x) & 1ull);
}

// lnorm_k = |L_k|_F (an upper bound on |L_k|_2), rounded up to FP32: kLnParts CTAs
// per component sum squares of the lower triangle over contiguous slices of the
// row-major matrix (partials in a fixed order), then one thread per component
// adds its partials in order.
constexpr int kLnParts = 64;
__global__ void __launch_bounds__(256) k_tc_lnorm_part(int d, const double *L, double *part) {
    const int k = blockIdx.y, b = blockIdx.x;
    const size_t dd = (size_t)d * d, per = (dd + kLnParts - 1) / kLnParts;
    const size_t e0 = (size_t)b * per, e1 = e0 + per < dd ? e0 + per : dd;
    const double *Lk = L + (size_t)k * dd;
    double acc = 0.0;
    for (size_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const size_t i = e / d, j = e % d;
        if (j <= i) acc = fma(Lk[e], Lk[e], acc);
    }
    __shared__ double w8[8];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) w8[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < 8; ++q) t += w8[q];
        part[(size_t)k * kLnParts + b] = t;
    }
}
__global__ void k_tc_lnorm_fin(int K, const double *part, float *lnorm) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    double t = 0.0;
    for (int b = 0; b < kLnParts; ++b) t += part[(size_t)k * kLnParts + b];
    lnorm[k] = __double2float_ru(sqrt(t) * (1.0 + 1e-6));
}

// Points whose centred rows for component k are the columns of L_k:
// X[(kk d + i)][j] = mu_k[j] + L_k[j][i] (j >= i; mu_k[j] above the diagonal),
// k = k0 + kk, so that the |z_k|^2 pass sums |L_k^T c_i|^2 = |L_k^T L_k|_F^2.
__global__ void k_tc_lcols(int d, int k0, int kc, const double *L, const float *mu32, float *X) {
    const size_t tot = (size_t)kc * d * d;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        const int kk = (int)(e / ((size_t)d * d));
        const size_t r = e % ((size_t)d * d);
        const int i = (int)(r / d), j = (int)(r % d);
        const int k = k0 + kk;
        const float m = mu32[(size_t)k * d + j];
        X[e] = j >= i ? m + (float)L[((size_t)k * d + j) * d + i] : m;
    }
}
// lnorm_k = min(|L_k|_F, (1.1 |L_k^T L_k|_F)^(1/2)) from the |z_k|^2 partials of the
// points above (the 10 % covers the rounding of the tensor-core operands; both are
// upper bounds on |L_k|_2 = lambda_max(P_k)^(1/2) <= |P_k|_F^(1/2)).
__global__ void __launch_bounds__(256) k_tc_lnorm_gram(int d, int K, int k0, int n_ntile, const float *qpart,
                                                       float *lnorm) {
    const int kk = blockIdx.x, k = k0 + kk;
    double acc = 0.0;
    for (int i = threadIdx.x; i < d; i += blockDim.x) {
        const float *qp = qpart + ((size_t)(kk * d + i) * K + k) * n_ntile;
        for (int t = 0; t < n_ntile; ++t) acc += (double)qp[t];
    }
    __shared__ double part[8];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double S = 0.0;
        for (int q = 0; q < 8; ++q) S += part[q];
        const float g = __double2float_ru(sqrt(1.1 * sqrt(S)));
        if (isfinite(g) && g > 0.f && g < lnorm[k]) lnorm[k] = g;
    }
}

// A operand of GEMM1: A1[k][n][i] = round(x_n[i] - mu_k[i]) formed in FP32; x_n is a
// walker row (through the active list).
// Rows from n_rows up to the next multiple of 128 and columns >= d are zeroed.
// One thread per (row, 16-byte column group): x is formed once and the thread
// writes that column group for every component.
template <int PREC>
__global__ void __launch_bounds__(256) k_tc_center(int d, int K, int rows_cap, int ldp, const int32_t *n_rows_dev,
                                                   int n_rows_max, const int32_t *act, const float *X, int ld,
                                                   const float *mu32, void *A1, const uint32_t *zmask) {
    constexpr int VE = (PREC == SB_PREC_BF16) ? 8 : 4;  // elements per 16-byte store
    const int n_rows = n_rows_dev ? *n_rows_dev : n_rows_max;
    int rows_pad = (n_rows + BM - 1) / BM * BM;
    if (rows_pad > rows_cap) rows_pad = rows_cap;
    const int ncg = ldp / VE;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = e / ncg, cg = e - n * ncg;
    if (n >= rows_pad) return;
    const int i0 = cg * VE;
    const bool live = n < n_rows;
    const bool vec = ((d & 3) == 0) && i0 + VE <= d;
    float x[VE];
#pragma unroll
    for (int q = 0; q < VE; ++q) x[q] = 0.f;
    if (live) {
        const float *xr = X + (size_t)(act ? act[n] : n) * ld;
        if (vec && (ld & 3) == 0) {
#pragma unroll
            for (int q = 0; q < VE; q += 4) {
                const float4 t = *reinterpret_cast<const float4 *>(xr + i0 + q);
                x[q] = t.x;
                x[q + 1] = t.y;
                x[q + 2] = t.z;
                x[q + 3] = t.w;
            }
        } else {
#pragma unroll
            for (int q = 0; q < VE; ++q)
                if (i0 + q < d) x[q] = xr[i0 + q];
        }
    }
    const uint64_t km = zmask ? block_kmask(zmask, n / BM, K) : ~0ull;  // pairs the |z|^2 pass visits
    for (int k = 0; k < K; ++k) {
        if (!((km >> k) & 1ull)) continue;
        float v[VE];
#pragma unroll
        for (int q = 0; q < VE; ++q) v[q] = 0.f;
        if (live) {
            const float *mk = mu32 + (size_t)k * d;
            if (vec) {
#pragma unroll
                for (int q = 0; q < VE; q += 4) {
                    const float4 m4 = *reinterpret_cast<const float4 *>(mk + i0 + q);
                    v[q] = x[q] - m4.x;
                    v[q + 1] = x[q + 1] - m4.y;
                    v[q + 2] = x[q + 2] - m4.z;
                    v[q + 3] = x[q + 3] - m4.w;
                }
            } else {
#pragma unroll
                for (int q = 0; q < VE; ++q) v[q] = (i0 + q < d) ? x[q] - mk[i0 + q] : 0.f;
            }
        }
        const size_t o = ((size_t)k * rows_cap + n) * ldp + i0;
        if (PREC == SB_PREC_BF16) {
            uint4 p;
            p.x = pack_bf16x2(v[0], v[1]);
            p.y = pack_bf16x2(v[2], v[3]);
            p.z = pack_bf16x2(v[4], v[5]);
            p.w = pack_bf16x2(v[6], v[7]);
            *reinterpret_cast<uint4 *>(reinterpret_cast<__nv_bfloat16 *>(A1) + o) = p;
        } else {
            *reinterpret_cast<float4 *>(reinterpret_cast<float *>(A1) + o) =
                make_float4(to_tf32(v[0]), to_tf32(v[1]), to_tf32(v[2]), to_tf32(v[3]));
        }
    }
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

__global__ void k_tc_to_f32(size_t n, const double *x, float *y) {
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x)
        y[e] = (float)x[e];
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

// 3-D map over [dim2][dim1][stride1] elements with box (128 bytes of dim0, box1 rows, 1).
bool make_map(CUtensorMap *m, void *base, int dim0, int dim1, int dim2, int stride1, int prec, int box1) {
    auto fn = encode_fn();
    if (!fn) return false;
    const int e = esz(prec);
    cuuint64_t dims[3] = {(cuuint64_t)dim0, (cuuint64_t)dim1, (cuuint64_t)dim2};
    cuuint64_t strides[2] = {(cuuint64_t)stride1 * e, (cuuint64_t)stride1 * e * dim1};
    cuuint32_t box[3] = {(cuuint32_t)(128 / e), (cuuint32_t)box1, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    const CUtensorMapDataType dt =
        prec == SB_PREC_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    return fn(m, dt, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN, int PREC, int MODE>
constexpr int smem_bytes() {
    constexpr int STAGES = (BN >= 256) ? 4 : 6;
    return 1024 + STAGES * (BM * ROWB + BN * ROWB) + (2 * STAGES + 5) * 8 + 64 +
           (MODE != MODE_G ? (9 + kMaxGroupList) * 4 : 0);
}

template <int BN, int PREC, int MODE>
void launch_gemm(const CUtensorMap &mapA, const CUtensorMap &map, const TcArgs &a, cudaStream_t s) {
    constexpr int SM = smem_bytes<BN, PREC, MODE>();
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(k_tc_gemm<BN, PREC, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, SM);
    });
    const int mb = (a.n_rows_max + BM - 1) / BM;
    const long long groups = (long long)mb * (MODE == MODE_G ? (a.d + BN - 1) / BN : a.K);
    int grid = num_sms();
    if (groups < grid) grid = (int)(groups > 0 ? groups : 1);
    ProfScope prof(a.prof >= 0 ? a.prof
                               : (MODE == MODE_ZW ? PROF_TC_Z_WALKERS
                                                  : ((MODE == MODE_ZR || MODE == MODE_Q) ? PROF_TC_Z_RAYS : PROF_TC_GRAD)),
                   s);
    note_launch();
    k_tc_gemm<BN, PREC, MODE><<<grid, THREADS, SM, s>>>(mapA, map, a);
}

template <int PREC, int MODE>
void launch_gemm_bn(int bn, const CUtensorMap &mapA, const CUtensorMap &map, const TcArgs &a, cudaStream_t s) {
    if (bn == 256)
        launch_gemm<256, PREC, MODE>(mapA, map, a, s);
    else if (bn == 128)
        launch_gemm<128, PREC, MODE>(mapA, map, a, s);
    else
        launch_gemm<64, PREC, MODE>(mapA, map, a, s);
}

void launch_gemm_any(int prec, int mode, int bn, const CUtensorMap &mapA, const CUtensorMap &map, const TcArgs &a,
                     cudaStream_t s) {
    if (prec == SB_PREC_BF16) {
        if (mode == MODE_ZW) launch_gemm_bn<SB_PREC_BF16, MODE_ZW>(bn, mapA, map, a, s);
        else if (mode == MODE_ZR) launch_gemm_bn<SB_PREC_BF16, MODE_ZR>(bn, mapA, map, a, s);
        else if (mode == MODE_Q) launch_gemm_bn<SB_PREC_BF16, MODE_Q>(bn, mapA, map, a, s);
        else launch_gemm_bn<SB_PREC_BF16, MODE_G>(bn, mapA, map, a, s);
    } else {
        if (mode == MODE_ZW) launch_gemm_bn<SB_PREC_TF32, MODE_ZW>(bn, mapA, map, a, s);
        else if (mode == MODE_ZR) launch_gemm_bn<SB_PREC_TF32, MODE_ZR>(bn, mapA, map, a, s);
        else if (mode == MODE_Q) launch_gemm_bn<SB_PREC_TF32, MODE_Q>(bn, mapA, map, a, s);
        else launch_gemm_bn<SB_PREC_TF32, MODE_G>(bn, mapA, map, a, s);
    }
}

void launch_center(const TcWs &t, int d, int K, const int32_t *n_rows_dev, int n_rows_max, const int32_t *act,
                   const float *X, cudaStream_t s, const uint32_t *zmask = nullptr) {
    const int ldp = ldp_of(d, t.prec);
    const int ncg = ldp / (t.prec == SB_PREC_BF16 ? 8 : 4);
    int rows = (n_rows_max + BM - 1) / BM * BM;
    if (rows > (int)t.rows) rows = (int)t.rows;
    const dim3 grid((unsigned)(((long long)rows * ncg + 255) / 256));
    note_launch();
    if (t.prec == SB_PREC_BF16)
        k_tc_center<SB_PREC_BF16><<<grid, 256, 0, s>>>(d, K, (int)t.rows, ldp, n_rows_dev, n_rows_max, act, X, d,
                                                      (const float *)t.p[2], t.p[9], zmask);
    else
        k_tc_center<SB_PREC_TF32><<<grid, 256, 0, s>>>(d, K, (int)t.rows, ldp, n_rows_dev, n_rows_max, act, X, d,
                                                      (const float *)t.p[2], t.p[9], zmask);
}

TcArgs base_args(const ProbView &pv, const TcWs &t) {
    TcArgs a{};
    a.d = pv.d;
    a.K = pv.K;
    a.Z = t.p[4];
    a.ldz = ldz_of(pv.d);
    a.z_rows = (int)t.rows;
    a.qpart = (float *)t.p[5];
    a.R = (const float *)t.p[6];
    a.rflag = (const uint32_t *)t.p[10];
    a.prof = -1;
    a.n_ntile = (pv.d + t.bn - 1) / t.bn;
    a.err = pv.status;
    return a;
}

void launch_scale_z(const ProbView &pv, const TcWs &t, const int32_t *n_rows_dev, int n_rows_max, cudaStream_t s) {
    const dim3 grid((unsigned)((n_rows_max + BM - 1) / BM), (unsigned)pv.K, 4u);
    note_launch();
    if (t.prec == SB_PREC_BF16)
        k_tc_scale_z<SB_PREC_BF16><<<grid, 256, 0, s>>>(pv.K, (int)t.ldz, (int)t.rows, n_rows_dev, n_rows_max,
                                                         (const float *)t.p[6], (const uint32_t *)t.p[10], t.p[4]);
    else
        k_tc_scale_z<SB_PREC_TF32><<<grid, 256, 0, s>>>(pv.K, (int)t.ldz, (int)t.rows, n_rows_dev, n_rows_max,
                                                         (const float *)t.p[6], (const uint32_t *)t.p[10], t.p[4]);
}

}  // namespace

bool tc_available(int prec) { return (prec == SB_PREC_BF16 || prec == SB_PREC_TF32) && encode_fn() != nullptr; }

// Layout: [0] LT, [1] LB, [2] mu32, [3] c32, [4] Z [K][rows][ldz], [5] qpart, [6] R,
// [7] X32 (points), [8] G32 (points), [9] A1 [K][rows][ldp] (centred GEMM1 operand),
// [10] rflag, and for the component skip of the walker rounds (k_tc_need):
// [11] zb [rows][K], [12] jst [rows], [13] zst [rows], [14] dist [rows],
// [15] lnorm [K], [16] zmask [row blocks][K]
void carve_tc(Carver &cv, TcWs &t, int rows, int d, int K, int prec) {
    const int e = esz(prec), ldp = ldp_of(d, prec), bn = bn_of(d);
    const int nct = (d + 63) / 64;  // partials sized for the narrowest tile the tuner may pick
    rows = (rows + BM - 1) / BM * BM;
    t.rows = rows;
    t.prec = prec;
    t.bn = bn;
    t.d = d;
    t.K = K;
    t.ldz = ldz_of(d);
    t.p[0] = cv.take<uint8_t>((size_t)K * d * ldp * e);
    t.p[1] = cv.take<uint8_t>((size_t)K * d * ldp * e);
    t.p[2] = cv.take<float>((size_t)K * d);
    t.p[3] = cv.take<float>((size_t)d);
    t.p[4] = cv.take<uint8_t>((size_t)rows * K * t.ldz * e);
    t.p[5] = cv.take<float>((size_t)rows * K * nct);
    t.p[6] = cv.take<float>((size_t)rows * K);
    t.p[7] = cv.take<float>((size_t)rows * d);
    t.p[8] = cv.take<float>((size_t)rows * d);
    t.p[9] = cv.take<uint8_t>((size_t)K * rows * ldp * e);
    t.p[10] = cv.take<uint32_t>((size_t)(rows / BM) * K);
    t.p[11] = cv.take<float>((size_t)rows * K);
    t.p[12] = cv.take<int32_t>((size_t)rows);
    t.p[13] = cv.take<float>((size_t)rows);
    t.p[14] = cv.take<float>((size_t)rows);
    t.p[15] = cv.take<float>((size_t)K);
    t.p[16] = cv.take<uint32_t>((size_t)(rows / BM) * K);
}

int tc_setup_rows(int64_t total) {
    // the tile autotuner times at most 16384 rows (enough row blocks for every SM)
    return (int)(total < 16384 ? total : 16384);
}

bool tc_maps_for_rows(TcWs &t) {
    const int ldp = ldp_of(t.d, t.prec);
    return make_map(&t.mapA1, t.p[9], t.d, (int)t.rows, t.K, ldp, t.prec, BM) &&
           make_map(&t.mapZ, t.p[4], t.d, (int)t.rows, t.K, t.ldz, t.prec, BM);
}

// ------------------------------------------------------------------ tile autotuner
// The output tile width BN of both GEMMs is picked per (d, K, precision) by
// timing GEMM1 + GEMM2 for every candidate on this call's scratch (MMA timing
// does not depend on the values), once per process; SB_TUNE=0 uses the
// heuristic instead, SB_TUNE_CACHE=<file> keeps the choices across processes.
namespace {
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int>, int> g_tune;
bool g_tune_loaded = false;

void tune_load_locked() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char *path = std::getenv("SB_TUNE_CACHE");
    if (!path) return;
    FILE *f = std::fopen(path, "r");
    if (!f) return;
    int d, K, p, bn;
    while (std::fscanf(f, " {\"d\": %d, \"K\": %d, \"prec\": %d, \"bn\": %d}", &d, &K, &p, &bn) == 4)
        g_tune[std::make_tuple(d, K, p)] = bn;
    std::fclose(f);
}

void tune_store_locked() {
    const char *path = std::getenv("SB_TUNE_CACHE");
    if (!path) return;
    FILE *f = std::fopen(path, "w");
    if (!f) return;
    for (auto &kv : g_tune)
        std::fprintf(f, "{\"d\": %d, \"K\": %d, \"prec\": %d, \"bn\": %d}\n", std::get<0>(kv.first),
                     std::get<1>(kv.first), std::get<2>(kv.first), kv.second);
    std::fclose(f);
}

float time_tile(const ProbView &pv, TcWs &t, int bn, cudaStream_t s) {
    const int d = pv.d, K = pv.K, ldp = ldp_of(d, t.prec);
    TcWs u = t;
    u.bn = bn;
    if (!make_map(&u.mapT, u.p[0], d, d, K, ldp, u.prec, bn) || !make_map(&u.mapB, u.p[1], d, d, K, ldp, u.prec, bn))
        return -1.f;
    TcArgs a = base_args(pv, u);
    // as many rows as the scratch holds, up to 16384: enough row blocks to fill
    // every SM, so the timing ranks the tiles as a full-size launch would
    a.n_rows_max = (int)(u.rows < 16384 ? u.rows : 16384);
    a.rflag = nullptr;  // time the dense case: every component visited
    a.G = (float *)u.p[8];
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return -1.f;
    float best = -1.f;
    for (int rep = 0; rep < 3; ++rep) {
        cudaEventRecord(e0, s);
        launch_gemm_any(u.prec, MODE_ZW, bn, u.mapA1, u.mapT, a, s);
        launch_gemm_any(u.prec, MODE_G, bn, u.mapZ, u.mapB, a, s);
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) break;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && (best < 0.f || ms < best)) best = ms;  // first repetition warms up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best;
}

int pick_tile(const ProbView &pv, TcWs &t, cudaStream_t s) {
    const auto key = std::make_tuple(pv.d, pv.K, t.prec);
    const char *off = std::getenv("SB_TUNE");
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_load_locked();
    auto it = g_tune.find(key);
    if (it != g_tune.end()) return it->second;
    int bn = bn_of(pv.d);
    cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cst) != cudaSuccess || cst != cudaStreamCaptureStatusNone)
        return bn;  // no timing inside a capture: the heuristic width, not remembered
    if (!(off && off[0] == '0')) {
        // widest tile first; a narrower one must be at least 3 % faster to win,
        // so timing noise between near-equal tiles does not flip the choice
        float best = -1.f;
        for (int cand : {256, 128, 64}) {
            if (cand > 64 && (pv.d + 63) / 64 * 64 <= cand / 2) continue;  // tile mostly padding
            const float ms = time_tile(pv, t, cand, s);
            if (ms > 0.f && (best < 0.f || ms < 0.97f * best)) {
                best = ms;
                bn = cand;
            }
        }
    }
    g_tune[key] = bn;
    tune_store_locked();
    return bn;
}
}  // namespace

int tc_tuned_tile(int d, int K, int prec) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(std::make_tuple(d, K, prec));
    return it == g_tune.end() ? 0 : it->second;
}

sb_status tc_prepare(const ProbView &pv, TcWs &t, cudaStream_t s, bool skip_bounds) {
    const int d = pv.d, K = pv.K;
    const int ldp = ldp_of(d, t.prec);
    note_launch();
    if (t.prec == SB_PREC_BF16)
        k_tc_convert_L<uint16_t><<<1184, 256, 0, s>>>(d, K, ldp, pv.L, (uint16_t *)t.p[0], (uint16_t *)t.p[1]);
    else
        k_tc_convert_L<float><<<1184, 256, 0, s>>>(d, K, ldp, pv.L, (float *)t.p[0], (float *)t.p[1]);
    note_launch();
    k_tc_convert_vec<<<(K * d + 255) / 256, 256, 0, s>>>(d, K, pv.mu, pv.c, (float *)t.p[2], (float *)t.p[3]);
    if (skip_bounds) {  // partials in the qpart scratch (the Gram pass below overwrites it later)
        note_launch();
        k_tc_lnorm_part<<<dim3(kLnParts, K), 256, 0, s>>>(d, pv.L, (double *)t.p[5]);
        note_launch();
        k_tc_lnorm_fin<<<(K + 63) / 64, 64, 0, s>>>(K, (const double *)t.p[5], (float *)t.p[15]);
    }
    if (!tc_maps_for_rows(t)) return SB_ERR_CUDA;
    t.bn = pick_tile(pv, t, s);
    if (!make_map(&t.mapT, t.p[0], d, d, K, ldp, t.prec, t.bn) || !make_map(&t.mapB, t.p[1], d, d, K, ldp, t.prec, t.bn))
        return SB_ERR_CUDA;
    // the component skip's |L_k|_2 bound, tightened through |L_k^T L_k|_F (one |z|^2
    // pass over d points per component, as many components per pass as the rows hold)
    const int per = skip_bounds ? (int)(t.rows / (size_t)d) : 0;
    for (int k0 = 0; per >= 1 && k0 < K; k0 += per) {
        const int kc = per < K - k0 ? per : K - k0, rows = kc * d;
        note_launch();
        k_tc_lcols<<<1184, 256, 0, s>>>(d, k0, kc, pv.L, (const float *)t.p[2], (float *)t.p[7]);
        TcArgs a = base_args(pv, t);
        a.n_rows_max = rows;
        launch_center(t, d, K, nullptr, rows, nullptr, (const float *)t.p[7], s);
        launch_gemm_any(t.prec, MODE_ZR, t.bn, t.mapA1, t.mapT, a, s);
        note_launch();
        k_tc_lnorm_gram<<<kc, 256, 0, s>>>(d, K, k0, a.n_ntile, a.qpart, (float *)t.p[15]);
    }
    return cudaGetLastError() == cudaSuccess ? SB_OK : SB_ERR_CUDA;
}

// ------------------------------------------------------------------ quadratic form of the rays
// x split into hi + lo of the operand precision: hi = round(x), lo = round(x - hi)
template <int PREC>
__device__ __forceinline__ void split_op(double x, float &hi, float &lo) {
    if (PREC == SB_PREC_BF16) {
        hi = __bfloat162float(__double2bfloat16(x));
        lo = __bfloat162float(__double2bfloat16(x - (double)hi));
    } else {
        hi = to_tf32((float)x);
        lo = to_tf32((float)(x - (double)hi));
    }
}
template <int PREC>
__device__ __forceinline__ void put_op(void *base, size_t e, float v) {
    if (PREC == SB_PREC_BF16)
        reinterpret_cast<__nv_bfloat16 *>(base)[e] = __float2bfloat16_rn(v);  // exact: v is a bf16 value
    else
        reinterpret_cast<float *>(base)[e] = v;
}

// A2[r][0 .. dK) = hi(u_r), A2[r][dK .. 2 dK) = lo(u_r); zeros past d and past the ray
// count (n_rays, or *n_dev when given), rows past the count's last 128-row block untouched
template <int PREC>
__global__ void k_q_split_rows(int n_rays, int rows, int d, int dK, const double *u, void *A2, const int32_t *n_dev) {
    if (n_dev) {
        const int c = *n_dev < n_rays ? *n_dev : n_rays;
        const int rb = (c + BM - 1) / BM * BM;
        n_rays = c;
        rows = rb < rows ? rb : rows;
    }
    const size_t tot = (size_t)rows * dK;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / dK), i = (int)(e % dK);
        float hi = 0.f, lo = 0.f;
        if (r < n_rays && i < d) split_op<PREC>(u[(size_t)r * d + i], hi, lo);
        put_op<PREC>(A2, (size_t)r * 2 * dK + i, hi);
        put_op<PREC>(A2, (size_t)r * 2 * dK + dK + i, lo);
    }
}

// B2[k][j][i] = hi(L_k[i][j]), B2[k][j][dK + i] = lo(L_k[i][j]) for i >= j (L_k^T, the
// operand of GEMM1), zeros elsewhere
template <int PREC>
__global__ void k_q_split_LT(int d, int K, int dK, const double *L, void *B2) {
    const size_t tot = (size_t)K * d * dK;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(e / ((size_t)d * dK));
        const size_t rem = e % ((size_t)d * dK);
        const int j = (int)(rem / dK), i = (int)(rem % dK);
        float hi = 0.f, lo = 0.f;
        if (i < d && i >= j) split_op<PREC>(L[((size_t)k * d + i) * d + j], hi, lo);
        const size_t row = ((size_t)k * d + j) * 2 * dK;
        put_op<PREC>(B2, row + i, hi);
        put_op<PREC>(B2, row + dK + i, lo);
    }
}

// z_k(c)_j = sum_{i >= j} (c_i - mu_k,i) L_k,ij in FP64 (c null: -mu_k L_k): one CTA per
// (32 columns, component), a lane per column (rows of L_k read 256 bytes at a time),
// the eight warps over interleaved rows, their partials summed in a fixed order
__global__ void __launch_bounds__(256) k_q_zc(int d, const double *c, const double *mu, const double *L,
                                              double *zc) {
    const int k = blockIdx.y, j0 = blockIdx.x * 32, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int j = j0 + lane;
    const double *Lk = L + (size_t)k * d * d;
    const double *mk = mu + (size_t)k * d;
    double s = 0.0;
    if (j < d)
        for (int i = j0 + w; i < d; i += 8)
            if (i >= j) s = fma(c ? c[i] - mk[i] : -mk[i], Lk[(size_t)i * d + j], s);
    __shared__ double part[8][32];
    part[w][lane] = s;
    __syncthreads();
    if (w == 0 && j < d) {
        double t = 0.0;
        for (int q = 0; q < 8; ++q) t += part[q][lane];
        zc[(size_t)k * d + j] = t;
    }
}

// alpha[k][j] = (float) z_k(c)_j (zero for d <= j < ald) and q0[k] = |z_k(c)|^2 (FP64,
// partials in a fixed order): one CTA per component
__global__ void __launch_bounds__(256) k_q_alpha(int d, int ald, const double *zc, float *alpha, double *q0) {
    const int k = blockIdx.x;
    double s = 0.0;
    for (int j = threadIdx.x; j < ald; j += blockDim.x) {
        const double z = j < d ? zc[(size_t)k * d + j] : 0.0;
        alpha[(size_t)k * ald + j] = (float)z;
        s = fma(z, z, s);
    }
    __shared__ double part[8];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < 8; ++q) t += part[q];
        q0[k] = t;
    }
}

// (q1, q2)[r][k]: the FP64 sums of ray r's column-tile partials (FP32) of z_k(c) . w_rk
// and |w_rk|^2, one thread per (ray, component)
// (qp0 given: also q0r[r][k], the sum of the origin pass's |z_k(o_r)|^2 partials; K and
// the ray count *n_dev bound the pairs when n_dev is given)
__global__ void __launch_bounds__(256) k_q_sum(int n_rk, int n_ntile, const float *qp1, const float *qp2,
                                               double2 *q12, const float *qp0, double *q0r, int K,
                                               const int32_t *n_dev) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_rk || (n_dev && e >= *n_dev * K)) return;
    const float *p1 = qp1 + (size_t)e * n_ntile;
    const float *p2 = qp2 + (size_t)e * n_ntile;
    double q1 = 0.0, q2 = 0.0;
    for (int t = 0; t < n_ntile; ++t) {
        q1 += (double)p1[t];
        q2 += (double)p2[t];
    }
    q12[e] = make_double2(q1, q2);
    if (qp0) {
        const float *p0 = qp0 + (size_t)e * n_ntile;
        double q0 = 0.0;
        for (int t = 0; t < n_ntile; ++t) q0 += (double)p0[t];
        q0r[e] = q0;
    }
}

// l at sample j of ray r: |z_k|^2 = q0_k + 2 tau q1_rk + tau^2 q2_rk in FP64,
// tau = ((j + 1) / n_steps) t_exit,r; the LSE as in k_tc_lse (FP64 terms, FP32
// exponentials of the shifted terms). The threads of a warp mostly share a ray, so
// its coefficients are broadcast loads.
// (q0r given: q0 of ray r is q0r[r][k], the ray's own origin; ns_dev given: samples
// past *ns_dev are skipped)
__global__ void __launch_bounds__(256) k_q_ell(int n_rays, int n_steps, int K, const double *a_k, const double *q0,
                                               const double2 *q12, const double *texit, double *ell,
                                               const double *q0r, const int32_t *ns_dev) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= (int64_t)n_rays * n_steps || (ns_dev && e >= *ns_dev)) return;
    const int r = (int)(e / n_steps), j = (int)(e - (int64_t)r * n_steps);
    const double tau = ((double)(j + 1) / (double)n_steps) * texit[r];
    const double2 *qr = q12 + (size_t)r * K;
    const double *q0k = q0r ? q0r + (size_t)r * K : q0;
    auto term = [&](int k) {
        const double2 q = qr[k];
        return a_k[k] - 0.5 * (q0k[k] + tau * (2.0 * q.x + tau * q.y));
    };
    double emax = -INFINITY;
    for (int k = 0; k < K; ++k) emax = fmax(emax, term(k));
    float s = 0.f;
    for (int k = 0; k < K; ++k) s += __expf((float)(term(k) - emax));
    ell[e] = emax + (double)__logf(s);
}

void carve_tc_quad(Carver &cv, TcQuadWs &q, int n_rays, int d, int K, int prec) {
    const int e = esz(prec), kc = 128 / e;
    const int nct = (d + 63) / 64;  // partials sized for the narrowest tile the tuner may pick
    q.rows = (n_rays + BM - 1) / BM * BM;
    q.dK = (d + kc - 1) / kc * kc;  // whole 128-byte chunks per segment: no chunk straddles two
    q.ald = (d + 255) / 256 * 256;  // the widest column tile's span
    q.A2 = cv.take<uint8_t>((size_t)q.rows * 2 * q.dK * e);
    q.B2 = cv.take<uint8_t>((size_t)K * d * 2 * q.dK * e);
    q.alpha = cv.take<float>((size_t)K * q.ald);
    q.qpart1 = cv.take<float>((size_t)q.rows * K * nct);
    q.qpart2 = cv.take<float>((size_t)q.rows * K * nct);
    q.zc = cv.take<double>((size_t)K * d);
    q.q0 = cv.take<double>((size_t)K);
    q.q12 = cv.take<double2>((size_t)n_rays * K);
}

sb_status tc_ray_loglik_quad(const ProbView &pv, int n_rays, int n_steps, int prec, int bn, TcQuadWs q,
                             const double *u, const double *texit, double *ell_all, cudaStream_t s) {
    const int d = pv.d, K = pv.K;
    if (bn <= 0) bn = tc_tuned_tile(d, K, prec);
    if (bn <= 0) bn = bn_of(d);
    const unsigned gs = 1184;
    note_launch();
    note_launch();
    if (prec == SB_PREC_BF16) {
        k_q_split_rows<SB_PREC_BF16><<<gs, 256, 0, s>>>(n_rays, q.rows, d, q.dK, u, q.A2, nullptr);
        k_q_split_LT<SB_PREC_BF16><<<gs, 256, 0, s>>>(d, K, q.dK, pv.L, q.B2);
    } else {
        k_q_split_rows<SB_PREC_TF32><<<gs, 256, 0, s>>>(n_rays, q.rows, d, q.dK, u, q.A2, nullptr);
        k_q_split_LT<SB_PREC_TF32><<<gs, 256, 0, s>>>(d, K, q.dK, pv.L, q.B2);
    }
    // z_k(c) in FP64 (one point), then its FP32 copy and |z_k(c)|^2
    note_launch();
    k_q_zc<<<dim3((unsigned)((d + 31) / 32), (unsigned)K), 256, 0, s>>>(d, pv.c, pv.mu, pv.L, q.zc);
    note_launch();
    k_q_alpha<<<K, 256, 0, s>>>(d, q.ald, q.zc, q.alpha, q.q0);
    if (!make_map(&q.mapU, q.A2, 2 * q.dK, q.rows, 1, 2 * q.dK, prec, BM) ||
        !make_map(&q.mapL, q.B2, 2 * q.dK, d, K, 2 * q.dK, prec, bn))
        return SB_ERR_CUDA;
    TcArgs a{};
    a.d = d;
    a.K = K;
    a.prof = -1;
    a.n_ntile = (d + bn - 1) / bn;
    a.err = pv.status;
    a.n_rows_max = n_rays;
    a.qpart = q.qpart2;
    a.qpart1 = q.qpart1;
    a.qalpha = q.alpha;
    a.qseg = q.dK;
    a.qald = q.ald;
    a.zmask = nullptr;
    a.rflag = nullptr;
    launch_gemm_any(prec, MODE_Q, bn, q.mapU, q.mapL, a, s);
    const int64_t ns = (int64_t)n_rays * n_steps;
    note_launch();
    k_q_sum<<<(unsigned)((n_rays * K + 255) / 256), 256, 0, s>>>(n_rays * K, a.n_ntile, q.qpart1, q.qpart2, q.q12,
                                                                 nullptr, nullptr, K, nullptr);
    note_launch();
    k_q_ell<<<(unsigned)((ns + 255) / 256), 256, 0, s>>>(n_rays, n_steps, K, pv.a, q.q0, q.q12, texit, ell_all,
                                                         nullptr, nullptr);
    return cudaGetLastError() == cudaSuccess ? SB_OK : SB_ERR_CUDA;
}

void carve_tc_origins(Carver &cv, TcOriginWs &o, int n_rays, int d, int K, int prec) {
    (void)prec;
    const int nct = (d + 63) / 64;
    const int rows = (n_rays + BM - 1) / BM * BM;
    const int ald = (d + 255) / 256 * 256;
    o.zo = cv.take<float>((size_t)rows * K * ald);
    o.off = cv.take<float>((size_t)K * ald);
    o.qp0 = cv.take<float>((size_t)rows * K * nct);
    o.negm = cv.take<double>((size_t)K * d);
    o.q0k = cv.take<double>((size_t)K);
    o.q0r = cv.take<double>((size_t)rows * K);
}

sb_status tc_quad_prepare_origins(const ProbView &pv, int prec, TcQuadWs q, TcOriginWs o, cudaStream_t s) {
    const int d = pv.d, K = pv.K;
    const unsigned gs = 1184;
    note_launch();
    if (prec == SB_PREC_BF16)
        k_q_split_LT<SB_PREC_BF16><<<gs, 256, 0, s>>>(d, K, q.dK, pv.L, q.B2);
    else
        k_q_split_LT<SB_PREC_TF32><<<gs, 256, 0, s>>>(d, K, q.dK, pv.L, q.B2);
    // -mu_k L_k in FP64, then its FP32 copy (the origin pass's offset)
    note_launch();
    k_q_zc<<<dim3((unsigned)((d + 31) / 32), (unsigned)K), 256, 0, s>>>(d, nullptr, pv.mu, pv.L, o.negm);
    note_launch();
    k_q_alpha<<<K, 256, 0, s>>>(d, q.ald, o.negm, o.off, o.q0k);
    return cudaGetLastError() == cudaSuccess ? SB_OK : SB_ERR_CUDA;
}

sb_status tc_ray_origins_quad(const ProbView &pv, int n_cap, int n_steps, int prec, int bn, TcQuadWs q, TcOriginWs o,
                              const double *O, const double *U, const double *texit, const int32_t *n_rays_dev,
                              const int32_t *n_samples_dev, double *ell, cudaStream_t s) {
    const int d = pv.d, K = pv.K;
    if (bn <= 0) bn = tc_tuned_tile(d, K, prec);
    if (bn <= 0) bn = bn_of(d);
    const unsigned gs = 1184;
    if (!make_map(&q.mapU, q.A2, 2 * q.dK, q.rows, 1, 2 * q.dK, prec, BM) ||
        !make_map(&q.mapL, q.B2, 2 * q.dK, d, K, 2 * q.dK, prec, bn))
        return SB_ERR_CUDA;
    auto split = [&](const double *src) {
        note_launch();
        if (prec == SB_PREC_BF16)
            k_q_split_rows<SB_PREC_BF16><<<gs, 256, 0, s>>>(n_cap, q.rows, d, q.dK, src, q.A2, n_rays_dev);
        else
            k_q_split_rows<SB_PREC_TF32><<<gs, 256, 0, s>>>(n_cap, q.rows, d, q.dK, src, q.A2, n_rays_dev);
    };
    TcArgs a{};
    a.d = d;
    a.K = K;
    a.prof = -1;
    a.n_ntile = (d + bn - 1) / bn;
    a.err = pv.status;
    a.n_rows_max = n_cap;
    a.n_rows_dev = n_rays_dev;
    a.qseg = q.dK;
    a.qald = q.ald;
    // origins: z_k(o_r) stored (FP32) with its |z|^2 partials
    split(O);
    a.qzout = o.zo;
    a.qoff = o.off;
    a.qpart = o.qp0;
    launch_gemm_any(prec, MODE_Q, bn, q.mapU, q.mapL, a, s);
    // directions: w_rk = L_k^T u_r, z_k(o_r) . w_rk and |w_rk|^2 partials
    split(U);
    a.qzout = nullptr;
    a.qoff = nullptr;
    a.qalpha = o.zo;
    a.qalpha_rows = 1;
    a.qpart = q.qpart2;
    a.qpart1 = q.qpart1;
    launch_gemm_any(prec, MODE_Q, bn, q.mapU, q.mapL, a, s);
    note_launch();
    k_q_sum<<<(unsigned)((n_cap * K + 255) / 256), 256, 0, s>>>(n_cap * K, a.n_ntile, q.qpart1, q.qpart2, q.q12, o.qp0,
                                                                o.q0r, K, n_rays_dev);
    const int64_t ns = (int64_t)n_cap * n_steps;
    note_launch();
    k_q_ell<<<(unsigned)((ns + 255) / 256), 256, 0, s>>>(n_cap, n_steps, K, pv.a, nullptr, q.q12, texit, ell, o.q0r,
                                                         n_samples_dev);
    return cudaGetLastError() == cudaSuccess ? SB_OK : SB_ERR_CUDA;
}

void tc_to_f32(const double *x, float *y, size_t n, cudaStream_t s) {
    note_launch();
    const size_t blocks = (n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096;
    k_tc_to_f32<<<(unsigned)(blocks > 0 ? blocks : 1), 256, 0, s>>>(n, x, y);
}

void tc_walkers_reset(const TcWs &t, int n, cudaStream_t s) {
    cudaMemsetAsync(t.p[12], 0xff, sizeof(int32_t) * (size_t)n, s);  // jst = -1: no bound yet
}

void tc_eval_walkers(const ProbView &pv, const sb_config *c, const TcWs &t, const float *XT, const int32_t *act,
                     const int32_t *n_act, int n, float *FT, float *GT, cudaStream_t s) {
    (void)c;
    TcArgs a = base_args(pv, t);
    a.act = act;
    a.n_rows_dev = n_act;
    a.n_rows_max = n;
    a.prof = PROF_TC_Z_WALKERS;
    // the (row block, component) pairs whose terms can still reach l (k_tc_need),
    // then their centred operand, |z|^2 and z, then l, r and the flags of the pairs
    // with r > 0, then r z for those pairs (GEMM2's A operand), then the gradient
    uint32_t *zmask = (uint32_t *)t.p[16];
    note_launch();
    k_tc_need<<<(n + 127) / 128, 128, 0, s>>>(pv.K, n_act, n, act, pv.a, (const float *)t.p[15], (float *)t.p[11],
                                              (const int32_t *)t.p[12], (const float *)t.p[13],
                                              (const float *)t.p[14], zmask);
    launch_center(t, pv.d, pv.K, n_act, n, act, XT, s, zmask);
    a.zmask = zmask;
    a.rflag = nullptr;  // GEMM1 over the kept pairs: |z|^2 partials and z itself
    launch_gemm_any(t.prec, MODE_ZW, t.bn, t.mapA1, t.mapT, a, s);
    a.zmask = nullptr;
    a.rflag = (const uint32_t *)t.p[10];  // written for every block by k_tc_lse
    note_launch();
    k_tc_lse<<<(n + 127) / 128, 128, 0, s>>>(0, pv.K, a.n_ntile, n_act, n, act, a.qpart, pv.a, (float *)t.p[6], FT,
                                             nullptr, (uint32_t *)t.p[10], zmask, (float *)t.p[11],
                                             (int32_t *)t.p[12], (float *)t.p[13]);
    launch_scale_z(pv, t, n_act, n, s);
    a.prof = -1;
    a.G = GT;
    launch_gemm_any(t.prec, MODE_G, t.bn, t.mapZ, t.mapB, a, s);
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
    a.n_rows_max = n;
    a.prof = PROF_TC_Z_WALKERS;
    launch_center(t, pv.d, pv.K, nullptr, n, nullptr, X, s);
    // with the gradient, GEMM1 also stores z (the A operand of GEMM2 once scaled by r)
    a.rflag = nullptr;
    launch_gemm_any(t.prec, grad ? MODE_ZW : MODE_ZR, t.bn, t.mapA1, t.mapT, a, s);
    a.rflag = (const uint32_t *)t.p[10];  // written for every block by k_tc_lse
    note_launch();
    k_tc_lse<<<(n + 127) / 128, 128, 0, s>>>(2, pv.K, a.n_ntile, nullptr, n, nullptr, a.qpart, pv.a,
                                             (float *)t.p[6], nullptr, ell, (uint32_t *)t.p[10], nullptr, nullptr,
                                             nullptr, nullptr);
    if (grad) {
        launch_scale_z(pv, t, nullptr, n, s);
        a.prof = -1;
        a.G = G;
        launch_gemm_any(t.prec, MODE_G, t.bn, t.mapZ, t.mapB, a, s);
        note_launch();
        k_tc_points_out<<<(unsigned)(((size_t)n * pv.d + 255) / 256 < 4096 ? ((size_t)n * pv.d + 255) / 256 : 4096),
                          256, 0, s>>>(n, pv.d, G, grad);
    }
    return cudaGetLastError() == cudaSuccess ? SB_OK : SB_ERR_CUDA;
}

}  // namespace sb
