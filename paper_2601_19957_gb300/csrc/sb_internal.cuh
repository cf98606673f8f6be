// sb_internal.cuh -- internal declarations shared by the CUDA translation units of libsb.
// Nothing here is part of the C ABI (include/sb.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

#include "sb.h"

#define SB_LOG_2PI 1.8378770664093454836
#define SB_TWO_PI 6.283185307179586477

// Device status word bits (stored in the workspace header).
enum : int32_t {
    SB_DEV_INVALID = 1,    // lo >= hi, L_kk <= 0
    SB_DEV_NONFINITE = 2,  // NaN/Inf in parameters
    SB_DEV_NO_MODES = 4,   // Laplace stage kept nothing
    SB_DEV_TIMEOUT = 8,    // a bounded loop hit its cap
};

#define SB_CUDA_TRY(expr)                                   \
    do {                                                    \
        cudaError_t _e = (expr);                            \
        if (_e != cudaSuccess) return SB_ERR_CUDA;          \
    } while (0)

namespace sb {

constexpr int kMaxD = 1024;
constexpr int kMaxK = 64;
constexpr int kMaxM = 64;

// ---------------------------------------------------------------- workspace carving
// Bump allocator over the caller's scratch. With base == nullptr it only measures.
struct Carver {
    char *base;
    size_t off = 0;
    explicit Carver(void *b) : base(static_cast<char *>(b)) {}
    template <typename T>
    T *take(size_t n) {
        off = (off + 255) & ~size_t(255);
        T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
        off += n * sizeof(T);
        return p;
    }
    size_t bytes() const { return (off + 255) & ~size_t(255); }
};

// Header at the start of every workspace.
struct WsHeader {
    int32_t status;  // SB_DEV_* bits
    int32_t pad[63];
};

// ---------------------------------------------------------------- device helpers
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ int warp_and(int v) { return __all_sync(0xffffffffu, v); }

// Round-to-nearest arithmetic without contraction, so update formulas match a
// plain evaluation order (x + a*p is a product rounded, then a sum rounded).
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double div_rn(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float div_rn(float a, float b) { return __fdiv_rn(a, b); }

// t_exit = min_i half_i / |u_i| over the coordinates i = lane, lane + 32, ... of one
// warp (u_i = 0 skipped; INFINITY when every u_i is 0), each quotient rounded to
// nearest in FP64, without dividing every coordinate in FP64: FP32 quotients (three
// roundings, relative error below 2^-21 when operands and quotient lie in
// [1e-30, 1e30]) bound the smallest one, and only coordinates within 2^-18 of that
// bound, or outside that range, are divided in FP64. The FP64 quotient is monotone in
// the exact one, so the result is the plain minimum of all of them.
__device__ __forceinline__ float exit_estimate(double au, double h64) {  // -1: always divide in FP64
    constexpr float kLo = 1e-30f, kHi = 1e30f;
    const float a = (float)au, h = (float)h64;
    if (!(a >= kLo && a <= kHi) || !(h >= kLo && h <= kHi)) return -1.f;
    const float e = __fdiv_rn(h, a);
    return e >= kLo && e <= kHi ? e : -1.f;
}
__device__ __forceinline__ double warp_exit_min(int lane, int d, const double *u, const double *half) {
    float est = INFINITY;
    for (int i = lane; i < d; i += 32) {
        const float e = exit_estimate(fabs(u[i]), half[i]);
        if (e >= 0.f) est = fminf(est, e);
    }
    const float thr = warp_min(est) * (1.0f + 0x1p-18f);
    double t = INFINITY;
    for (int i = lane; i < d; i += 32) {
        const double au = fabs(u[i]);
        if (!(au > 0.0)) continue;
        const float e = exit_estimate(au, half[i]);
        if (e >= 0.f && e > thr) continue;
        t = fmin(t, __ddiv_rn(half[i], au));
    }
    return warp_min(t);
}

__device__ __forceinline__ bool is_finite(double v) { return isfinite(v); }
__device__ __forceinline__ bool is_finite(float v) { return isfinite(v); }

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds, Weyl key bumps.
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        const uint32_t lo0 = 0xD2511F53u * c[0];
        const uint32_t hi0 = __umulhi(0xD2511F53u, c[0]);
        const uint32_t lo1 = 0xCD9E8D57u * c[2];
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]);
        const uint32_t n0 = hi1 ^ c[1] ^ k0;
        const uint32_t n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// Uniform in (0,1) from the top 52 bits of (hi:lo).
__device__ __forceinline__ double unit_from_words(uint32_t hi, uint32_t lo) {
    const uint64_t a = (uint64_t(hi) << 32) | uint64_t(lo);
    return (double(a >> 12) + 0.5) * (1.0 / 4503599627370496.0);
}

// Order-preserving map of a double to uint64 (ascending), for radix selection.
__device__ __forceinline__ uint64_t ordered_bits(double v) {
    uint64_t b = (uint64_t)__double_as_longlong(v);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

// ---------------------------------------------------------------- problem views
// Device-side view of one problem plus setup-derived quantities.
struct ProbView {
    int d, K;
    const double *log_w, *mu, *L, *lo, *hi;
    double *a;     // [K] log w_k - (d/2) log 2pi + sum_i log L_k,ii
    double *c;     // [d] box centre
    double *half;  // [d] half widths
    double *logV;  // [1] sum_i log(hi_i - lo_i)
    double *wmax;  // [1] max_i (hi_i - lo_i)
    int32_t *status;
};

// Host-side count of kernel launches issued by the library (diagnostics).
void note_launch(int64_t n = 1);

// Optional per-class device timing of launches (CUDA events on the launching
// stream, recorded only while profiling is enabled through the C ABI).
enum ProfClass {
    PROF_TC_Z_WALKERS = 0,
    PROF_TC_Z_RAYS = 1,
    PROF_TC_GRAD = 2,
    PROF_LBFGS_STEP = 3,
    PROF_F64_Z = 4,
    PROF_F64_GRAD = 5,
    PROF_CHOLESKY = 6,
    PROF_OTHER = 7,
    PROF_NCLASS = 8
};
bool prof_enabled();           // some class is being timed
bool prof_class_on(int cls);   // launches of class cls are being timed
struct ProfScope {
    int cls;
    cudaStream_t s;
    cudaEvent_t a, b;
    ProfScope(int c, cudaStream_t st);
    ~ProfScope();
};

// ---------------------------------------------------------------- launchers (host)
// setup.cu
void launch_setup(const ProbView &pv, cudaStream_t s);

// lik_f64.cu: FP64 batched log-likelihood pieces.
struct LikF64Args {
    int d, K;
    const double *mu, *L, *a;
    // row source: gather (X[rows[n]]) or ray samples
    const double *X;          // [*][d] gather source
    const int32_t *rows;      // row -> walker id (may be null: identity)
    const int32_t *n_rows_dev;// device count of rows (may be null: use n_rows)
    int n_rows;               // max rows (grid size)
    // ray source
    const double *u;          // [n_rays][d]
    const double *texit;      // [n_rays]
    const double *c;          // [d]
    int n_steps;
    int64_t flat0;            // first flat sample index of the chunk
    // outputs
    double *qpart;            // [out_rows][K][nJT]
    double *Z;                // [out_rows][K][d] (optional)
    double *R;                // [out_rows][K] responsibilities (optional)
    double *ell;              // [out_rows] (sign applied)
    double ell_sign;
    double *G;                // [out_rows][d] gradient (sign applied)
    double grad_sign;
    int out_by_walker;        // 1: outputs indexed by rows[n]; 0: by n
};
void launch_lik_f64_rays(const LikF64Args &a, cudaStream_t s);                 // values at ray samples
void launch_lik_f64_points(const LikF64Args &a, bool want_grad, cudaStream_t s);// values (+grads) at points
size_t lik_f64_qpart_elems(int d, int K, int rows);
// z_nk = L_k^T (x_n - mu_k) stored in Z (and the |z|^2 partials in qpart) for gathered rows, no l.
void launch_lik_f64_z(const LikF64Args &a, cudaStream_t s);
// Same outputs for a handful of points (GEMV-shaped work split; n_rows is the capacity).
void launch_lik_f64_few(const LikF64Args &a, bool want_grad, cudaStream_t s);

// rays.cu
// Unit directions u [n_rays][d] and their exit lengths from the box centre: FP64
// Box-Muller (fp32 = false, the oracle's directions) or FP32 Box-Muller widened to FP64
// (fp32 = true, for the mixed-precision path; t_exit exact for the widened directions).
void launch_ray_dirs(int d, int n_rays, uint64_t seed, const ProbView &pv, double *u, double *texit, bool fp32,
                     cudaStream_t s);
struct SelectWs {
    int32_t *bucket;     // [total]
    uint32_t *hist;      // [max(2*S, 256)]
    uint64_t *state;     // [8]
    int32_t *blockcnt;   // [nblocks]
    int64_t *idx;        // [n_starts]
};
void launch_select_starts(const double *ell_all, int n_rays, int n_steps, int n_starts, const SelectWs &w,
                          cudaStream_t s);
void launch_gather_starts(const ProbView &pv, const double *u, const double *texit, int n_steps, const int64_t *idx,
                          const double *ell_all, int n_starts, double *starts, double *ell_starts, cudaStream_t s);
size_t select_blocks(int64_t total);

}  // namespace sb
