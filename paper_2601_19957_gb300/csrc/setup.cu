// setup.cu -- per-problem constants of the likelihood and the prior box.
//   a_k  = log w_k - (d/2) log 2pi + sum_i log L_k,ii   (normalised Gaussian, Sec. 3.2)
//   c    = (lo + hi) / 2, half = (hi - lo) / 2          (prior centre, Sec. 3.4.1)
//   logV = sum_i log(hi_i - lo_i)                        (prior volume, Sec. 3.2)
// It also validates what only the device can see: lo < hi, L_k,ii > 0, finite values.
#include "sb_internal.cuh"

namespace sb {

template <typename T, typename Op>
__device__ T block_reduce(T v, Op op, T *sh, T identity) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    if (wid == 0) {
        v = lane < nw ? sh[lane] : identity;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
        if (lane == 0) sh[0] = v;
    }
    __syncthreads();
    T r = sh[0];
    __syncthreads();
    return r;
}

struct AddOp {
    __device__ double operator()(double a, double b) const { return a + b; }
};
struct MaxOp {
    __device__ double operator()(double a, double b) const { return fmax(a, b); }
};
struct OrOp {
    __device__ int operator()(int a, int b) const { return a | b; }
};

// Finiteness of the lower triangles of all L_k, spread over many blocks.
__global__ void __launch_bounds__(256) k_check_L(ProbView pv) {
    const int d = pv.d;
    const size_t tot = (size_t)pv.K * d * d;
    int bad = 0;
    for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        const size_t r = e % ((size_t)d * d);
        const int i = (int)(r / d), j = (int)(r % d);
        if (j <= i && !isfinite(pv.L[e])) bad = 1;
    }
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(pv.status, SB_DEV_NONFINITE);
}

__global__ void __launch_bounds__(256) k_setup(ProbView pv) {
    __shared__ double shd[32];
    __shared__ int shi[32];
    const int d = pv.d;
    if (blockIdx.x == 0) {
        double lsum = 0.0, wm = 0.0;
        int bad = 0;
        for (int i = threadIdx.x; i < d; i += blockDim.x) {
            const double lo = pv.lo[i], hi = pv.hi[i];
            const double w = hi - lo;
            if (!isfinite(lo) || !isfinite(hi)) bad |= SB_DEV_NONFINITE;
            if (!(w > 0.0)) bad |= SB_DEV_INVALID;
            pv.c[i] = 0.5 * (lo + hi);
            pv.half[i] = 0.5 * (hi - lo);
            lsum += log(w);
            wm = fmax(wm, w);
        }
        lsum = block_reduce(lsum, AddOp(), shd, 0.0);
        wm = block_reduce(wm, MaxOp(), shd, 0.0);
        bad = block_reduce(bad, OrOp(), shi, 0);
        if (threadIdx.x == 0) {
            pv.logV[0] = lsum;
            pv.wmax[0] = wm;
            if (bad) atomicOr(pv.status, bad);
        }
    } else {
        const int k = blockIdx.x - 1;
        const double *Lk = pv.L + (size_t)k * d * d;
        double s = 0.0;
        int bad = 0;
        for (int i = threadIdx.x; i < d; i += blockDim.x) {
            const double l = Lk[(size_t)i * d + i];
            if (!(l > 0.0)) bad |= SB_DEV_INVALID;
            s += log(l);
            if (!isfinite(pv.mu[(size_t)k * d + i])) bad |= SB_DEV_NONFINITE;
        }
        s = block_reduce(s, AddOp(), shd, 0.0);
        bad = block_reduce(bad, OrOp(), shi, 0);
        if (threadIdx.x == 0) {
            const double lw = pv.log_w[k];
            if (!isfinite(lw)) bad |= SB_DEV_NONFINITE;
            pv.a[k] = (lw - 0.5 * (double)d * SB_LOG_2PI) + s;
            if (bad) atomicOr(pv.status, bad);
        }
    }
}

void launch_setup(const ProbView &pv, cudaStream_t s) {
    note_launch();
    k_setup<<<pv.K + 1, 256, 0, s>>>(pv);
    const size_t tot = (size_t)pv.K * pv.d * pv.d;
    size_t blocks = (tot + 1023) / 1024;
    if (blocks > 1184) blocks = 1184;
    note_launch();
    k_check_L<<<(unsigned)(blocks > 0 ? blocks : 1), 256, 0, s>>>(pv);
}

}  // namespace sb
