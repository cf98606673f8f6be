// lbfgs.cu -- batched L-BFGS with Armijo backtracking (Sec. 3.6.2, App. A.5).
//
// Walkers minimise f = -l. Every round evaluates f and grad f at each active
// walker's trial point (the likelihood kernels), then one warp per walker runs
// the state machine below; finished walkers drop out of the active list, so
// the next round's contractions only see running walkers.
//
//   trial accepted (Armijo f_t <= f + c1 alpha grad f . p, finite):
//       s = x_t - x, y = g_t - g; store (s, y, 1/s.y) in the ring if
//       s.y > 1e-10 |s| |y|; x, g, f <- trial; start a new iteration.
//   trial rejected: alpha *= backtrack while backtracks <= max_backtracks;
//       then clear the history and retry once with steepest descent; a
//       second failure (or one with no history) stops the walker: STALLED.
//   new iteration: CONVERGED if |grad l|_inf <= gtol (1 + |l|); STALLED after
//       two accepted steps in a row without a decrease of f; MAXITER after
//       max_iter accepted steps; else direction p = -H grad f by the two-loop
//       recursion (H0 = gamma I, gamma = s.y / y.y of the newest pair), or
//       p = -g/|g| without history or when g.p >= 0; trial x + p.
//
// Layout: one warp per walker; coordinate i lives in lane i % 32, slot i / 32,
// so every vector and history read is a coalesced 32-wide access. The history
// ring S, Y is walker-major [walker][slot][d]; dot products are warp
// shuffle reductions.
#include "sb_lbfgs.cuh"

namespace sb {

namespace {

constexpr int WPB = 8;  // walkers (warps) per block

template <typename T>
struct Ctx {
    const LbfgsArgs<T> *a;
    int lane, d, m;
    T *X, *G, *P, *XT;
    const T *GT;
    T *S, *Y, *rho;
};

template <typename T, int VPL>
__device__ __forceinline__ void steepest(const Ctx<T> &c) {
    T gg = 0;
#pragma unroll
    for (int v = 0; v < VPL; ++v) {
        const int i = c.lane + 32 * v;
        if (i < c.d) {
            const T g = c.G[i];
            gg += g * g;
        }
    }
    const T gn = sqrt(warp_sum(gg));
#pragma unroll
    for (int v = 0; v < VPL; ++v) {
        const int i = c.lane + 32 * v;
        if (i < c.d) c.P[i] = -div_rn(c.G[i], gn);
    }
}

// p = -H g by the two-loop recursion over `count` pairs starting at ring slot `head`.
template <typename T, int VPL>
__device__ __forceinline__ void two_loop(const Ctx<T> &c, int count, int head, T *al) {
    T q[VPL];
#pragma unroll
    for (int v = 0; v < VPL; ++v) {
        const int i = c.lane + 32 * v;
        q[v] = i < c.d ? c.G[i] : T(0);
    }
    for (int t = count - 1; t >= 0; --t) {
        const int slot = (head + t) % c.m;
        const T *s = c.S + (size_t)slot * c.d;
        const T *y = c.Y + (size_t)slot * c.d;
        T sq = 0;
#pragma unroll
        for (int v = 0; v < VPL; ++v) {
            const int i = c.lane + 32 * v;
            if (i < c.d) sq += s[i] * q[v];
        }
        const T alpha = mul_rn(c.rho[slot], warp_sum(sq));
        if (c.lane == 0) al[t] = alpha;
#pragma unroll
        for (int v = 0; v < VPL; ++v) {
            const int i = c.lane + 32 * v;
            if (i < c.d) q[v] = sub_rn(q[v], mul_rn(alpha, y[i]));
        }
    }
    const int newest = (head + count - 1) % c.m;
    T sy = 0, yy = 0;
    {
        const T *s = c.S + (size_t)newest * c.d;
        const T *y = c.Y + (size_t)newest * c.d;
#pragma unroll
        for (int v = 0; v < VPL; ++v) {
            const int i = c.lane + 32 * v;
            if (i < c.d) {
                const T yi = y[i];
                sy += s[i] * yi;
                yy += yi * yi;
            }
        }
    }
    const T gamma = div_rn(warp_sum(sy), warp_sum(yy));
#pragma unroll
    for (int v = 0; v < VPL; ++v) q[v] = mul_rn(gamma, q[v]);
    __syncwarp();
    for (int t = 0; t < count; ++t) {
        const int slot = (head + t) % c.m;
        const T *s = c.S + (size_t)slot * c.d;
        const T *y = c.Y + (size_t)slot * c.d;
        T yr = 0;
#pragma unroll
        for (int v = 0; v < VPL; ++v) {
            const int i = c.lane + 32 * v;
            if (i < c.d) yr += y[i] * q[v];
        }
        const T beta = mul_rn(c.rho[slot], warp_sum(yr));
        const T coef = sub_rn(al[t], beta);
#pragma unroll
        for (int v = 0; v < VPL; ++v) {
            const int i = c.lane + 32 * v;
            if (i < c.d) q[v] = add_rn(q[v], mul_rn(s[i], coef));
        }
    }
#pragma unroll
    for (int v = 0; v < VPL; ++v) {
        const int i = c.lane + 32 * v;
        if (i < c.d) c.P[i] = -q[v];
    }
}

// Direction for a new attempt, the descent check, and the unit trial x + p.
template <typename T, int VPL>
__device__ __forceinline__ void new_direction(const Ctx<T> &c, WalkerState<T> &st, T *al) {
    if (st.count == 0)
        steepest<T, VPL>(c);
    else
        two_loop<T, VPL>(c, st.count, st.head, al);
    __syncwarp();
    T gp = 0;
#pragma unroll
    for (int v = 0; v < VPL; ++v) {
        const int i = c.lane + 32 * v;
        if (i < c.d) gp += c.G[i] * c.P[i];
    }
    T dphi = warp_sum(gp);
    if (!(dphi < T(0))) {
        st.count = 0;
        st.head = 0;
        __syncwarp();
        steepest<T, VPL>(c);
        __syncwarp();
        gp = 0;
#pragma unroll
        for (int v = 0; v < VPL; ++v) {
            const int i = c.lane + 32 * v;
            if (i < c.d) gp += c.G[i] * c.P[i];
        }
        dphi = warp_sum(gp);
    }
    st.dphi = dphi;
    st.alpha = T(1);
    st.bt = 0;
#pragma unroll
    for (int v = 0; v < VPL; ++v) {
        const int i = c.lane + 32 * v;
        if (i < c.d) c.XT[i] = add_rn(c.X[i], c.P[i]);
    }
}

template <typename T, int VPL>
__global__ void __launch_bounds__(32 * WPB) k_lbfgs_step(LbfgsArgs<T> a) {
    __shared__ T s_al[WPB][kMaxM];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const int n = blockIdx.x * WPB + wl;
    if (n >= *a.n_act) return;
    const int w = a.act[n];
    const int d = a.d;
    Ctx<T> c;
    c.a = &a;
    c.lane = lane;
    c.d = d;
    c.m = a.m;
    c.X = a.X + (size_t)w * d;
    c.G = a.G + (size_t)w * d;
    c.P = a.P + (size_t)w * d;
    c.XT = a.XT + (size_t)w * d;
    c.GT = a.GT + (size_t)w * d;
    c.S = a.S + (size_t)w * a.m * d;
    c.Y = a.Y + (size_t)w * a.m * d;
    c.rho = a.rho + (size_t)w * a.m;
    T *al = s_al[wl];

    WalkerState<T> st = a.st[w];
    const T ft = a.FT[w];
    bool newiter = false;

    if (st.phase == 0) {  // first evaluation at the start point
        int fin = is_finite(ft);
#pragma unroll
        for (int v = 0; v < VPL; ++v) {
            const int i = lane + 32 * v;
            if (i < d) {
                const T gt = c.GT[i];
                c.X[i] = c.XT[i];
                c.G[i] = gt;
                fin &= is_finite(gt) ? 1 : 0;
            }
        }
        fin = warp_and(fin);
        st.f = ft;
        st.phase = 1;
        if (!fin) {
            st.status = SB_WALKER_NONFINITE;
        } else {
            newiter = true;
        }
    } else {
        int fin = is_finite(ft);
#pragma unroll
        for (int v = 0; v < VPL; ++v) {
            const int i = lane + 32 * v;
            if (i < d) fin &= is_finite(c.GT[i]) ? 1 : 0;
        }
        fin = warp_and(fin);
        const T bound = add_rn(st.f, mul_rn(mul_rn(a.c1, st.alpha), st.dphi));
        if (fin && ft <= bound) {
            T ss = 0, yy = 0, sy = 0;
            T sv[VPL], yv[VPL];
#pragma unroll
            for (int v = 0; v < VPL; ++v) {
                const int i = lane + 32 * v;
                sv[v] = yv[v] = 0;
                if (i < d) {
                    sv[v] = sub_rn(c.XT[i], c.X[i]);
                    yv[v] = sub_rn(c.GT[i], c.G[i]);
                    ss += sv[v] * sv[v];
                    yy += yv[v] * yv[v];
                    sy += sv[v] * yv[v];
                }
            }
            ss = warp_sum(ss);
            yy = warp_sum(yy);
            sy = warp_sum(sy);
            if (sy > T(1e-10) * sqrt(ss) * sqrt(yy)) {
                int slot;
                if (st.count < a.m) {
                    slot = (st.head + st.count) % a.m;
                    ++st.count;
                } else {
                    slot = st.head;
                    st.head = (st.head + 1) % a.m;
                }
                T *s = c.S + (size_t)slot * d;
                T *y = c.Y + (size_t)slot * d;
#pragma unroll
                for (int v = 0; v < VPL; ++v) {
                    const int i = lane + 32 * v;
                    if (i < d) {
                        s[i] = sv[v];
                        y[i] = yv[v];
                    }
                }
                if (lane == 0) c.rho[slot] = div_rn(T(1), sy);
            }
            st.flat = (ft >= st.f) ? st.flat + 1 : 0;
#pragma unroll
            for (int v = 0; v < VPL; ++v) {
                const int i = lane + 32 * v;
                if (i < d) {
                    c.X[i] = c.XT[i];
                    c.G[i] = c.GT[i];
                }
            }
            st.f = ft;
            ++st.it;
            newiter = true;
        } else {
            ++st.bt;
            if (st.bt <= a.max_backtracks) {
                st.alpha = mul_rn(st.alpha, a.backtrack);
#pragma unroll
                for (int v = 0; v < VPL; ++v) {
                    const int i = lane + 32 * v;
                    if (i < d) c.XT[i] = add_rn(c.X[i], mul_rn(st.alpha, c.P[i]));
                }
            } else if (st.count > 0 && st.attempt == 0) {
                st.count = 0;
                st.head = 0;
                st.attempt = 1;
                __syncwarp();
                new_direction<T, VPL>(c, st, al);
            } else {
                st.status = SB_WALKER_STALLED;
            }
        }
    }

    if (newiter) {
        __syncwarp();
        T gm = 0;
#pragma unroll
        for (int v = 0; v < VPL; ++v) {
            const int i = lane + 32 * v;
            if (i < d) gm = fmax(gm, fabs(c.G[i]));
        }
        gm = warp_max(gm);
        if (gm <= a.gtol * (T(1) + fabs(st.f))) {
            st.status = SB_WALKER_CONVERGED;
        } else if (st.flat >= 2) {
            st.status = SB_WALKER_STALLED;
        } else if (st.it >= a.max_iter) {
            st.status = SB_WALKER_MAXITER;
        } else {
            st.attempt = 0;
            new_direction<T, VPL>(c, st, al);
        }
    }
    __syncwarp();
    if (lane == 0) a.st[w] = st;
}

template <typename T>
__global__ void k_lbfgs_init(int n, int d, const double *starts, T *XT, WalkerState<T> *st, int32_t *act,
                             int32_t *n_act, int64_t *n_evals) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < (int64_t)n * d) XT[e] = (T)starts[e];
    if (e < n) {
        WalkerState<T> s{};
        s.status = SB_WALKER_RUNNING;
        s.phase = 0;
        st[e] = s;
        act[e] = (int32_t)e;
    }
    if (e == 0) {
        *n_act = n;
        if (n_evals) *n_evals = 0;
    }
}

// Ordered in-place compaction of the active list; counts the evaluations of the round.
// One CTA of 1024 threads over super-chunks of 8 x 1024 entries: every thread
// first loads its 8 walker ids and their statuses (two memory round trips per
// super-chunk instead of two per 1024 entries), a barrier, then per 1024-entry
// chunk a ballot per warp, one warp scans the 32 warp counts with shuffles, two
// barriers. All reads of a super-chunk precede its writes and every output
// position is <= its input position, so later super-chunks read untouched entries.
constexpr int kCompactR = 8;
template <typename T>
__global__ void __launch_bounds__(1024) k_lbfgs_compact(const WalkerState<T> *st, int32_t *act, int32_t *n_act,
                                                        int64_t *n_evals) {
    __shared__ int warp_off[32];
    __shared__ int s_base[2];
    const int prev = *n_act;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        s_base[0] = 0;
        if (n_evals) *n_evals += prev;
    }
    __syncthreads();
    int par = 0;
    for (int s0 = 0; s0 < prev; s0 += 1024 * kCompactR) {
        int wv[kCompactR];
        bool kp[kCompactR];
#pragma unroll
        for (int r = 0; r < kCompactR; ++r) {
            const int nidx = s0 + r * 1024 + (int)threadIdx.x;
            wv[r] = nidx < prev ? act[nidx] : -1;
        }
#pragma unroll
        for (int r = 0; r < kCompactR; ++r) kp[r] = wv[r] >= 0 && st[wv[r]].status == SB_WALKER_RUNNING;
        __syncthreads();  // the super-chunk's reads are done before any of its writes
#pragma unroll
        for (int r = 0; r < kCompactR; ++r, par ^= 1) {
            const unsigned bal = __ballot_sync(0xffffffffu, kp[r]);
            if (lane == 0) warp_off[wid] = __popc(bal);
            __syncthreads();
            const int base = s_base[par];
            if (wid == 0) {
                const int c = warp_off[lane];
                int incl = c;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                warp_off[lane] = incl - c;  // exclusive offsets of the warps
                if (lane == 31) s_base[par ^ 1] = base + incl;
            }
            __syncthreads();
            const int pos = base + warp_off[wid] + __popc(bal & ((1u << lane) - 1u));
            if (kp[r]) act[pos] = wv[r];
            // warp_off is rewritten only after the next chunk's first barrier, which
            // every thread reaches after this read; s_base alternates between two slots
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) *n_act = s_base[par];
}

template <typename T>
__global__ void k_lbfgs_finish(int n, int d, const T *X, const WalkerState<T> *st, double *x_out, double *ell_out,
                               int8_t *status_out, int32_t *iters_out, int32_t *dev_status) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < (int64_t)n * d) x_out[e] = (double)X[e];
    if (e < n) {
        WalkerState<T> s = st[e];
        int8_t status = s.status;
        if (status == SB_WALKER_RUNNING) {
            status = SB_WALKER_MAXITER;
            atomicOr(dev_status, SB_DEV_TIMEOUT);
        }
        status_out[e] = status;
        ell_out[e] = -(double)s.f;
        if (iters_out) iters_out[e] = s.it;
    }
}

template <typename T, int VPL>
void step_vpl(const LbfgsArgs<T> &a, int n, cudaStream_t s) {
    ProfScope prof(PROF_LBFGS_STEP, s);
    note_launch();
    k_lbfgs_step<T, VPL><<<(n + WPB - 1) / WPB, 32 * WPB, 0, s>>>(a);
}

}  // namespace

template <typename T>
void launch_lbfgs_init(int n, int d, const double *starts, const LbfgsArgs<T> &a, int64_t *n_evals,
                       cudaStream_t s) {
    const int64_t tot = (int64_t)n * d > n ? (int64_t)n * d : n;
    note_launch();
    k_lbfgs_init<T><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(n, d, starts, a.XT, a.st, a.act, a.n_act,
                                                                   n_evals);
}

template <typename T>
void launch_lbfgs_step(const LbfgsArgs<T> &a, int n, cudaStream_t s) {
    const int vpl = (a.d + 31) / 32;
    if (vpl <= 1)
        step_vpl<T, 1>(a, n, s);
    else if (vpl <= 2)
        step_vpl<T, 2>(a, n, s);
    else if (vpl <= 4)
        step_vpl<T, 4>(a, n, s);
    else if (vpl <= 8)
        step_vpl<T, 8>(a, n, s);
    else if (vpl <= 16)
        step_vpl<T, 16>(a, n, s);
    else
        step_vpl<T, 32>(a, n, s);
}

template <typename T>
void launch_lbfgs_compact(const LbfgsArgs<T> &a, int64_t *n_evals, cudaStream_t s) {
    note_launch();
    k_lbfgs_compact<T><<<1, 1024, 0, s>>>(a.st, a.act, a.n_act, n_evals);
}

template <typename T>
void launch_lbfgs_finish(int n, int d, const LbfgsArgs<T> &a, double *x_out, double *ell_out, int8_t *status_out,
                         int32_t *iters_out, int32_t *dev_status, cudaStream_t s) {
    const int64_t tot = (int64_t)n * d > n ? (int64_t)n * d : n;
    note_launch();
    k_lbfgs_finish<T><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(n, d, a.X, a.st, x_out, ell_out, status_out,
                                                                     iters_out, dev_status);
}

#define SB_INST(T)                                                                                          \
    template void launch_lbfgs_init<T>(int, int, const double *, const LbfgsArgs<T> &, int64_t *,           \
                                       cudaStream_t);                                                       \
    template void launch_lbfgs_step<T>(const LbfgsArgs<T> &, int, cudaStream_t);                            \
    template void launch_lbfgs_compact<T>(const LbfgsArgs<T> &, int64_t *, cudaStream_t);                   \
    template void launch_lbfgs_finish<T>(int, int, const LbfgsArgs<T> &, double *, double *, int8_t *,      \
                                         int32_t *, int32_t *, cudaStream_t);
SB_INST(double)
SB_INST(float)
#undef SB_INST

}  // namespace sb
