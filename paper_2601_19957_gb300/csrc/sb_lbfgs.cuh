// sb_lbfgs.cuh -- walker state and launch interface of the batched L-BFGS kernels.
#pragma once
#include "sb_internal.cuh"

namespace sb {

template <typename T>
struct WalkerState {
    T f;        // f = -l at the accepted point
    T alpha;    // step of the pending trial
    T dphi;     // grad f . p of the current direction
    int32_t it;     // accepted steps
    int32_t count;  // stored pairs
    int32_t head;   // ring slot of the oldest pair
    int16_t bt;     // backtracks in the current line search
    int8_t status;  // SB_WALKER_*
    int8_t phase;   // 0: start point pending evaluation, 1: trial pending
    int8_t attempt; // 0 first line search of the iteration, 1 retry without history
    int8_t flat;    // consecutive accepted steps without a decrease of f
    int8_t pad[2];
    T pn;           // |p| of the current direction (CTA step)
};

template <typename T>
struct LbfgsArgs {
    int d, m, max_iter, max_backtracks;
    T c1, backtrack, gtol;
    T *X, *G, *P, *XT, *GT, *FT;  // [N][d] (FT: [N])
    T *S, *Y, *rho;               // [N][m][d] (bf16 [N][m][hist_ld(d)] for the CTA step), [N][m]: 1 / s^T y
                                  // (two-loop step) or s^T y (CTA step)
    WalkerState<T> *st;           // [N]
    int32_t *act;                 // [N] active walker ids
    int32_t *n_act;               // device scalar
    int32_t *err;                 // device status word (SB_DEV_TIMEOUT from bounded waits), may be null
    T *dist;                      // [N] upper bound on |new trial - previous trial| (CTA step), may be null
};

template <typename T>
void launch_lbfgs_init(int n, int d, const double *starts, const LbfgsArgs<T> &a, int64_t *n_evals, cudaStream_t s);
template <typename T>
void launch_lbfgs_step(const LbfgsArgs<T> &a, int n, cudaStream_t s);
template <typename T>
void launch_lbfgs_compact(const LbfgsArgs<T> &a, int64_t *n_evals, cudaStream_t s);
// Row pitch (elements) of the mixed path's stored bf16 pairs: whole 16-byte chunks, so
// that every stored row is moved in aligned 16-byte copies; coordinates d .. pitch - 1 hold zeros.
__host__ __device__ __forceinline__ int hist_ld(int d) { return (d + 7) / 8 * 8; }
// FP32 step, one CTA per walker, compact-representation direction (lbfgs_cta.cu);
// the stored pairs S, Y are bf16 ([N][m][hist_ld(d)]). MRI, MYY: per-walker [N][m][m] R^-1
// (R = upper(S^T Y)) and Y^T Y, slot-indexed.
void launch_lbfgs_step_cta(const LbfgsArgs<float> &a, int n, float *MRI, float *MYY, int num_sms, cudaStream_t s);
// Compaction of the mixed path's active list (at most n entries), grouped by key[w]
// (the walker's dominant component, 0..K-1; others last), the list order kept inside a
// group; tmp: [n] scratch, cnt: lbfgs_compact_cnt_elems(n) scratch.
void launch_lbfgs_compact_by_key(const LbfgsArgs<float> &a, int n, int64_t *n_evals, const int32_t *key, int K,
                                 int32_t *tmp, int32_t *cnt, cudaStream_t s);
int lbfgs_compact_blocks(int n);
size_t lbfgs_compact_cnt_elems(int n);
// Whether n walkers fit the keyed compaction (walker ids below 2^25; else the plain
// compaction runs, with the same results).
bool lbfgs_compact_by_key_fits(int n);
// Algorithmic bytes moved by the FP32 step launches while profiling was on
// (synchronises the device, then clears the counter); -1 on a CUDA error.
double lbfgs_bytes_take();

template <typename T>
void launch_lbfgs_finish(int n, int d, const LbfgsArgs<T> &a, double *x_out, double *ell_out, int8_t *status_out,
                         int32_t *iters_out, int32_t *dev_status, cudaStream_t s);

}  // namespace sb
