// sb_capi.cu -- the C ABI of libsb (declared in include/sb.h): argument
// validation, workspace carving and the host-side orchestration of the
// discover -> refine -> laplace stages.
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <map>
#include <mutex>
#include <type_traits>
#include <vector>

#include "sb_adjoint.cuh"
#include "sb_chisao.cuh"
#include "sb_precheck.cuh"
#include "sb_segments.cuh"
#include "sb_fd.cuh"
#include "sb_raysq.cuh"
#include "sb_internal.cuh"
#include "sb_laplace.cuh"
#include "sb_lbfgs.cuh"
#include "sb_tc.cuh"
#include "sb_graph.cuh"

using namespace sb;

namespace {
std::atomic<int64_t> g_launches{0};
std::atomic<uint32_t> g_prof_mask{0};  // bit c: time the launches of class c
std::mutex g_prof_mu;
struct ProfRec {
    int cls;
    cudaEvent_t a, b;
};
std::vector<ProfRec> g_prof;
std::vector<cudaEvent_t> g_ev_pool;  // events of read records, reused (no create per launch)

cudaEvent_t pooled_event() {
    {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        if (!g_ev_pool.empty()) {
            cudaEvent_t e = g_ev_pool.back();
            g_ev_pool.pop_back();
            return e;
        }
    }
    cudaEvent_t e = nullptr;
    return cudaEventCreate(&e) == cudaSuccess ? e : nullptr;
}
}  // namespace
void sb::note_launch(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

sb::ProfScope::ProfScope(int c, cudaStream_t st) : cls(c), s(st), a(nullptr), b(nullptr) {
    if (!prof_class_on(c)) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    a = pooled_event();
    b = a ? pooled_event() : nullptr;
    if (!b) {
        if (a) cudaEventDestroy(a);
        a = nullptr;
        return;
    }
    cudaEventRecord(a, s);
}
sb::ProfScope::~ProfScope() {
    if (!a) return;
    cudaEventRecord(b, s);
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof.push_back({cls, a, b});
}

bool sb::prof_enabled() { return g_prof_mask.load(std::memory_order_relaxed) != 0; }
bool sb::prof_class_on(int cls) { return (g_prof_mask.load(std::memory_order_relaxed) >> cls) & 1u; }

extern "C" void sb_profile_enable(int on) { g_prof_mask.store(on ? 0xFFu : 0u); }
extern "C" void sb_profile_classes(uint32_t mask) { g_prof_mask.store(mask & 0xFFu); }

extern "C" double sb_profile_bytes(int32_t cls) {
    if (cls == PROF_LBFGS_STEP) return lbfgs_bytes_take();
    return 0.0;
}

extern "C" int32_t sb_profile_read(double *ms, int64_t *launches) {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (int c = 0; c < PROF_NCLASS; ++c) {
        if (ms) ms[c] = 0.0;
        if (launches) launches[c] = 0;
    }
    int32_t bad = 0;
    for (auto &r : g_prof) {
        float t = 0.f;
        if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
            if (ms) ms[r.cls] += t;
            if (launches) launches[r.cls] += 1;
        } else {
            ++bad;
        }
        g_ev_pool.push_back(r.a);
        g_ev_pool.push_back(r.b);
    }
    g_prof.clear();
    return bad;
}

extern "C" int64_t sb_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

extern "C" const char *sb_status_string(sb_status s) {
    switch (s) {
        case SB_OK: return "SB_OK";
        case SB_ERR_INVALID_ARG: return "SB_ERR_INVALID_ARG";
        case SB_ERR_CUDA: return "SB_ERR_CUDA";
        case SB_ERR_WORKSPACE: return "SB_ERR_WORKSPACE";
        case SB_ERR_NONFINITE: return "SB_ERR_NONFINITE";
        case SB_ERR_NO_MODES: return "SB_ERR_NO_MODES";
        case SB_ERR_TIMEOUT: return "SB_ERR_TIMEOUT";
        case SB_ERR_UNSUPPORTED: return "SB_ERR_UNSUPPORTED";
    }
    return "SB_ERR_UNKNOWN";
}

namespace {

constexpr int kRoundsPerPoll = 8;  // L-BFGS rounds between host reads of the active count

inline int njt(int d) { return (d + 63) / 64; }

sb_status check_problem(const sb_problem *p) {
    if (!p || !p->log_w || !p->mu || !p->L || !p->lo || !p->hi) return SB_ERR_INVALID_ARG;
    if (p->d < 1 || p->K < 1) return SB_ERR_INVALID_ARG;
    if (p->d > kMaxD || p->K > kMaxK) return SB_ERR_UNSUPPORTED;
    return SB_OK;
}

sb_status check_config(const sb_config *c) {
    if (!c) return SB_ERR_INVALID_ARG;
    if (c->n_rays < 1 || c->n_steps < 1 || c->n_steps > 1024 || c->n_starts < 1) return SB_ERR_INVALID_ARG;
    const int64_t total = (int64_t)c->n_rays * c->n_steps;
    if (total > 0x7fffffffLL || c->n_starts > total) return SB_ERR_INVALID_ARG;
    if (c->m < 1 || c->m > kMaxM || c->max_iter < 0 || c->max_backtracks < 0 || c->max_backtracks > 10000)
        return SB_ERR_INVALID_ARG;
    if (c->newton_steps < 0 || c->newton_steps > 64 || c->cand_cap < 1 || c->cand_cap > 4096)
        return SB_ERR_INVALID_ARG;
    if (!(c->gtol >= 0) || !(c->armijo_c1 > 0 && c->armijo_c1 < 1) || !(c->backtrack > 0 && c->backtrack < 1))
        return SB_ERR_INVALID_ARG;
    if (!(c->dedup_coarse >= 0) || !(c->dedup_tol >= 0) || !(c->eps_grad >= 0)) return SB_ERR_INVALID_ARG;
    if (c->prec < SB_PREC_FP64 || c->prec > SB_PREC_BF16 || c->reserved != 0) return SB_ERR_INVALID_ARG;
    return SB_OK;
}

// ------------------------------------------------------------------ workspace layout
struct SetupWs {
    WsHeader *hdr;
    double *a, *c, *half, *logV, *wmax;
};

struct DiscoverWs {
    double *u, *texit, *ell_all, *qpart;
    int chunk;
    SelectWs sel;
    TcWs tc;        // tensor-core scratch (mixed precision)
    TcQuadWs quad;  // the rays' quadratic form (mixed precision)
};

template <typename T>
struct RefineWs {
    LbfgsArgs<T> lb;
    float *MRI, *MYY;  // [N][m][m] R^-1 (R = upper(S^T Y)) and Y^T Y, slot-indexed (FP32 compact-form step)
    int64_t *n_evals;
    int64_t *round;         // rounds run (device-decided loop)
    int32_t *act_tmp;       // [N] scratch of the grouped compaction (mixed path)
    int32_t *act_cnt;       // its per-CTA bucket counts
    double *qpart, *Z, *R;  // FP64 evaluation
    TcWs tc;                // mixed-precision evaluation
};

struct LaplaceWs {
    double *P, *XC, *LC, *GC, *Z, *R, *qpart, *GK, *H, *delta, *XN, *LN, *XN2, *LN2, *qpart2, *logZk_c, *t, *pred;
    int32_t *reps, *n_reps, *info, *halvings, *rows2, *n_rows2, *reps2, *n_reps2;
    uint8_t *assigned, *active, *searching, *keep;
    double *dd_l;
    int32_t *dd_i;
    uint32_t *dd_bar;
    int32_t *p_done, *p_need;  // [K] P_k formed / to form now
    int32_t *n_live;           // candidates still moving in a Newton step
    int32_t *onehot;           // [cap] component k when a candidate's responsibilities are one-hot, else -1
    int32_t *n_eff;            // candidates a Newton step's evaluations run on (0 once none moves)
};

struct EvidenceWs {
    double *starts, *ell_starts, *x_out, *ell_out;
    int8_t *status;
};

struct Layout {
    SetupWs su;
    DiscoverWs di;
    RefineWs<double> r64;
    RefineWs<float> r32;
    LaplaceWs la;
    EvidenceWs ev;
    size_t bytes;
};

int discover_chunk(int d, int K, int64_t total) {
    const int64_t per = (int64_t)K * njt(d);
    int64_t b = ((int64_t)8 << 20) / per;  // qpart <= 64 MB
    if (b < 64) b = 64;
    if (b > total) b = total;
    return (int)b;
}

template <typename T>
void carve_refine(Carver &cv, RefineWs<T> &r, int n, int d, int K, int m, bool fp64_eval, int prec) {
    auto &a = r.lb;
    a.X = cv.take<T>((size_t)n * d);
    a.G = cv.take<T>((size_t)n * d);
    a.P = cv.take<T>((size_t)n * d);
    a.XT = cv.take<T>((size_t)n * d);
    a.GT = cv.take<T>((size_t)n * d);
    a.FT = cv.take<T>((size_t)n);
    // the mixed path's pairs are bf16 rows of hist_ld(d) elements (as many T = float
    // as half of that)
    const size_t hist = fp64_eval ? (size_t)n * m * d : (size_t)n * m * (hist_ld(d) / 2);
    a.S = cv.take<T>(hist);
    a.Y = cv.take<T>(hist);
    a.rho = cv.take<T>((size_t)n * m);
    a.st = cv.take<WalkerState<T>>((size_t)n);
    a.act = cv.take<int32_t>((size_t)n);
    a.n_act = cv.take<int32_t>(1);
    r.n_evals = cv.take<int64_t>(1);
    r.round = cv.take<int64_t>(1);
    if (fp64_eval) {
        r.qpart = cv.take<double>(lik_f64_qpart_elems(d, K, n));
        r.Z = cv.take<double>((size_t)n * K * d);
        r.R = cv.take<double>((size_t)n * K);
    } else {
        carve_tc(cv, r.tc, n, d, K, prec);
        r.act_tmp = cv.take<int32_t>((size_t)n);
        r.act_cnt = cv.take<int32_t>(lbfgs_compact_cnt_elems(n));
        r.MRI = cv.take<float>((size_t)n * m * m);
        r.MYY = cv.take<float>((size_t)n * m * m);
    }
}

// One layout serves every entry point: the stages' regions never overlap.
Layout layout(void *base, const sb_problem *p, const sb_config *c) {
    Layout L{};
    Carver cv(base);
    const int d = p->d, K = p->K;
    L.su.hdr = cv.take<WsHeader>(1);
    L.su.a = cv.take<double>(K);
    L.su.c = cv.take<double>(d);
    L.su.half = cv.take<double>(d);
    L.su.logV = cv.take<double>(1);
    L.su.wmax = cv.take<double>(1);

    const int64_t total = (int64_t)c->n_rays * c->n_steps;
    const bool fp64 = c->prec == SB_PREC_FP64;
    L.di.u = cv.take<double>((size_t)c->n_rays * d);
    L.di.texit = cv.take<double>(c->n_rays);
    L.di.ell_all = cv.take<double>(total);
    L.di.chunk = discover_chunk(d, K, total);
    if (fp64)
        L.di.qpart = cv.take<double>(lik_f64_qpart_elems(d, K, L.di.chunk));
    else {
        carve_tc(cv, L.di.tc, tc_setup_rows(total), d, K, c->prec);
        carve_tc_quad(cv, L.di.quad, c->n_rays, d, K, c->prec);
    }
    L.di.sel.bucket = cv.take<int32_t>(total);
    L.di.sel.hist = cv.take<uint32_t>(c->n_steps * 2 > 256 ? c->n_steps * 2 : 256);
    L.di.sel.state = cv.take<uint64_t>(8);
    L.di.sel.blockcnt = cv.take<int32_t>(select_blocks(total));
    L.di.sel.idx = cv.take<int64_t>(c->n_starts);

    const int n = c->n_starts;
    if (fp64)
        carve_refine(cv, L.r64, n, d, K, c->m, true, c->prec);
    else
        carve_refine(cv, L.r32, n, d, K, c->m, false, c->prec);

    const int cap = c->cand_cap;
    const int nJT = njt(d);
    const int H2 = kHalvings - 1;
    auto &la = L.la;
    la.P = cv.take<double>((size_t)K * d * d);
    la.reps = cv.take<int32_t>(cap);
    la.n_reps = cv.take<int32_t>(1);
    la.assigned = cv.take<uint8_t>(n > cap ? n : cap);
    la.dd_l = cv.take<double>(2 * kDedupMaxGrid);
    la.dd_i = cv.take<int32_t>(2 * kDedupMaxGrid);
    la.dd_bar = cv.take<uint32_t>(2);
    la.p_done = cv.take<int32_t>(kMaxK);
    la.p_need = cv.take<int32_t>(kMaxK);
    la.n_live = cv.take<int32_t>(1);
    la.onehot = cv.take<int32_t>(cap);
    la.n_eff = cv.take<int32_t>(1);
    la.XC = cv.take<double>((size_t)cap * d);
    la.LC = cv.take<double>(cap);
    la.GC = cv.take<double>((size_t)cap * d);
    la.Z = cv.take<double>((size_t)cap * K * d);
    la.R = cv.take<double>((size_t)cap * K);
    la.qpart = cv.take<double>((size_t)cap * K * nJT);
    la.GK = cv.take<double>((size_t)cap * K * d);
    la.H = cv.take<double>((size_t)cap * d * d);
    la.info = cv.take<int32_t>(cap);
    la.active = cv.take<uint8_t>(cap);
    la.searching = cv.take<uint8_t>(cap);
    la.halvings = cv.take<int32_t>(cap);
    la.t = cv.take<double>(cap);
    la.pred = cv.take<double>(cap);
    la.delta = cv.take<double>((size_t)cap * d);
    la.XN = cv.take<double>((size_t)cap * d);
    la.LN = cv.take<double>(cap);
    la.XN2 = cv.take<double>((size_t)cap * H2 * d);
    la.LN2 = cv.take<double>((size_t)cap * H2);
    la.qpart2 = cv.take<double>((size_t)cap * H2 * K * nJT);
    la.rows2 = cv.take<int32_t>((size_t)cap * H2);
    la.n_rows2 = cv.take<int32_t>(1);
    la.keep = cv.take<uint8_t>(cap);
    la.logZk_c = cv.take<double>(cap);
    la.reps2 = cv.take<int32_t>(cap);
    la.n_reps2 = cv.take<int32_t>(1);

    L.ev.starts = cv.take<double>((size_t)n * d);
    L.ev.ell_starts = cv.take<double>(n);
    L.ev.x_out = cv.take<double>((size_t)n * d);
    L.ev.ell_out = cv.take<double>(n);
    L.ev.status = cv.take<int8_t>(n);
    L.bytes = cv.bytes();
    return L;
}

ProbView make_view(const sb_problem *p, const Layout &L) {
    ProbView v;
    v.d = p->d;
    v.K = p->K;
    v.log_w = p->log_w;
    v.mu = p->mu;
    v.L = p->L;
    v.lo = p->lo;
    v.hi = p->hi;
    v.a = L.su.a;
    v.c = L.su.c;
    v.half = L.su.half;
    v.logV = L.su.logV;
    v.wmax = L.su.wmax;
    v.status = &L.su.hdr->status;
    return v;
}

// ------------------------------------------------------------------ FP64 evaluation helpers
LikF64Args f64_args(const ProbView &pv) {
    LikF64Args a{};
    a.d = pv.d;
    a.K = pv.K;
    a.mu = pv.mu;
    a.L = pv.L;
    a.a = pv.a;
    a.c = pv.c;
    a.ell_sign = 1.0;
    a.grad_sign = -1.0;
    return a;
}

// ------------------------------------------------------------------ stages
sb_status run_discover(const ProbView &pv, const sb_config *c, const Layout &L, double *starts, double *ell,
                       cudaStream_t s) {
    const int d = pv.d;
    const int64_t total = (int64_t)c->n_rays * c->n_steps;
    launch_ray_dirs(d, c->n_rays, c->seed, pv, L.di.u, L.di.texit, c->prec != SB_PREC_FP64, s);
    if (c->prec == SB_PREC_FP64) {
        for (int64_t f0 = 0; f0 < total; f0 += L.di.chunk) {
            const int rows = (int)((total - f0) < L.di.chunk ? (total - f0) : L.di.chunk);
            LikF64Args a = f64_args(pv);
            a.u = L.di.u;
            a.texit = L.di.texit;
            a.n_steps = c->n_steps;
            a.flat0 = f0;
            a.n_rows = rows;
            a.qpart = L.di.qpart;
            a.ell = L.di.ell_all + f0;
            a.out_by_walker = 0;
            launch_lik_f64_rays(a, s);
        }
    } else {
        // one GEMM of the directions, l at the samples from three scalars per (ray, component)
        const sb_status st = tc_ray_loglik_quad(pv, c->n_rays, c->n_steps, c->prec, L.di.tc.bn, L.di.quad, L.di.u,
                                                L.di.texit, L.di.ell_all, s);
        if (st != SB_OK) return st;
    }
    launch_select_starts(L.di.ell_all, c->n_rays, c->n_steps, c->n_starts, L.di.sel, s);
    launch_gather_starts(pv, L.di.u, L.di.texit, c->n_steps, L.di.sel.idx, L.di.ell_all, c->n_starts, starts, ell, s);
    SB_CUDA_TRY(cudaGetLastError());
    return SB_OK;
}

template <typename T>
void eval_round(const ProbView &pv, const sb_config *c, const RefineWs<T> &r, int n, cudaStream_t s);

template <>
void eval_round<double>(const ProbView &pv, const sb_config *c, const RefineWs<double> &r, int n, cudaStream_t s) {
    (void)c;
    LikF64Args a = f64_args(pv);
    a.X = r.lb.XT;
    a.rows = r.lb.act;
    a.n_rows_dev = r.lb.n_act;
    a.n_rows = n;
    a.qpart = r.qpart;
    a.Z = r.Z;
    a.R = r.R;
    a.ell = r.lb.FT;
    a.ell_sign = -1.0;  // f = -l
    a.G = r.lb.GT;
    a.grad_sign = 1.0;  // grad f = -grad l
    a.out_by_walker = 1;
    launch_lik_f64_points(a, true, s);
}

template <>
void eval_round<float>(const ProbView &pv, const sb_config *c, const RefineWs<float> &r, int n, cudaStream_t s) {
    tc_eval_walkers(pv, c, r.tc, r.lb.XT, r.lb.act, r.lb.n_act, n, r.lb.FT, r.lb.GT, s);
}

int device_sms() {
    static const int n = [] {  // thread-safe one-time query
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        return v > 0 ? v : 1;
    }();
    return n;
}


template <typename T>
void step_round(const RefineWs<T> &r, const LbfgsArgs<T> &a, int n, cudaStream_t s);
template <>
void step_round<double>(const RefineWs<double> &, const LbfgsArgs<double> &a, int n, cudaStream_t s) {
    launch_lbfgs_step<double>(a, n, s);  // two-loop recursion, warp per walker
}
template <>
void step_round<float>(const RefineWs<float> &r, const LbfgsArgs<float> &a, int n, cudaStream_t s) {
    // compact form, CTA per walker; it leaves the trial-point distance bounds the
    // next round's component skip reads
    LbfgsArgs<float> b = a;
    b.dist = (float *)r.tc.p[kTcDistSlot];
    launch_lbfgs_step_cta(b, n, r.MRI, r.MYY, device_sms(), s);
}

template <typename T>
sb_status run_refine(const ProbView &pv, const sb_config *c, const RefineWs<T> &r, const double *starts, int n,
                     double *x_out, double *ell_out, int8_t *status_out, int32_t *iters_out, int64_t *n_evals,
                     cudaStream_t s) {
    LbfgsArgs<T> a = r.lb;
    a.d = pv.d;
    a.m = c->m;
    a.max_iter = c->max_iter;
    a.max_backtracks = c->max_backtracks;
    a.c1 = (T)c->armijo_c1;
    a.backtrack = (T)c->backtrack;
    a.gtol = (T)c->gtol;
    a.err = pv.status;
    RefineWs<T> rr = r;
    rr.lb = a;
    int64_t *ev = n_evals ? n_evals : r.n_evals;
    launch_lbfgs_init<T>(n, pv.d, starts, a, ev, s);
    if constexpr (std::is_same<T, float>::value) tc_walkers_reset(r.tc, n, s);
    // every accepted step takes at most 2 (max_backtracks + 2) rounds
    const int64_t cap_rounds = 2 + (int64_t)(c->max_iter + 1) * 2 * (c->max_backtracks + 2);
    auto batch = [&](cudaStream_t bs) {
        for (int b = 0; b < kRoundsPerPoll; ++b) {
            eval_round<T>(pv, c, rr, n, bs);
            step_round<T>(rr, a, n, bs);
            bool keyed = false;
            if constexpr (std::is_same<T, float>::value) {  // walkers grouped by dominant component
                if (lbfgs_compact_by_key_fits(n)) {
                    launch_lbfgs_compact_by_key(a, n, ev, static_cast<const int32_t *>(r.tc.p[12]), pv.K, r.act_tmp,
                                                r.act_cnt, bs);
                    keyed = true;
                }
            }
            if (!keyed) launch_lbfgs_compact<T>(a, ev, bs);
        }
    };
    if (stream_capturing(s)) {
        // the rounds as the body of a WHILE node whose condition the device sets after
        // every batch (walkers still active and the round cap not reached)
        SB_CUDA_TRY(cudaMemsetAsync(r.round, 0, sizeof(int64_t), s));
        const sb_status st = capture_while(s, [&](cudaStream_t bs, cudaGraphConditionalHandle h) {
            batch(bs);
            launch_loop_cond(h, r.round, kRoundsPerPoll, cap_rounds, a.n_act, pv.status, bs);
            return cudaGetLastError() == cudaSuccess ? SB_OK : SB_ERR_CUDA;
        });
        if (st != SB_OK) return st;
    } else {
        // eager: the host reads the active count after every batch of rounds
        int64_t round = 0;
        while (true) {
            batch(s);
            round += kRoundsPerPoll;
            int32_t h_act = 0;
            SB_CUDA_TRY(cudaMemcpyAsync(&h_act, a.n_act, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            SB_CUDA_TRY(cudaStreamSynchronize(s));
            if (h_act == 0 || round >= cap_rounds) break;
        }
    }
    launch_lbfgs_finish<T>(n, pv.d, a, x_out, ell_out, status_out, iters_out, pv.status, s);
    SB_CUDA_TRY(cudaGetLastError());
    return SB_OK;
}

// l and grad l (FP64) at the Laplace stage's candidates (few points): rows of X listed in
// rows[0..*n_rows) (or 0..n), outputs by row id.
void f64_points(const ProbView &pv, const double *X, const int32_t *rows, const int32_t *n_rows_dev, int n_rows,
                double *qpart, double *Z, double *R, double *ell, double *G, cudaStream_t s) {
    LikF64Args a = f64_args(pv);
    a.X = X;
    a.rows = rows;
    a.n_rows_dev = n_rows_dev;
    a.n_rows = n_rows;
    a.qpart = qpart;
    a.Z = Z;
    a.R = R;
    a.ell = ell;
    a.G = G;
    a.out_by_walker = 1;
    launch_lik_f64_few(a, G != nullptr, s);
}

sb_status run_laplace(const ProbView &pv, const sb_config *c, const Layout &L, const double *x, const double *ell,
                      const int8_t *status, int n, double *modes, double *logZk, double *ell_modes, int cap_out,
                      int32_t *n_modes, double *logZ, cudaStream_t s) {
    const int d = pv.d, K = pv.K, cap = c->cand_cap;
    const auto &la = L.la;
    SB_CUDA_TRY(cudaMemsetAsync(la.p_done, 0, sizeof(int32_t) * kMaxK, s));
    const DedupScratch dds{la.dd_l, la.dd_i, la.dd_bar, pv.status};
    launch_dedup(n, d, x, ell, status, nullptr, c->dedup_coarse, pv.wmax, cap, la.reps, la.n_reps, la.assigned, dds,
                 s);
    launch_gather_rows(d, cap, x, la.reps, la.n_reps, la.XC, ell, la.LC, s);
    // Every candidate kernel below is sized by cand_cap and reads the candidate count
    // (n_reps, or n_eff inside a Newton step) on the device: no host read, so the
    // stage can sit in a captured graph.
    SB_CUDA_TRY(cudaMemsetAsync(la.active, 1, cap, s));
    // l, grad l, H and its Cholesky factor at every candidate (of the first *nc)
    auto eval_full = [&](const int32_t *nc) {
        f64_points(pv, la.XC, nullptr, nc, cap, la.qpart, la.Z, la.R, la.LC, la.GC, s);
        launch_onehot(K, la.R, nc, cap, la.onehot, s);
        launch_precision_needed(d, K, pv.L, la.R, nc, la.p_done, la.p_need, la.P, s, la.onehot);
        launch_hessian_chol(d, K, cap, pv.L, la.P, la.Z, la.R, la.GC, nc, la.GK, la.H, la.info, la.dd_bar, pv.status, s,
                            la.onehot);
    };
    eval_full(la.n_reps);
    // Newton polish, newton_steps steps; a step's evaluations run on n_eff candidates,
    // which drops to zero once no candidate's Newton step is above the convergence
    // threshold (the rest of the polish is then empty launches)
    launch_set_eff(la.n_eff, la.n_reps, nullptr, s);
    for (int step = 0; step < c->newton_steps; ++step) {
        launch_chol_solve_coop(d, cap, la.H, la.GC, la.n_eff, la.info, la.active, la.delta, la.pred, la.dd_bar,
                               pv.status, s);
        SB_CUDA_TRY(cudaMemsetAsync(la.n_live, 0, sizeof(int32_t), s));
        launch_newton_ls(d, cap, 0, la.n_eff, la.info, la.active, la.searching, la.halvings, la.t, la.XC, la.LC,
                         la.delta, la.XN, la.LN, la.pred, la.n_live, s);
        launch_set_eff(la.n_eff, la.n_reps, la.n_live, s);
        f64_points(pv, la.XN, nullptr, la.n_eff, cap, la.qpart, nullptr, nullptr, la.LN, nullptr, s);
        launch_newton_ls(d, cap, 1, la.n_eff, la.info, la.active, la.searching, la.halvings, la.t, la.XC, la.LC,
                         la.delta, la.XN, la.LN, la.pred, la.n_live, s);
        launch_ls_batch_setup(d, cap, la.n_eff, la.searching, la.XC, la.delta, la.XN2, la.rows2, la.n_rows2, s);
        f64_points(pv, la.XN2, la.rows2, la.n_rows2, cap * (kHalvings - 1), la.qpart2, nullptr, nullptr, la.LN2,
                   nullptr, s);
        launch_ls_batch_decide(d, cap, la.n_eff, la.searching, la.active, la.XC, la.LC, la.XN2, la.LN2, s);
        eval_full(la.n_eff);
    }
    SB_CUDA_TRY(cudaMemsetAsync(la.keep, 0, cap, s));
    launch_cand_stats(d, cap, la.XC, la.LC, la.GC, la.H, la.info, pv.lo, pv.hi, c->eps_grad, la.n_reps, la.keep,
                      la.logZk_c, s);
    launch_dedup(cap, d, la.XC, la.LC, nullptr, la.keep, c->dedup_tol, pv.wmax, cap, la.reps2, la.n_reps2,
                 la.assigned, dds, s);
    launch_laplace_final(d, la.XC, la.LC, la.logZk_c, la.n_reps, la.reps2, la.n_reps2, pv.logV, cap_out, modes, logZk,
                         ell_modes, n_modes, logZ, pv.status, s);
    SB_CUDA_TRY(cudaGetLastError());
    return SB_OK;
}

struct Prelude {
    Layout L;
    ProbView pv;
    cudaStream_t s;
};

sb_status prelude(const sb_problem *p, const sb_config *c, void *ws, size_t ws_bytes, void *stream, Prelude &out) {
    sb_status st = check_problem(p);
    if (st != SB_OK) return st;
    st = check_config(c);
    if (st != SB_OK) return st;
    if (!ws) return SB_ERR_INVALID_ARG;
    if (c->prec != SB_PREC_FP64 && !tc_available(c->prec)) return SB_ERR_UNSUPPORTED;
    Layout L = layout(ws, p, c);
    if (ws_bytes < L.bytes) return SB_ERR_WORKSPACE;
    out.L = L;
    out.pv = make_view(p, L);
    out.s = static_cast<cudaStream_t>(stream);
    SB_CUDA_TRY(cudaMemsetAsync(L.su.hdr, 0, sizeof(WsHeader), out.s));
    launch_setup(out.pv, out.s);
    if (c->prec != SB_PREC_FP64) {
        // one converted copy of L_k, mu, c serves discover and refine
        st = tc_prepare(out.pv, out.L.di.tc, out.s);
        if (st != SB_OK) return st;
        for (int i = 0; i < 4; ++i) out.L.r32.tc.p[i] = out.L.di.tc.p[i];
        out.L.r32.tc.p[15] = out.L.di.tc.p[15];  // |L_k|_F
        out.L.r32.tc.mapT = out.L.di.tc.mapT;
        out.L.r32.tc.mapB = out.L.di.tc.mapB;
        out.L.r32.tc.bn = out.L.di.tc.bn;
        if (!tc_maps_for_rows(out.L.r32.tc)) return SB_ERR_CUDA;
    }
    SB_CUDA_TRY(cudaGetLastError());
    return SB_OK;
}

// Host-side checks of a solve call (the size of the workspace included).
sb_status check_call(const sb_problem *p, const sb_config *c, const void *ws, size_t ws_bytes, bool chisao);

// Key of a graph-mode call: the entry point, the problem's shape and arrays, the knobs
// and the workspace (the caller adds its own outputs).
GraphKey call_key(int fn, const sb_problem *p, const sb_config *c, const void *ws, size_t ws_bytes) {
    GraphKey k;
    k.add((uint64_t)fn);
    k.add((uint64_t)p->d);
    k.add((uint64_t)p->K);
    for (const void *q : {(const void *)p->log_w, (const void *)p->mu, (const void *)p->L, (const void *)p->lo,
                          (const void *)p->hi})
        k.add_ptr(q);
    k.add_bytes(*c);
    k.add_ptr(ws);
    k.add((uint64_t)ws_bytes);
    return k;
}

// Before a graph-mode capture of a mixed-precision call whose shape the tile autotuner
// has not seen: one eager prelude on the caller's stream, which times the tiles (the
// capture itself cannot synchronise).
void pretune(const sb_problem *p, const sb_config *c, void *ws, size_t ws_bytes, cudaStream_t s) {
    if (c->prec == SB_PREC_FP64 || stream_capturing(s) || !graph_mode_for(s)) return;
    if (tc_tuned_tile(p->d, p->K, c->prec) != 0) return;
    Prelude P;
    (void)prelude(p, c, ws, ws_bytes, s, P);
}

}  // namespace

extern "C" size_t sb_workspace_bytes(const sb_problem *p, const sb_config *c) {
    if (check_problem(p) != SB_OK || check_config(c) != SB_OK) return 0;
    return layout(nullptr, p, c).bytes;
}

extern "C" sb_status sb_discover(const sb_problem *p, const sb_config *c, double *starts, double *ell, void *ws,
                                 size_t ws_bytes, void *stream) {
    if (!starts || !ell) return SB_ERR_INVALID_ARG;
    Prelude P;
    sb_status st = prelude(p, c, ws, ws_bytes, stream, P);
    if (st != SB_OK) return st;
    return run_discover(P.pv, c, P.L, starts, ell, P.s);
}

extern "C" sb_status sb_refine(const sb_problem *p, const sb_config *c, const double *starts, int32_t n,
                               double *x_out, double *ell_out, int8_t *status_out, int32_t *iters_out,
                               int64_t *n_evals, void *ws, size_t ws_bytes, void *stream) {
    if (!starts || !x_out || !ell_out || !status_out) return SB_ERR_INVALID_ARG;
    if (!c || n < 1 || n > c->n_starts) return SB_ERR_INVALID_ARG;
    sb_status st = check_call(p, c, ws, ws_bytes, false);
    if (st != SB_OK) return st;
    cudaStream_t s0 = static_cast<cudaStream_t>(stream);
    GraphKey key = call_key(3, p, c, ws, ws_bytes);
    for (const void *q : {(const void *)starts, (const void *)x_out, (const void *)ell_out, (const void *)status_out,
                          (const void *)iters_out, (const void *)n_evals})
        key.add_ptr(q);
    key.add((uint64_t)n);
    pretune(p, c, ws, ws_bytes, s0);
    return run_graph_or_direct(s0, key, [&](cudaStream_t s) {
        Prelude P;
        sb_status r = prelude(p, c, ws, ws_bytes, s, P);
        if (r != SB_OK) return r;
        if (c->prec == SB_PREC_FP64)
            return run_refine<double>(P.pv, c, P.L.r64, starts, n, x_out, ell_out, status_out, iters_out, n_evals, s);
        return run_refine<float>(P.pv, c, P.L.r32, starts, n, x_out, ell_out, status_out, iters_out, n_evals, s);
    });
}

extern "C" sb_status sb_laplace(const sb_problem *p, const sb_config *c, const double *x, const double *ell,
                                const int8_t *status, int32_t n, double *modes, double *logZk, double *ell_modes,
                                int32_t cap, int32_t *n_modes, double *logZ, void *ws, size_t ws_bytes,
                                void *stream) {
    if (!x || !ell || !modes || !logZk || !n_modes || !logZ || cap < 1) return SB_ERR_INVALID_ARG;
    if (!c || n < 1 || n > (c->n_starts > c->cand_cap ? c->n_starts : c->cand_cap)) return SB_ERR_INVALID_ARG;
    Prelude P;
    sb_status st = prelude(p, c, ws, ws_bytes, stream, P);
    if (st != SB_OK) return st;
    return run_laplace(P.pv, c, P.L, x, ell, status, n, modes, logZk, ell_modes, cap, n_modes, logZ, P.s);
}

// discover + refine + laplace on one prelude (the whole hot path), no host read.
static sb_status enqueue_evidence(const sb_problem *p, const sb_config *c, double *logZ, double *modes, double *logZk,
                           int32_t cap, int32_t *n_modes, void *ws, size_t ws_bytes, cudaStream_t s) {
    Prelude P;
    sb_status st = prelude(p, c, ws, ws_bytes, s, P);
    if (st != SB_OK) return st;
    const auto &ev = P.L.ev;
    st = run_discover(P.pv, c, P.L, ev.starts, ev.ell_starts, s);
    if (st != SB_OK) return st;
    if (c->prec == SB_PREC_FP64)
        st = run_refine<double>(P.pv, c, P.L.r64, ev.starts, c->n_starts, ev.x_out, ev.ell_out, ev.status, nullptr,
                                nullptr, s);
    else
        st = run_refine<float>(P.pv, c, P.L.r32, ev.starts, c->n_starts, ev.x_out, ev.ell_out, ev.status, nullptr,
                               nullptr, s);
    if (st != SB_OK) return st;
    return run_laplace(P.pv, c, P.L, ev.x_out, ev.ell_out, ev.status, c->n_starts, modes, logZk, nullptr, cap,
                       n_modes, logZ, s);
}

extern "C" sb_status sb_evidence(const sb_problem *p, const sb_config *c, double *logZ, double *modes,
                                 double *logZk, int32_t cap, int32_t *n_modes, void *ws, size_t ws_bytes,
                                 void *stream) {
    if (!logZ || !modes || !logZk || !n_modes || cap < 1) return SB_ERR_INVALID_ARG;
    sb_status st = check_call(p, c, ws, ws_bytes, false);
    if (st != SB_OK) return st;
    cudaStream_t s0 = static_cast<cudaStream_t>(stream);
    GraphKey key = call_key(4, p, c, ws, ws_bytes);
    for (const void *q : {(const void *)logZ, (const void *)modes, (const void *)logZk, (const void *)n_modes})
        key.add_ptr(q);
    key.add((uint64_t)cap);
    pretune(p, c, ws, ws_bytes, s0);
    return run_graph_or_direct(s0, key, [&](cudaStream_t s) {
        return enqueue_evidence(p, c, logZ, modes, logZk, cap, n_modes, ws, ws_bytes, s);
    });
}

extern "C" sb_status sb_check(void *ws, size_t ws_bytes, void *stream) {
    if (!ws || ws_bytes < sizeof(WsHeader)) return SB_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int32_t word = 0;
    SB_CUDA_TRY(cudaMemcpyAsync(&word, ws, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    SB_CUDA_TRY(cudaStreamSynchronize(s));
    SB_CUDA_TRY(cudaMemsetAsync(ws, 0, sizeof(int32_t), s));
    if (word & SB_DEV_NONFINITE) return SB_ERR_NONFINITE;
    if (word & SB_DEV_INVALID) return SB_ERR_INVALID_ARG;
    if (word & SB_DEV_TIMEOUT) return SB_ERR_TIMEOUT;
    if (word & SB_DEV_NO_MODES) return SB_ERR_NO_MODES;
    return SB_OK;
}

// ------------------------------------------------------------------ host-buffer entry points
namespace {
struct HostLayout {
    double *log_w, *mu, *L, *lo, *hi, *logZ, *modes, *logZk;
    int32_t *n_modes;
    void *inner;
    size_t inner_bytes, bytes;
};

// Device copies of the problem arrays and of the outputs, then `inner_bytes` of
// scratch for the solve itself.
HostLayout host_layout(void *base, const sb_problem *p, int cap, size_t inner_bytes) {
    HostLayout h{};
    Carver cv(base);
    const int d = p->d, K = p->K;
    h.log_w = cv.take<double>(K);
    h.mu = cv.take<double>((size_t)K * d);
    h.L = cv.take<double>((size_t)K * d * d);
    h.lo = cv.take<double>(d);
    h.hi = cv.take<double>(d);
    h.logZ = cv.take<double>(1);
    h.n_modes = cv.take<int32_t>(1);
    h.modes = cv.take<double>((size_t)cap * d);
    h.logZk = cv.take<double>(cap);
    h.inner_bytes = inner_bytes;
    h.inner = cv.take<char>(h.inner_bytes);
    h.bytes = cv.bytes();
    return h;
}

// Copies the host problem in, runs `solve` on device buffers, copies log Z, the mode
// count, the modes and their log Z_k out, and returns the device status word.
template <typename Solve>
sb_status host_solve(const sb_problem *hp, const sb_config *c, size_t inner_bytes, double *logZ, double *modes,
                     double *logZk, int32_t cap, int32_t *n_modes, void *ws, size_t ws_bytes, void *stream,
                     Solve solve) {
    if (!logZ || !n_modes || !ws || cap < 1) return SB_ERR_INVALID_ARG;
    const int ccap = c->cand_cap;
    HostLayout h = host_layout(ws, hp, ccap, inner_bytes);
    if (ws_bytes < h.bytes) return SB_ERR_WORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int d = hp->d, K = hp->K;
    SB_CUDA_TRY(cudaMemcpyAsync(h.log_w, hp->log_w, sizeof(double) * K, cudaMemcpyHostToDevice, s));
    SB_CUDA_TRY(cudaMemcpyAsync(h.mu, hp->mu, sizeof(double) * K * d, cudaMemcpyHostToDevice, s));
    SB_CUDA_TRY(cudaMemcpyAsync(h.L, hp->L, sizeof(double) * (size_t)K * d * d, cudaMemcpyHostToDevice, s));
    SB_CUDA_TRY(cudaMemcpyAsync(h.lo, hp->lo, sizeof(double) * d, cudaMemcpyHostToDevice, s));
    SB_CUDA_TRY(cudaMemcpyAsync(h.hi, hp->hi, sizeof(double) * d, cudaMemcpyHostToDevice, s));
    sb_problem dp{d, K, h.log_w, h.mu, h.L, h.lo, h.hi};
    sb_status st = solve(&dp, h.logZ, h.modes, h.logZk, ccap, h.n_modes, h.inner, h.inner_bytes, stream);
    if (st != SB_OK) return st;
    SB_CUDA_TRY(cudaMemcpyAsync(logZ, h.logZ, sizeof(double), cudaMemcpyDeviceToHost, s));
    SB_CUDA_TRY(cudaMemcpyAsync(n_modes, h.n_modes, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    SB_CUDA_TRY(cudaStreamSynchronize(s));
    const int nm = *n_modes < cap ? *n_modes : cap;
    const int nc = nm < ccap ? nm : ccap;
    if (modes && nc > 0)
        SB_CUDA_TRY(cudaMemcpyAsync(modes, h.modes, sizeof(double) * (size_t)nc * d, cudaMemcpyDeviceToHost, s));
    if (logZk && nc > 0) SB_CUDA_TRY(cudaMemcpyAsync(logZk, h.logZk, sizeof(double) * nc, cudaMemcpyDeviceToHost, s));
    SB_CUDA_TRY(cudaStreamSynchronize(s));
    return sb_check(h.inner, h.inner_bytes, stream);
}
}  // namespace

extern "C" size_t sb_evidence_host_workspace_bytes(const sb_problem *hp, const sb_config *c) {
    if (check_problem(hp) != SB_OK || check_config(c) != SB_OK) return 0;
    return host_layout(nullptr, hp, c->cand_cap, layout(nullptr, hp, c).bytes).bytes;
}

extern "C" sb_status sb_evidence_host(const sb_problem *hp, const sb_config *c, double *logZ, double *modes,
                                      double *logZk, int32_t cap, int32_t *n_modes, void *ws, size_t ws_bytes,
                                      void *stream) {
    sb_status st = check_problem(hp);
    if (st != SB_OK) return st;
    st = check_config(c);
    if (st != SB_OK) return st;
    return host_solve(hp, c, layout(nullptr, hp, c).bytes, logZ, modes, logZk, cap, n_modes, ws, ws_bytes, stream,
                      [c](const sb_problem *dp, double *lz, double *md, double *zk, int32_t cp, int32_t *nm,
                          void *in, size_t inb, void *str) { return sb_evidence(dp, c, lz, md, zk, cp, nm, in, inb, str); });
}

// ------------------------------------------------------------------ batched log-likelihood
extern "C" size_t sb_loglik_workspace_bytes(const sb_problem *p, int32_t prec, int32_t n) {
    if (check_problem(p) != SB_OK || n < 1) return 0;
    Carver cv(nullptr);
    cv.take<WsHeader>(1);
    cv.take<double>(p->K);
    if (prec == SB_PREC_FP64) {
        cv.take<double>(lik_f64_qpart_elems(p->d, p->K, n));
        cv.take<double>((size_t)n * p->K * p->d);
        cv.take<double>((size_t)n * p->K);
    } else if (prec == SB_PREC_TF32 || prec == SB_PREC_BF16) {
        TcWs t;
        carve_tc(cv, t, n, p->d, p->K, prec);
        cv.take<float>((size_t)n);
        cv.take<float>((size_t)n * p->d);
        cv.take<double>(2 * (size_t)p->d + 3);
    } else {
        return 0;
    }
    return cv.bytes();
}

extern "C" sb_status sb_loglik(const sb_problem *p, int32_t prec, const double *x, int32_t n, double *ell,
                               double *grad, void *ws, size_t ws_bytes, void *stream) {
    sb_status st = check_problem(p);
    if (st != SB_OK) return st;
    if (!x || !ell || !ws || n < 1) return SB_ERR_INVALID_ARG;
    if (prec < SB_PREC_FP64 || prec > SB_PREC_BF16) return SB_ERR_INVALID_ARG;
    if (prec != SB_PREC_FP64 && !tc_available(prec)) return SB_ERR_UNSUPPORTED;
    if (ws_bytes < sb_loglik_workspace_bytes(p, prec, n)) return SB_ERR_WORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Carver cv(ws);
    WsHeader *hdr = cv.take<WsHeader>(1);
    double *a = cv.take<double>(p->K);
    SB_CUDA_TRY(cudaMemsetAsync(hdr, 0, sizeof(WsHeader), s));
    ProbView pv{};
    pv.d = p->d;
    pv.K = p->K;
    pv.log_w = p->log_w;
    pv.mu = p->mu;
    pv.L = p->L;
    pv.lo = p->lo;
    pv.hi = p->hi;
    pv.a = a;
    pv.status = &hdr->status;
    if (prec == SB_PREC_FP64) {
        double *qpart = cv.take<double>(lik_f64_qpart_elems(p->d, p->K, n));
        double *Z = cv.take<double>((size_t)n * p->K * p->d);
        double *R = cv.take<double>((size_t)n * p->K);
        // setup needs c/half/logV/wmax only for box work; give it scratch inside Z (overwritten later)
        pv.c = Z;
        pv.half = Z + p->d;
        pv.logV = Z + 2 * p->d;
        pv.wmax = Z + 2 * p->d + 1;
        launch_setup(pv, s);
        LikF64Args la = f64_args(pv);
        la.X = x;
        la.n_rows = n;
        la.qpart = qpart;
        la.Z = Z;
        la.R = R;
        la.ell = ell;
        la.G = grad;
        la.out_by_walker = 0;
        launch_lik_f64_points(la, grad != nullptr, s);
    } else {
        TcWs t;
        carve_tc(cv, t, n, p->d, p->K, prec);
        float *f = cv.take<float>((size_t)n);
        float *g = cv.take<float>((size_t)n * p->d);
        double *box = cv.take<double>(2 * (size_t)p->d + 3);
        pv.c = box;
        pv.half = box + p->d;
        pv.logV = box + 2 * p->d;
        pv.wmax = box + 2 * p->d + 1;
        launch_setup(pv, s);
        sb_config c{};
        c.prec = prec;
        st = tc_prepare(pv, t, s, false);  // no walker rounds here
        if (st != SB_OK) return st;
        st = tc_loglik_points(pv, &c, t, x, n, f, grad ? g : nullptr, ell, grad, s);
        if (st != SB_OK) return st;
    }
    SB_CUDA_TRY(cudaGetLastError());
    return SB_OK;
}

extern "C" sb_status sb_evidence_stats(const sb_problem *p, const sb_config *c, void *ws, size_t ws_bytes,
                                       int64_t *out, void *stream) {
    sb_status st = check_problem(p);
    if (st != SB_OK) return st;
    st = check_config(c);
    if (st != SB_OK) return st;
    if (!ws || !out) return SB_ERR_INVALID_ARG;
    const Layout L = layout(ws, p, c);
    if (ws_bytes < L.bytes) return SB_ERR_WORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int64_t ev = 0;
    int32_t nc = 0, nm = 0;
    const int64_t *evp = c->prec == SB_PREC_FP64 ? L.r64.n_evals : L.r32.n_evals;
    SB_CUDA_TRY(cudaMemcpyAsync(&ev, evp, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SB_CUDA_TRY(cudaMemcpyAsync(&nc, L.la.n_reps, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    SB_CUDA_TRY(cudaMemcpyAsync(&nm, L.la.n_reps2, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    SB_CUDA_TRY(cudaStreamSynchronize(s));
    out[0] = (int64_t)c->n_rays * c->n_steps;
    out[1] = ev;
    out[2] = nc;
    out[3] = nm;
    return SB_OK;
}

// ------------------------------------------------------------------ adjoint
namespace {
struct BwdLayout {
    WsHeader *hdr;
    double *a, *c, *half, *logV, *wmax;
    AdjWs adj;
    size_t bytes;
};
BwdLayout bwd_layout(void *base, const sb_problem *p) {
    BwdLayout B{};
    Carver cv(base);
    B.hdr = cv.take<WsHeader>(1);
    B.a = cv.take<double>(p->K);
    B.c = cv.take<double>(p->d);
    B.half = cv.take<double>(p->d);
    B.logV = cv.take<double>(1);
    B.wmax = cv.take<double>(1);
    adjoint_carve(cv, B.adj, p->d, p->K);
    B.bytes = cv.bytes();
    return B;
}
}  // namespace

extern "C" size_t sb_evidence_backward_workspace_bytes(const sb_problem *p) {
    if (check_problem(p) != SB_OK) return 0;
    return bwd_layout(nullptr, p).bytes;
}

extern "C" sb_status sb_evidence_backward(const sb_problem *p, const double *modes, const double *logZk,
                                          int32_t n_modes, double grad_logZ, double *dmu, double *dL, void *ws,
                                          size_t ws_bytes, void *stream) {
    sb_status st = check_problem(p);
    if (st != SB_OK) return st;
    if (!modes || !logZk || !dmu || !dL || !ws || n_modes < 1 || n_modes > kMaxAdjModes) return SB_ERR_INVALID_ARG;
    const BwdLayout B = bwd_layout(ws, p);
    if (ws_bytes < B.bytes) return SB_ERR_WORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    SB_CUDA_TRY(cudaMemsetAsync(B.hdr, 0, sizeof(WsHeader), s));
    ProbView pv{};
    pv.d = p->d;
    pv.K = p->K;
    pv.log_w = p->log_w;
    pv.mu = p->mu;
    pv.L = p->L;
    pv.lo = p->lo;
    pv.hi = p->hi;
    pv.a = B.a;
    pv.c = B.c;
    pv.half = B.half;
    pv.logV = B.logV;
    pv.wmax = B.wmax;
    pv.status = &B.hdr->status;
    launch_setup(pv, s);
    return adjoint_run(pv, B.adj, modes, logZk, n_modes, grad_logZ, dmu, dL, s);
}

extern "C" int32_t sb_tuned_tile(int32_t d, int32_t K, int32_t prec) { return tc_tuned_tile(d, K, prec); }

// ------------------------------------------------------------------ ChiSao (Sec. 3.5.5)
namespace {

struct ChisaoWs {
    double *X, *V, *G, *ell, *ellg, *O, *U, *texit, *Q, *P, *ellp, *qp;
    float *O32, *U32;  // FP32 copies of the reseeding rays (mixed path)
    int8_t *status;
    uint8_t *conv, *stuck, *lost;
    int32_t *reps, *n_reps, *lost_list, *unconv_list, *moving_list, *cnt;
    int32_t *job_start, *job_pk, *job_b, *job_cols;
    int64_t *job_off;
    int64_t *stats;  // [4] l-only ray evaluations, L-BFGS l+grad, anti-convergence l+grad, -
    int32_t *state;  // [8] the oscillations' device-side state (see launch_cs_state_init)
    int32_t *rows;   // [0] ray samples of the current reseeding chunk (all rays: mixed path), [1] its rays
    int lc;  // lost samples per chunk of ray samples (FP64 path)
    TcQuadWs quad;    // mixed path: the reseeding rays' quadratic form (split operands, partials)
    TcOriginWs orig;  // mixed path: z_k at the rays' origins
    size_t bytes;
};

// Carved after the solve stages' layout (offset `off`), for up to n_starts samples.
ChisaoWs chisao_layout(void *base, size_t off, const sb_problem *p, const sb_config *c) {
    ChisaoWs w{};
    Carver cv(base ? static_cast<char *>(base) + off : nullptr);
    const int n = c->n_starts, d = p->d, K = p->K;
    w.lc = n / c->n_steps > 0 ? n / c->n_steps : 1;
    const int rows = w.lc * c->n_steps;
    w.X = cv.take<double>((size_t)n * d);
    w.V = cv.take<double>((size_t)n * d);
    w.G = cv.take<double>((size_t)n * d);
    w.O = cv.take<double>((size_t)n * d);
    w.U = cv.take<double>((size_t)n * d);
    w.Q = cv.take<double>((size_t)n * d);  // Golden Rooster bases: at most one column per lost sample
    w.ell = cv.take<double>(n);
    w.ellg = cv.take<double>(n);
    w.texit = cv.take<double>(n);
    const bool mixed = c->prec != SB_PREC_FP64;
    if (!mixed) {
        w.P = cv.take<double>((size_t)rows * d);
        w.qp = cv.take<double>(lik_f64_qpart_elems(d, K, rows));
    }
    // the mixed path evaluates every reseeding ray in one pass
    w.ellp = cv.take<double>(mixed ? (size_t)n * c->n_steps : (size_t)rows);
    w.status = cv.take<int8_t>(n);
    w.conv = cv.take<uint8_t>(n);
    w.stuck = cv.take<uint8_t>(n);
    w.lost = cv.take<uint8_t>(n);
    w.reps = cv.take<int32_t>(n);
    w.n_reps = cv.take<int32_t>(1);
    w.lost_list = cv.take<int32_t>(n);
    w.unconv_list = cv.take<int32_t>(n);
    w.moving_list = cv.take<int32_t>(n);
    w.cnt = cv.take<int32_t>(4);
    w.job_start = cv.take<int32_t>((size_t)n + 1);
    w.job_pk = cv.take<int32_t>(n);
    w.job_b = cv.take<int32_t>(n);
    w.job_cols = cv.take<int32_t>(n);
    w.job_off = cv.take<int64_t>(n);
    w.stats = cv.take<int64_t>(4);
    w.state = cv.take<int32_t>(8);
    w.rows = cv.take<int32_t>(2);
    if (mixed) {
        w.O32 = cv.take<float>((size_t)n * d);
        w.U32 = cv.take<float>((size_t)n * d);
        carve_tc_quad(cv, w.quad, n, d, K, c->prec);
        carve_tc_origins(cv, w.orig, n, d, K, c->prec);
    }
    w.bytes = cv.bytes();
    return w;
}

sb_status check_chisao(const sb_chisao_config *cc) {
    if (!cc) return SB_ERR_INVALID_ARG;
    if (cc->n_osc < 1 || cc->n_osc > 1024 || cc->conv_iters < 0 || cc->anti_steps < 0 || cc->anti_steps > 100000 ||
        cc->min_unconverged < 1)
        return SB_ERR_INVALID_ARG;
    if (!std::isfinite(cc->momentum) || !std::isfinite(cc->anti_alpha)) return SB_ERR_INVALID_ARG;
    return SB_OK;
}

}  // namespace

namespace {
sb_status check_call(const sb_problem *p, const sb_config *c, const void *ws, size_t ws_bytes, bool chisao) {
    sb_status st = check_problem(p);
    if (st != SB_OK) return st;
    st = check_config(c);
    if (st != SB_OK) return st;
    if (!ws) return SB_ERR_INVALID_ARG;
    if (c->prec != SB_PREC_FP64 && !tc_available(c->prec)) return SB_ERR_UNSUPPORTED;
    size_t need = layout(nullptr, p, c).bytes;
    if (chisao) need += chisao_layout(nullptr, need, p, c).bytes;
    return ws_bytes < need ? SB_ERR_WORKSPACE : SB_OK;
}
}  // namespace

extern "C" size_t sb_chisao_workspace_bytes(const sb_problem *p, const sb_config *c) {
    if (check_problem(p) != SB_OK || check_config(c) != SB_OK) return 0;
    const size_t base = layout(nullptr, p, c).bytes;
    return base + chisao_layout(nullptr, base, p, c).bytes;
}

namespace {

// The ChiSao oscillation (Sec. 3.5.5, Algorithm 1) of the n samples at x0 after a
// prelude: every decision that depends on device state (which samples stick, are
// lost or move, which reseeding branch runs, the Golden Rooster groups) is taken by
// kernels, so the host only enqueues and the whole loop can sit in a captured graph.
sb_status run_chisao(const Prelude &P, const sb_config *c, const sb_chisao_config *cc, const ChisaoWs &w,
                     const double *x0, int n, double *x_out, double *ell_out, int8_t *stuck_out, int32_t *n_peaks,
                     cudaStream_t s) {
    const int d = P.pv.d;
    const ProbView &pv = P.pv;
    const auto &la = P.L.la;
    const auto &r = P.L.r64;
    const bool mixed = c->prec != SB_PREC_FP64;
    sb_status st = SB_OK;
    sb_config c2 = *c;
    c2.max_iter = cc->conv_iters;
    const DedupScratch dds{la.dd_l, la.dd_i, la.dd_bar, pv.status};
    SB_CUDA_TRY(cudaMemsetAsync(w.stats, 0, sizeof(int64_t) * 4, s));
    launch_cs_state_init(w.state, s);
    if (mixed) {
        st = tc_quad_prepare_origins(pv, c->prec, w.quad, w.orig, s);
        if (st != SB_OK) return st;
    }
    SB_CUDA_TRY(cudaMemcpyAsync(w.X, x0, sizeof(double) * n * d, cudaMemcpyDeviceToDevice, s));
    // l and grad l at the samples listed in rows (all n when rows is null)
    auto grad_at = [&](const int32_t *rows, const int32_t *n_rows_dev, int n_rows) {
        LikF64Args a = f64_args(pv);
        a.X = w.X;
        a.rows = rows;
        a.n_rows_dev = n_rows_dev;
        a.n_rows = n_rows;
        a.qpart = r.qpart;
        a.Z = r.Z;
        a.R = r.R;
        a.ell = w.ellg;
        a.G = w.G;
        a.out_by_walker = 1;
        launch_lik_f64_points(a, true, s);
    };
    for (int osc = 0; osc < cc->n_osc; ++osc) {
        // convergence phase: every sample released, L-BFGS from where it is
        if (mixed)
            st = run_refine<float>(pv, &c2, P.L.r32, w.X, n, w.X, w.ell, w.status, nullptr, nullptr, s);
        else
            st = run_refine<double>(pv, &c2, r, w.X, n, w.X, w.ell, w.status, nullptr, nullptr, s);
        if (st != SB_OK) return st;
        launch_cs_stat_add(w.stats + 1, mixed ? P.L.r32.n_evals : r.n_evals, 0, s);
        // stick test, then the dedup of the stuck samples (representatives stay stuck); the
        // mixed path's gradients are too coarse for the FP64 gradient test, so there the
        // refinement's CONVERGED / STALLED state is the test
        if (mixed) {
            launch_cs_conv_status(n, w.status, w.ell, w.conv, s);
        } else {
            grad_at(nullptr, nullptr, n);
            launch_cs_conv(n, d, w.G, w.ell, c->eps_grad, w.conv, s);
        }
        launch_cs_stick(n, w.ell, w.conv, w.stuck, s);
        launch_dedup(n, d, w.X, w.ell, nullptr, w.stuck, c->dedup_coarse, pv.wmax, n, w.reps, w.n_reps, la.assigned,
                     dds, s);
        launch_cs_split(n, w.reps, w.n_reps, w.stuck, w.lost, s);
        launch_cs_osc_state(w.n_reps, w.state, s);
        if (osc == cc->n_osc - 1) break;
        // reseeding of the lost samples: the branch and its job tables on the device
        launch_cs_lists(n, w.lost, w.conv, w.stuck, w.status, w.ell, w.lost_list, w.unconv_list, w.moving_list, w.cnt,
                        s);
        launch_cs_branch(w.cnt, w.n_reps, cc->min_unconverged, d, c->n_steps, w.state, w.job_start, w.job_pk, w.job_b,
                         w.job_cols, w.job_off, w.stats, s);
        launch_cs_rm_rays(n, d, c->seed, osc, w.unconv_list, w.cnt, w.state, w.X, pv.lo, pv.hi, w.O, w.U, w.texit,
                          s);
        launch_cs_bases(n, d, c->seed, osc, w.job_pk, w.job_b, w.job_cols, w.job_off, w.state, w.Q, mixed, s);
        launch_cs_gr_rays(n, d, w.n_reps, w.reps, w.X, pv.lo, pv.hi, w.job_start, w.job_off, w.Q, w.cnt, w.state, w.O,
                          w.U, w.texit, s);
        if (mixed) {
            // every ray in one quadratic-form pass: two split GEMMs over the rays (origins,
            // directions), then l at each sample from three scalars per (ray, component)
            launch_cs_chunk_rows(w.cnt, w.state, 0, n, c->n_steps, w.rows, s);
            launch_cs_chunk_rows(w.cnt, w.state, 0, n, 1, w.rows + 1, s);
            st = tc_ray_origins_quad(pv, n, c->n_steps, c->prec, P.L.r32.tc.bn, w.quad, w.orig, w.O, w.U, w.texit,
                                     w.rows + 1, w.rows, w.ellp, s);
            if (st != SB_OK) return st;
            launch_cs_ray_pick(0, n, c->n_steps, d, w.rows, w.state, w.ellp, w.lost_list, w.O, w.U, w.texit, w.X, s);
        }
        for (int l0 = 0; !mixed && l0 < n; l0 += w.lc) {
            const int lc = n - l0 < w.lc ? n - l0 : w.lc;
            launch_cs_chunk_rows(w.cnt, w.state, l0, lc, c->n_steps, w.rows, s);
            {
                launch_cs_ray_points(l0, lc, c->n_steps, d, w.O, w.U, w.texit, w.rows, w.P, s);
                LikF64Args a = f64_args(pv);
                a.X = w.P;
                a.n_rows = lc * c->n_steps;
                a.n_rows_dev = w.rows;
                a.qpart = w.qp;
                a.ell = w.ellp;
                a.out_by_walker = 0;
                launch_lik_f64_points(a, false, s);
            }
            launch_cs_ray_pick(l0, lc, c->n_steps, d, w.rows, w.state, w.ellp, w.lost_list, w.O, w.U, w.texit, w.X,
                               s);
        }
        // anti-convergence of every sample that is not stuck (the moving list)
        if (cc->anti_steps > 0) {
            launch_cs_stat_add32(w.stats + 2, w.cnt + 2, cc->anti_steps, s);
            if (mixed) {
                // in FP32 on the walker evaluation of the refinement: the moving samples
                // only, with the component skip (every component at the first step, then
                // the bounds moved by the distance of each momentum step)
                const TcWs &t = P.L.r32.tc;
                float *X32 = w.O32, *V32 = w.U32;  // free once the reseeding rays are evaluated
                tc_to_f32(w.X, X32, (size_t)n * d, s);
                SB_CUDA_TRY(cudaMemsetAsync(V32, 0, sizeof(float) * n * d, s));
                tc_walkers_reset(t, n, s);
                for (int step = 0; step < cc->anti_steps; ++step) {
                    tc_eval_walkers(pv, c, t, X32, w.moving_list, w.cnt + 2, n, P.L.r32.lb.FT, P.L.r32.lb.GT, s);
                    launch_cs_momentum_f32(n, d, w.moving_list, w.cnt + 2, cc->momentum, cc->anti_alpha,
                                           P.L.r32.lb.GT, V32, X32, pv.lo, pv.hi,
                                           static_cast<float *>(t.p[kTcDistSlot]), s);
                }
                launch_cs_scatter_moving(n, d, w.moving_list, w.cnt + 2, X32, w.X, s);
            } else {
                SB_CUDA_TRY(cudaMemsetAsync(w.V, 0, sizeof(double) * n * d, s));
                for (int step = 0; step < cc->anti_steps; ++step) {
                    grad_at(w.moving_list, w.cnt + 2, n);
                    launch_cs_momentum(n, d, w.moving_list, w.cnt + 2, cc->momentum, cc->anti_alpha, w.G, w.V, w.X,
                                       pv.lo, pv.hi, s);
                }
            }
        }
        SB_CUDA_TRY(cudaGetLastError());
    }
    SB_CUDA_TRY(cudaMemcpyAsync(x_out, w.X, sizeof(double) * n * d, cudaMemcpyDeviceToDevice, s));
    SB_CUDA_TRY(cudaMemcpyAsync(ell_out, w.ell, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    SB_CUDA_TRY(cudaMemcpyAsync(stuck_out, w.stuck, n, cudaMemcpyDeviceToDevice, s));
    SB_CUDA_TRY(cudaMemcpyAsync(n_peaks, w.n_reps, sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    SB_CUDA_TRY(cudaGetLastError());
    return SB_OK;
}

}  // namespace

extern "C" sb_status sb_chisao(const sb_problem *p, const sb_config *c, const sb_chisao_config *cc, const double *x0,
                               int32_t n, double *x_out, double *ell_out, int8_t *stuck_out, int32_t *n_peaks,
                               void *ws, size_t ws_bytes, void *stream) {
    if (!x0 || !x_out || !ell_out || !stuck_out || !n_peaks) return SB_ERR_INVALID_ARG;
    if (!c || n < 1 || n > c->n_starts) return SB_ERR_INVALID_ARG;
    sb_status st = check_chisao(cc);
    if (st != SB_OK) return st;
    // the mixed path evaluates ray samples in chunks of at most n_starts rows
    if (c->prec != SB_PREC_FP64 && c->n_starts < c->n_steps) return SB_ERR_UNSUPPORTED;
    st = check_call(p, c, ws, ws_bytes, true);
    if (st != SB_OK) return st;
    cudaStream_t s0 = static_cast<cudaStream_t>(stream);
    GraphKey key = call_key(1, p, c, ws, ws_bytes);
    key.add_bytes(*cc);
    for (const void *q : {(const void *)x0, (const void *)x_out, (const void *)ell_out, (const void *)stuck_out,
                          (const void *)n_peaks})
        key.add_ptr(q);
    key.add((uint64_t)n);
    pretune(p, c, ws, ws_bytes, s0);
    return run_graph_or_direct(s0, key, [&](cudaStream_t s) {
        Prelude P;
        sb_status r = prelude(p, c, ws, ws_bytes, s, P);
        if (r != SB_OK) return r;
        const ChisaoWs w = chisao_layout(ws, P.L.bytes, p, c);
        return run_chisao(P, c, cc, w, x0, n, x_out, ell_out, stuck_out, n_peaks, s);
    });
}

namespace {
// discover + ChiSao + Laplace over every final sample, on one prelude, no host read.
sb_status enqueue_evidence_chisao(const sb_problem *p, const sb_config *c, const sb_chisao_config *cc, double *logZ,
                                  double *modes, double *logZk, int32_t cap, int32_t *n_modes, void *ws,
                                  size_t ws_bytes, cudaStream_t s) {
    Prelude P;
    sb_status r = prelude(p, c, ws, ws_bytes, s, P);
    if (r != SB_OK) return r;
    const auto &ev = P.L.ev;
    const int n = c->n_starts;
    r = run_discover(P.pv, c, P.L, ev.starts, ev.ell_starts, s);
    if (r != SB_OK) return r;
    const ChisaoWs w = chisao_layout(ws, P.L.bytes, p, c);
    r = run_chisao(P, c, cc, w, ev.starts, n, ev.x_out, ev.ell_out, ev.status, n_modes, s);
    if (r != SB_OK) return r;
    launch_cs_stat_add(w.stats + 0, nullptr, (int64_t)c->n_rays * c->n_steps, s);
    return run_laplace(P.pv, c, P.L, ev.x_out, ev.ell_out, nullptr, n, modes, logZk, nullptr, cap, n_modes, logZ, s);
}
}  // namespace

extern "C" sb_status sb_evidence_chisao(const sb_problem *p, const sb_config *c, const sb_chisao_config *cc,
                                        double *logZ, double *modes, double *logZk, int32_t cap, int32_t *n_modes,
                                        void *ws, size_t ws_bytes, void *stream) {
    if (!logZ || !modes || !logZk || !n_modes || cap < 1) return SB_ERR_INVALID_ARG;
    sb_status st = check_chisao(cc);
    if (st != SB_OK) return st;
    if (c && c->prec != SB_PREC_FP64 && c->n_starts < c->n_steps) return SB_ERR_UNSUPPORTED;
    st = check_call(p, c, ws, ws_bytes, true);
    if (st != SB_OK) return st;
    cudaStream_t s0 = static_cast<cudaStream_t>(stream);
    GraphKey key = call_key(2, p, c, ws, ws_bytes);
    key.add_bytes(*cc);
    for (const void *q : {(const void *)logZ, (const void *)modes, (const void *)logZk, (const void *)n_modes})
        key.add_ptr(q);
    key.add((uint64_t)cap);
    pretune(p, c, ws, ws_bytes, s0);
    // discovery into the evidence buffers, ChiSao from its starts (its peak count goes to
    // n_modes for now), then the Laplace stage over every final sample; one prelude, so
    // the device status word collects what every stage records
    return run_graph_or_direct(s0, key, [&](cudaStream_t s) {
        return enqueue_evidence_chisao(p, c, cc, logZ, modes, logZk, cap, n_modes, ws, ws_bytes, s);
    });
}

extern "C" size_t sb_evidence_chisao_host_workspace_bytes(const sb_problem *hp, const sb_config *c) {
    const size_t inner = sb_chisao_workspace_bytes(hp, c);
    if (inner == 0) return 0;
    return host_layout(nullptr, hp, c->cand_cap, inner).bytes;
}

extern "C" sb_status sb_evidence_chisao_host(const sb_problem *hp, const sb_config *c, const sb_chisao_config *cc,
                                             double *logZ, double *modes, double *logZk, int32_t cap,
                                             int32_t *n_modes, void *ws, size_t ws_bytes, void *stream) {
    sb_status st = check_problem(hp);
    if (st != SB_OK) return st;
    st = check_config(c);
    if (st != SB_OK) return st;
    st = check_chisao(cc);
    if (st != SB_OK) return st;
    return host_solve(hp, c, sb_chisao_workspace_bytes(hp, c), logZ, modes, logZk, cap, n_modes, ws, ws_bytes, stream,
                      [c, cc](const sb_problem *dp, double *lz, double *md, double *zk, int32_t cp, int32_t *nm,
                              void *in, size_t inb, void *str) {
                          return sb_evidence_chisao(dp, c, cc, lz, md, zk, cp, nm, in, inb, str);
                      });
}

extern "C" sb_status sb_chisao_stats(const sb_problem *p, const sb_config *c, void *ws, size_t ws_bytes, int64_t *out,
                                     void *stream) {
    sb_status st = check_problem(p);
    if (st != SB_OK) return st;
    st = check_config(c);
    if (st != SB_OK) return st;
    if (!ws || !out) return SB_ERR_INVALID_ARG;
    const Layout L = layout(ws, p, c);
    const ChisaoWs w = chisao_layout(ws, L.bytes, p, c);
    if (ws_bytes < L.bytes + w.bytes) return SB_ERR_WORKSPACE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int32_t nm = 0;
    SB_CUDA_TRY(cudaMemcpyAsync(out, w.stats, sizeof(int64_t) * 3, cudaMemcpyDeviceToHost, s));
    SB_CUDA_TRY(cudaMemcpyAsync(&nm, L.la.n_reps2, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    SB_CUDA_TRY(cudaStreamSynchronize(s));
    out[3] = nm;
    return SB_OK;
}

// ------------------------------------------------------------------ batched problems
// Independent problems of uneven d and K run on `n_workers` worker streams,
// each with its own host thread (the refine stage polls its stream) and its own
// slice of the workspace; problem i goes to worker i % n_workers.
namespace {
size_t batched_slice_bytes(const sb_problem *probs, int32_t P, const sb_config *c, bool chisao) {
    size_t mx = 0;
    for (int32_t i = 0; i < P; ++i) {
        size_t b = layout(nullptr, &probs[i], c).bytes;
        if (chisao) b += chisao_layout(nullptr, b, &probs[i], c).bytes;
        if (b > mx) mx = b;
    }
    // per-problem modes buffer [cand_cap][d_max] and logZk [cand_cap]
    int dmax = 1;
    for (int32_t i = 0; i < P; ++i) dmax = probs[i].d > dmax ? probs[i].d : dmax;
    const size_t extra = ((size_t)c->cand_cap * dmax * sizeof(double) + 255) / 256 * 256 +
                         ((size_t)c->cand_cap * sizeof(double) + 255) / 256 * 256;
    return (mx + extra + 255) / 256 * 256;
}
}  // namespace

extern "C" size_t sb_evidence_batched_workspace_bytes(const sb_problem *probs, int32_t P, const sb_config *c,
                                                      int32_t n_workers) {
    if (!probs || P < 1 || n_workers < 1 || check_config(c) != SB_OK) return 0;
    for (int32_t i = 0; i < P; ++i)
        if (check_problem(&probs[i]) != SB_OK) return 0;
    const int32_t w = n_workers < P ? n_workers : P;
    return (size_t)w * batched_slice_bytes(probs, P, c, false);
}

extern "C" size_t sb_evidence_chisao_batched_workspace_bytes(const sb_problem *probs, int32_t P, const sb_config *c,
                                                             int32_t n_workers) {
    if (!probs || P < 1 || n_workers < 1 || check_config(c) != SB_OK) return 0;
    for (int32_t i = 0; i < P; ++i)
        if (check_problem(&probs[i]) != SB_OK) return 0;
    const int32_t w = n_workers < P ? n_workers : P;
    return (size_t)w * batched_slice_bytes(probs, P, c, true);
}

namespace {
// Worker streams and fork / join events of this host thread (created once per device).
struct Workers {
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> joins;
    cudaEvent_t fork = nullptr;
};
Workers *workers_for(int W) {
    thread_local std::map<int, Workers> pools;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    Workers &wk = pools[dev];
    if (!wk.fork && cudaEventCreateWithFlags(&wk.fork, cudaEventDisableTiming) != cudaSuccess) return nullptr;
    while ((int)wk.streams.size() < W) {
        cudaStream_t st = nullptr;
        cudaEvent_t ev = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return nullptr;
        wk.streams.push_back(st);
        wk.joins.push_back(ev);
    }
    return &wk;
}
}  // namespace

namespace {
// The batch of P problems (with ChiSao when cc is given) on W worker streams forked from
// and joined into the caller's stream; one cached graph in graph mode.
sb_status batched(const sb_problem *probs, int32_t P, const sb_config *c, const sb_chisao_config *cc, double *logZ,
                  int32_t *n_modes, int32_t n_workers, void *ws, size_t ws_bytes, void *stream) {
    if (!probs || P < 1 || n_workers < 1 || !logZ || !n_modes || !ws) return SB_ERR_INVALID_ARG;
    sb_status st = check_config(c);
    if (st != SB_OK) return st;
    if (cc) {
        st = check_chisao(cc);
        if (st != SB_OK) return st;
        if (c->prec != SB_PREC_FP64 && c->n_starts < c->n_steps) return SB_ERR_UNSUPPORTED;
    }
    for (int32_t i = 0; i < P; ++i) {
        st = check_problem(&probs[i]);
        if (st != SB_OK) return st;
    }
    if (c->prec != SB_PREC_FP64 && !tc_available(c->prec)) return SB_ERR_UNSUPPORTED;
    const int32_t W = n_workers < P ? n_workers : P;
    const size_t slice = batched_slice_bytes(probs, P, c, cc != nullptr);
    if (ws_bytes < (size_t)W * slice) return SB_ERR_WORKSPACE;
    int dmax = 1;
    for (int32_t i = 0; i < P; ++i) dmax = probs[i].d > dmax ? probs[i].d : dmax;
    cudaStream_t s0 = static_cast<cudaStream_t>(stream);
    Workers *wk = workers_for(W);
    if (!wk) return SB_ERR_CUDA;
    // the tile autotuner times each new shape once, outside the capture, on the slice of
    // the worker that will solve it
    for (int32_t i = 0; i < P; ++i) pretune(&probs[i], c, static_cast<char *>(ws) + (size_t)(i % W) * slice, slice, s0);
    GraphKey key;
    key.add(cc ? 6 : 5);
    key.add((uint64_t)P);
    key.add((uint64_t)W);
    for (int32_t i = 0; i < P; ++i) key.add_bytes(probs[i]);
    key.add_bytes(*c);
    if (cc) key.add_bytes(*cc);
    for (const void *q : {(const void *)logZ, (const void *)n_modes, (const void *)ws}) key.add_ptr(q);
    key.add((uint64_t)ws_bytes);
    // problem i on worker i % W, in order (the worker's problems share its workspace
    // slice); the workers fork from the caller's stream and join back into it
    return run_graph_or_direct(s0, key, [&](cudaStream_t s) {
        SB_CUDA_TRY(cudaEventRecord(wk->fork, s));
        for (int32_t w = 0; w < W; ++w) SB_CUDA_TRY(cudaStreamWaitEvent(wk->streams[w], wk->fork, 0));
        for (int32_t i = 0; i < P; ++i) {
            const int32_t w = i % W;
            char *base = static_cast<char *>(ws) + (size_t)w * slice;
            Carver cv(base);
            double *modes = cv.take<double>((size_t)c->cand_cap * dmax);
            double *zk = cv.take<double>((size_t)c->cand_cap);
            void *inner = base + cv.bytes();
            const size_t inner_bytes = slice - cv.bytes();
            const sb_status r =
                cc ? enqueue_evidence_chisao(&probs[i], c, cc, logZ + i, modes, zk, c->cand_cap, n_modes + i, inner,
                                             inner_bytes, wk->streams[w])
                   : enqueue_evidence(&probs[i], c, logZ + i, modes, zk, c->cand_cap, n_modes + i, inner, inner_bytes,
                                      wk->streams[w]);
            if (r != SB_OK) return r;
        }
        for (int32_t w = 0; w < W; ++w) {
            SB_CUDA_TRY(cudaEventRecord(wk->joins[w], wk->streams[w]));
            SB_CUDA_TRY(cudaStreamWaitEvent(s, wk->joins[w], 0));
        }
        return SB_OK;
    });
}
}  // namespace

extern "C" sb_status sb_evidence_batched(const sb_problem *probs, int32_t P, const sb_config *c, double *logZ,
                                         int32_t *n_modes, int32_t n_workers, void *ws, size_t ws_bytes,
                                         void *stream) {
    return batched(probs, P, c, nullptr, logZ, n_modes, n_workers, ws, ws_bytes, stream);
}

extern "C" sb_status sb_evidence_chisao_batched(const sb_problem *probs, int32_t P, const sb_config *c,
                                                const sb_chisao_config *cc, double *logZ, int32_t *n_modes,
                                                int32_t n_workers, void *ws, size_t ws_bytes, void *stream) {
    if (!cc) return SB_ERR_INVALID_ARG;
    return batched(probs, P, c, cc, logZ, n_modes, n_workers, ws, ws_bytes, stream);
}

// ------------------------------------------------------------------ setup-only entry points
namespace {

// Carves the per-problem constants (a_k, centre, half-widths, log V) at the start of a
// workspace; used by the entry points that need no solve-stage layout.
void carve_setup(Carver &cv, const sb_problem *p, SetupWs &su) {
    su.hdr = cv.take<WsHeader>(1);
    su.a = cv.take<double>(p->K);
    su.c = cv.take<double>(p->d);
    su.half = cv.take<double>(p->d);
    su.logV = cv.take<double>(1);
    su.wmax = cv.take<double>(1);
}

// The problem view over those constants, computed on `cs` (status word cleared first).
cudaError_t setup_only(const sb_problem *p, const SetupWs &su, cudaStream_t cs, ProbView &pv) {
    pv.d = p->d;
    pv.K = p->K;
    pv.log_w = p->log_w;
    pv.mu = p->mu;
    pv.L = p->L;
    pv.lo = p->lo;
    pv.hi = p->hi;
    pv.a = su.a;
    pv.c = su.c;
    pv.half = su.half;
    pv.logV = su.logV;
    pv.wmax = su.wmax;
    pv.status = &su.hdr->status;
    const cudaError_t e = cudaMemsetAsync(su.hdr, 0, sizeof(WsHeader), cs);
    if (e != cudaSuccess) return e;
    launch_setup(pv, cs);
    return cudaGetLastError();
}

}  // namespace

// ------------------------------------------------------------------ preprocessing (Sec. 3.4)
namespace {

struct PrecheckWs {
    SetupWs su;
    double *scratch;
    size_t bytes;
};

PrecheckWs precheck_layout(void *base, const sb_problem *p) {
    PrecheckWs w{};
    Carver cv(base);
    carve_setup(cv, p, w.su);
    w.scratch = cv.take<double>(precheck_scratch_elems(p->d, p->K));
    w.bytes = cv.bytes();
    return w;
}

}  // namespace

extern "C" size_t sb_precheck_workspace_bytes(const sb_problem *p) {
    if (check_problem(p) != SB_OK) return 0;
    return precheck_layout(nullptr, p).bytes;
}

extern "C" sb_status sb_precheck(const sb_problem *p, double eps_flat, double eps_soft, double *s, int8_t *cls,
                                 double *log_int, double *log_vol, int32_t *n_active, void *ws, size_t ws_bytes,
                                 void *stream) {
    sb_status st = check_problem(p);
    if (st != SB_OK) return st;
    if (!s || !cls || !log_int || !log_vol || !n_active || !ws) return SB_ERR_INVALID_ARG;
    if (!(eps_flat >= 0.0) || !(eps_soft >= 0.0) || !std::isfinite(eps_flat) || !std::isfinite(eps_soft))
        return SB_ERR_INVALID_ARG;
    const PrecheckWs w = precheck_layout(ws, p);
    if (ws_bytes < w.bytes) return SB_ERR_WORKSPACE;
    const cudaStream_t cs = static_cast<cudaStream_t>(stream);
    ProbView pv;
    SB_CUDA_TRY(setup_only(p, w.su, cs, pv));
    launch_precheck(pv, eps_flat, eps_soft, w.scratch, s, cls, log_int, log_vol, n_active, cs);
    SB_CUDA_TRY(cudaGetLastError());
    return SB_OK;
}

// ------------------------------------------------------------------ other ray families (Sec. 3.5.1-3.5.2)
namespace {

struct SegmentsWs {
    SetupWs su;
    double *scratch;
    size_t bytes;
};

SegmentsWs segments_layout(void *base, const sb_problem *p, int n_rays, int n_steps) {
    SegmentsWs w{};
    Carver cv(base);
    carve_setup(cv, p, w.su);
    w.scratch = cv.take<double>(segments_scratch_elems(n_rays, n_steps, p->d, p->K));
    w.bytes = cv.bytes();
    return w;
}

bool segments_sizes_ok(int n_rays, int n_steps) {
    return n_rays >= 1 && n_steps >= 1 && n_rays <= (1 << 24) && (int64_t)n_rays * (n_steps + 1) <= 0x7fffffffLL;
}

}  // namespace

extern "C" size_t sb_segments_workspace_bytes(const sb_problem *p, int32_t n_rays, int32_t n_steps) {
    if (check_problem(p) != SB_OK || !segments_sizes_ok(n_rays, n_steps)) return 0;
    return segments_layout(nullptr, p, n_rays, n_steps).bytes;
}

extern "C" sb_status sb_segments(const sb_problem *p, int32_t family, uint64_t seed, int32_t n_rays, int32_t n_steps,
                                 double delta, int32_t n_ref, double *ends, double *ell_coarse, double *t_ref,
                                 double *ell_ref, void *ws, size_t ws_bytes, void *stream) {
    sb_status st = check_problem(p);
    if (st != SB_OK) return st;
    if (family != SB_RAY_V2V && family != SB_RAY_V2E && family != SB_RAY_W2W) return SB_ERR_INVALID_ARG;
    if (!segments_sizes_ok(n_rays, n_steps) || n_ref < 0 || (int64_t)n_rays * n_ref > 0x7fffffffLL)
        return SB_ERR_INVALID_ARG;
    if (!(delta >= 0.0)) return SB_ERR_INVALID_ARG;  // +inf allowed, NaN refused
    if (!ends || !ell_coarse || !ws || (n_ref > 0 && (!t_ref || !ell_ref))) return SB_ERR_INVALID_ARG;
    const SegmentsWs w = segments_layout(ws, p, n_rays, n_steps);
    if (ws_bytes < w.bytes) return SB_ERR_WORKSPACE;
    const cudaStream_t cs = static_cast<cudaStream_t>(stream);
    ProbView pv;
    SB_CUDA_TRY(setup_only(p, w.su, cs, pv));
    launch_segments(pv, family, seed, n_rays, n_steps, delta, n_ref, w.scratch, ends, ell_coarse, t_ref, ell_ref, cs);
    SB_CUDA_TRY(cudaGetLastError());
    return SB_OK;
}

// ------------------------------------------------------------------ black-box derivatives (App. A.4)
namespace {

struct FdWs {
    SetupWs su;
    double *scratch;
    size_t bytes;
};

FdWs fd_layout(void *base, const sb_problem *p, bool full) {
    FdWs w{};
    Carver cv(base);
    carve_setup(cv, p, w.su);
    w.scratch = cv.take<double>(fd_scratch_elems(p->d, p->K, full));
    w.bytes = cv.bytes();
    return w;
}

}  // namespace

extern "C" size_t sb_fd_workspace_bytes(const sb_problem *p, int32_t full) {
    if (check_problem(p) != SB_OK) return 0;
    return fd_layout(nullptr, p, full != 0).bytes;
}

extern "C" sb_status sb_fd_derivatives(const sb_problem *p, const double *x, double eps_g, double eps_h, int32_t full,
                                       double *grad, double *hdiag, double *H, double *b, void *ws, size_t ws_bytes,
                                       void *stream) {
    sb_status st = check_problem(p);
    if (st != SB_OK) return st;
    if (!x || !hdiag || !ws || (full && !H)) return SB_ERR_INVALID_ARG;
    if (!(eps_g > 0.0) || !(eps_h > 0.0) || !std::isfinite(eps_g) || !std::isfinite(eps_h)) return SB_ERR_INVALID_ARG;
    const FdWs w = fd_layout(ws, p, full != 0);
    if (ws_bytes < w.bytes) return SB_ERR_WORKSPACE;
    const cudaStream_t cs = static_cast<cudaStream_t>(stream);
    ProbView pv;
    SB_CUDA_TRY(setup_only(p, w.su, cs, pv));
    launch_fd(pv, x, eps_g, eps_h, full != 0, w.scratch, grad, hdiag, H, b, cs);
    SB_CUDA_TRY(cudaGetLastError());
    return SB_OK;
}

// ------------------------------------------------------------------ ray likelihoods by the quadratic in t
namespace {

struct RayqWs {
    SetupWs su;
    double *scratch;  // forms 0, 1: the FP64 / FP32 forms' scratch; forms 2, 3: t_exit
    TcQuadWs quad;    // forms 2, 3 (tensor-core GEMM of the split directions)
    size_t bytes;
};

RayqWs rayq_layout(void *base, const sb_problem *p, int n_rays, int form) {
    RayqWs w{};
    Carver cv(base);
    carve_setup(cv, p, w.su);
    if (form <= 1)
        w.scratch = cv.take<double>(rayq_scratch_elems(n_rays, p->d, p->K, form));
    else {
        w.scratch = cv.take<double>(n_rays);
        carve_tc_quad(cv, w.quad, n_rays, p->d, p->K, form == 2 ? SB_PREC_BF16 : SB_PREC_TF32);
    }
    w.bytes = cv.bytes();
    return w;
}

struct RayoWs {
    SetupWs su;
    double *texit;
    TcQuadWs quad;
    TcOriginWs orig;
    size_t bytes;
};

RayoWs rayo_layout(void *base, const sb_problem *p, int n_rays, int form) {
    RayoWs w{};
    Carver cv(base);
    carve_setup(cv, p, w.su);
    const int prec = form == 2 ? SB_PREC_BF16 : SB_PREC_TF32;
    w.texit = cv.take<double>(n_rays);
    carve_tc_quad(cv, w.quad, n_rays, p->d, p->K, prec);
    carve_tc_origins(cv, w.orig, n_rays, p->d, p->K, prec);
    w.bytes = cv.bytes();
    return w;
}

}  // namespace

extern "C" size_t sb_ray_loglik_origins_workspace_bytes(const sb_problem *p, int32_t form, int32_t n_rays) {
    if (check_problem(p) != SB_OK || (form != 2 && form != 3) || n_rays < 1 || n_rays > (1 << 24)) return 0;
    return rayo_layout(nullptr, p, n_rays, form).bytes;
}

extern "C" sb_status sb_ray_loglik_origins(const sb_problem *p, int32_t form, const double *o, const double *u,
                                           int32_t n_rays, int32_t n_steps, double *ell, double *texit, void *ws,
                                           size_t ws_bytes, void *stream) {
    sb_status st = check_problem(p);
    if (st != SB_OK) return st;
    if ((form != 2 && form != 3) || !o || !u || !ell || !ws) return SB_ERR_INVALID_ARG;
    if (n_rays < 1 || n_rays > (1 << 24) || n_steps < 1 || (int64_t)n_rays * n_steps > 0x7fffffffLL)
        return SB_ERR_INVALID_ARG;
    const RayoWs w = rayo_layout(ws, p, n_rays, form);
    if (ws_bytes < w.bytes) return SB_ERR_WORKSPACE;
    const int prec = form == 2 ? SB_PREC_BF16 : SB_PREC_TF32;
    if (!tc_available(prec)) return SB_ERR_UNSUPPORTED;
    const cudaStream_t cs = static_cast<cudaStream_t>(stream);
    ProbView pv;
    SB_CUDA_TRY(setup_only(p, w.su, cs, pv));
    launch_cs_exit(n_rays, p->d, o, u, pv.lo, pv.hi, w.texit, cs);
    st = tc_quad_prepare_origins(pv, prec, w.quad, w.orig, cs);
    if (st != SB_OK) return st;
    st = tc_ray_origins_quad(pv, n_rays, n_steps, prec, 0, w.quad, w.orig, o, u, w.texit, nullptr, nullptr, ell, cs);
    if (st != SB_OK) return st;
    if (texit) SB_CUDA_TRY(cudaMemcpyAsync(texit, w.texit, sizeof(double) * n_rays, cudaMemcpyDeviceToDevice, cs));
    SB_CUDA_TRY(cudaGetLastError());
    return SB_OK;
}

extern "C" size_t sb_ray_loglik_quad_workspace_bytes(const sb_problem *p, int32_t form, int32_t n_rays) {
    if (check_problem(p) != SB_OK || form < 0 || form > 3 || n_rays < 1 || n_rays > (1 << 24)) return 0;
    return rayq_layout(nullptr, p, n_rays, form).bytes;
}

extern "C" sb_status sb_ray_loglik_quad(const sb_problem *p, int32_t form, const double *u, int32_t n_rays,
                                        int32_t n_steps, double *ell, void *ws, size_t ws_bytes, void *stream) {
    sb_status st = check_problem(p);
    if (st != SB_OK) return st;
    if (form < 0 || form > 3 || !u || !ell || !ws) return SB_ERR_INVALID_ARG;
    if (n_rays < 1 || n_rays > (1 << 24) || n_steps < 1 || (int64_t)n_rays * n_steps > 0x7fffffffLL)
        return SB_ERR_INVALID_ARG;
    const RayqWs w = rayq_layout(ws, p, n_rays, form);
    if (ws_bytes < w.bytes) return SB_ERR_WORKSPACE;
    const cudaStream_t cs = static_cast<cudaStream_t>(stream);
    ProbView pv;
    SB_CUDA_TRY(setup_only(p, w.su, cs, pv));
    if (form <= 1)
        launch_ray_loglik_quad(pv, form, u, n_rays, n_steps, w.scratch, ell, cs);
    else {
        const int prec = form == 2 ? SB_PREC_BF16 : SB_PREC_TF32;
        if (!tc_available(prec)) return SB_ERR_UNSUPPORTED;
        launch_ray_texit(pv, u, n_rays, w.scratch, cs);
        st = tc_ray_loglik_quad(pv, n_rays, n_steps, prec, 0, w.quad, u, w.scratch, ell, cs);
        if (st != SB_OK) return st;
    }
    SB_CUDA_TRY(cudaGetLastError());
    return SB_OK;
}
