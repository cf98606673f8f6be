// graph.cu -- graph mode of the solve stages: capture streams, the executable
// graph cache and the condition kernel of the device-decided refinement loop.
#include <cstdlib>
#include <map>
#include <mutex>

#include "sb_graph.cuh"

namespace sb {

namespace {

__global__ void k_loop_cond(cudaGraphConditionalHandle h, int64_t *round, int per_batch, int64_t cap,
                            const int32_t *n_act, int32_t *err) {
    if (threadIdx.x != 0) return;
    const int64_t r = *round + per_batch;
    *round = r;
    const bool active = *n_act > 0;
    if (active && r >= cap) atomicOr(err, SB_DEV_TIMEOUT);
    cudaGraphSetConditional(h, (active && r < cap) ? 1u : 0u);
}

// Streams of this host thread, one per device: bodies of conditional nodes, and the
// library's own captures of calls made outside a capture.
cudaStream_t thread_stream(int which) {
    thread_local std::map<int, cudaStream_t> streams[2];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    auto it = streams[which].find(dev);
    if (it != streams[which].end()) return it->second;
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return nullptr;
    streams[which][dev] = s;
    return s;
}

struct Entry {
    cudaGraphExec_t exec;
    cudaEvent_t done;  // recorded after the latest launch
    uint64_t last;
};
std::mutex g_mu;
std::map<std::vector<uint64_t>, Entry> g_cache;
uint64_t g_tick = 0;
constexpr size_t kMaxCached = 32;

}  // namespace

bool stream_capturing(cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
}

bool graph_mode_for(cudaStream_t s) {
    (void)s;
    static const bool eager = [] {
        const char *e = std::getenv("SB_EAGER");
        return e && e[0] == '1';
    }();
    return !eager && !prof_enabled();
}

cudaStream_t body_stream() { return thread_stream(0); }

sb_status launch_cached_graph(const GraphKey &key0, EnqueueFn fn, void *ctx, cudaStream_t s) {
    int dev = 0;
    SB_CUDA_TRY(cudaGetDevice(&dev));
    std::vector<uint64_t> key = key0.v;
    key.push_back((uint64_t)dev);
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_cache.find(key);
        if (it != g_cache.end()) {
            it->second.last = ++g_tick;
            SB_CUDA_TRY(cudaGraphLaunch(it->second.exec, s));
            SB_CUDA_TRY(cudaEventRecord(it->second.done, s));
            return SB_OK;
        }
    }
    cudaStream_t cs = thread_stream(1);
    if (!cs) return SB_ERR_CUDA;
    SB_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
    const sb_status st = fn(ctx, cs);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(cs, &g);
    if (st != SB_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return st != SB_OK ? st : SB_ERR_CUDA;
    }
    Entry en{};
    const cudaError_t ie = cudaGraphInstantiate(&en.exec, g, 0);
    cudaGraphDestroy(g);
    SB_CUDA_TRY(ie);
    if (cudaEventCreateWithFlags(&en.done, cudaEventDisableTiming) != cudaSuccess) {
        cudaGraphExecDestroy(en.exec);
        return SB_ERR_CUDA;
    }
    SB_CUDA_TRY(cudaGraphLaunch(en.exec, s));
    SB_CUDA_TRY(cudaEventRecord(en.done, s));
    std::lock_guard<std::mutex> lk(g_mu);
    en.last = ++g_tick;
    auto ins = g_cache.emplace(key, en);
    if (!ins.second) {  // another thread cached the same key meanwhile: keep one
        cudaEventSynchronize(en.done);
        cudaGraphExecDestroy(en.exec);
        cudaEventDestroy(en.done);
    }
    while (g_cache.size() > kMaxCached) {
        auto lru = g_cache.begin();
        for (auto i = g_cache.begin(); i != g_cache.end(); ++i)
            if (i->second.last < lru->second.last) lru = i;
        cudaEventSynchronize(lru->second.done);  // its last launch has finished
        cudaGraphExecDestroy(lru->second.exec);
        cudaEventDestroy(lru->second.done);
        g_cache.erase(lru);
    }
    return SB_OK;
}

void launch_loop_cond(cudaGraphConditionalHandle h, int64_t *round, int per_batch, int64_t cap_rounds,
                      const int32_t *n_act, int32_t *err, cudaStream_t s) {
    note_launch();
    k_loop_cond<<<1, 32, 0, s>>>(h, round, per_batch, cap_rounds, n_act, err);
}

}  // namespace sb
