// sb_graph.cuh -- device-decided control flow for the solve stages (CUDA graphs).
//
// The refinement runs until no walker is active; the number of rounds is known
// only on the device. In graph mode that loop is a WHILE conditional node whose
// body (a batch of rounds) ends with a kernel setting the condition, so no
// host read is needed and a caller can capture any entry point into its own
// graph. A call made outside a capture is captured by the library on a stream
// of its own, instantiated once per distinct argument set, and replayed on the
// caller's stream. Eager mode (host reads of the active count every batch of
// rounds, no graph) serves the per-launch profiling, whose CUDA events cannot
// sit in a graph, and SB_EAGER=1.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "sb_internal.cuh"

namespace sb {

// True when work enqueued on s is being captured into a graph.
bool stream_capturing(cudaStream_t s);

// Whether a call on stream s (not capturing) runs as a graph (true) or eagerly.
bool graph_mode_for(cudaStream_t s);

// A stream of this host thread on which conditional bodies are captured.
cudaStream_t body_stream();

// Adds a WHILE node to the capture in progress on s (its condition is 1 at every
// launch of the graph) whose body is what body(cs, h) enqueues on the stream cs; the
// work captured on s afterwards depends on the node. The body must set the
// condition through h from a kernel (cudaGraphSetConditional).
template <typename F>
sb_status capture_while(cudaStream_t s, F body) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    const cudaGraphEdgeData *edata = nullptr;
    size_t nd = 0;
    if (cudaStreamGetCaptureInfo(s, &st, nullptr, &g, &deps, &edata, &nd) != cudaSuccess ||
        st != cudaStreamCaptureStatusActive)
        return SB_ERR_CUDA;
    std::vector<cudaGraphNode_t> dv(deps, deps + nd);
    std::vector<cudaGraphEdgeData> ev;
    if (edata) ev.assign(edata, edata + nd);
    cudaGraphConditionalHandle h;
    if (cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault) != cudaSuccess) return SB_ERR_CUDA;
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeWhile;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    if (cudaGraphAddNode(&node, g, dv.data(), edata ? ev.data() : nullptr, nd, &p) != cudaSuccess) return SB_ERR_CUDA;
    cudaGraph_t bg = p.conditional.phGraph_out[0];
    cudaStream_t cs = body_stream();
    if (!cs || cudaStreamBeginCaptureToGraph(cs, bg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) != cudaSuccess)
        return SB_ERR_CUDA;
    const sb_status bst = body(cs, h);
    cudaGraph_t out = nullptr;
    const cudaError_t e = cudaStreamEndCapture(cs, &out);
    if (bst != SB_OK) return bst;
    if (e != cudaSuccess) return SB_ERR_CUDA;
    if (cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies) != cudaSuccess)
        return SB_ERR_CUDA;
    return SB_OK;
}

// Adds to the capture in progress on s an IF node whose body is what body(cs) enqueues
// on the stream cs. set_cond(s, h) enqueues, before the node, a kernel that sets the
// condition through h (it is 0 at every launch of the graph until then).
template <typename C, typename F>
sb_status capture_if(cudaStream_t s, C set_cond, F body) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    cudaGraph_t g = nullptr;
    if (cudaStreamGetCaptureInfo(s, &st, nullptr, &g) != cudaSuccess || st != cudaStreamCaptureStatusActive)
        return SB_ERR_CUDA;
    cudaGraphConditionalHandle h;
    if (cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault) != cudaSuccess) return SB_ERR_CUDA;
    set_cond(s, h);
    const cudaGraphNode_t *deps = nullptr;
    const cudaGraphEdgeData *edata = nullptr;
    size_t nd = 0;
    if (cudaStreamGetCaptureInfo(s, &st, nullptr, &g, &deps, &edata, &nd) != cudaSuccess ||
        st != cudaStreamCaptureStatusActive)
        return SB_ERR_CUDA;
    std::vector<cudaGraphNode_t> dv(deps, deps + nd);
    std::vector<cudaGraphEdgeData> ev;
    if (edata) ev.assign(edata, edata + nd);
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = cudaGraphCondTypeIf;
    p.conditional.size = 1;
    cudaGraphNode_t node;
    if (cudaGraphAddNode(&node, g, dv.data(), edata ? ev.data() : nullptr, nd, &p) != cudaSuccess) return SB_ERR_CUDA;
    cudaGraph_t bg = p.conditional.phGraph_out[0];
    cudaStream_t cs = body_stream();
    if (!cs || cudaStreamBeginCaptureToGraph(cs, bg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) != cudaSuccess)
        return SB_ERR_CUDA;
    body(cs);
    cudaGraph_t out = nullptr;
    if (cudaStreamEndCapture(cs, &out) != cudaSuccess) return SB_ERR_CUDA;
    if (cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies) != cudaSuccess)
        return SB_ERR_CUDA;
    return SB_OK;
}

// Cached executable graphs, keyed by every argument that shapes the captured work
// (pointers, sizes, knobs). Runs `enqueue` on a capture stream the first time a key
// is seen, instantiates the graph, and launches the instance on s (each time).
// Entries beyond a small number are evicted after their last launch completes.
struct GraphKey {
    std::vector<uint64_t> v;
    void add(uint64_t x) { v.push_back(x); }
    void add_ptr(const void *p) { v.push_back((uint64_t)(uintptr_t)p); }
    void add_f(double x) {
        uint64_t u;
        static_assert(sizeof(u) == sizeof(x), "64-bit doubles");
        __builtin_memcpy(&u, &x, sizeof(u));
        v.push_back(u);
    }
    template <typename T>
    void add_bytes(const T &t) {
        const unsigned char *b = reinterpret_cast<const unsigned char *>(&t);
        for (size_t i = 0; i < sizeof(T); i += 8) {
            uint64_t u = 0;
            __builtin_memcpy(&u, b + i, sizeof(T) - i < 8 ? sizeof(T) - i : 8);
            v.push_back(u);
        }
    }
};

using EnqueueFn = sb_status (*)(void *ctx, cudaStream_t s);
sb_status launch_cached_graph(const GraphKey &key, EnqueueFn fn, void *ctx, cudaStream_t s);

// Runs enqueue(s) directly when s is capturing or the call is eager, else as a cached
// graph launched on s.
template <typename F>
sb_status run_graph_or_direct(cudaStream_t s, const GraphKey &key, F enqueue) {
    if (stream_capturing(s) || !graph_mode_for(s)) return enqueue(s);
    struct Ctx {
        F *f;
    } ctx{&enqueue};
    return launch_cached_graph(
        key, [](void *c, cudaStream_t cs) { return (*static_cast<Ctx *>(c)->f)(cs); }, &ctx, s);
}

// Sets the WHILE condition of a refinement loop: *round += per_batch, condition =
// (*n_act > 0 && *round < cap_rounds); the cap (a bound no run reaches: every
// accepted step takes at most 2 (max_backtracks + 2) rounds) reached with walkers
// still active records SB_DEV_TIMEOUT.
void launch_loop_cond(cudaGraphConditionalHandle h, int64_t *round, int per_batch, int64_t cap_rounds,
                      const int32_t *n_act, int32_t *err, cudaStream_t s);

}  // namespace sb
