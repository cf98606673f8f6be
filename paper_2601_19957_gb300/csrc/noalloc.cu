// noalloc.cu -- sb_loglik for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code running while a CUDA graph is being
// captured with a relaxed allocator policy, plugins that run inside a host
// application which owns every device allocation, or tight loops that must not
// touch the allocator. sb_loglik_noalloc runs the same batched likelihood as
// sb_loglik, with its scratch in a fixed array compiled into this library
// instead of a caller-provided workspace. The caller still passes inputs and
// outputs. The array is 32 MiB and is held by every GPU that loads the library
// until the process exits.
#include <mutex>

#include "sb_internal.cuh"

namespace {

constexpr size_t kScratchBytes = size_t(32) << 20;
constexpr int kMaxDevices = 64;

// Shared by every call on a device; it keeps the previous call's contents.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device. Host code holds only the
// symbol's host-side stand-in, which is not a device address, so the address is
// asked of the runtime: on every call made outside a stream capture (so that a
// context that was reset and reloaded the module is seen), and from the value
// cached by the last such call while the stream is being captured.
sb_status scratch_address(cudaStream_t s, void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SB_ERR_CUDA;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return SB_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (cs == cudaStreamCaptureStatusNone) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return SB_ERR_CUDA;
        g_addr[dev] = p;
    }
    if (!g_addr[dev]) return SB_ERR_INVALID_ARG;  // first call on this device made inside a capture
    *out = g_addr[dev];
    return SB_OK;
}

}  // namespace

extern "C" sb_status sb_loglik_noalloc(const sb_problem *prob, int32_t prec, const double *x, int32_t n, double *ell,
                                       double *grad, void *stream) {
    const size_t need = sb_loglik_workspace_bytes(prob, prec, n);
    if (need == 0) return SB_ERR_INVALID_ARG;
    if (need > kScratchBytes) return SB_ERR_WORKSPACE;
    void *ws = nullptr;
    const sb_status st = scratch_address(static_cast<cudaStream_t>(stream), &ws);
    if (st != SB_OK) return st;
    // sb_loglik clears its status header and overwrites every scratch region it reads.
    return sb_loglik(prob, prec, x, n, ell, grad, ws, kScratchBytes, stream);
}

extern "C" sb_status sb_loglik_noalloc_check(void *stream) {
    void *ws = nullptr;
    const sb_status st = scratch_address(static_cast<cudaStream_t>(stream), &ws);
    if (st != SB_OK) return st;
    return sb_check(ws, kScratchBytes, stream);
}
