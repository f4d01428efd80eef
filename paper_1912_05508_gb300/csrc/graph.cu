// Replay of whole factorizations / solves as CUDA graphs.
//
// A solve enqueues ~10^3 small kernels from a host-side recursion; issuing them one by one
// leaves the GPU waiting on the host. The first call with a given argument set (sizes,
// options, every pointer, workspace size, device) is captured from the caller's stream into
// a graph; later identical calls launch the instantiated graph. Graphs are not used when
// the stream is a legacy/per-thread default stream, when the stream is already being
// captured by the caller (their capture then records the kernels directly), or when
// LLS_NO_GRAPH or LLS_TRACE is set. Up to kMaxGraphs recent argument sets are kept.
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <list>
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"

namespace lls {

extern std::atomic<unsigned long long> g_launches;

namespace {
constexpr size_t kMaxGraphs = 16;
struct Entry {
    GraphKey key;
    cudaGraphExec_t exec;
    cudaEvent_t ev[3];
    unsigned long long launches;
};
std::mutex g_mu;
std::list<Entry> g_cache;

bool graphs_enabled() {
    static const bool on = getenv("LLS_NO_GRAPH") == nullptr && getenv("LLS_TRACE") == nullptr;
    return on;
}

bool same_key(const GraphKey& a, const GraphKey& b) { return memcmp(&a, &b, sizeof(GraphKey)) == 0; }
}  // namespace

void record_phase(cudaEvent_t ev, cudaStream_t st, bool capturing) {
    if (!ev) return;
    if (capturing) cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal);
    else cudaEventRecord(ev, st);
}

int run_graphed(const GraphKey& key, cudaStream_t st, EnqueueFn fn, void* ctx, cudaEvent_t* ev_out) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const bool can = graphs_enabled() && st != 0 && st != cudaStreamLegacy && st != cudaStreamPerThread &&
                     cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone;
    if (!can) {
        // direct enqueue; phase events (if wanted) are the caller's
        return fn(ctx, st, ev_out, false);
    }
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto it = g_cache.begin(); it != g_cache.end(); ++it) {
        if (same_key(it->key, key)) {
            g_cache.splice(g_cache.begin(), g_cache, it);
            Entry& e = g_cache.front();
            LLS_CUDA_TRY(cudaGraphLaunch(e.exec, st));
            g_launches.fetch_add(e.launches, std::memory_order_relaxed);
            if (ev_out) for (int i = 0; i < 3; ++i) ev_out[i] = e.ev[i];
            return LLS_OK;
        }
    }
    Entry e;
    e.key = key;
    for (auto& v : e.ev) LLS_CUDA_TRY(cudaEventCreate(&v));
    const unsigned long long before = g_launches.load();
    LLS_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    int rc = fn(ctx, st, e.ev, true);
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamEndCapture(st, &g);
    e.launches = g_launches.load() - before;
    g_launches.fetch_sub(e.launches, std::memory_order_relaxed);
    if (rc != LLS_OK || ce != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        for (auto& v : e.ev) cudaEventDestroy(v);
        cudaGetLastError();
        if (rc != LLS_OK) return rc;
        return fn(ctx, st, ev_out, false);     // capture refused: run directly
    }
    ce = cudaGraphInstantiate(&e.exec, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) {
        for (auto& v : e.ev) cudaEventDestroy(v);
        cudaGetLastError();
        return fn(ctx, st, ev_out, false);
    }
    if (g_cache.size() >= kMaxGraphs) {
        Entry& old = g_cache.back();
        cudaGraphExecDestroy(old.exec);
        for (auto& v : old.ev) cudaEventDestroy(v);
        g_cache.pop_back();
    }
    g_cache.push_front(e);
    LLS_CUDA_TRY(cudaGraphLaunch(e.exec, st));
    g_launches.fetch_add(e.launches, std::memory_order_relaxed);
    if (ev_out) for (int i = 0; i < 3; ++i) ev_out[i] = e.ev[i];
    return LLS_OK;
}

}  // namespace lls
