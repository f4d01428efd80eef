// Launch counting, optional per-kernel tracing, and the registry of the debug build's
// per-unit index-check words.
//
// Every launch goes through note_launch(name, stream). With the environment variable
// LLS_TRACE set, an event is recorded after each launch; trace_flush() (called at the end of
// the public entry points) turns consecutive events on a stream into per-kernel times
// (end-to-end on the stream, so launch gaps are charged to the kernel that follows them)
// and a table is printed to stderr at process exit.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"

namespace lls {

std::atomic<unsigned long long> g_launches{0};

namespace {
struct Rec { const char* name; cudaEvent_t ev; cudaStream_t st; };
struct Acc { unsigned long long count = 0; double ms = 0.0; };
std::mutex g_mu;
std::vector<Rec> g_pending;
std::map<cudaStream_t, cudaEvent_t> g_last;
std::map<std::string, Acc> g_acc;

bool trace_on() {
    static const bool on = getenv("LLS_TRACE") != nullptr;
    return on;
}

void report() {
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_acc.empty()) return;
    double tot = 0.0;
    for (auto& kv : g_acc) tot += kv.second.ms;
    fprintf(stderr, "[lls trace] %-22s %10s %12s %10s %7s\n", "kernel", "launches", "total_ms", "avg_us", "share");
    for (auto& kv : g_acc)
        fprintf(stderr, "[lls trace] %-22s %10llu %12.3f %10.2f %6.1f%%\n", kv.first.c_str(), kv.second.count,
                kv.second.ms, 1e3 * kv.second.ms / (double)kv.second.count, 100.0 * kv.second.ms / tot);
}
}  // namespace

void note_launch(const char* name, cudaStream_t st) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (!trace_on()) return;
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    cudaEventRecord(e, st);
    std::lock_guard<std::mutex> lk(g_mu);
    g_pending.push_back({name, e, st});
}

void trace_mark(cudaStream_t st) {
    if (!trace_on()) return;
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    cudaEventRecord(e, st);
    std::lock_guard<std::mutex> lk(g_mu);
    g_pending.push_back({nullptr, e, st});
}

void trace_flush() {
    if (!trace_on()) return;
    static bool registered = false;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!registered) { atexit(report); registered = true; }
    for (auto& r : g_pending) {
        cudaEventSynchronize(r.ev);
        auto it = g_last.find(r.st);
        if (it != g_last.end()) {
            if (r.name) {
                float ms = 0.f;
                cudaEventElapsedTime(&ms, it->second, r.ev);
                Acc& a = g_acc[r.name];
                a.count++;
                a.ms += ms;
            }
            cudaEventDestroy(it->second);
        }
        g_last[r.st] = r.ev;
    }
    g_pending.clear();
}

// ---- LLS_DEBUG index checks: one word per translation unit -------------------------------
namespace {
struct DebugUnit { DebugFetch fetch; const char* file; };
std::vector<DebugUnit>& debug_units() {
    static std::vector<DebugUnit> u;   // filled by static initializers, before any call
    return u;
}
}  // namespace

bool debug_register(DebugFetch f, const char* file) {
    debug_units().push_back({f, file});
    return true;
}

void debug_reset(cudaStream_t st) {
    for (auto& u : debug_units()) u.fetch(st, 1);
}

int debug_collect(cudaStream_t st) {
    int status = LLS_OK;
    for (auto& u : debug_units()) {
        const int line = u.fetch(st, 0);
        if (line != 0) {
            const char* base = strrchr(u.file, '/');
            fprintf(stderr, "[lls debug] index check failed at %s:%d (the access was skipped)\n",
                    base ? base + 1 : u.file, line);
            status = LLS_ERR_BOUNDS;
            u.fetch(st, 1);
        }
    }
    return status;
}

}  // namespace lls
