// Shared device/host helpers for the GB300 least-squares library.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/lls_gb300.h"

#define LLS_CUDA_TRY(expr)                                  \
    do {                                                     \
        cudaError_t _e = (expr);                             \
        if (_e != cudaSuccess) return LLS_ERR_CUDA;          \
    } while (0)

namespace lls {
void note_launch(const char* name, cudaStream_t st);
void trace_mark(cudaStream_t st);
void trace_flush();
}
// After every kernel launch: count it (and, under LLS_TRACE, time it) and surface
// launch-configuration errors.
#define LLS_LAUNCH_CHECK(name, st)                           \
    do {                                                     \
        ::lls::note_launch(name, st);                        \
        LLS_CUDA_TRY(cudaGetLastError());                    \
    } while (0)

#define LLS_TRY(expr)                                        \
    do {                                                     \
        int _s = (expr);                                     \
        if (_s != LLS_OK) return _s;                         \
    } while (0)

namespace lls {

constexpr unsigned kFullMask = 0xffffffffu;

// Device error word values (written by kernels that hit a bounded-wait limit or bad data).
enum DevErr : int { DEV_OK = 0, DEV_TIMEOUT = 1, DEV_SINGULAR = 2 };

// ---------------------------------------------------------------------------------------
// Index checks of the LLS_DEBUG build (liblls_gb300_debug.so). LLS_INB(cond) guards one
// global-memory access. In the release build it is the constant true and compiles away. In
// the debug build a false condition records the source line of the first failed check in
// the translation unit's debug word, and the caller skips the access; no kernel returns
// early on a failed check, so its barriers stay matched. The public entry points clear the
// words before a call and read them after it (a stream synchronization), returning
// LLS_ERR_BOUNDS and naming the file and line on stderr. Debug calls cannot be captured
// into a caller's CUDA graph.
// ---------------------------------------------------------------------------------------
#ifndef LLS_DEBUG
#define LLS_DEBUG 0
#endif
// Reads (reset = 0: the recorded line, 0 if none) or clears (reset = 1) one unit's word.
using DebugFetch = int (*)(cudaStream_t st, int reset);
bool debug_register(DebugFetch f, const char* file);
int debug_collect(cudaStream_t st);   // LLS_OK, or LLS_ERR_BOUNDS after naming the site
void debug_reset(cudaStream_t st);
#if LLS_DEBUG
namespace {
__device__ int g_debug_line;     // one per translation unit (no relocatable device code)
__device__ __forceinline__ bool debug_check(bool ok, int line) {
    if (!ok) atomicCAS(&g_debug_line, 0, line);
    return ok;
}
int debug_fetch(cudaStream_t st, int reset) {
    int v = 0;
    if (reset) {
        cudaMemcpyToSymbolAsync(g_debug_line, &v, sizeof(v), 0, cudaMemcpyHostToDevice, st);
        return 0;
    }
    cudaMemcpyFromSymbolAsync(&v, g_debug_line, sizeof(v), 0, cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    return v;
}
[[maybe_unused]] const bool g_debug_registered = debug_register(debug_fetch, __BASE_FILE__);
}  // namespace
#define LLS_INB(cond) (::lls::debug_check((cond), __LINE__))
#else
#define LLS_INB(cond) true
#endif

// Maximum wait of any device-side spin before it gives up, in nanoseconds.
constexpr unsigned long long kSpinLimitNs = 2000000000ull;

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---------------------------------------------------------------------------------------
// Double-float arithmetic: a value is hi + lo with two FP32 numbers. GB300's FP64 rate is
// about 1/70 of its FP32 rate, so the FP64-accurate Krylov products use error-free
// transformations on FP32 instead: TwoProduct via FMA (exact a*b = p + e) and Knuth's
// TwoSum (exact a + b = s + e). The _rn intrinsics keep the compiler from contracting or
// reassociating the steps.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    float z = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

// Compensated dot-product step (Ogita, Rump, Oishi 2005, "Dot2"): accumulates
// a * (th + tl) into the running sum s with the rounding errors collected in c.
__device__ __forceinline__ void dot2_step(float& s, float& c, float a, float th, float tl) {
    float p = __fmul_rn(a, th);
    float e = __fmaf_rn(a, th, -p);       // exact: a*th = p + e
    e = __fmaf_rn(a, tl, e);              // low part of t, product rounded once (~u^2 relative)
    float s2, e2;
    two_sum(s, p, s2, e2);
    s = s2;
    c = __fadd_rn(c, __fadd_rn(e, e2));
}

// Warp-wide sum of double-float values (s, c) with TwoSum at every butterfly level.
__device__ __forceinline__ void warp_sum_df(float& s, float& c) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float s2 = __shfl_xor_sync(kFullMask, s, o);
        const float c2 = __shfl_xor_sync(kFullMask, c, o);
        float t, e;
        two_sum(s, s2, t, e);
        s = t;
        c = __fadd_rn(__fadd_rn(c, c2), e);
    }
}

__device__ __forceinline__ void split_df(double v, float& hi, float& lo) {
    hi = __double2float_rn(v);
    lo = __double2float_rn(__dsub_rn(v, (double)hi));
}

__device__ __forceinline__ double join_df(float s, float c) {
    return __dadd_rn((double)s, (double)c);
}

// ---------------------------------------------------------------------------------------
// Low-precision element types of the tensor-core products.
// ---------------------------------------------------------------------------------------
template <typename T> struct LowPrec;
template <> struct LowPrec<__half> {
    static __device__ __forceinline__ __half from_float(float x) { return __float2half_rn(x); }
    static __device__ __forceinline__ float to_float(__half x) { return __half2float(x); }
};
template <> struct LowPrec<__nv_bfloat16> {
    static __device__ __forceinline__ __nv_bfloat16 from_float(float x) { return __float2bfloat16_rn(x); }
    static __device__ __forceinline__ float to_float(__nv_bfloat16 x) { return __bfloat162float(x); }
};
template <> struct LowPrec<__nv_fp8_e4m3> {   // round to nearest even, saturating to +-448
    static __device__ __forceinline__ __nv_fp8_e4m3 from_float(float x) { return __nv_fp8_e4m3(x); }
    static __device__ __forceinline__ float to_float(__nv_fp8_e4m3 x) { return float(x); }
};
template <> struct LowPrec<float> {
    static __device__ __forceinline__ float from_float(float x) { return x; }
    static __device__ __forceinline__ float to_float(float x) { return x; }
};

// Column scale exponent e with max|x| * 2^e in [2^14, 2^15) (FP16 target range, largest
// finite FP16 is 65504). Zero (or non-finite) maximum gives 0; clamped to [-100, 100].
__device__ __forceinline__ int fp16_scale_exponent(float mx) {
    if (!(mx > 0.0f) || !isfinite(mx)) return 0;
    int ex;
    frexpf(mx, &ex);                      // mx = f * 2^ex, f in [0.5, 1)
    int e = 15 - ex;
    return e < -100 ? -100 : (e > 100 ? 100 : e);
}

// Column scale exponent e with max|x| * 2^e in [2^7, 2^8) (FP8 E4M3 target range, largest
// finite E4M3 is 448). Zero (or non-finite) maximum gives 0; clamped to [-100, 100].
__device__ __forceinline__ int fp8_scale_exponent(float mx) {
    if (!(mx > 0.0f) || !isfinite(mx)) return 0;
    int ex;
    frexpf(mx, &ex);
    int e = 8 - ex;
    return e < -100 ? -100 : (e > 100 ? 100 : e);
}

// Scale kinds of the low-precision copies: 0 none (BF16, FP32), 1 FP16 range, 2 FP8 range.
__device__ __forceinline__ int scale_exponent(int kind, float mx) {
    return kind == 1 ? fp16_scale_exponent(mx) : (kind == 2 ? fp8_scale_exponent(mx) : 0);
}

// 2^e as an FP32 number for e in [-126, 127] (exponent field only): multiplying by it is exact
// whenever the product is a normal number.
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((e + 127) << 23); }

// ---------------------------------------------------------------------------------------
// Warp reductions.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_xor_sync(kFullMask, v, o));
    return v;
}
__device__ __forceinline__ float warp_max_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFullMask, v, o));
    return v;
}

// ---------------------------------------------------------------------------------------
// Grid-wide barrier for cooperative (co-resident) launches. bar[0..1] form one 8-byte-aligned
// 64-bit word: the arrival count in its low half, the generation in its high half. A CTA
// arrives with one atomic add, which also tells it the generation it waits to see change; the
// last arrival resets the count and advances the generation with a single add of
// 2^32 - nblocks. The count is left at zero. The wait is bounded by kSpinLimitNs, after which
// the error word is set and the caller must return. Returns false when the barrier timed out
// or an error was flagged before this arrival. The error word is read together with the
// arrival (both loads in flight at once), so a flag raised by another CTA while this one
// waits is seen at the next barrier: a CTA that returned on an error never arrives there,
// and the waiting CTAs read the error word while they poll.
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned nblocks, int* err) {
    __syncthreads();
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        unsigned long long* word = reinterpret_cast<unsigned long long*>(bar);
        __threadfence();
        const int e0 = *(volatile int*)err;
        const unsigned long long old = atomicAdd(word, 1ull);
        const unsigned gen = (unsigned)(old >> 32);
        int ok = e0 == DEV_OK ? 1 : 0;
        if ((unsigned)(old & 0xffffffffull) == nblocks - 1) {
            atomicAdd(word, (1ull << 32) - (unsigned long long)nblocks);
        } else {
            const volatile unsigned* genp = bar + 1;
            const unsigned long long t0 = globaltimer_ns();
            int spins = 0;
            while (*genp == gen) {
                if (++spins < 64) continue;         // a first short burst of polls, then paced
                if (*(volatile int*)err != DEV_OK) { ok = 0; break; }
                if (globaltimer_ns() - t0 > kSpinLimitNs) {
                    atomicCAS(err, DEV_OK, DEV_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

}  // namespace lls

// Host-side helpers shared by the translation units.
namespace lls {

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }
inline int ceil_div(int a, int b) { return (a + b - 1) / b; }

// Bump allocator over the caller's workspace (all offsets 256-B aligned).
struct WsArena {
    char* base;
    size_t cap;
    size_t off;
    bool ok;
    WsArena(void* p, size_t c) : base((char*)p), cap(c), off(0), ok(true) {}
    template <typename T> T* take(size_t count) {
        size_t bytes = align_up(count * sizeof(T), 256);
        if (off + bytes > cap) { ok = false; off += bytes; return nullptr; }
        T* r = base ? (T*)(base + off) : nullptr;
        off += bytes;
        return r;
    }
};

}  // namespace lls
