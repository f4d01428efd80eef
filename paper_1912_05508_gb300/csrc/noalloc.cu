// lls_lowp_projection_noalloc: the projection product of one recursion step (R12 = Q1^T A2
// with its scaled low-precision copy) for callers that cannot allocate device memory.
//
// lls_lowp_projection takes a caller-allocated workspace for its split-K partial sums and
// its device error word. Some callers have no way to provide one at the point of the call:
// code running inside a framework's custom-op or plugin hook that owns the memory pool and
// forbids allocation in its execute step, real-time paths where cudaMalloc's implicit device
// synchronisation is not acceptable, or host code that only holds borrowed device pointers.
// This variant takes the same scratch from one fixed array compiled into the library and so
// calls no allocator at all. The kernels and the order of summation are those of
// lls_lowp_projection; only the origin of the scratch differs.
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"

namespace lls {

// The fixed scratch, laid out like the workspace of lls_lowp_projection: split-K partial sums
// first, then the 16-word device error word after a 256-byte boundary. Every GPU that loads
// the library holds these bytes until the process exits.
constexpr size_t kNoallocBytes = LLS_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {};

// The name g_noalloc_scratch in host code is only a host-side stand-in for the array; the
// device address differs per device and must be asked for with that device current. This is
// done on the first call on each device and cached for the life of the process. A
// cudaDeviceReset discards the device's context and with it the array, so the cached address
// is then stale: the entry point is not to be used after a reset of that device.
int scratch_address(void** out) {
    int dev = 0;
    LLS_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return LLS_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        LLS_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return LLS_OK;
}
}  // namespace

}  // namespace lls

using namespace lls;

extern "C" int lls_lowp_projection_noalloc(int m, int w1, int w2, int prec, const void* Q1l, const void* A2l,
                                           int ldh, const int* e, float* R12, int ldr, void* R12l, int ldrl,
                                           int* f, cudaStream_t stream) {
    if (m < 1 || w1 < 1 || w2 < 1 || ldh < m || ldr < w1 || ldrl < w1 || (ldrl & 7) != 0) return LLS_ERR_ARG;
    if (prec != LLS_PREC_FP16 && prec != LLS_PREC_BF16) return LLS_ERR_ARG;
    if (!Q1l || !A2l || !e || !R12 || !R12l || !f) return LLS_ERR_ARG;
    // same scratch need as lls_lowp_projection_workspace_size(m, w1, w2)
    const size_t partials = proj_partial_floats(m, w1, w2);
    if (align_up(sizeof(float) * partials, 256) + 256 > kNoallocBytes) return LLS_ERR_TOO_LARGE;
    void* base = nullptr;
    LLS_TRY(scratch_address(&base));
    WsArena ar(base, kNoallocBytes);
    ProjCall pc;
    pc.part_floats = partials;
    pc.part = ar.take<float>(partials);
    pc.err = ar.take<int>(16);
    if (!ar.ok) return LLS_ERR_TOO_LARGE;
    // The array keeps whatever the previous call left. The error word must start at zero. The
    // partial sums are fully written by the product kernel before the reduction reads them,
    // except when a bounded wait of the product gives up: it then leaves its partials
    // unwritten and sets the error word, and the reduction, seeing the word, writes R12 and
    // R12l as NaN (f = 0) instead of summing what an earlier call left there.
    LLS_CUDA_TRY(cudaMemsetAsync(pc.err, 0, sizeof(int) * 16, stream));
    pc.Q1l = Q1l; pc.A2l = A2l; pc.ldh = ldh; pc.m = m; pc.w1 = w1; pc.w2 = w2; pc.e = e;
    pc.R12 = R12; pc.ldr = ldr; pc.R12l = R12l; pc.ldrl = ldrl; pc.f = f;
    pc.lowp = prec == LLS_PREC_FP16 ? 0 : 1;
    return gemm_projection(pc, stream);
}
