// Self-test of the failure path of the bounded device waits: a cooperative launch whose grid
// barrier expects one CTA more than the grid holds, so the barrier can never complete. Every
// wait gives up after its time limit (common.cuh, kSpinLimitNs), sets the device error word
// and returns; the host reads the word and reports LLS_ERR_TIMEOUT. Nothing faults and the
// context stays usable.
#include "common.cuh"
#include "kernels.cuh"

namespace lls {
namespace {

__global__ void barrier_timeout_kernel(unsigned* bar, int* err) {
    grid_barrier(bar, gridDim.x + 1, err);      // one arrival short: the wait runs out
}

}  // namespace
}  // namespace lls

using namespace lls;

extern "C" int lls_selftest_wait_timeout(void* ws, size_t ws_bytes, cudaStream_t stream) {
    if (!ws || ws_bytes < 256 || ((uintptr_t)ws & 255) != 0) return LLS_ERR_ARG;
    unsigned* bar = (unsigned*)ws;               // count, generation
    int* err = (int*)((char*)ws + 128);
    LLS_CUDA_TRY(cudaMemsetAsync(ws, 0, 256, stream));
    void* args[] = {&bar, &err};
    LLS_CUDA_TRY(cudaLaunchCooperativeKernel((void*)barrier_timeout_kernel, dim3(2), dim3(32), args, 0, stream));
    LLS_LAUNCH_CHECK("barrier_timeout", stream);
    int herr = 0;
    LLS_CUDA_TRY(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, stream));
    LLS_CUDA_TRY(cudaStreamSynchronize(stream));
    return herr == DEV_TIMEOUT ? LLS_ERR_TIMEOUT : (herr == DEV_OK ? LLS_OK : LLS_ERR_CUDA);
}
