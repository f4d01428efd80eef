// The direct solve with the mixed-precision factors, x0 = R^{-1} (Q^T b): the last two steps
// of the direct least-squares method (Alg. 1: b <- Q^T b, then the triangular solve) applied to
// the Q and R of RGSQRF (Alg. 2). Its accuracy is limited by the low-precision products
// (Sec. 4.2.2 finds it about two orders of magnitude less accurate than a single-precision
// Householder solve), so the library uses it only as the starting point of the Krylov
// iteration (lls_options.x0 = 2): CGLS then starts with ||A (x0 - x*)|| at the level of the
// factorization error instead of ||b||.
//
//   c = Q^T b     row-chunk partial sums: one warp per column and chunk, four FP32
//                 accumulation chains per lane over 16-byte loads of Q, then a fixed-order
//                 FP64 sum over the chunks;
//   x0 = M c      M = R^{-1} (upper triangular, formed for the preconditioner):
//                 x0_i = sum_{k >= i} M_ik c_k, read from column i of M^T, FP64 sums.
// FP32 products suffice: the error of x0 only changes the number of iterations, never the
// solution the iteration converges to.
#include "common.cuh"
#include "kernels.cuh"

namespace lls {

constexpr int kDirRows = 2048;      // rows per Q^T b work item (64 per lane)

__global__ void __launch_bounds__(256) qtb_partial_kernel(const float* __restrict__ Q, int ldq, int m, int n,
                                                          const double* __restrict__ b, double* __restrict__ part,
                                                          int vec4) {
    const int lane = threadIdx.x & 31;
    const int j = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (j >= n) return;
    const int r0 = blockIdx.y * kDirRows, r1 = min(m, r0 + kDirRows);
    const float* q = Q + (size_t)j * ldq;
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
    if (vec4) {
        for (int i = r0 + 4 * lane; i + 3 < r1; i += 128) {
            const float4 v = __ldg(reinterpret_cast<const float4*>(q + i));
            const double2 b01 = __ldg(reinterpret_cast<const double2*>(b + i));
            const double2 b23 = __ldg(reinterpret_cast<const double2*>(b + i + 2));
            s0 = fmaf(v.x, (float)b01.x, s0);
            s1 = fmaf(v.y, (float)b01.y, s1);
            s2 = fmaf(v.z, (float)b23.x, s2);
            s3 = fmaf(v.w, (float)b23.y, s3);
        }
        // rows past the last full group of four (only in the last chunk of a ragged m)
        const int tail = r0 + ((r1 - r0) & ~3);
        for (int i = tail + lane; i < r1; i += 32) s0 = fmaf(q[i], (float)b[i], s0);
    } else {
        for (int i = r0 + lane; i < r1; i += 32) s0 = fmaf(q[i], (float)b[i], s0);
    }
    double s = (double)s0 + (double)s1 + ((double)s2 + (double)s3);
    s = warp_sum_d(s);
    if (lane == 0 && LLS_INB(r0 < m && ldq >= m)) part[(size_t)blockIdx.y * n + j] = s;
}

__global__ void __launch_bounds__(256) qtb_sum_kernel(const double* __restrict__ part, int chunks, int n,
                                                      double* __restrict__ c) {
    const int j = blockIdx.x * 256 + threadIdx.x;
    if (j >= n) return;
    double s = 0.0;
    for (int k = 0; k < chunks; ++k) s += part[(size_t)k * n + j];
    c[j] = s;
}

__global__ void __launch_bounds__(256) tri_apply_kernel(const float* __restrict__ Mt, int n,
                                                        const double* __restrict__ c, double* __restrict__ x) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * 8 + (threadIdx.x >> 5);
    if (i >= n) return;
    const float* col = Mt + (size_t)i * n;       // column i of M^T = row i of M
    double s = 0.0;
    for (int k = i + lane; k < n; k += 32) s = fma((double)col[k], c[k], s);
    s = warp_sum_d(s);
    if (lane == 0) x[i] = s;
}

size_t direct_start_scratch_bytes(int m, int n) {
    const size_t chunks = (size_t)ceil_div(m, kDirRows);
    return sizeof(double) * (chunks * (size_t)n + (size_t)n) + 256;
}

int direct_start(const float* Q, int ldq, int m, int n, const double* b, const float* Mt, double* x, void* scratch,
                 size_t scratch_bytes, cudaStream_t st) {
    if (scratch_bytes < direct_start_scratch_bytes(m, n)) return LLS_ERR_WORKSPACE;
    const int chunks = ceil_div(m, kDirRows);
    double* part = (double*)scratch;
    double* c = part + (size_t)chunks * n;
    const int vec4 = (((uintptr_t)Q & 15) == 0 && ldq % 4 == 0 && ((uintptr_t)b & 15) == 0) ? 1 : 0;
    qtb_partial_kernel<<<dim3(ceil_div(n, 8), chunks), 256, 0, st>>>(Q, ldq, m, n, b, part, vec4);
    LLS_LAUNCH_CHECK("qtb_partial", st);
    qtb_sum_kernel<<<ceil_div(n, 256), 256, 0, st>>>(part, chunks, n, c);
    LLS_LAUNCH_CHECK("qtb_sum", st);
    tri_apply_kernel<<<ceil_div(n, 8), 256, 0, st>>>(Mt, n, c, x);
    LLS_LAUNCH_CHECK("tri_apply", st);
    return LLS_OK;
}

}  // namespace lls
