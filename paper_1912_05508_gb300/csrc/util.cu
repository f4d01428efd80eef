// Small helper kernels: matrix copies, R diagonal check, Frobenius norm.
#include "common.cuh"
#include "kernels.cuh"

namespace lls {

int copy_matrix(const float* src, int lds, float* dst, int ldd, int m, int n, cudaStream_t st) {
    if (m <= 0 || n <= 0) return LLS_OK;
    LLS_CUDA_TRY(cudaMemcpy2DAsync(dst, sizeof(float) * (size_t)ldd, src, sizeof(float) * (size_t)lds,
                                   sizeof(float) * (size_t)m, (size_t)n, cudaMemcpyDeviceToDevice, st));
    return LLS_OK;
}

__global__ void check_diag_kernel(const float* __restrict__ R, int ldr, int n, int* err) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float d = R[(size_t)i + (size_t)i * ldr];
        if (!(d > 0.f) || !isfinite(d)) atomicCAS(err, DEV_OK, DEV_SINGULAR);
    }
}

int check_diag(const float* R, int ldr, int n, int* dev_err, cudaStream_t st) {
    check_diag_kernel<<<ceil_div(n, 256) < 64 ? ceil_div(n, 256) : 64, 256, 0, st>>>(R, ldr, n, dev_err);
    LLS_LAUNCH_CHECK("check_diag", st);
    return LLS_OK;
}

// After a factorization whose device error word is set (a bounded wait gave up, so R and Q
// are incomplete): R's diagonal becomes NaN, which the caller sees without synchronizing.
__global__ void poison_diag_kernel(float* R, int ldr, int n, const int* err) {
    if (*(volatile const int*)err == DEV_OK) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        R[(size_t)i + (size_t)i * ldr] = __int_as_float(0x7fc00000);
}

int poison_diag_on_error(float* R, int ldr, int n, const int* dev_err, cudaStream_t st) {
    if (n <= 0) return LLS_OK;
    poison_diag_kernel<<<ceil_div(n, 256) < 16 ? ceil_div(n, 256) : 16, 256, 0, st>>>(R, ldr, n, dev_err);
    LLS_LAUNCH_CHECK("poison_diag", st);
    return LLS_OK;
}

__global__ void zero_lower_kernel(float* R, int ldr, int n) {
    int j = blockIdx.y;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x + j + 1; i < n; i += gridDim.x * blockDim.x)
        R[(size_t)i + (size_t)j * ldr] = 0.f;
}

int zero_lower(float* R, int ldr, int n, cudaStream_t st) {
    if (n <= 1) return LLS_OK;
    dim3 grid(ceil_div(n, 256) < 16 ? ceil_div(n, 256) : 16, n);
    zero_lower_kernel<<<grid, 256, 0, st>>>(R, ldr, n);
    LLS_LAUNCH_CHECK("zero_lower", st);
    return LLS_OK;
}

// Sum of squares of an m x n FP32 matrix: compensated (double-float) accumulation per
// thread, FP64 across threads; per-block partials, then one warp sums them in a fixed order.
__global__ void sumsq_kernel(const float* __restrict__ A, int lda, int m, int n, double* part) {
    // compensated FP32 accumulation (FP64 arithmetic is ~70x slower on this GPU)
    float hs = 0.f, hc = 0.f;
    for (int j = blockIdx.y; j < n; j += gridDim.y) {
        const float* col = A + (size_t)j * lda;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
            float v = col[i];
            dot2_step(hs, hc, v, v, 0.f);
        }
    }
    double s = warp_sum_d(join_df(hs, hc));
    __shared__ double sh[8];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        part[blockIdx.x + blockIdx.y * gridDim.x] = t;
    }
}

__global__ void sum_parts_kernel(const double* part, int np, double* out) {
    double s = 0.0;
    for (int i = threadIdx.x; i < np; i += 32) s += part[i];
    s = warp_sum_d(s);
    if (threadIdx.x == 0) *out = s;
}

// W = A (m x n) and, in the same pass over A, out = ||A||_F^2 (the copy into the work matrix
// and the norm the stop test needs, one read of A instead of two). With W null only the norm is
// formed, with the same partition and order of the sums. 16-byte loads and stores when both
// matrices allow them.
__global__ void copy_sumsq_kernel(const float* __restrict__ A, int lda, float* __restrict__ W, int ldw, int m, int n,
                                  double* part, int vec4) {
    // every thread takes groups of four consecutive rows, then the rows past the last group:
    // the same sums in the same order whether the 16-byte path is taken or not
    float hs = 0.f, hc = 0.f;
    const int m4 = m >> 2;
    for (int j = blockIdx.y; j < n; j += gridDim.y) {
        const float* a = A + (size_t)j * lda;
        float* w = W ? W + (size_t)j * ldw : nullptr;
        for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < m4; q += gridDim.x * blockDim.x) {
            if (!LLS_INB(4 * q + 3 < m && (W == nullptr || ldw >= m) && lda >= m)) continue;
            float4 v;
            if (vec4) {
                v = __ldg(reinterpret_cast<const float4*>(a) + q);
                if (w) reinterpret_cast<float4*>(w)[q] = v;
            } else {
                v = make_float4(a[4 * q], a[4 * q + 1], a[4 * q + 2], a[4 * q + 3]);
                if (w) { w[4 * q] = v.x; w[4 * q + 1] = v.y; w[4 * q + 2] = v.z; w[4 * q + 3] = v.w; }
            }
            dot2_step(hs, hc, v.x, v.x, 0.f);
            dot2_step(hs, hc, v.y, v.y, 0.f);
            dot2_step(hs, hc, v.z, v.z, 0.f);
            dot2_step(hs, hc, v.w, v.w, 0.f);
        }
        for (int i = 4 * m4 + blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
            const float v = a[i];
            if (w) w[i] = v;
            dot2_step(hs, hc, v, v, 0.f);
        }
    }
    double s = warp_sum_d(join_df(hs, hc));
    __shared__ double sh[8];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w2 = 0; w2 < (int)(blockDim.x >> 5); ++w2) t += sh[w2];
        part[blockIdx.x + blockIdx.y * gridDim.x] = t;
    }
}

int copy_fro_sumsq(const float* A, int lda, float* W, int ldw, int m, int n, double* part, double* out,
                   cudaStream_t st) {
    if (m <= 0 || n <= 0) return LLS_OK;
    const int vec4 = ((uintptr_t)A & 15) == 0 && (lda & 3) == 0 &&
                     (!W || (((uintptr_t)W & 15) == 0 && (ldw & 3) == 0));
    dim3 grid(ceil_div(m, 1024) < 8 ? ceil_div(m, 1024) : 8, n < 512 ? n : 512);
    copy_sumsq_kernel<<<grid, 256, 0, st>>>(A, lda, W, ldw, m, n, part, vec4);
    LLS_LAUNCH_CHECK("copy_sumsq", st);
    sum_parts_kernel<<<1, 32, 0, st>>>(part, (int)(grid.x * grid.y), out);
    LLS_LAUNCH_CHECK("sum_parts", st);
    return LLS_OK;
}

// out = ||A||_F^2 (FP64, device). part: >= 64*64 doubles.
int fro_sumsq(const float* A, int lda, int m, int n, double* part, double* out, cudaStream_t st) {
    dim3 grid(ceil_div(m, 256) < 8 ? ceil_div(m, 256) : 8, n < 512 ? n : 512);
    sumsq_kernel<<<grid, 256, 0, st>>>(A, lda, m, n, part);
    LLS_LAUNCH_CHECK("sumsq", st);
    sum_parts_kernel<<<1, 32, 0, st>>>(part, (int)(grid.x * grid.y), out);
    LLS_LAUNCH_CHECK("sum_parts", st);
    return LLS_OK;
}

}  // namespace lls
