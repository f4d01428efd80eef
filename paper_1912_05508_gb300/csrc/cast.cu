// Per-column power-of-two scaling and rounding to the tensor-core input type.
//
// The paper runs the recursion's products with FP16 inputs (Sec. 2.1, Sec. 3.1.2) and
// points out FP16's narrow range; it does not say how range is handled. Here each column
// j of the operand is multiplied by 2^e_j, chosen from the column's largest magnitude so
// that it lands in [2^14, 2^15) (FP16; BF16 needs no scale), then rounded to nearest even.
// A power of two changes no significand bit, so dividing the product by 2^e_j is exact.
#include "common.cuh"
#include "kernels.cuh"

namespace lls {

constexpr int kCastThreads = 256;

template <typename TL>
__global__ void __launch_bounds__(kCastThreads)
scale_cast_kernel(const float* __restrict__ X, int ldx, int m, int c0, TL* __restrict__ Xh,
                  int ldh, int want_scale, int* __restrict__ exps) {
    const int j = c0 + blockIdx.x;
    const float* col = X + (size_t)j * ldx;
    __shared__ float s_red[kCastThreads / 32];
    __shared__ int s_e;
    int e = 0;
    if (want_scale) {
        float mx = 0.f;
        for (int i = threadIdx.x; i < m; i += kCastThreads) mx = fmaxf(mx, fabsf(col[i]));
        mx = warp_max_f(mx);
        if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = mx;
        __syncthreads();
        if (threadIdx.x == 0) {
            float t = 0.f;
            for (int w = 0; w < kCastThreads / 32; ++w) t = fmaxf(t, s_red[w]);
            s_e = fp16_scale_exponent(t);
            exps[blockIdx.x] = s_e;
        }
        __syncthreads();
        e = s_e;
    } else if (threadIdx.x == 0) {
        exps[blockIdx.x] = 0;
    }
    const float sc = pow2f(e);
    TL* out = Xh + (size_t)j * ldh;
    for (int i = threadIdx.x; i < m; i += kCastThreads)
        out[i] = LowPrec<TL>::from_float(col[i] * sc);
}

int scale_cast_columns(const float* X, int ldx, int m, int c0, int w, void* Xh, int ldh,
                       int lowp, int* exps, cudaStream_t st) {
    if (w <= 0) return LLS_OK;
    if (lowp == 0)
        scale_cast_kernel<__half><<<w, kCastThreads, 0, st>>>(X, ldx, m, c0, (__half*)Xh, ldh, 1, exps);
    else if (lowp == 1)
        scale_cast_kernel<__nv_bfloat16><<<w, kCastThreads, 0, st>>>(X, ldx, m, c0, (__nv_bfloat16*)Xh, ldh, 0, exps);
    else
        return LLS_ERR_UNSUPPORTED;
    LLS_LAUNCH_CHECK("scale_cast", st);
    return LLS_OK;
}

}  // namespace lls
