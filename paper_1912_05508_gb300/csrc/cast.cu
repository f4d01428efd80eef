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

constexpr int kCastThreads = 512;

template <typename TL> struct Pack4;
template <> struct Pack4<__half> {
    static __device__ __forceinline__ uint2 make(float4 v) {
        __half2 a = __floats2half2_rn(v.x, v.y), b = __floats2half2_rn(v.z, v.w);
        return make_uint2(*reinterpret_cast<unsigned*>(&a), *reinterpret_cast<unsigned*>(&b));
    }
};
template <> struct Pack4<__nv_bfloat16> {
    static __device__ __forceinline__ uint2 make(float4 v) {
        __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
        return make_uint2(*reinterpret_cast<unsigned*>(&a), *reinterpret_cast<unsigned*>(&b));
    }
};
template <> struct Pack4<__nv_fp8_e4m3> {
    static __device__ __forceinline__ unsigned make(float4 v) {
        const __nv_fp8_e4m3 a(v.x), b(v.y), c(v.z), d(v.w);
        return (unsigned)a.__x | ((unsigned)b.__x << 8) | ((unsigned)c.__x << 16) | ((unsigned)d.__x << 24);
    }
};
// The 4-element packed store type of each format (8 bytes for 16-bit, 4 bytes for 8-bit).
template <typename TL> struct PackT { using type = uint2; };
template <> struct PackT<__nv_fp8_e4m3> { using type = unsigned; };

// One CTA per column: the column maximum (FP16 only), then the scaled cast. With 16-byte
// aligned columns both passes move 16-byte vectors, four independent loads per thread per
// trip, so each CTA keeps enough loads in flight; the second pass re-reads the column from L2.
template <typename TL>
__global__ void __launch_bounds__(kCastThreads)
scale_cast_kernel(const float* __restrict__ X, int ldx, int m, int c0, TL* __restrict__ Xh,
                  int ldh, int kind, int* __restrict__ exps, int vec) {
    const int j = c0 + blockIdx.x;
    const float* col = X + (size_t)j * ldx;
    TL* out = Xh + (size_t)j * ldh;
    __shared__ float s_red[kCastThreads / 32];
    __shared__ int s_e;
    const int t = threadIdx.x;
    const int m4 = vec ? m / 4 : 0;                 // float4 part; the tail goes element-wise
    const float4* col4 = reinterpret_cast<const float4*>(col);
    int e = 0;
    if (kind != 0) {
        float mx = 0.f;
        int q = t;
        for (; q + 3 * kCastThreads < m4; q += 4 * kCastThreads) {
            const float4 a = __ldg(col4 + q), b = __ldg(col4 + q + kCastThreads);
            const float4 c = __ldg(col4 + q + 2 * kCastThreads), d = __ldg(col4 + q + 3 * kCastThreads);
            mx = fmaxf(mx, fmaxf(fmaxf(fmaxf(fabsf(a.x), fabsf(a.y)), fmaxf(fabsf(a.z), fabsf(a.w))),
                                 fmaxf(fmaxf(fabsf(b.x), fabsf(b.y)), fmaxf(fabsf(b.z), fabsf(b.w)))));
            mx = fmaxf(mx, fmaxf(fmaxf(fmaxf(fabsf(c.x), fabsf(c.y)), fmaxf(fabsf(c.z), fabsf(c.w))),
                                 fmaxf(fmaxf(fabsf(d.x), fabsf(d.y)), fmaxf(fabsf(d.z), fabsf(d.w)))));
        }
        for (; q < m4; q += kCastThreads) {
            const float4 a = __ldg(col4 + q);
            mx = fmaxf(mx, fmaxf(fmaxf(fabsf(a.x), fabsf(a.y)), fmaxf(fabsf(a.z), fabsf(a.w))));
        }
        for (int i = 4 * m4 + t; i < m; i += kCastThreads) mx = fmaxf(mx, fabsf(col[i]));
        mx = warp_max_f(mx);
        if ((t & 31) == 0) s_red[t >> 5] = mx;
        __syncthreads();
        if (t == 0) {
            float tm = 0.f;
            for (int w = 0; w < kCastThreads / 32; ++w) tm = fmaxf(tm, s_red[w]);
            s_e = scale_exponent(kind, tm);
            exps[blockIdx.x] = s_e;
        }
        __syncthreads();
        e = s_e;
    } else if (t == 0) {
        exps[blockIdx.x] = 0;
    }
    const float sc = pow2f(e);
    using P = typename PackT<TL>::type;
    P* out2 = reinterpret_cast<P*>(out);
    int q = t;
    for (; q + kCastThreads < m4; q += 2 * kCastThreads) {
        float4 a = __ldg(col4 + q), b = __ldg(col4 + q + kCastThreads);
        a.x *= sc; a.y *= sc; a.z *= sc; a.w *= sc;
        b.x *= sc; b.y *= sc; b.z *= sc; b.w *= sc;
        out2[q] = Pack4<TL>::make(a);
        out2[q + kCastThreads] = Pack4<TL>::make(b);
    }
    for (; q < m4; q += kCastThreads) {
        float4 a = __ldg(col4 + q);
        a.x *= sc; a.y *= sc; a.z *= sc; a.w *= sc;
        out2[q] = Pack4<TL>::make(a);
    }
    for (int i = 4 * m4 + t; i < m; i += kCastThreads) out[i] = LowPrec<TL>::from_float(col[i] * sc);
}

int scale_cast_columns(const float* X, int ldx, int m, int c0, int w, void* Xh, int ldh,
                       int lowp, int* exps, cudaStream_t st) {
    if (w <= 0) return LLS_OK;
    // 16-byte vectors need 16-byte aligned columns in X and 4-element aligned ones in Xh
    const int esz = lowp == 2 ? 1 : 2;
    const int vec = (((uintptr_t)X & 15) == 0) && (ldx % 4 == 0) && (((uintptr_t)Xh & (4 * esz - 1)) == 0) &&
                    (ldh % 4 == 0);
    if (lowp == 0)
        scale_cast_kernel<__half><<<w, kCastThreads, 0, st>>>(X, ldx, m, c0, (__half*)Xh, ldh, 1, exps, vec);
    else if (lowp == 1)
        scale_cast_kernel<__nv_bfloat16><<<w, kCastThreads, 0, st>>>(X, ldx, m, c0, (__nv_bfloat16*)Xh, ldh, 0, exps, vec);
    else if (lowp == 2)
        scale_cast_kernel<__nv_fp8_e4m3><<<w, kCastThreads, 0, st>>>(X, ldx, m, c0, (__nv_fp8_e4m3*)Xh, ldh, 2, exps, vec);
    else
        return LLS_ERR_UNSUPPORTED;
    LLS_LAUNCH_CHECK("scale_cast", st);
    return LLS_OK;
}

// Row-major copy of columns [c0, c0 + w) of a column-major 8-bit matrix (the K-major A operand
// of the FP8 update product): T[i * ldt + c] = X[i + c * ldx]. One thread per row; a warp
// reads 32 consecutive bytes of each column and writes 16-byte row segments when aligned.
__global__ void __launch_bounds__(256)
rowmajor_copy8_kernel(const uint8_t* __restrict__ X, int ldx, int m, int c0, int w, uint8_t* __restrict__ T,
                      int ldt) {
    const int i = blockIdx.x * 256 + threadIdx.x;
    if (i >= m) return;
    uint8_t* row = T + (size_t)i * ldt + c0;
    int c = 0;
    if (((c0 | ldt) & 15) == 0) {
        for (; c + 16 <= w; c += 16) {
            uint32_t wd[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                uint32_t v = 0;
#pragma unroll
                for (int b = 0; b < 4; ++b) v |= (uint32_t)X[(size_t)i + (size_t)(c0 + c + 4 * q + b) * ldx] << (8 * b);
                wd[q] = v;
            }
            *reinterpret_cast<uint4*>(row + c) = make_uint4(wd[0], wd[1], wd[2], wd[3]);
        }
    }
    for (; c < w; ++c) row[c] = X[(size_t)i + (size_t)(c0 + c) * ldx];
}

int rowmajor_copy8(const void* X, int ldx, int m, int c0, int w, void* T, int ldt, cudaStream_t st) {
    if (w <= 0 || m <= 0) return LLS_OK;
    rowmajor_copy8_kernel<<<ceil_div(m, 256), 256, 0, st>>>((const uint8_t*)X, ldx, m, c0, w, (uint8_t*)T, ldt);
    LLS_LAUNCH_CHECK("rowmajor_copy8", st);
    return LLS_OK;
}

}  // namespace lls
