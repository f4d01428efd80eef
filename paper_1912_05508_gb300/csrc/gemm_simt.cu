// FP32-accumulating GEMMs on the CUDA cores (SIMT), column-major.
//
// Used for (a) the FP32 reference precision of the recursion's products (no input
// rounding), (b) the R^{-1} recursion M12 = -M11 R12 M22 of the preconditioner set-up,
// and (c) the split-K reduction / epilogues shared with the tensor-core kernels.
#include "common.cuh"
#include "kernels.cuh"

namespace lls {

constexpr int kSB = 64;      // output tile (square)
constexpr int kSK = 16;      // K step
constexpr int kSThreads = 256;

enum SimtEpi { EPI_PARTIAL = 0, EPI_AXPBY = 1, EPI_UPDATE = 2 };

// op(A)[i,k] = TA ? A[k + i*lda] : A[i + k*lda];  op(B)[k,j] = TB ? B[j + k*ldb] : B[k + j*ldb]
template <typename TIA, typename TIB, bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(kSThreads)
gemm_simt_kernel(int M, int N, int K, int kchunk, const TIA* __restrict__ A, int lda,
                 const TIB* __restrict__ B, int ldb, float* __restrict__ C, int ldc,
                 float alpha, float beta, const int* __restrict__ fexp) {
    __shared__ float As[kSK][kSB + 4];
    __shared__ float Bs[kSK][kSB + 4];
    const int t = threadIdx.x;
    const int i0 = blockIdx.x * kSB, j0 = blockIdx.y * kSB;
    const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
    const int ti = (t % 16) * 4, tj = (t / 16) * 4;
    float acc[4][4] = {};
    for (int k0 = kb; k0 < ke; k0 += kSK) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            int idx = t + r * kSThreads;            // 0..1023
            int ii, kk;
            if (TA) { kk = idx % kSK; ii = idx / kSK; } else { ii = idx % kSB; kk = idx / kSB; }
            int gi = i0 + ii, gk = k0 + kk;
            float v = 0.f;
            if (gi < M && gk < ke)
                v = LowPrec<TIA>::to_float(TA ? A[(size_t)gk + (size_t)gi * lda] : A[(size_t)gi + (size_t)gk * lda]);
            As[kk][ii] = v;
            int jj;
            if (TB) { jj = idx % kSB; kk = idx / kSB; } else { kk = idx % kSK; jj = idx / kSK; }
            int gj = j0 + jj;
            gk = k0 + kk;
            float w = 0.f;
            if (gj < N && gk < ke)
                w = LowPrec<TIB>::to_float(TB ? B[(size_t)gj + (size_t)gk * ldb] : B[(size_t)gk + (size_t)gj * ldb]);
            Bs[kk][jj] = w;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kSK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) { a[u] = As[kk][ti + u]; b[u] = Bs[kk][tj + u]; }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        int j = j0 + tj + v;
        if (j >= N) continue;
        float fs = (EPI == EPI_UPDATE && fexp) ? pow2f(-fexp[j]) : 1.f;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            int i = i0 + ti + u;
            if (i >= M) continue;
            if (EPI == EPI_PARTIAL) {
                C[(size_t)blockIdx.z * M * N + (size_t)i + (size_t)j * M] = acc[u][v];
            } else if (EPI == EPI_AXPBY) {
                size_t idx = (size_t)i + (size_t)j * ldc;
                C[idx] = beta == 0.f ? alpha * acc[u][v] : fmaf(alpha, acc[u][v], beta * C[idx]);
            } else {
                size_t idx = (size_t)i + (size_t)j * ldc;
                C[idx] = C[idx] - acc[u][v] * fs;
            }
        }
    }
}

int sgemm(bool ta, bool tb, int M, int N, int K, float alpha, const float* A, int lda,
          const float* B, int ldb, float beta, float* C, int ldc, cudaStream_t st) {
    if (M <= 0 || N <= 0) return LLS_OK;
    dim3 grid(ceil_div(M, kSB), ceil_div(N, kSB), 1);
    int kc = K > 0 ? K : 1;
#define LLS_SG(TAv, TBv) gemm_simt_kernel<float, float, TAv, TBv, EPI_AXPBY><<<grid, kSThreads, 0, st>>>(M, N, K, kc, A, lda, B, ldb, C, ldc, alpha, beta, nullptr)
    if (!ta && !tb) LLS_SG(false, false);
    else if (ta && !tb) LLS_SG(true, false);
    else if (!ta && tb) LLS_SG(false, true);
    else LLS_SG(true, true);
#undef LLS_SG
    LLS_LAUNCH_CHECK("sgemm", st);
    return LLS_OK;
}

// ---------------------------------------------------------------------------------------
// Split-K reduction and epilogue of the projection R12 = Q1^T A2 (the projection step of Alg. 2):
// R12[i, j] = (sum_s part[s][i, j]) * 2^-e_j in a fixed order, stored in FP32; then the
// column exponent f_j of R12 and R12l = round(R12 * 2^f_j) for the update product.
// One CTA per column j. When the product kernel before it gave up a bounded wait (err set),
// its partial sums are incomplete: the column is then written as NaN (R12, R12l) with f_j = 0,
// so the failure shows in the caller's outputs and in anything computed from them.
// ---------------------------------------------------------------------------------------
template <typename TL>
__global__ void __launch_bounds__(256)
proj_reduce_kernel(const float* __restrict__ part, int splits, int w1, int w2,
                   const int* __restrict__ e, const int* __restrict__ sq, float* __restrict__ R12, int ldr,
                   TL* __restrict__ R12l, int ldrl, int* __restrict__ f, int kind, const int* __restrict__ err) {
    // Threads split as (row slot i0 < rp) x (split group g < G): group g sums splits
    // g, g + G, ... in that order (sixteen loads issued per trip before they are added); the
    // groups are then added in order g = 0, 1, ..., so the result does not depend on timing.
    __shared__ float s_part[256];
    __shared__ float s_red[8];
    __shared__ int s_f;
    const int j = blockIdx.x;
    if (err && *(volatile const int*)err != DEV_OK) {
        for (int i = threadIdx.x; i < w1; i += 256) {
            R12[(size_t)i + (size_t)j * ldr] = __int_as_float(0x7fc00000);
            if (R12l) R12l[(size_t)i + (size_t)j * ldrl] = LowPrec<TL>::from_float(__int_as_float(0x7fc00000));
        }
        if (threadIdx.x == 0 && f) f[j] = 0;
        return;
    }
    const float se = e ? pow2f(-e[j]) : 1.f;
    const size_t plane = (size_t)w1 * w2;
    int rp = 1;
    while (rp < w1 && rp < 256) rp <<= 1;
    const int G = 256 / rp;
    const int t = threadIdx.x, i0 = t % rp, g = t / rp;
    float mx = 0.f;
    for (int ib = 0; ib < w1; ib += rp) {
        const int i = ib + i0;
        float s = 0.f;
        if (i < w1) {
            const float* p = part + (size_t)i + (size_t)j * w1;
            int z = g;
            for (; z + 15 * G < splits; z += 16 * G) {
                float x[16];
#pragma unroll
                for (int u = 0; u < 16; ++u) x[u] = __ldg(p + (size_t)(z + u * G) * plane);
#pragma unroll
                for (int u = 0; u < 16; ++u) s += x[u];
            }
            for (; z + 3 * G < splits; z += 4 * G) {
                const float a = __ldg(p + (size_t)z * plane), b = __ldg(p + (size_t)(z + G) * plane);
                const float c = __ldg(p + (size_t)(z + 2 * G) * plane), d = __ldg(p + (size_t)(z + 3 * G) * plane);
                s += a; s += b; s += c; s += d;
            }
            for (; z < splits; z += G) s += __ldg(p + (size_t)z * plane);
        }
        if (G > 1) {
            __syncthreads();
            s_part[t] = s;
            __syncthreads();
            if (g == 0) {
                for (int q = 1; q < G; ++q) s += s_part[q * rp + i0];
            }
        }
        if (g == 0 && i < w1) {
            // FP8: Q1 column i was scaled by 2^sq_i, so R12 row i is unscaled by it, and the
            // update operand carries it once more (Q1 R12 = (Q1 2^sq) (2^-sq R12))
            const float rs = sq ? pow2f(-sq[i]) : 1.f;
            s *= se * rs;
            R12[(size_t)i + (size_t)j * ldr] = s;
            mx = fmaxf(mx, fabsf(s * rs));
        }
    }
    if (!R12l) return;
    mx = warp_max_f(mx);
    if ((t & 31) == 0) s_red[t >> 5] = mx;
    __syncthreads();
    if (t == 0) {
        float tm = 0.f;
        for (int w = 0; w < 8; ++w) tm = fmaxf(tm, s_red[w]);
        s_f = scale_exponent(kind, tm);
        f[j] = s_f;
    }
    __syncthreads();
    const float sc = pow2f(s_f);
    for (int i = t; i < w1; i += 256) {
        const float rs = sq ? pow2f(-sq[i]) : 1.f;
        R12l[(size_t)i + (size_t)j * ldrl] = LowPrec<TL>::from_float(R12[(size_t)i + (size_t)j * ldr] * rs * sc);
    }
}

int proj_reduce(const float* part, int splits, int w1, int w2, const int* e, const int* sq, float* R12, int ldr,
                void* R12l, int ldrl, int* f, int lowp, cudaStream_t st, const int* err) {
    if (lowp == 0)
        proj_reduce_kernel<__half><<<w2, 256, 0, st>>>(part, splits, w1, w2, e, nullptr, R12, ldr, (__half*)R12l, ldrl, f, 1,
                                                       err);
    else if (lowp == 1)
        proj_reduce_kernel<__nv_bfloat16><<<w2, 256, 0, st>>>(part, splits, w1, w2, e, nullptr, R12, ldr,
                                                              (__nv_bfloat16*)R12l, ldrl, f, 0, err);
    else if (lowp == 2)
        proj_reduce_kernel<__nv_fp8_e4m3><<<w2, 256, 0, st>>>(part, splits, w1, w2, e, sq, R12, ldr,
                                                              (__nv_fp8_e4m3*)R12l, ldrl, f, 2, err);
    else
        proj_reduce_kernel<float><<<w2, 256, 0, st>>>(part, splits, w1, w2, nullptr, nullptr, R12, ldr, (float*)nullptr,
                                                      0, f, 0, err);
    LLS_LAUNCH_CHECK("proj_reduce", st);
    return LLS_OK;
}

// Number of K splits for a projection of M = w1, N = w2, K = m: enough CTAs to fill the GPU.
int proj_splits_simt(int m, int w1, int w2) {
    int tiles = ceil_div(w1, kSB) * ceil_div(w2, kSB);
    int want = ceil_div(4 * 152, tiles);
    int maxs = ceil_div(m, 512);
    int s = want < maxs ? want : maxs;
    return s < 1 ? 1 : s;
}

// SIMT projection / update for the FP32 reference precision (inputs are the FP32 matrices).
int simt_projection_f32(const float* Q1, const float* A2, int ldw, int m, int w1, int w2,
                        float* R12, int ldr, float* part, cudaStream_t st) {
    int splits = proj_splits_simt(m, w1, w2);
    int kc = align_up((size_t)ceil_div(m, splits), kSK);
    splits = ceil_div(m, kc);
    dim3 grid(ceil_div(w1, kSB), ceil_div(w2, kSB), splits);
    gemm_simt_kernel<float, float, true, false, EPI_PARTIAL><<<grid, kSThreads, 0, st>>>(
        w1, w2, m, kc, Q1, ldw, A2, ldw, part, 0, 1.f, 0.f, nullptr);
    LLS_LAUNCH_CHECK("simt_proj_f32", st);
    return proj_reduce(part, splits, w1, w2, nullptr, nullptr, R12, ldr, nullptr, 0, nullptr, 3, st, nullptr);
}

int simt_update_f32(const float* Q1, int ldw, const float* R12, int ldr, float* A2, int m, int w1,
                    int w2, cudaStream_t st) {
    dim3 grid(ceil_div(m, kSB), ceil_div(w2, kSB), 1);
    gemm_simt_kernel<float, float, false, false, EPI_UPDATE><<<grid, kSThreads, 0, st>>>(
        m, w2, w1, w1, Q1, ldw, R12, ldr, A2, ldw, 1.f, 0.f, nullptr);
    LLS_LAUNCH_CHECK("simt_proj_f32", st);
    return LLS_OK;
}

// Low-precision operands on the CUDA cores (products of FP16/BF16 values are exact in FP32,
// accumulation in FP32 as on the tensor cores).
template <typename TL>
static int simt_lowp_projection(const ProjCall& c, cudaStream_t st) {
    int splits = proj_splits_simt(c.m, c.w1, c.w2);
    int kc = align_up((size_t)ceil_div(c.m, splits), kSK);
    splits = ceil_div(c.m, kc);
    if ((size_t)splits * c.w1 * c.w2 > c.part_floats) return LLS_ERR_WORKSPACE;
    dim3 grid(ceil_div(c.w1, kSB), ceil_div(c.w2, kSB), splits);
    gemm_simt_kernel<TL, TL, true, false, EPI_PARTIAL><<<grid, kSThreads, 0, st>>>(
        c.w1, c.w2, c.m, kc, (const TL*)c.Q1l, c.ldh, (const TL*)c.A2l, c.ldh, c.part, 0, 1.f, 0.f, nullptr);
    LLS_LAUNCH_CHECK("simt_upd_f32", st);
    return proj_reduce(c.part, splits, c.w1, c.w2, c.e, c.sq, c.R12, c.ldr, c.R12l, c.ldrl, c.f, c.lowp, st, nullptr);
}

template <typename TL>
static int simt_lowp_update(const UpdCall& c, cudaStream_t st) {
    dim3 grid(ceil_div(c.m, kSB), ceil_div(c.w2, kSB), 1);
    gemm_simt_kernel<TL, TL, false, false, EPI_UPDATE><<<grid, kSThreads, 0, st>>>(
        c.m, c.w2, c.w1, c.w1, (const TL*)c.Q1l, c.ldh, (const TL*)c.R12l, c.ldrl, c.A2, c.ldw, 1.f, 0.f, c.f);
    LLS_LAUNCH_CHECK("simt_proj_lowp", st);
    return LLS_OK;
}

int simt_projection_lowp(const ProjCall& c, cudaStream_t st) {
    return c.lowp == 0 ? simt_lowp_projection<__half>(c, st) : simt_lowp_projection<__nv_bfloat16>(c, st);
}
int simt_update_lowp(const UpdCall& c, cudaStream_t st) {
    return c.lowp == 0 ? simt_lowp_update<__half>(c, st) : simt_lowp_update<__nv_bfloat16>(c, st);
}

size_t simt_partial_floats(int m, int w1, int w2) {
    int splits = proj_splits_simt(m, w1, w2);
    int kc = align_up((size_t)ceil_div(m, splits), kSK);
    splits = ceil_div(m, kc);
    return (size_t)splits * w1 * w2;
}

}  // namespace lls
