// CGS2 factorization of a register-resident block of up to 1024 x 32 (shared by the CAQR
// panel kernels and the batched solver). 256 threads, 4 rows per thread.
#pragma once
#include "common.cuh"

namespace lls {

constexpr int kPanelThreads = 256;
constexpr int kPanelWarps = kPanelThreads / 32;
constexpr int kRPT = 4;                               // rows per thread
constexpr int kNodeRows = kPanelThreads * kRPT;       // 1024-row blocks and tree nodes

__host__ __device__ constexpr int pow2ceil(int x) { return x <= 1 ? 1 : 2 * pow2ceil((x + 1) / 2); }

// Butterfly transpose-reduction of S values held by every lane: afterwards lane L holds the
// warp-wide sum of value index (L mod S).
template <int S>
__device__ __forceinline__ float warp_transpose_reduce(float (&x)[S]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = S / 2; o >= 1; o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < o; ++i) {
            const float send = up ? x[i] : x[i + o];
            const float keep = up ? x[i + o] : x[i];
            x[i] = keep + __shfl_xor_sync(kFullMask, send, o);
        }
    }
    float r = x[0];
#pragma unroll
    for (int o = S; o < 32; o <<= 1) r += __shfl_xor_sync(kFullMask, r, o);
    return r;
}

// Block-wide sum of S values (index j valid for j < S); returns, in every lane L, the block
// total of index (L mod S). red: two buffers of kPanelWarps x 32 floats, alternated.
template <int S>
__device__ __forceinline__ float block_reduce_vec(float (&x)[S], float* red, int& parity) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float w = warp_transpose_reduce<S>(x);
    float* rb = red + parity * (kPanelWarps * 32);
    parity ^= 1;
    rb[warp * 32 + lane] = w;
    __syncthreads();
    float t = 0.f;
#pragma unroll
    for (int q = 0; q < kPanelWarps; ++q) t += rb[q * 32 + (lane % S)];
    return t;
}

// CGS2 on the register-resident block v (see file comment), one column per loop trip.
// The block is kept rotated so that every register index is a compile-time constant: at step
// k the column being orthogonalised is at position 0, the raw columns a_{k+1..} follow, and
// q_0..q_{k-1} occupy positions B-k..B-1 (q_j at B-k+j). After normalising, the block is
// rotated left by one, which appends q_k at position B-1. After b steps q_j is at B-b+j.
// Rs (32 x 33, row-major) receives R.
template <int B>
__device__ void cgs2_block(float (&v)[kRPT][B], int b, float* red, float* Rs) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int parity = 0;
#pragma unroll 1
    for (int k = 0; k < b; ++k) {
        const int qs = B - k;              // first position holding a finished q
        float hacc = 0.f;                  // lane p (p >= qs): R[p - qs][k]
        if (k > 0) {
            float p1[B];
            p1[0] = 0.f;
#pragma unroll
            for (int j = 1; j < B; ++j) {
                float s = 0.f;
#pragma unroll
                for (int r = 0; r < kRPT; ++r) s = fmaf(v[r][j], v[r][0], s);
                p1[j] = j >= qs ? s : 0.f;
            }
            const float h = block_reduce_vec<B>(p1, red, parity);
            hacc = h;
            float acc[kRPT];
#pragma unroll
            for (int r = 0; r < kRPT; ++r) acc[r] = v[r][0];
#pragma unroll
            for (int j = 1; j < B; ++j) {
                const float hj = j >= qs ? __shfl_sync(kFullMask, h, j) : 0.f;
#pragma unroll
                for (int r = 0; r < kRPT; ++r) acc[r] = fmaf(-v[r][j], hj, acc[r]);
            }
#pragma unroll
            for (int r = 0; r < kRPT; ++r) v[r][0] = acc[r];
        }
        // second pass together with ||a_k||^2 at index 0
        float p2[B];
#pragma unroll
        for (int j = 0; j < B; ++j) {
            float s = 0.f;
#pragma unroll
            for (int r = 0; r < kRPT; ++r) s = fmaf(v[r][j], v[r][0], s);
            p2[j] = (j == 0 || j >= qs) ? s : 0.f;
        }
        const float h2 = block_reduce_vec<B>(p2, red, parity);
        const float nn = __shfl_sync(kFullMask, h2, 0);
        float normsq = nn;
        if (k > 0) {
            float acc[kRPT];
#pragma unroll
            for (int r = 0; r < kRPT; ++r) acc[r] = v[r][0];
            float hh = 0.f;
#pragma unroll
            for (int j = 1; j < B; ++j) {
                const float hj = j >= qs ? __shfl_sync(kFullMask, h2, j) : 0.f;
                hh = fmaf(hj, hj, hh);
#pragma unroll
                for (int r = 0; r < kRPT; ++r) acc[r] = fmaf(-v[r][j], hj, acc[r]);
            }
#pragma unroll
            for (int r = 0; r < kRPT; ++r) v[r][0] = acc[r];
            hacc += h2;
            normsq = nn - hh;
            if (!(normsq >= 0.25f * nn)) {     // the second pass removed a large part: reduce directly
                float d[1];
                d[0] = 0.f;
#pragma unroll
                for (int r = 0; r < kRPT; ++r) d[0] = fmaf(v[r][0], v[r][0], d[0]);
                normsq = block_reduce_vec<1>(d, red, parity);
            }
        }
        const float nrm = sqrtf(fmaxf(normsq, 0.f));
        const float inv = nrm > 0.f ? 1.f / nrm : 0.f;
        if (warp == 0) {
            if (lane < B && lane >= qs) Rs[(lane - qs) * 33 + k] = hacc;
            if (lane == 0) Rs[k * 33 + k] = nrm;
        }
#pragma unroll
        for (int r = 0; r < kRPT; ++r) {
            const float q = v[r][0] * inv;
#pragma unroll
            for (int j = 0; j < B - 1; ++j) v[r][j] = v[r][j + 1];
            v[r][B - 1] = q;
        }
    }
    __syncthreads();   // Rs complete
}


}  // namespace lls
