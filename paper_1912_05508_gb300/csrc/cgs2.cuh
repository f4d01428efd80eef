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

// The same butterfly with max instead of sum: lane L ends with the warp-wide maximum of value
// index (L mod S), S a power of two <= 32.
template <int S>
__device__ __forceinline__ float warp_transpose_max(float (&x)[S]) {
    static_assert(S >= 1 && S <= 32 && (S & (S - 1)) == 0, "one power-of-two chunk of at most 32 values");
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = S / 2; o >= 1; o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < o; ++i) {
            const float send = up ? x[i] : x[i + o];
            const float keep = up ? x[i + o] : x[i];
            x[i] = fmaxf(keep, __shfl_xor_sync(kFullMask, send, o));
        }
    }
    float r = x[0];
#pragma unroll
    for (int o = S; o < 32; o <<= 1) r = fmaxf(r, __shfl_xor_sync(kFullMask, r, o));
    return r;
}

// Reduction scratch: two alternating buffers, each with room for two vectors of 32 per warp.
constexpr int kRedStride = 2 * kPanelWarps * 32;
constexpr int kRedFloats = 2 * kRedStride;

// Block-wide sum of S values (index j valid for j < S); returns, in every lane L, the block
// total of index (L mod S). red: kRedFloats floats; the two halves alternate with `parity`,
// so one barrier per reduction suffices.
template <int S>
__device__ __forceinline__ float block_reduce_vec(float (&x)[S], float* red, int& parity) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float w = warp_transpose_reduce<S>(x);
    float* rb = red + parity * kRedStride;
    parity ^= 1;
    rb[warp * 32 + lane] = w;
    __syncthreads();
    float t = 0.f;
#pragma unroll
    for (int q = 0; q < kPanelWarps; ++q) t += rb[q * 32 + (lane % S)];
    return t;
}

// Two independent block-wide sums behind one barrier.
template <int S>
__device__ __forceinline__ void block_reduce_two(float (&x)[S], float (&y)[S], float* red, int& parity,
                                                 float& ox, float& oy) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float wx = warp_transpose_reduce<S>(x);
    const float wy = warp_transpose_reduce<S>(y);
    float* rb = red + parity * kRedStride;
    parity ^= 1;
    rb[warp * 32 + lane] = wx;
    rb[(kPanelWarps + warp) * 32 + lane] = wy;
    __syncthreads();
    float tx = 0.f, ty = 0.f;
#pragma unroll
    for (int q = 0; q < kPanelWarps; ++q) {
        tx += rb[q * 32 + (lane % S)];
        ty += rb[(kPanelWarps + q) * 32 + (lane % S)];
    }
    ox = tx;
    oy = ty;
}

// CGS2 on the register-resident block v (see file comment), one column per loop trip, with
// ONE block-wide reduction per column: the second projection of column k and the first
// projection of column k+1 share it (the lagged form of CGS2). At step k the reduction gives
//   h2 = Q_<k^T a_k',  nn = ||a_k'||^2,  g = Q_<k^T a_{k+1},  c = a_k'^T a_{k+1},
// where a_k' is column k after its first projection. Then
//   a_k'' = a_k' - Q_<k h2,  R_kk^2 = nn - ||h2||^2 (reduced directly if the second pass
//   removed more than 3/4 of the norm),  q_k = a_k'' / R_kk,  R_<k,k = h1 + h2,
// and column k+1's first projection uses g for q_<k and, for q_k,
//   q_k^T a_{k+1} = (c - h2^T g) / R_kk
// (exact in exact arithmetic, since a_k'' = a_k' - Q_<k h2). Column k+1 then gets its own
// full second projection against q_0..q_k at step k+1, so every column is orthogonalised
// twice, as in CGS2. In exact arithmetic Q and R equal those of CGS2.
// Register layout: the block is kept rotated so that every register index is a compile-time
// constant: at step k the column being finished is at position 0, the next raw columns
// follow, and q_0..q_{k-1} occupy positions B-k..B-1 (q_j at B-k+j). After normalising, the
// block is rotated left by one, which appends q_k at position B-1. After b steps q_j is at
// B-b+j. Rs (32 x 33, row-major) receives R.
// CGS2 on the register-resident block v (see file comment), one column per loop trip, with
// ONE block-wide reduction per column: the second projection of column k and the first
// projection of column k+1 share it (the lagged form of CGS2). At step k the reduction gives
//   h2 = Q_<k^T a_k',  nn = ||a_k'||^2,  g = Q_<k^T a_{k+1},  c = a_k'^T a_{k+1},
// where a_k' is column k after its first projection. Then
//   a_k'' = a_k' - Q_<k h2,  R_kk^2 = nn - ||h2||^2 (reduced directly if the second pass
//   removed more than 3/4 of the norm),  q_k = a_k'' / R_kk,  R_<k,k = h1 + h2,
// and column k+1's first projection uses g for q_<k and, for q_k,
//   q_k^T a_{k+1} = (c - h2^T g) / R_kk
// (exact in exact arithmetic, since a_k'' = a_k' - Q_<k h2). Column k+1 then gets its own
// full second projection against q_0..q_k at step k+1, so every column is orthogonalised
// twice, as in CGS2. In exact arithmetic Q and R equal those of CGS2.
// Register layout: the block is kept rotated so that every register index is a compile-time
// constant: at step k the column being finished is at position 0, the next raw columns
// follow, and q_0..q_{k-1} occupy positions B-k..B-1 (q_j at B-k+j). After normalising, the
// block is rotated left by one, which appends q_k at position B-1. After b steps q_j is at
// B-b+j. Rs (32 x 33, row-major) receives R.
template <int B>
__device__ void cgs2_block(float (&v)[kRPT][B], int b, float* red, float* Rs) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int parity = 0;
    float h1 = 0.f;   // lane p (a q position): first-pass coefficient of the current column
#pragma unroll 1
    for (int k = 0; k < b; ++k) {
        const int qs = B - k;              // first position holding a finished q
        const bool next = k + 1 < b;       // column k+1 exists (then position 1 is raw, qs >= 2)
        float x1[B], x2[B];
#pragma unroll
        for (int j = 0; j < B; ++j) {
            float s1 = 0.f, s2 = 0.f;
#pragma unroll
            for (int r = 0; r < kRPT; ++r) {
                s1 = fmaf(v[r][j], v[r][0], s1);
                s2 = fmaf(v[r][j], v[r][1 < B ? 1 : 0], s2);
            }
            const bool use = j == 0 || j >= qs;
            x1[j] = use ? s1 : 0.f;
            x2[j] = (use && next) ? s2 : 0.f;
        }
        float o1, o2;
        block_reduce_two<B>(x1, x2, red, parity, o1, o2);
        const float nn = __shfl_sync(kFullMask, o1, 0);
        const float c = __shfl_sync(kFullMask, o2, 0);
        float acc[kRPT], nxt[kRPT];
#pragma unroll
        for (int r = 0; r < kRPT; ++r) { acc[r] = v[r][0]; nxt[r] = v[r][1 < B ? 1 : 0]; }
        float hh = 0.f, hg = 0.f;
#pragma unroll
        for (int j = 1; j < B; ++j) {
            const bool isq = j >= qs;
            const float hj = isq ? __shfl_sync(kFullMask, o1, j) : 0.f;
            const float gj = (isq && next) ? __shfl_sync(kFullMask, o2, j) : 0.f;
            hh = fmaf(hj, hj, hh);
            hg = fmaf(hj, gj, hg);
#pragma unroll
            for (int r = 0; r < kRPT; ++r) {
                acc[r] = fmaf(-v[r][j], hj, acc[r]);
                nxt[r] = fmaf(-v[r][j], gj, nxt[r]);
            }
        }
        float normsq = nn - hh;
        if (!(normsq >= 0.25f * nn)) {     // the second pass removed a large part: reduce directly
            float d[1];
            d[0] = 0.f;
#pragma unroll
            for (int r = 0; r < kRPT; ++r) d[0] = fmaf(acc[r], acc[r], d[0]);
            normsq = block_reduce_vec<1>(d, red, parity);
        }
        const float nrm = sqrtf(fmaxf(normsq, 0.f));
        const float inv = nrm > 0.f ? 1.f / nrm : 0.f;
        const float gq = next ? (c - hg) * inv : 0.f;     // q_k^T a_{k+1}
        if (warp == 0) {
            if (lane < B && lane >= qs) Rs[(lane - qs) * 33 + k] = h1 + o1;
            if (lane == 0) Rs[k * 33 + k] = nrm;
        }
        // next step's first-pass coefficients, re-indexed to the rotated positions
        const float sh = __shfl_sync(kFullMask, o2, (lane + 1) & 31);
        h1 = (lane >= qs - 1 && lane < B - 1) ? sh : (lane == B - 1 ? gq : 0.f);
#pragma unroll
        for (int r = 0; r < kRPT; ++r) {
            const float q = acc[r] * inv;
            const float a1 = fmaf(-q, gq, nxt[r]);
#pragma unroll
            for (int j = 0; j < B - 1; ++j) v[r][j] = (j == 0) ? a1 : v[r][j + 1];
            v[r][B - 1] = q;
        }
    }
    __syncthreads();   // Rs complete
}


}  // namespace lls
