// R-preconditioned CGLS (Alg. 5, Sec. 3.2.3) as one persistent cooperative kernel.
//
// Products with A: the default engine makes two passes over A per iteration: q = A t as
// per-column-chunk partial sums over 1024-row tiles (columns in increasing order over the
// grid's waves), then, after the r update, u = A^T r as per-row-chunk partial sums, each CTA
// staying on one row chunk and taking groups of 8 columns from the last column down; every
// partial is summed in a fixed order. An optional one-pass engine (LLS_KRYLOV=onepass, CGLS with n <= 4096) streams a
// row-block copy of A in 4-row blocks through a double-buffered shared-memory ring
// (cp.async); for each block the CTA forms q = A t on those rows (block-wide reduction),
// then accumulates A^T q and A^T r for its columns from the same shared-memory copy, and
// after the pass u = A^T r_new = A^T r - alpha A^T q.
//
// The loop of Alg. 5, with the slips of the printed listing read as: step length
// alpha = gamma / delta, solution update x += alpha R^{-1} p, and the preconditioned
// start s = R^{-T} A^T r:
//   t = R^{-1} p;  q = A t;  delta = ||q||^2;  alpha = gamma / delta
//   x += alpha t;  r -= alpha q;  s = R^{-T} A^T r;  gamma' = ||s||^2
//   beta = gamma' / gamma;  p = s + beta p
// R^{-1} is applied as a product with the explicit inverse M (and M^T), formed once.
//
// Precision: A is FP32 and exact; every product with A or M accumulates with the
// compensated dot product (Ogita-Rump-Oishi Dot2) in double-float, i.e. to about 2^-48
// relative, because GB300's FP64 rate is ~1/70 of its FP32 rate. Vectors are stored FP64.
//
// Stop test (the paper omits it): eta_est = ||s|| / (||A||_F ||x||) <= tol for the FP64
// target (an upper bound, up to the preconditioner's quality, on the Karlson-Walden
// least-squares backward error); ||M||_F ||s|| / ||x|| <= tol for the FP32 target (a
// bound on the relative forward error). Convergence on the recursively updated residual
// is confirmed with a freshly computed b - A x; if that fails the iteration restarts
// from the current x (at most kMaxRestarts times).
//
// All CTAs compute every reduction in the same fixed order, so they take identical
// branch decisions; the grid barriers are bounded (common.cuh) and report a timeout.
#include <stdlib.h>

#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"

namespace lls {

constexpr int kKThreads = 256;
constexpr int kKWarps = kKThreads / 32;
constexpr int kRowTile = 1024;    // rows per A t work item (four rows per thread)
constexpr int kColChunkMin = 48;  // columns per A t work item: chosen per launch in [48, 96]
constexpr int kColChunkMax = 96;  // so that the items fill whole waves of the grid
constexpr int kRowChunkCap = 4096;   // rows of r a CTA stages for the A^T r pass (at least; n when wider)
constexpr int kMaxRestarts = 3;
constexpr int kPrefetchCols = 8;  // L2 prefetch distance of the A passes (columns, or 32-lane steps)
constexpr int kNPart = 4;         // block-partial slots

struct KArgs {
    int m, n, lda;
    const float* A;
    const double* b;
    double* x;
    const float* M;
    const float* Mt;
    double *r, *q, *t, *p, *s, *u, *d, *qpart, *upart, *bpart;
    unsigned* bar;
    int* err;
    double* info;
    const double* anorm2;
    const double* mnorm2;
    double tol;
    int max_iter, target, x_zero;
    int nrt, nck, nrc, ncg;
    int colchunk;                // columns per A t work item
    int at_rows, at_cpr;         // A^T r pass: rows per row chunk, CTAs per row chunk
    double *v1part, *v2part;     // fused engine: per-CTA partial A^T q and A^T r, [grid][n]
    int aligned16;               // A and lda allow 16-byte copies of 4-row column segments
    const float4* At;            // row-block copy of A: At[blk * n + j] = A[4 blk .. 4 blk + 3, j], or null
    float2 *rdf, *tdf, *udf, *pdf;   // double-float copies (hi, lo) of r, t, u, p, written where the
                                     // vectors are produced so no CTA re-splits a whole vector
    int vec_floats;              // floats reserved at the start of dynamic smem for vectors
    double* hist;                // the stop quantity after each iteration (kHistLen entries), or null
    unsigned long long* phases;  // CGLS phase log (kPhaseLen entries), or null
};

// The stop quantity of iteration `it` into the history (block 0, thread 0; the value is the
// same in every CTA).
__device__ __forceinline__ void log_hist(const KArgs& a, int it, double v) {
    if (a.hist && blockIdx.x == 0 && threadIdx.x == 0 && it < kHistLen) a.hist[it] = v;
}

// A non-finite ||b - A x||^2 at the start (a NaN or infinity in b, or in the starting x) is
// reported like a non-finite R: the same value in every CTA, so every CTA returns here.
__device__ __forceinline__ bool finite_start(const KArgs& a, double rn2) {
    if (isfinite(rn2)) return true;
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(a.err, DEV_OK, DEV_SINGULAR);
    return false;
}

extern __shared__ __align__(16) float2 k_dsm[];

__device__ __forceinline__ void stage_vec(const double* __restrict__ v, int len) {
    for (int i = threadIdx.x; i < len; i += kKThreads) {
        float hi, lo;
        split_df(__ldcg(v + i), hi, lo);
        k_dsm[i] = make_float2(hi, lo);
    }
    __syncthreads();
}

// Copy a vector already split into double-float pairs into shared memory. Sixteen loads per
// thread are issued before the first is stored, so a vector of up to 4096 entries costs one
// round trip to L2 instead of one per 256 entries.
__device__ __forceinline__ void stage_df(const float2* __restrict__ v, int len) {
    int i = threadIdx.x;
    for (; i + 15 * kKThreads < len; i += 16 * kKThreads) {
        float2 x[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) x[u] = __ldcg(v + i + u * kKThreads);
#pragma unroll
        for (int u = 0; u < 16; ++u) k_dsm[i + u * kKThreads] = x[u];
    }
    {
        float2 x[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) x[u] = i + u * kKThreads < len ? __ldcg(v + i + u * kKThreads) : float2{};
#pragma unroll
        for (int u = 0; u < 16; ++u)
            if (i + u * kKThreads < len) k_dsm[i + u * kKThreads] = x[u];
    }
    __syncthreads();
}

__device__ __forceinline__ float2 to_df(double v) {
    float2 r;
    split_df(v, r.x, r.y);
    return r;
}

// Sum of one double per thread over the block, written to slot (k, blockIdx.x).
__device__ __forceinline__ void block_partial(double v, double* bpart, int k) {
    __shared__ double sh[kKWarps];
    v = warp_sum_d(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kKWarps; ++w) s += sh[w];
        bpart[(size_t)k * gridDim.x + blockIdx.x] = s;
    }
}

// Fixed-order sum of slot k over all blocks (identical in every CTA). Lane l adds the blocks
// l, l + 32, ... in that order; its first sixteen loads are all issued before the additions.
__device__ __forceinline__ double grid_total(const double* bpart, int k) {
    __shared__ double s_tot;
    if (threadIdx.x < 32) {
        const double* p = bpart + (size_t)k * gridDim.x;
        const int g = (int)gridDim.x;
        double x[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int i = (int)threadIdx.x + 32 * u;
            x[u] = i < g ? __ldcg(p + i) : 0.0;
        }
        double s = 0.0;
#pragma unroll
        for (int u = 0; u < 16; ++u)
            if ((int)threadIdx.x + 32 * u < g) s += x[u];
        for (int i = (int)threadIdx.x + 512; i < g; i += 32) s += __ldcg(p + i);
        s = warp_sum_d(s);
        if (threadIdx.x == 0) s_tot = s;
    }
    __syncthreads();
    double r = s_tot;
    __syncthreads();
    return r;
}

// sum_{k < count} p[k * stride] in a fixed order: eight interleaved accumulators (k mod 8),
// combined pairwise, so eight loads are in flight at a time.
__device__ __forceinline__ double sum_parts(const double* __restrict__ p, int count, size_t stride) {
    double acc[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    int k = 0;
    for (; k + 7 < count; k += 8) {
#pragma unroll
        for (int u = 0; u < 8; ++u) acc[u] += __ldcg(p + (size_t)(k + u) * stride);
    }
#pragma unroll
    for (int u = 0; u < 7; ++u)
        if (k + u < count) acc[u] += __ldcg(p + (size_t)(k + u) * stride);
    return ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
}

// The same sum spread over the four lanes of an aligned lane quad (lane k of the quad takes
// partials k, k + 4, ...); the quad combines its four sums as (s0 + s1) + (s2 + s3), so every
// lane returns the same total in a fixed order. All 32 lanes of the warp must call it;
// `valid` false contributes nothing.
__device__ __forceinline__ double sum_parts_quad(const double* __restrict__ p, int count, size_t stride,
                                                 bool valid) {
    const int sub = threadIdx.x & 3;
    double s0 = 0.0, s1 = 0.0;
    if (valid) {
        int k = sub;
        // the first eight trips' sixteen loads are all issued before the (ordered) additions
        if (k + 60 < count) {
            double x0[8], x1[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                x0[u] = __ldcg(p + (size_t)(k + 8 * u) * stride);
                x1[u] = __ldcg(p + (size_t)(k + 8 * u + 4) * stride);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                s0 += x0[u];
                s1 += x1[u];
            }
            k += 64;
        }
#pragma unroll 4   // loads of later trips issue ahead of the (ordered) additions
        for (; k + 4 < count; k += 8) {
            s0 += __ldcg(p + (size_t)k * stride);
            s1 += __ldcg(p + (size_t)(k + 4) * stride);
        }
        if (k < count) s0 += __ldcg(p + (size_t)k * stride);
    }
    double s = s0 + s1;
    s += __shfl_xor_sync(kFullMask, s, 1);
    s += __shfl_xor_sync(kFullMask, s, 2);
    return s;
}

// out_c = sum over r in [lo(c), hi(c)) of X[r + c n] * v_r, v staged in k_dsm.
// upper: rows 0..c (column c of an upper-triangular X); lower: rows c..n-1.
// One warp per column: 16-byte loads over the aligned body of the column (four compensated
// chains, so four loads are in flight per lane), single elements at the ragged ends, and a
// double-float warp sum joined to FP64 once.
__device__ double tri_gemv(const float* __restrict__ X, int n, bool upper, double* __restrict__ out,
                          float2* __restrict__ outdf = nullptr) {
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * kKWarps + (threadIdx.x >> 5), nw = gridDim.x * kKWarps;
    const bool vec = (n & 3) == 0 && ((uintptr_t)X & 15) == 0;
    double sq = 0.0;
    // columns by decreasing length, the odd rounds in reverse warp order: the warps whose first
    // column is longest take the shortest (or no) second one
    for (int k = 0; (long long)k * nw < n; ++k) {
        const int p = k * nw + ((k & 1) ? nw - 1 - gw : gw);
        if (p >= n) continue;
        const int c = upper ? n - 1 - p : p;
        const int lo = upper ? 0 : c, hi = upper ? c + 1 : n;
        const float* col = X + (size_t)c * n;
        float s0 = 0.f, c0 = 0.f, s1 = 0.f, c1 = 0.f, s2 = 0.f, c2 = 0.f, s3 = 0.f, c3 = 0.f;
        int blo = lo, bhi = lo;                       // aligned body [blo, bhi), multiples of 4
        if (vec) {
            blo = min((lo + 3) & ~3, hi);
            bhi = max(blo, hi & ~3);
            const float4* col4 = reinterpret_cast<const float4*>(col);
            const int qe = bhi / 4;
            int q = blo / 4 + lane;
            // four 16-byte loads per trip (a column of 4096 entries is 8 trips); the next trip's
            // loads are issued before this trip's products, so eight are in flight per lane
            auto trip = [&](const float4& a0, const float4& a1, const float4& a2, const float4& a3, int qq) {
                const float2* v = k_dsm + 4 * qq;
                dot2_step(s0, c0, a0.x, v[0].x, v[0].y);
                dot2_step(s1, c1, a1.x, v[128].x, v[128].y);
                dot2_step(s2, c2, a2.x, v[256].x, v[256].y);
                dot2_step(s3, c3, a3.x, v[384].x, v[384].y);
                dot2_step(s0, c0, a0.y, v[1].x, v[1].y);
                dot2_step(s1, c1, a1.y, v[129].x, v[129].y);
                dot2_step(s2, c2, a2.y, v[257].x, v[257].y);
                dot2_step(s3, c3, a3.y, v[385].x, v[385].y);
                dot2_step(s0, c0, a0.z, v[2].x, v[2].y);
                dot2_step(s1, c1, a1.z, v[130].x, v[130].y);
                dot2_step(s2, c2, a2.z, v[258].x, v[258].y);
                dot2_step(s3, c3, a3.z, v[386].x, v[386].y);
                dot2_step(s0, c0, a0.w, v[3].x, v[3].y);
                dot2_step(s1, c1, a1.w, v[131].x, v[131].y);
                dot2_step(s2, c2, a2.w, v[259].x, v[259].y);
                dot2_step(s3, c3, a3.w, v[387].x, v[387].y);
            };
            if (q + 96 < qe) {
                float4 a0 = __ldg(col4 + q), a1 = __ldg(col4 + q + 32);
                float4 a2 = __ldg(col4 + q + 64), a3 = __ldg(col4 + q + 96);
                for (;;) {
                    const int qn = q + 128;
                    if (qn + 96 < qe) {
                        const float4 b0 = __ldg(col4 + qn), b1 = __ldg(col4 + qn + 32);
                        const float4 b2 = __ldg(col4 + qn + 64), b3 = __ldg(col4 + qn + 96);
                        trip(a0, a1, a2, a3, q);
                        a0 = b0; a1 = b1; a2 = b2; a3 = b3;
                        q = qn;
                    } else {
                        trip(a0, a1, a2, a3, q);
                        q = qn;
                        break;
                    }
                }
            }
            for (; q < qe; q += 32) {
                const float4 a0 = __ldg(col4 + q);
                const float2* v = k_dsm + 4 * q;
                dot2_step(s0, c0, a0.x, v[0].x, v[0].y);
                dot2_step(s0, c0, a0.y, v[1].x, v[1].y);
                dot2_step(s0, c0, a0.z, v[2].x, v[2].y);
                dot2_step(s0, c0, a0.w, v[3].x, v[3].y);
            }
        }
        // ragged ends: [lo, blo) and [bhi, hi) (the whole range when not vectorized)
        {
            const int r = lo + lane;
            if (r < blo) {
                const float2 v = k_dsm[r];
                dot2_step(s1, c1, __ldg(col + r), v.x, v.y);
            }
            for (int r2 = bhi + lane; r2 < hi; r2 += 32) {
                const float2 v = k_dsm[r2];
                dot2_step(s1, c1, __ldg(col + r2), v.x, v.y);
            }
        }
        float t, e;
        two_sum(s0, s1, t, e); s0 = t; c0 = __fadd_rn(__fadd_rn(c0, c1), e);
        two_sum(s2, s3, t, e); s2 = t; c2 = __fadd_rn(__fadd_rn(c2, c3), e);
        two_sum(s0, s2, t, e); s0 = t; c0 = __fadd_rn(__fadd_rn(c0, c2), e);
        warp_sum_df(s0, c0);
        if (lane == 0 && LLS_INB(c >= 0 && c < n)) {
            const double val = join_df(s0, c0);
            out[c] = val;
            if (outdf) outdf[c] = to_df(val);
            sq += val * val;
        }
    }
    return sq;
}

// qpart[cc][i] = sum_{j in chunk cc} A[i, j] * v_j, v staged in k_dsm. Each thread owns 4
// consecutive rows (one 16-byte load per column when A is 16-byte aligned), giving four
// independent compensated accumulation chains.
__device__ void a_times_partials(const KArgs& a) {
    const int items = a.nrt * a.nck;
    for (int it = blockIdx.x; it < items; it += gridDim.x) {
        const int rt = it % a.nrt, cc = it / a.nrt;
        const int i0 = rt * kRowTile + 4 * threadIdx.x;
        if (i0 >= a.m) continue;
        const int j0 = cc * a.colchunk, j1 = min(a.n, j0 + a.colchunk);
        if (!LLS_INB(j0 >= 0 && j1 <= a.n && a.lda >= a.m)) continue;
        const bool full = a.aligned16 && i0 + 4 <= a.m;
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f, c0 = 0.f, c1 = 0.f, c2 = 0.f, c3 = 0.f;
        if (full) {
            const float4* colp = reinterpret_cast<const float4*>(a.A + i0);
            const size_t step = (size_t)a.lda / 4;
#pragma unroll 4
            for (int j = j0; j < j1; ++j) {
                // pull column j + 8 of this thread's rows into L2 (deepens the loads in flight
                // beyond the unrolled register loads)
                if (j + kPrefetchCols < j1)
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(colp + (size_t)(j + kPrefetchCols) * step));
                const float4 v = __ldg(colp + (size_t)j * step);
                const float2 t = k_dsm[j];
                dot2_step(s0, c0, v.x, t.x, t.y);
                dot2_step(s1, c1, v.y, t.x, t.y);
                dot2_step(s2, c2, v.z, t.x, t.y);
                dot2_step(s3, c3, v.w, t.x, t.y);
            }
        } else {
            for (int j = j0; j < j1; ++j) {
                const float* col = a.A + (size_t)j * a.lda + i0;
                const float2 t = k_dsm[j];
                dot2_step(s0, c0, col[0], t.x, t.y);
                if (i0 + 1 < a.m) dot2_step(s1, c1, col[1], t.x, t.y);
                if (i0 + 2 < a.m) dot2_step(s2, c2, col[2], t.x, t.y);
                if (i0 + 3 < a.m) dot2_step(s3, c3, col[3], t.x, t.y);
            }
        }
        if (!LLS_INB(cc < a.nck && i0 < a.m)) continue;
        double* out = a.qpart + (size_t)cc * a.m + i0;
        out[0] = join_df(s0, c0);
        if (i0 + 1 < a.m) out[1] = join_df(s1, c1);
        if (i0 + 2 < a.m) out[2] = join_df(s2, c2);
        if (i0 + 3 < a.m) out[3] = join_df(s3, c3);
    }
}

// upart[rc][j] = sum_{i in row chunk rc} A[i, j] * v_i for v (length m) in global memory.
// The m rows are cut into nrc chunks of at_rows rows; CTA c works on chunk c / at_cpr only, so
// it stages that chunk of v in shared memory once per pass (CTAs from nrc * at_cpr on have no
// work here). A work item is one column per warp: the column group g covers columns
// 8 g .. 8 g + 7. The at_cpr CTAs of a chunk take the groups in interleaved order from the last
// group down (CTA k of the chunk: g = ncg - 1 - k, then g - at_cpr, ...), so at any time the
// grid reads one band of columns, and the pass starts with the columns that the A t pass before
// it (increasing columns) read last and that are still in L2. Each lane reads 4 consecutive
// rows per step.
__device__ void at_times_partials(const KArgs& a, const double* __restrict__ v,
                                  const float2* __restrict__ vdf = nullptr) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int K = a.at_cpr, L = a.at_rows;
    const int k = (int)blockIdx.x % K;
    // one chunk per CTA when the chunks' CTAs fit the grid (the step then passes nrc), else
    // (K = 1) the chunks c, c + grid, ...; uniform across the CTA
    for (int rc = (int)blockIdx.x / K; rc < a.nrc; rc += (int)gridDim.x / K) {
        const int r0 = rc * L, rows = min(a.m - r0, L);
        if (rows <= 0) break;
        __syncthreads();                              // earlier users of k_dsm are done
        if (!LLS_INB(r0 >= 0 && r0 + rows <= a.m && rows <= L && 2 * rows <= a.vec_floats)) break;
        if (vdf) {
            for (int i = threadIdx.x; i < rows; i += kKThreads) k_dsm[i] = __ldcg(vdf + r0 + i);
        } else {
            for (int i = threadIdx.x; i < rows; i += kKThreads) {
                float hi, lo;
                split_df(__ldcg(v + r0 + i), hi, lo);
                k_dsm[i] = make_float2(hi, lo);
            }
        }
        __syncthreads();
        const bool full = a.aligned16 && (rows & 3) == 0;
        const int nq = rows >> 2;
        for (int g = a.ncg - 1 - k; g >= 0; g -= K) {
            const int j = g * kKWarps + warp;
            if (j >= a.n) continue;
            const float* col = a.A + (size_t)j * a.lda + r0;
            float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f, c0 = 0.f, c1 = 0.f, c2 = 0.f, c3 = 0.f;
            if (full) {
                const float4* col4 = reinterpret_cast<const float4*>(col);
#pragma unroll 4
                for (int q = lane; q < nq; q += 32) {
                    if (q + 32 * kPrefetchCols < nq)
                        asm volatile("prefetch.global.L2 [%0];" ::"l"(col4 + q + 32 * kPrefetchCols));
                    const float4 av = __ldg(col4 + q);
                    const float2 w0 = k_dsm[4 * q], w1 = k_dsm[4 * q + 1], w2 = k_dsm[4 * q + 2], w3 = k_dsm[4 * q + 3];
                    dot2_step(s0, c0, av.x, w0.x, w0.y);
                    dot2_step(s1, c1, av.y, w1.x, w1.y);
                    dot2_step(s2, c2, av.z, w2.x, w2.y);
                    dot2_step(s3, c3, av.w, w3.x, w3.y);
                }
                // the start of this warp's next column (4 KB) into L2
                if (g - K >= 0 && (g - K) * kKWarps + warp < a.n && 32 * lane < rows)
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(col - (size_t)K * kKWarps * a.lda + 32 * lane));
            } else {
                for (int i = lane; i < rows; i += 32) {
                    const float2 w = k_dsm[i];
                    dot2_step(s0, c0, __ldg(col + i), w.x, w.y);
                }
            }
            // combine the four chains, then the 32 lanes, in double-float
            float t, e;
            two_sum(s0, s1, t, e); s0 = t; c0 = __fadd_rn(__fadd_rn(c0, c1), e);
            two_sum(s2, s3, t, e); s2 = t; c2 = __fadd_rn(__fadd_rn(c2, c3), e);
            two_sum(s0, s2, t, e); s0 = t; c0 = __fadd_rn(__fadd_rn(c0, c2), e);
            warp_sum_df(s0, c0);
            if (lane == 0 && LLS_INB(rc < a.nrc && j < a.n)) a.upart[(size_t)rc * a.n + j] = join_df(s0, c0);
        }
    }
}

// ---------------------------------------------------------------------------------------
// Fused engine (n <= 256 * NC): one pass over A per call.
// ---------------------------------------------------------------------------------------
constexpr int kRB = 4;   // rows per streamed block

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(uint32_t dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Two compensated dot-product steps at once (dot2_step on each lane of a float2), with the
// paired FP32 instructions of sm_100 and later; every operation rounds to nearest, so the
// error-free transformations hold lane by lane.
__device__ __forceinline__ float2 neg2(float2 v) { return make_float2(-v.x, -v.y); }
__device__ __forceinline__ void dot2_step2(float2& s, float2& c, float2 a, float2 th, float2 tl) {
    const float2 p = __fmul2_rn(a, th);
    float2 e = __ffma2_rn(a, th, neg2(p));           // exact: a*th = p + e
    e = __ffma2_rn(a, tl, e);
    const float2 s2 = __fadd2_rn(s, p);              // TwoSum(s, p) = s2 + e2
    const float2 z = __fadd2_rn(s2, neg2(s));
    const float2 e2 = __fadd2_rn(__fadd2_rn(s, neg2(__fadd2_rn(s2, neg2(z)))), __fadd2_rn(p, neg2(z)));
    s = s2;
    c = __fadd2_rn(c, __fadd2_rn(e, e2));
}

// Row block `blk` (rows 4 blk .. 4 blk + 3) of the CTA's own columns into buffer `dst`,
// stored column by column: dst[j] = (A[i0, j], A[i0+1, j], A[i0+2, j], A[i0+3, j]).
template <int NC>
__device__ __forceinline__ void prefetch_rows(const KArgs& a, int blk, float4* dst) {
    if (a.At) {   // the block is one contiguous run of n 16-byte segments
        const float4* src = a.At + (size_t)blk * a.n;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int j = threadIdx.x + c * kKThreads;
            if (j >= a.n) break;
            cp_async16((uint32_t)__cvta_generic_to_shared(dst + j), src + j);
        }
        cp_async_commit();
        return;
    }
    const int i0 = blk * kRB;
    const bool full = a.aligned16 && (i0 + kRB <= a.m);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const int j = threadIdx.x + c * kKThreads;
        if (j >= a.n) break;
        const float* src = a.A + (size_t)i0 + (size_t)j * a.lda;
        const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst + j);
        if (full) {
            cp_async16(d, src);
        } else {
#pragma unroll
            for (int r = 0; r < kRB; ++r) {
                if (i0 + r < a.m) cp_async4(d + 4 * r, src + r);
                else reinterpret_cast<float*>(dst + j)[r] = 0.f;
            }
        }
    }
    cp_async_commit();
}

// One pass over A. doA: q = A t (written to a.q, ||q||^2 added to dsum by threads 0..3);
// doB1: per-CTA partial of A^T q into v1part; doB2: per-CTA partial of A^T r into v2part.
// Thread t owns columns t + 256 c (c < NC); the products of two columns (A^T) or two rows
// (A t) advance together in the paired FP32 instructions.
template <int NC>
__device__ void fused_pass(const KArgs& a, const double* __restrict__ tvec, const double* __restrict__ rvec,
                           bool doA, bool doB1, bool doB2, double& dsum) {
    constexpr int NP = (NC + 1) / 2;   // column pairs; an odd last pair carries one column
    float4* ring = reinterpret_cast<float4*>(reinterpret_cast<float*>(k_dsm) + a.vec_floats);
    __shared__ float2 s_red[kKWarps][kRB];
    __shared__ float4 s_qr[kRB];   // per row of the block: q and r as double-float (qh, ql, rh, rl)
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const float2 z2 = make_float2(0.f, 0.f);
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float th[NC], tl[NC];
    float2 v1s[NP], v1c[NP], v2s[NP], v2c[NP];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const int j = t + c * kKThreads;
        th[c] = tl[c] = 0.f;
        if (doA && j < a.n) {
            if (tvec == a.t) {
                const float2 d = __ldcg(a.tdf + j);
                th[c] = d.x; tl[c] = d.y;
            } else {
                split_df(__ldcg(tvec + j), th[c], tl[c]);
            }
        }
    }
#pragma unroll
    for (int p = 0; p < NP; ++p) v1s[p] = v1c[p] = v2s[p] = v2c[p] = z2;
    const int nblk = (a.m + kRB - 1) / kRB;
    const int per = (nblk + gridDim.x - 1) / gridDim.x;
    const int b0 = blockIdx.x * per, b1 = min(nblk, b0 + per);
    __syncthreads();   // the ring is free (previous users of dynamic smem are done)
    if (b0 < b1) prefetch_rows<NC>(a, b0, ring);
    int buf = 0;
    for (int blk = b0; blk < b1; ++blk, buf ^= 1) {
        if (blk + 1 < b1) {
            prefetch_rows<NC>(a, blk + 1, ring + (buf ^ 1) * a.n);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const float4* rb = ring + buf * a.n;
        const int i0 = blk * kRB;
        if (doA) {
            float2 s01 = z2, c01 = z2, s23 = z2, c23 = z2;   // rows (0, 1) and (2, 3)
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                const int j = t + c * kKThreads;
                const float4 av = j < a.n ? rb[j] : z4;
                const float2 h2 = make_float2(th[c], th[c]), l2 = make_float2(tl[c], tl[c]);
                dot2_step2(s01, c01, make_float2(av.x, av.y), h2, l2);
                dot2_step2(s23, c23, make_float2(av.z, av.w), h2, l2);
            }
            float qs[kRB] = {s01.x, s01.y, s23.x, s23.y}, qc[kRB] = {c01.x, c01.y, c23.x, c23.y};
#pragma unroll
            for (int r = 0; r < kRB; ++r) {
                warp_sum_df(qs[r], qc[r]);
                if (lane == 0) s_red[warp][r] = make_float2(qs[r], qc[r]);
            }
            __syncthreads();
        }
        // the block's row scalars q_i and r_i, split once (FP64 work is scarce on this GPU)
        if (t < kRB) {
            double v = 0.0;
            if (doA) {
#pragma unroll
                for (int w = 0; w < kKWarps; ++w) v += join_df(s_red[w][t].x, s_red[w][t].y);
                if (i0 + t < a.m) {
                    a.q[i0 + t] = v;
                    dsum += v * v;
                }
            }
            const double rv = (doB2 && i0 + t < a.m) ? __ldcg(rvec + i0 + t) : 0.0;
            float4 o;
            split_df(v, o.x, o.y);
            split_df(rv, o.z, o.w);
            s_qr[t] = o;
        }
        __syncthreads();
        if (doB1 || doB2) {
            float qh[kRB], ql[kRB], rh[kRB], rl[kRB];
#pragma unroll
            for (int r = 0; r < kRB; ++r) {
                const float4 o = s_qr[r];
                qh[r] = o.x; ql[r] = o.y; rh[r] = o.z; rl[r] = o.w;
            }
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const int j0 = t + (2 * p) * kKThreads, j1 = j0 + kKThreads;
                const float4 A0 = j0 < a.n ? rb[j0] : z4;
                const float4 A1 = (2 * p + 1 < NC && j1 < a.n) ? rb[j1] : z4;
                const float2 a2[kRB] = {make_float2(A0.x, A1.x), make_float2(A0.y, A1.y),
                                        make_float2(A0.z, A1.z), make_float2(A0.w, A1.w)};
#pragma unroll
                for (int r = 0; r < kRB; ++r) {
                    if (doB1) dot2_step2(v1s[p], v1c[p], a2[r], make_float2(qh[r], qh[r]), make_float2(ql[r], ql[r]));
                    if (doB2) dot2_step2(v2s[p], v2c[p], a2[r], make_float2(rh[r], rh[r]), make_float2(rl[r], rl[r]));
                }
            }
        }
        __syncthreads();   // this buffer is overwritten by the prefetch two blocks ahead
    }
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const int j0 = t + (2 * p) * kKThreads, j1 = j0 + kKThreads;
        if (j0 < a.n) {
            if (doB1) a.v1part[(size_t)blockIdx.x * a.n + j0] = join_df(v1s[p].x, v1c[p].x);
            if (doB2) a.v2part[(size_t)blockIdx.x * a.n + j0] = join_df(v2s[p].x, v2c[p].x);
        }
        if (2 * p + 1 < NC && j1 < a.n) {
            if (doB1) a.v1part[(size_t)blockIdx.x * a.n + j1] = join_df(v1s[p].y, v1c[p].y);
            if (doB2) a.v2part[(size_t)blockIdx.x * a.n + j1] = join_df(v2s[p].y, v2c[p].y);
        }
    }
}

// u_j = sum_cta v2part[cta][j] - alpha * sum_cta v1part[cta][j], fixed order; returns the
// thread's part of ||u||^2.
__device__ double reduce_u(const KArgs& a, double alpha, bool use_v1, int gtid, int gthreads) {
    double sq = 0.0;
    for (int j = gtid; j < a.n; j += gthreads) {
        double s2 = 0.0, s1 = 0.0;
        for (int c = 0; c < (int)gridDim.x; ++c) {
            s2 += __ldcg(a.v2part + (size_t)c * a.n + j);
            if (use_v1) s1 += __ldcg(a.v1part + (size_t)c * a.n + j);
        }
        const double v = use_v1 ? s2 - alpha * s1 : s2;
        a.u[j] = v;
        sq += v * v;
    }
    return sq;
}

#define KB_SYNC() do { if (!grid_barrier(a.bar, gridDim.x, a.err)) return; KB_AFTER_SYNC; } while (0)
#define KB_AFTER_SYNC ((void)0)

// Phase log of the CGLS iteration (LLS_LOG=2): CTA 0 appends %globaltimer after every grid
// barrier and, with the top bit set, at the top of every iteration of the loop.
__device__ __forceinline__ void phase_stamp(const KArgs& a, int& ph, bool top) {
    if (a.phases && blockIdx.x == 0 && threadIdx.x == 0 && ph < kPhaseLen)
        a.phases[ph] = globaltimer_ns() | (top ? (1ull << 63) : 0ull);
    ++ph;
}

// NC > 0: fused engine with NC columns per thread; NC == 0: two-pass engine.
template <int NC>
__global__ void __launch_bounds__(kKThreads, NC > 0 ? 1 : 3)
cgls_kernel(KArgs a) {
    const int gtid = blockIdx.x * kKThreads + threadIdx.x, gthreads = gridDim.x * kKThreads;
    const double anorm = sqrt(*a.anorm2);
    const double mnorm = sqrt(*a.mnorm2);
    int iters = 0, status = 1, apasses = 0, mpasses = 0;
    double eta = 0.0, fwd = 0.0, rn2 = 0.0, un2 = 0.0, xn2 = 0.0, gamma = 0.0;
    bool xzero = a.x_zero != 0;
    int ph = 0;                    // entries of the phase log so far
#undef KB_AFTER_SYNC
#define KB_AFTER_SYNC phase_stamp(a, ph, false)

    for (int restart = 0; restart <= kMaxRestarts; ++restart) {
        // ---- true residual r = b - A x ----
        if (xzero) {
            double sq = 0.0;
            for (int i = gtid; i < a.m; i += gthreads) {
                const double bi = a.b[i];
                a.r[i] = bi;
                a.rdf[i] = to_df(bi);
                sq += bi * bi;
            }
            block_partial(sq, a.bpart, 0);
            for (int j = gtid; j < a.n; j += gthreads) a.x[j] = 0.0;
        } else {
            if constexpr (NC > 0) {
                double dummy = 0.0;
                fused_pass<NC>(a, a.x, nullptr, true, false, false, dummy);
                ++apasses;
                KB_SYNC();
                double sq = 0.0;
                for (int i = gtid; i < a.m; i += gthreads) {
                    double ri = a.b[i] - __ldcg(a.q + i);
                    a.r[i] = ri;
                    a.rdf[i] = to_df(ri);
                    sq += ri * ri;
                }
                block_partial(sq, a.bpart, 0);
            } else {
                stage_vec(a.x, a.n);
                a_times_partials(a);
                ++apasses;
                KB_SYNC();
                double sq = 0.0;
                for (int base = (gtid >> 5) * 8; base < a.m; base += (gthreads >> 5) * 8) {
                    const int i = base + ((threadIdx.x & 31) >> 2);
                    const double ax = sum_parts_quad(a.qpart + i, a.nck, (size_t)a.m, i < a.m);
                    if ((threadIdx.x & 3) == 0 && i < a.m) {
                        const double ri = a.b[i] - ax;
                        a.r[i] = ri;
                        a.rdf[i] = to_df(ri);
                        sq += ri * ri;
                    }
                }
                block_partial(sq, a.bpart, 0);
            }
        }
        xzero = false;
        KB_SYNC();
        rn2 = grid_total(a.bpart, 0);
        if (!finite_start(a, rn2)) return;
        // ---- u = A^T r, s = M^T u, gamma = ||s||^2 ----
        if constexpr (NC > 0) {
            double dummy = 0.0;
            fused_pass<NC>(a, nullptr, a.r, false, false, true, dummy);
        } else {
            at_times_partials(a, a.r, a.rdf);
        }
        ++apasses;
        KB_SYNC();
        {
            double sq = 0.0;
            if constexpr (NC > 0) {
                sq = reduce_u(a, 0.0, false, gtid, gthreads);
            } else {
                for (int base = (gtid >> 5) * 8; base < a.n; base += (gthreads >> 5) * 8) {
                    const int j = base + ((threadIdx.x & 31) >> 2);
                    const double v = sum_parts_quad(a.upart + j, a.nrc, (size_t)a.n, j < a.n);
                    if ((threadIdx.x & 3) == 0 && j < a.n) {
                        a.u[j] = v;
                        a.udf[j] = to_df(v);
                        sq += v * v;
                    }
                }
            }
            block_partial(sq, a.bpart, 1);
            double xs = 0.0;
            for (int j = gtid; j < a.n; j += gthreads) { double xv = __ldcg(a.x + j); xs += xv * xv; }
            block_partial(xs, a.bpart, 3);
        }
        KB_SYNC();
        un2 = grid_total(a.bpart, 1);
        xn2 = grid_total(a.bpart, 3);
        if constexpr (NC > 0) stage_vec(a.u, a.n);
        else stage_df(a.udf, a.n);
        block_partial(tri_gemv(a.M, a.n, true, a.s), a.bpart, 2);
        ++mpasses;
        KB_SYNC();
        gamma = grid_total(a.bpart, 2);
        {
            const double xn = sqrt(xn2), sn = sqrt(gamma);
            eta = xn > 0.0 ? sn / (anorm * xn) : (sn == 0.0 ? 0.0 : INFINITY);
            fwd = xn > 0.0 ? mnorm * sn / xn : (sn == 0.0 ? 0.0 : INFINITY);
        }
        const double crit = a.target == LLS_TARGET_FP64 ? eta : fwd;
        log_hist(a, iters, crit);
        if (crit <= a.tol) { status = 0; break; }
        if (iters >= a.max_iter || restart == kMaxRestarts) { status = 1; break; }
        for (int j = gtid; j < a.n; j += gthreads) {
            const double pj = __ldcg(a.s + j);
            a.p[j] = pj;
            a.pdf[j] = to_df(pj);
        }
        KB_SYNC();

        // ---- iterate ----
        while (iters < a.max_iter) {
            phase_stamp(a, ph, true);
            // t = M p
            stage_df(a.pdf, a.n);
            tri_gemv(a.Mt, a.n, false, a.t, a.tdf);
            ++mpasses;
            KB_SYNC();
            double delta;
            if constexpr (NC > 0) {
                // one pass: q = A t, A^T q, A^T r
                double dsum = 0.0;
                fused_pass<NC>(a, a.t, a.r, true, true, true, dsum);
                ++apasses;
                block_partial(dsum, a.bpart, 0);
                KB_SYNC();
                delta = grid_total(a.bpart, 0);
            } else {
                stage_df(a.tdf, a.n);
                a_times_partials(a);
                ++apasses;
                KB_SYNC();
                double sq = 0.0;
                for (int base = (gtid >> 5) * 8; base < a.m; base += (gthreads >> 5) * 8) {
                    const int i = base + ((threadIdx.x & 31) >> 2);
                    const double v = sum_parts_quad(a.qpart + i, a.nck, (size_t)a.m, i < a.m);
                    if ((threadIdx.x & 3) == 0 && i < a.m) {
                        a.q[i] = v;
                        sq += v * v;
                    }
                }
                block_partial(sq, a.bpart, 0);
                KB_SYNC();
                delta = grid_total(a.bpart, 0);
            }
            ++iters;
            if (!(delta > 0.0)) break;
            const double alpha = gamma / delta;
            {
                double xs = 0.0;
                for (int j = gtid; j < a.n; j += gthreads) {
                    double xv = a.x[j] + alpha * __ldcg(a.t + j);
                    a.x[j] = xv;
                    xs += xv * xv;
                }
                block_partial(xs, a.bpart, 3);
                for (int i = gtid; i < a.m; i += gthreads) {
                    const double ri = a.r[i] - alpha * __ldcg(a.q + i);
                    a.r[i] = ri;
                    a.rdf[i] = to_df(ri);
                }
                if constexpr (NC > 0) reduce_u(a, alpha, true, gtid, gthreads);
            }
            KB_SYNC();
            if constexpr (NC == 0) {
                // s = M^T (A^T r) with a second pass over A
                at_times_partials(a, a.r, a.rdf);
                ++apasses;
                KB_SYNC();
                for (int base = (gtid >> 5) * 8; base < a.n; base += (gthreads >> 5) * 8) {
                    const int j = base + ((threadIdx.x & 31) >> 2);
                    const double v = sum_parts_quad(a.upart + j, a.nrc, (size_t)a.n, j < a.n);
                    if ((threadIdx.x & 3) == 0 && j < a.n) {
                        a.u[j] = v;
                        a.udf[j] = to_df(v);
                    }
                }
                KB_SYNC();
            }
            if constexpr (NC > 0) stage_vec(a.u, a.n);
            else stage_df(a.udf, a.n);
            block_partial(tri_gemv(a.M, a.n, true, a.s), a.bpart, 2);
            ++mpasses;
            KB_SYNC();
            const double gnew = grid_total(a.bpart, 2);
            const double xn = sqrt(grid_total(a.bpart, 3));
            const double beta = gnew / gamma;
            gamma = gnew;
            for (int j = gtid; j < a.n; j += gthreads) {
                const double pj = __ldcg(a.s + j) + beta * a.p[j];
                a.p[j] = pj;
                a.pdf[j] = to_df(pj);
            }
            const double sn = sqrt(gnew);
            const double e1 = xn > 0.0 ? sn / (anorm * xn) : INFINITY;
            const double f1 = xn > 0.0 ? mnorm * sn / xn : INFINITY;
            KB_SYNC();
            log_hist(a, iters, a.target == LLS_TARGET_FP64 ? e1 : f1);
            if ((a.target == LLS_TARGET_FP64 ? e1 : f1) <= a.tol) break;
        }
        // loop back: the top of the restart loop recomputes b - A x and re-tests
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.info[0] = iters;
        a.info[1] = eta;
        a.info[2] = fwd;
        a.info[3] = sqrt(rn2);
        a.info[4] = sqrt(un2);
        a.info[5] = anorm;
        a.info[6] = sqrt(xn2);
        a.info[7] = status;
        a.info[10] = apasses + (a.At ? 2 : 0);   // the row-block copy reads and writes A once
        a.info[11] = mpasses;
    }
}

#undef KB_AFTER_SYNC
#define KB_AFTER_SYNC ((void)0)

// ---------------------------------------------------------------------------------------
// LSQR (Paige and Saunders; Sec. 5 names it as the stable equivalent of CGLS) on the same
// right-preconditioned operator B = A M, M = R^{-1}, with x = M y kept directly.
// Golub-Kahan bidiagonalization started from the current residual r = b - A x:
//   beta u = r,  alpha v = M^T A^T u,  t = M v,  d = t,  phibar = beta,  rhobar = alpha
//   loop: w = A t - alpha u;  beta = ||w||;  u = w / beta
//         s = M^T A^T u - beta v;  alpha = ||s||;  v = s / alpha
//         rho = hypot(rhobar, beta);  c = rhobar / rho;  sn = beta / rho
//         theta = sn alpha;  rhobar = -c alpha;  phi = c phibar;  phibar = sn phibar
//         x += (phi / rho) d;  t = M v;  d = t - (theta / rho) d
// ||B^T r|| = phibar alpha |c| is the same quantity as CGLS's ||s||, so the stop tests and
// the fresh-residual confirmation (with restarts from the current x) are those of CGLS.
// Per iteration: one pass over A for A t, one for A^T u, one product each with M and M^T.
// Vector roles: u -> r (m), w -> q (m), v -> p, A^T u -> u, s -> s, t -> t, d -> d (n).
__global__ void __launch_bounds__(kKThreads, 2)
lsqr_kernel(KArgs a) {
    const int gtid = blockIdx.x * kKThreads + threadIdx.x, gthreads = gridDim.x * kKThreads;
    const double anorm = sqrt(*a.anorm2);
    const double mnorm = sqrt(*a.mnorm2);
    int iters = 0, status = 1, apasses = 0, mpasses = 0;
    double eta = 0.0, fwd = 0.0, rn2 = 0.0, un2 = 0.0, xn2 = 0.0;
    bool xzero = a.x_zero != 0;

    for (int restart = 0; restart <= kMaxRestarts; ++restart) {
        // ---- r = b - A x, beta = ||r|| ----
        if (xzero) {
            double sq = 0.0;
            for (int i = gtid; i < a.m; i += gthreads) { double bi = a.b[i]; a.r[i] = bi; sq += bi * bi; }
            block_partial(sq, a.bpart, 0);
            for (int j = gtid; j < a.n; j += gthreads) a.x[j] = 0.0;
        } else {
            stage_vec(a.x, a.n);
            a_times_partials(a);
            ++apasses;
            KB_SYNC();
            double sq = 0.0;
            for (int i = gtid; i < a.m; i += gthreads) {
                double ax = 0.0;
                ax += sum_parts(a.qpart + i, a.nck, (size_t)a.m);
                double ri = a.b[i] - ax;
                a.r[i] = ri;
                sq += ri * ri;
            }
            block_partial(sq, a.bpart, 0);
        }
        xzero = false;
        KB_SYNC();
        rn2 = grid_total(a.bpart, 0);
        if (!finite_start(a, rn2)) return;
        double beta = sqrt(rn2);
        // ---- A^T r (scaled to A^T u below), ||x||^2 ----
        at_times_partials(a, a.r);
        ++apasses;
        {
            double xs = 0.0;
            for (int j = gtid; j < a.n; j += gthreads) { double xv = __ldcg(a.x + j); xs += xv * xv; }
            block_partial(xs, a.bpart, 3);
        }
        KB_SYNC();
        xn2 = grid_total(a.bpart, 3);
        {
            const double ib = beta > 0.0 ? 1.0 / beta : 0.0;
            double sq = 0.0;
            for (int j = gtid; j < a.n; j += gthreads) {
                double v = 0.0;
                v += sum_parts(a.upart + j, a.nrc, (size_t)a.n);
                sq += v * v;
                a.u[j] = v * ib;
            }
            block_partial(sq, a.bpart, 1);
            for (int i = gtid; i < a.m; i += gthreads) a.r[i] *= ib;
        }
        KB_SYNC();
        un2 = grid_total(a.bpart, 1);
        // ---- alpha v = M^T A^T u ----
        stage_vec(a.u, a.n);
        block_partial(tri_gemv(a.M, a.n, true, a.s), a.bpart, 2);
        ++mpasses;
        KB_SYNC();
        double alpha = sqrt(grid_total(a.bpart, 2));
        {
            const double xn = sqrt(xn2), sn = alpha * beta;
            eta = xn > 0.0 ? sn / (anorm * xn) : (sn == 0.0 ? 0.0 : INFINITY);
            fwd = xn > 0.0 ? mnorm * sn / xn : (sn == 0.0 ? 0.0 : INFINITY);
        }
        const double crit = a.target == LLS_TARGET_FP64 ? eta : fwd;
        log_hist(a, iters, crit);
        if (crit <= a.tol) { status = 0; break; }
        if (iters >= a.max_iter || restart == kMaxRestarts || !(alpha > 0.0)) { status = 1; break; }
        {
            const double ia = 1.0 / alpha;
            for (int j = gtid; j < a.n; j += gthreads) a.p[j] = __ldcg(a.s + j) * ia;
        }
        KB_SYNC();
        stage_vec(a.p, a.n);
        tri_gemv(a.Mt, a.n, false, a.t);
        ++mpasses;
        KB_SYNC();
        for (int j = gtid; j < a.n; j += gthreads) a.d[j] = __ldcg(a.t + j);
        double phibar = beta, rhobar = alpha;

        // ---- iterate ----
        while (iters < a.max_iter) {
            // w = A t - alpha u, beta = ||w||
            stage_vec(a.t, a.n);
            a_times_partials(a);
            ++apasses;
            KB_SYNC();
            {
                double sq = 0.0;
                for (int i = gtid; i < a.m; i += gthreads) {
                    double v = 0.0;
                    v += sum_parts(a.qpart + i, a.nck, (size_t)a.m);
                    v -= alpha * a.r[i];
                    a.q[i] = v;
                    sq += v * v;
                }
                block_partial(sq, a.bpart, 0);
            }
            KB_SYNC();
            beta = sqrt(grid_total(a.bpart, 0));
            const double ib = beta > 0.0 ? 1.0 / beta : 0.0;
            // u = w / beta;  A^T u = (A^T w) / beta
            at_times_partials(a, a.q);
            ++apasses;
            for (int i = gtid; i < a.m; i += gthreads) a.r[i] = __ldcg(a.q + i) * ib;
            KB_SYNC();
            for (int j = gtid; j < a.n; j += gthreads) {
                double v = 0.0;
                v += sum_parts(a.upart + j, a.nrc, (size_t)a.n);
                a.u[j] = v * ib;
            }
            KB_SYNC();
            // s = M^T A^T u - beta v, alpha = ||s||
            stage_vec(a.u, a.n);
            tri_gemv(a.M, a.n, true, a.s);
            ++mpasses;
            KB_SYNC();
            {
                double sq = 0.0;
                for (int j = gtid; j < a.n; j += gthreads) {
                    const double v = __ldcg(a.s + j) - beta * a.p[j];
                    a.s[j] = v;
                    sq += v * v;
                }
                block_partial(sq, a.bpart, 1);
            }
            KB_SYNC();
            alpha = sqrt(grid_total(a.bpart, 1));
            ++iters;
            // plane rotation of the bidiagonal (every CTA computes the same scalars)
            const double rho = hypot(rhobar, beta);
            const double c = rho > 0.0 ? rhobar / rho : 1.0, sn = rho > 0.0 ? beta / rho : 0.0;
            const double theta = sn * alpha;
            rhobar = -c * alpha;
            const double phi = c * phibar;
            phibar = sn * phibar;
            const double step = rho > 0.0 ? phi / rho : 0.0, dcoef = rho > 0.0 ? theta / rho : 0.0;
            const double ia = alpha > 0.0 ? 1.0 / alpha : 0.0;
            {
                double xs = 0.0;
                for (int j = gtid; j < a.n; j += gthreads) {
                    const double xv = a.x[j] + step * a.d[j];
                    a.x[j] = xv;
                    xs += xv * xv;
                    a.p[j] = __ldcg(a.s + j) * ia;
                }
                block_partial(xs, a.bpart, 3);
            }
            KB_SYNC();
            const double xn = sqrt(grid_total(a.bpart, 3));
            const double atr = phibar * alpha * fabs(c);
            const double e1 = xn > 0.0 ? atr / (anorm * xn) : INFINITY;
            const double f1 = xn > 0.0 ? mnorm * atr / xn : INFINITY;
            log_hist(a, iters, a.target == LLS_TARGET_FP64 ? e1 : f1);
            if ((a.target == LLS_TARGET_FP64 ? e1 : f1) <= a.tol || !(alpha > 0.0) || !(beta > 0.0)) break;
            // t = M v, d = t - (theta / rho) d
            stage_vec(a.p, a.n);
            tri_gemv(a.Mt, a.n, false, a.t);
            ++mpasses;
            KB_SYNC();
            for (int j = gtid; j < a.n; j += gthreads) a.d[j] = __ldcg(a.t + j) - dcoef * a.d[j];
        }
        // loop back: the top of the restart loop recomputes b - A x and re-tests
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.info[0] = iters;
        a.info[1] = eta;
        a.info[2] = fwd;
        a.info[3] = sqrt(rn2);
        a.info[4] = sqrt(un2);
        a.info[5] = anorm;
        a.info[6] = sqrt(xn2);
        a.info[7] = status;
        a.info[10] = apasses;
        a.info[11] = mpasses;
    }
}

// ---------------------------------------------------------------------------------------
// Adjoint of the least-squares solution map (for the differentiable solve).
//
// For a loss L(x*) with g = dL/dx, z = (A^T A)^{-1} g; then dL/db = A z and
// dL/dA = r z^T - (A z) x^T with r = b - A x (differentiate A^T (b - A x) = 0). z comes from
// preconditioned CG on A^T A z = g with the preconditioner M M^T = (R^T R)^{-1}, reusing the
// solve's R; each iteration applies A and A^T with the same compensated products as CGLS.
//   res = g, u = M^T res, y = M u, rho = ||u||^2, p = y
//   loop: q = A p, w = A^T q, alpha = rho / (p . w), z += alpha p, res -= alpha w,
//         u = M^T res, rho' = ||u||^2, beta = rho' / rho, y = M u, p = y + beta p
//   stop when ||M^T res|| <= tol ||M^T g||.
// Then r = b - A x and A z are formed and the rank-2 gradient is written in one sweep.
// Vector roles: z -> x, res -> s, y -> t, q -> q, w -> u, u -> r (n entries), g -> b.
struct AdjArgs {
    KArgs k;
    const double* g;
    const double* bvec;
    const double* xsol;
    float* gA; int ldga;
    double* gb;
};

__global__ void __launch_bounds__(kKThreads, 1)
adjoint_kernel(AdjArgs aa) {
    KArgs& a = aa.k;
    const int gtid = blockIdx.x * kKThreads + threadIdx.x, gthreads = gridDim.x * kKThreads;
    const int n = a.n, m = a.m;
    double* z = a.x;
    double* res = a.s;
    double* y = a.t;
    double* w = a.u;
    double* uu = a.r;
    int iters = 0, status = 1, apasses = 0, mpasses = 0;
    // res = g, z = 0
    for (int j = gtid; j < n; j += gthreads) { res[j] = aa.g[j]; z[j] = 0.0; }
    KB_SYNC();
    // u = M^T res, rho = ||u||^2
    stage_vec(res, n);
    block_partial(tri_gemv(a.M, n, true, uu), a.bpart, 0);
    ++mpasses;
    KB_SYNC();
    double rho = grid_total(a.bpart, 0);
    const double rho0 = rho;
    // y = M u, p = y
    stage_vec(uu, n);
    tri_gemv(a.Mt, n, false, y);
    ++mpasses;
    KB_SYNC();
    for (int j = gtid; j < n; j += gthreads) a.p[j] = __ldcg(y + j);
    KB_SYNC();
    if (!(rho0 > 0.0)) status = 0;
    while (status != 0 && iters < a.max_iter) {
        // q = A p
        stage_vec(a.p, n);
        a_times_partials(a);
        ++apasses;
        KB_SYNC();
        for (int i = gtid; i < m; i += gthreads) {
            double v = 0.0;
            v += sum_parts(a.qpart + i, a.nck, (size_t)m);
            a.q[i] = v;
        }
        KB_SYNC();
        // w = A^T q, pw = p . w
        at_times_partials(a, a.q);
        ++apasses;
        KB_SYNC();
        {
            double pw = 0.0;
            for (int j = gtid; j < n; j += gthreads) {
                double v = 0.0;
                v += sum_parts(a.upart + j, a.nrc, (size_t)n);
                w[j] = v;
                pw += v * __ldcg(a.p + j);
            }
            block_partial(pw, a.bpart, 1);
        }
        KB_SYNC();
        const double pw = grid_total(a.bpart, 1);
        ++iters;
        if (!(pw > 0.0)) { status = 0; break; }
        const double alpha = rho / pw;
        for (int j = gtid; j < n; j += gthreads) {
            z[j] += alpha * __ldcg(a.p + j);
            res[j] -= alpha * __ldcg(w + j);
        }
        KB_SYNC();
        stage_vec(res, n);
        block_partial(tri_gemv(a.M, n, true, uu), a.bpart, 0);
        ++mpasses;
        KB_SYNC();
        const double rnew = grid_total(a.bpart, 0);
        const double beta = rnew / rho;
        rho = rnew;
        stage_vec(uu, n);
        tri_gemv(a.Mt, n, false, y);
        ++mpasses;
        KB_SYNC();
        for (int j = gtid; j < n; j += gthreads) a.p[j] = __ldcg(y + j) + beta * a.p[j];
        KB_SYNC();
        if (sqrt(rho) <= a.tol * sqrt(rho0)) { status = 0; break; }
    }
    // r = b - A x  (into q), then A z (into qpart reduce -> gb)
    stage_vec(aa.xsol, n);
    a_times_partials(a);
    ++apasses;
    KB_SYNC();
    for (int i = gtid; i < m; i += gthreads) {
        double v = 0.0;
        v += sum_parts(a.qpart + i, a.nck, (size_t)m);
        a.q[i] = aa.bvec[i] - v;
    }
    KB_SYNC();
    stage_vec(z, n);
    a_times_partials(a);
    ++apasses;
    KB_SYNC();
    for (int i = gtid; i < m; i += gthreads) {
        double v = 0.0;
        v += sum_parts(a.qpart + i, a.nck, (size_t)m);
        aa.gb[i] = v;
    }
    KB_SYNC();
    // dL/dA[i, j] = r_i z_j - (A z)_i x_j, column by column (coalesced over i)
    for (size_t e = (size_t)gtid; e < (size_t)m * n; e += (size_t)gthreads) {
        const int i = (int)(e % m), j = (int)(e / m);
        const double val = __ldcg(a.q + i) * __ldcg(z + j) - __ldcg(aa.gb + i) * __ldcg(aa.xsol + j);
        aa.gA[(size_t)i + (size_t)j * aa.ldga] = (float)val;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.info[0] = iters;
        a.info[1] = rho0 > 0.0 ? sqrt(rho / rho0) : 0.0;
        a.info[7] = status;
        a.info[10] = apasses;
        a.info[11] = mpasses;
    }
}

// ---------------------------------------------------------------------------------------
struct KLayout {
    int nrt, nck, nrc, ncg, colchunk, at_rows, at_cpr;
    size_t off_r, off_q, off_t, off_p, off_s, off_u, off_d, off_qpart, off_upart, off_v1, off_v2, off_bpart,
        off_bar, off_rdf, off_tdf, off_udf, off_pdf, off_tile, total;
};

// The one-pass engine streams A from a copy in 4-row blocks (tiled = true): block blk is the
// contiguous run At[blk * n .. blk * n + n) of 16-byte segments (A[4 blk .. 4 blk + 3, j]).
// Width of the A t work items: a grid barrier follows the pass, so its time is the number of
// waves of items times the item's time, and the width that minimises waves x width wins
// (at m = 32768, n = 4096 on 456 CTAs: 72 columns, 1824 items in exactly 4 waves, where 64
// columns gave 2048 items in 4.5 waves).
static int pick_col_chunk(int m, int n, int grid) {
    const long long nrt = ceil_div(m, kRowTile);
    int best = 64;
    long long best_cost = -1;
    for (int c = kColChunkMin; c <= kColChunkMax; c += 8) {
        const long long items = nrt * ceil_div(n, c);
        const long long waves = (items + grid - 1) / grid;
        const long long cost = waves * (c < n ? c : n);
        if (best_cost < 0 || cost < best_cost || (cost == best_cost && c > best)) {
            best_cost = cost;
            best = c;
        }
    }
    return best;
}

// Rows staged for the A^T r pass at most (the vector space reserved in shared memory).
static int at_rows_cap(int n) { return n > kRowChunkCap ? n : kRowChunkCap; }

// The A^T r pass: R row chunks of L rows (L a multiple of 4, at most at_rows_cap(n) rounded down
// to a multiple of 4, the rows a CTA can stage), K = grid / R CTAs per chunk, groups of 8 columns.
// Every CTA streams L x 8 elements per item, so the pass takes about ceil(ncg / K) * L; the R
// with the least such time wins (fewest chunks on ties). At m = 32768, n = 4096 on 456 CTAs:
// 8 chunks of 4096 rows, 57 CTAs each, 512 groups in at most 9 items per CTA (8.98 on average).
// When even R = grid leaves chunks taller than the staging room, R is the fewest chunks that fit
// and each CTA takes the chunks c, c + grid, ... one after another (K = 1).
static int at_rows_fit(int n) { return at_rows_cap(n) & ~3; }

static void at_plan(int m, int n, int grid, int& R, int& L, int& K) {
    const long long ncg = ceil_div(n, kKWarps);
    const int cap = at_rows_fit(n);
    if (grid < 1) grid = 1;
    long long best = -1;
    for (int r = 1; r <= grid; ++r) {
        const int l = (ceil_div(m, r) + 3) & ~3;
        if (l > cap) continue;
        if ((long long)(r - 1) * l >= m) break;   // the last chunk would be empty
        const int k = grid / r;
        const long long cost = (ncg + k - 1) / k * l;
        if (best < 0 || cost < best) { best = cost; R = r; L = l; K = k; }
    }
    if (best < 0) {   // more chunks than CTAs
        R = ceil_div(m, cap);
        L = (ceil_div(m, R) + 3) & ~3;
        K = 1;
    }
}

// Row chunks the A^T r pass can take on grids of at most `grid` CTAs (room for its partials).
static long long at_rows_max_chunks(int m, int n, int grid) {
    const long long a = std::min<long long>(grid < 1 ? 1 : grid, ceil_div(m, 4));
    const long long b = ceil_div(m, at_rows_fit(n)) + 1;
    return a > b ? a : b;
}

static KLayout k_layout(int m, int n, int grid, bool tiled = false) {
    KLayout L;
    L.nrt = ceil_div(m, kRowTile);
    L.colchunk = pick_col_chunk(m, n, grid < 1 ? 1 : grid);
    L.nck = ceil_div(n, L.colchunk);
    at_plan(m, n, grid < 1 ? 1 : grid, L.nrc, L.at_rows, L.at_cpr);
    L.ncg = ceil_div(n, kKWarps);
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o = align_up(o + bytes, 256); return r; };
    L.off_r = take(8ull * m);
    L.off_q = take(8ull * m);
    L.off_t = take(8ull * n);
    L.off_p = take(8ull * n);
    L.off_s = take(8ull * n);
    L.off_u = take(8ull * n);
    L.off_d = take(8ull * n);
    L.off_qpart = take(8ull * m * ceil_div(n, kColChunkMin));   // room for the narrowest width (most partials)
    // room for the most row chunks any grid up to this one can take, so a scratch sized for
    // the largest grid holds every smaller grid's layout
    L.off_upart = take(8ull * n * (size_t)at_rows_max_chunks(m, n, grid));
    L.off_v1 = take(8ull * n * grid);
    L.off_v2 = take(8ull * n * grid);
    L.off_bpart = take(8ull * kNPart * grid);
    L.off_bar = take(64);
    L.off_rdf = take(8ull * m);
    L.off_tdf = take(8ull * n);
    L.off_udf = take(8ull * n);
    L.off_pdf = take(8ull * n);
    L.off_tile = tiled ? take(16ull * (size_t)ceil_div(m, kRB) * n) : 0;
    L.total = o;
    return L;
}

// At[blk * n + j] = (A[4 blk + r, j], r = 0..3), rows beyond m as zero. 64 row blocks x 32
// columns per CTA through shared memory, so both the column reads and the block writes are
// contiguous.
__global__ void __launch_bounds__(256) tile_rows_kernel(const float* __restrict__ A, int lda, int m, int n,
                                                        float4* __restrict__ At, int aligned16) {
    __shared__ float4 tile[64][33];
    const int nblk = (m + kRB - 1) / kRB;
    const int blk0 = blockIdx.x * 64, j0 = blockIdx.y * 32;
#pragma unroll
    for (int it = 0; it < 8; ++it) {
        const int bb = threadIdx.x % 64, jj = threadIdx.x / 64 + 4 * it;
        const int j = j0 + jj, i = kRB * (blk0 + bb);
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (j < n && i < m) {
            const float* src = A + (size_t)j * lda + i;
            if (aligned16 && i + kRB <= m) {
                v = __ldg(reinterpret_cast<const float4*>(src));
            } else {
                v.x = src[0];
                if (i + 1 < m) v.y = src[1];
                if (i + 2 < m) v.z = src[2];
                if (i + 3 < m) v.w = src[3];
            }
        }
        tile[bb][jj] = v;
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < 8; ++it) {
        const int jj = threadIdx.x % 32, bb = threadIdx.x / 32 + 8 * it;
        const int j = j0 + jj, blk = blk0 + bb;
        if (j < n && blk < nblk) At[(size_t)blk * n + j] = tile[bb][jj];
    }
}

static int sm_count() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 0;
    return sms;
}

constexpr int kMaxGridPerSm = 3;

// The one-pass engine (CGLS, n <= 4096) and its copy of A are used when the scratch holds it.
static int fused_nc(int n);
static bool tiled_engine_allowed(int n) {
    static const bool onepass = [] {
        const char* v = getenv("LLS_KRYLOV");
        return v && v[0] == 'o';   // LLS_KRYLOV=onepass: the one-pass engine for CGLS, n <= 4096
    }();
    return onepass && fused_nc(n) > 0;
}

size_t krylov_scratch_bytes(int m, int n, int grid, bool one_pass) {
    if (grid <= 0) {
        int sms = sm_count();
        grid = kMaxGridPerSm * (sms > 0 ? sms : 160);
    }
    return k_layout(m, n, grid, one_pass && tiled_engine_allowed(n)).total;
}

// One CTA per 64 Ki elements of A (the passes' work items are 1024-row tiles); the caller
// caps it at three CTAs per SM.
int krylov_default_ctas(int m, int n) {
    const long long work = (long long)m * n;
    const long long g = (work + (1 << 16) - 1) >> 16;
    return g < 1 ? 1 : (g > (1 << 20) ? (1 << 20) : (int)g);
}

static int fused_nc(int n) {
    const int need = ceil_div(n, kKThreads);
    if (need <= 1) return 1;
    if (need <= 2) return 2;
    if (need <= 4) return 4;
    if (need <= 8) return 8;
    if (need <= 16) return 16;
    return 0;
}

template <int NC>
static int launch_cgls(KArgs& a, const KrylovCall& c, char* base, size_t smem, int sms, cudaStream_t st,
                       bool lsqr = false) {
    void (*kern)(KArgs) = lsqr ? lsqr_kernel : cgls_kernel<NC>;
    LLS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    LLS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kKThreads, smem));
    if (per_sm < 1) return LLS_ERR_UNSUPPORTED;
    const int maxg = sms * (per_sm < kMaxGridPerSm ? per_sm : kMaxGridPerSm);
    int grid;
    if (NC > 0) {
        const int nblk = ceil_div(c.m, kRB);
        grid = ceil_div(nblk, 8);            // at least 8 row blocks per CTA
    } else {
        grid = c.ctas > 0 ? c.ctas : krylov_default_ctas(c.m, c.n);
    }
    if (grid < 1) grid = 1;
    if (grid > maxg) grid = maxg;
    KLayout L = k_layout(c.m, c.n, grid, NC > 0);
    if (L.total > c.scratch_bytes) return LLS_ERR_WORKSPACE;
    a.At = nullptr;
    if (NC > 0) {
        a.At = reinterpret_cast<const float4*>(base + L.off_tile);
        dim3 tg(ceil_div(ceil_div(c.m, kRB), 64), ceil_div(c.n, 32));
        tile_rows_kernel<<<tg, 256, 0, st>>>(c.A, c.lda, c.m, c.n, const_cast<float4*>(a.At), a.aligned16);
        LLS_LAUNCH_CHECK("tile_rows", st);
    }
    a.r = (double*)(base + L.off_r); a.q = (double*)(base + L.off_q);
    a.t = (double*)(base + L.off_t); a.p = (double*)(base + L.off_p);
    a.s = (double*)(base + L.off_s); a.u = (double*)(base + L.off_u); a.d = (double*)(base + L.off_d);
    a.qpart = (double*)(base + L.off_qpart); a.upart = (double*)(base + L.off_upart);
    a.v1part = (double*)(base + L.off_v1); a.v2part = (double*)(base + L.off_v2);
    a.bpart = (double*)(base + L.off_bpart);
    a.bar = (unsigned*)(base + L.off_bar);
    a.rdf = (float2*)(base + L.off_rdf); a.tdf = (float2*)(base + L.off_tdf);
    a.udf = (float2*)(base + L.off_udf); a.pdf = (float2*)(base + L.off_pdf);
    a.nrt = L.nrt; a.nck = L.nck; a.nrc = L.nrc; a.ncg = L.ncg; a.colchunk = L.colchunk;
    a.at_rows = L.at_rows; a.at_cpr = L.at_cpr;
    LLS_CUDA_TRY(cudaMemsetAsync(a.bar, 0, 64, st));
    void* args[] = {&a};
    LLS_CUDA_TRY(cudaLaunchCooperativeKernel((void*)kern, dim3(grid), dim3(kKThreads), args, smem, st));
    note_launch(lsqr ? "lsqr" : "cgls", st);
    return LLS_OK;
}

int krylov_solve(const KrylovCall& c, cudaStream_t st) {
    if (c.method != LLS_KRYLOV_CGLS && c.method != LLS_KRYLOV_LSQR) return LLS_ERR_UNSUPPORTED;
    const bool lsqr = c.method == LLS_KRYLOV_LSQR;
    const int sms = sm_count();
    if (sms <= 0) return LLS_ERR_CUDA;
    int nc = (!lsqr && tiled_engine_allowed(c.n)) ? fused_nc(c.n) : 0;
    if (nc > 0) {   // the one-pass engine needs its copy of A in the scratch
        const int maxg = kMaxGridPerSm * sms;
        if (k_layout(c.m, c.n, maxg, true).total > c.scratch_bytes) nc = 0;
    }
    KArgs a;
    a.m = c.m; a.n = c.n; a.lda = c.lda; a.A = c.A; a.b = c.b; a.x = c.x;
    a.M = c.Minv; a.Mt = c.Mt;
    a.err = c.dev_err;
    a.info = c.dev_info;
    a.anorm2 = c.dev_info + 8;
    a.mnorm2 = c.dev_info + 9;
    a.tol = c.tol; a.max_iter = c.max_iter; a.target = c.target; a.x_zero = c.x_zero;
    a.hist = c.hist;
    a.phases = c.phases;
    a.aligned16 = (((uintptr_t)c.A & 15) == 0) && (c.lda % 4 == 0);
    char* base = (char*)c.scratch;
    if (nc > 0) {
        a.vec_floats = (int)align_up((size_t)2 * c.n, 4);
        const size_t smem = sizeof(float) * ((size_t)a.vec_floats + (size_t)2 * kRB * c.n);
        if (smem > 220 * 1024) return LLS_ERR_UNSUPPORTED;
        switch (nc) {
            case 1: return launch_cgls<1>(a, c, base, smem, sms, st);
            case 2: return launch_cgls<2>(a, c, base, smem, sms, st);
            case 4: return launch_cgls<4>(a, c, base, smem, sms, st);
            case 8: return launch_cgls<8>(a, c, base, smem, sms, st);
            default: return launch_cgls<16>(a, c, base, smem, sms, st);
        }
    }
    a.vec_floats = 2 * at_rows_cap(c.n);
    const size_t smem = sizeof(float) * (size_t)a.vec_floats;
    if (smem > 220 * 1024) return LLS_ERR_UNSUPPORTED;
    return launch_cgls<0>(a, c, base, smem, sms, st, lsqr);
}

int adjoint_solve(const AdjointCall& c, cudaStream_t st) {
    const int sms = sm_count();
    if (sms <= 0) return LLS_ERR_CUDA;
    AdjArgs aa;
    KArgs& a = aa.k;
    a.m = c.m; a.n = c.n; a.lda = c.lda; a.A = c.A; a.b = nullptr; a.x = c.z;
    a.M = c.Minv; a.Mt = c.Mt;
    a.err = c.dev_err; a.info = c.dev_info; a.anorm2 = nullptr; a.mnorm2 = nullptr;
    a.tol = c.tol; a.max_iter = c.max_iter; a.target = LLS_TARGET_FP64; a.x_zero = 1;
    a.hist = nullptr;
    a.phases = nullptr;
    a.aligned16 = (((uintptr_t)c.A & 15) == 0) && (c.lda % 4 == 0);
    a.vec_floats = 2 * at_rows_cap(c.n);
    const size_t smem = sizeof(float) * (size_t)a.vec_floats;
    if (smem > 220 * 1024) return LLS_ERR_UNSUPPORTED;
    aa.g = c.g; aa.bvec = c.b; aa.xsol = c.x; aa.gA = c.gA; aa.ldga = c.ldga; aa.gb = c.gb;
    LLS_CUDA_TRY(cudaFuncSetAttribute(adjoint_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    LLS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, adjoint_kernel, kKThreads, smem));
    if (per_sm < 1) return LLS_ERR_UNSUPPORTED;
    const int maxg = sms * (per_sm < kMaxGridPerSm ? per_sm : kMaxGridPerSm);
    const long long work = (long long)c.m * c.n;
    int grid = (int)((work + (1 << 16) - 1) >> 16);
    if (grid < 1) grid = 1;
    if (grid > maxg) grid = maxg;
    KLayout L = k_layout(c.m, c.n, grid);
    if (L.total > c.scratch_bytes) return LLS_ERR_WORKSPACE;
    a.At = nullptr;
    char* base = (char*)c.scratch;
    a.r = (double*)(base + L.off_r); a.q = (double*)(base + L.off_q);
    a.t = (double*)(base + L.off_t); a.p = (double*)(base + L.off_p);
    a.s = (double*)(base + L.off_s); a.u = (double*)(base + L.off_u); a.d = (double*)(base + L.off_d);
    a.qpart = (double*)(base + L.off_qpart); a.upart = (double*)(base + L.off_upart);
    a.v1part = (double*)(base + L.off_v1); a.v2part = (double*)(base + L.off_v2);
    a.bpart = (double*)(base + L.off_bpart);
    a.bar = (unsigned*)(base + L.off_bar);
    a.rdf = (float2*)(base + L.off_rdf); a.tdf = (float2*)(base + L.off_tdf);
    a.udf = (float2*)(base + L.off_udf); a.pdf = (float2*)(base + L.off_pdf);
    a.nrt = L.nrt; a.nck = L.nck; a.nrc = L.nrc; a.ncg = L.ncg; a.colchunk = L.colchunk;
    a.at_rows = L.at_rows; a.at_cpr = L.at_cpr;
    LLS_CUDA_TRY(cudaMemsetAsync(a.bar, 0, 64, st));
    void* args[] = {&aa};
    LLS_CUDA_TRY(cudaLaunchCooperativeKernel((void*)adjoint_kernel, dim3(grid), dim3(kKThreads), args, smem, st));
    note_launch("adjoint", st);
    return LLS_OK;
}

}  // namespace lls
